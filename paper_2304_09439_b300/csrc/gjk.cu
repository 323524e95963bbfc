// UCF-GJK: the analytical comparator of the paper (Sec. IV-B, Claim 1; the
// "range of parameters in UCF-GJK" of its hyper-parameter table): every
// non-convex shape is a union of convex elements (a convex decomposition), a
// pair collides when any pair of elements intersects, and each element pair
// is tested by GJK run for a fixed number of iterations -- a uniform
// computational flow, the same work for every pair, which is what lets it run
// batched on a GPU.  Its accuracy is traded against time through the number
// of iterations, of elements and of hull vertices.
//
// GJK (Gilbert, Johnson, Keerthi 1988) on the Minkowski difference A - B of
// two convex hulls, written in A's body frame: support s(d) = argmax_a a.d -
// argmax_b b.(-d); the simplex (point, segment, triangle, tetrahedron) is
// reduced after each new support point to the feature closest to the origin
// and the search direction points from that feature towards the origin; a
// support point that does not pass the origin along d proves separation, a
// tetrahedron that encloses the origin proves intersection.  After the fixed
// number of iterations an undecided pair counts as intersecting (reading: the
// test has not found a separating direction).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "handle.cuh"

namespace locc {
namespace {

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator-(V3 a) { return v3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// (a x b) x a: the component of b orthogonal to a, scaled
__device__ __forceinline__ V3 triple(V3 a, V3 b) { return cross(cross(a, b), a); }

struct GjkFrame {
  float R[9];  // R_rel = R_A^T R_B (B's body frame -> A's)
  V3 t;        // t_rel = R_A^T (t_B - t_A)
};

__device__ __forceinline__ V3 support_A(const float4* v, int n, V3 d) {
  float best = -INFINITY;
  V3 s = v3(0.f, 0.f, 0.f);
  for (int i = 0; i < n; ++i) {
    const float4 p = v[i];
    const float h = p.x * d.x + p.y * d.y + p.z * d.z;
    if (h > best) best = h, s = v3(p.x, p.y, p.z);
  }
  return s;
}

// support of B's element in A's frame along d: R (argmax_b b . R^T d) + t
__device__ __forceinline__ V3 support_B(const float4* v, int n, V3 d, const GjkFrame& f) {
  const V3 db = v3(f.R[0] * d.x + f.R[3] * d.y + f.R[6] * d.z, f.R[1] * d.x + f.R[4] * d.y + f.R[7] * d.z,
                   f.R[2] * d.x + f.R[5] * d.y + f.R[8] * d.z);
  const V3 b = support_A(v, n, db);
  return v3(f.R[0] * b.x + f.R[1] * b.y + f.R[2] * b.z + f.t.x,
            f.R[3] * b.x + f.R[4] * b.y + f.R[5] * b.z + f.t.y,
            f.R[6] * b.x + f.R[7] * b.y + f.R[8] * b.z + f.t.z);
}

// Reduce the simplex s[0..n) (s[0] the newest point) to the feature nearest
// the origin and set the new direction; true when the origin is enclosed (or
// lies on the simplex).  A tetrahedron is first cut to the face whose outside
// holds the origin, which the triangle case then reduces further.
__device__ __forceinline__ bool reduce(V3* s, int& n, V3& d) {
  const V3 a = s[0], ao = -a;
  if (n == 4) {
    const V3 b = s[1], c = s[2], dd = s[3];
    const V3 ab = b - a, ac = c - a, ad = dd - a;
    const V3 abc = cross(ab, ac), acd = cross(ac, ad), adb = cross(ad, ab);
    // orient each face normal away from the opposite vertex
    const float sabc = dot(abc, ad) > 0.f ? -1.f : 1.f;
    const float sacd = dot(acd, ab) > 0.f ? -1.f : 1.f;
    const float sadb = dot(adb, ac) > 0.f ? -1.f : 1.f;
    if (sabc * dot(abc, ao) > 0.f) {
      n = 3;  // a, b, c
    } else if (sacd * dot(acd, ao) > 0.f) {
      s[1] = c;
      s[2] = dd;
      n = 3;
    } else if (sadb * dot(adb, ao) > 0.f) {
      s[1] = dd;
      s[2] = b;
      n = 3;
    } else {
      return true;  // inside all four faces
    }
  }
  if (n == 3) {
    const V3 b = s[1], c = s[2];
    const V3 ab = b - a, ac = c - a, abc = cross(ab, ac);
    if (dot(cross(abc, ac), ao) > 0.f) {
      if (dot(ac, ao) > 0.f) {
        s[1] = c;
        n = 2;
        d = triple(ac, ao);
      } else if (dot(ab, ao) > 0.f) {
        n = 2;
        d = triple(ab, ao);
      } else {
        n = 1;
        d = ao;
      }
    } else if (dot(cross(ab, abc), ao) > 0.f) {
      if (dot(ab, ao) > 0.f) {
        n = 2;
        d = triple(ab, ao);
      } else {
        n = 1;
        d = ao;
      }
    } else if (dot(abc, ao) > 0.f) {
      d = abc;
    } else {
      s[1] = c;
      s[2] = b;
      d = -abc;
    }
  } else if (n == 2) {
    const V3 ab = s[1] - a;
    if (dot(ab, ao) > 0.f) {
      d = triple(ab, ao);
    } else {
      n = 1;
      d = ao;
    }
  }
  return dot(d, d) <= 1e-12f;  // the origin lies on the current feature
}

// GJK with a fixed iteration count on element A (A's frame) and element B.
__device__ __forceinline__ bool gjk_pair(const float4* va, int na, const float4* vb, int nb,
                                         const GjkFrame& f, int iters) {
  V3 d = v3(1.f, 0.f, 0.f);
  V3 s[4];
  s[0] = support_A(va, na, d) - support_B(vb, nb, -d, f);
  int n = 1;
  d = -s[0];
  bool decided = false, hit = true;
  if (dot(d, d) <= 1e-12f) decided = true;  // the origin is a support point
  for (int it = 0; it < iters; ++it) {
    if (decided) continue;  // same trip count for every pair
    const V3 p = support_A(va, na, d) - support_B(vb, nb, -d, f);
    if (dot(p, d) < 0.f) {
      decided = true;
      hit = false;
      continue;
    }
    for (int k = n; k > 0; --k) s[k] = s[k - 1];
    s[0] = p;
    ++n;
    if (reduce(s, n, d)) decided = true;
  }
  return hit;
}

// One warp per pair; lanes take the element pairs.  collide[p] = 1 when any
// element pair intersects, 0 otherwise, 0xff for an out-of-range pair.
__global__ void __launch_bounds__(256)
    gjk_kernel(PairInputs in, int n_shapes, const int32_t* __restrict__ elem_off,
               const int32_t* __restrict__ vert_off, const float4* __restrict__ verts, int iters,
               uint8_t* __restrict__ collide, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < in.n_pairs; p += warps) {
    int a, b, sa, sb;
    if (!load_pair(in, n_shapes, p, &a, &b, &sa, &sb, lane == 0 ? err : nullptr)) {
      if (lane == 0) collide[p] = 0xff;
      continue;
    }
    GjkFrame f;
    {
      float RA[9], RB[9];
      const float* pa = in.poses + 7 * (size_t)a;
      const float* pb = in.poses + 7 * (size_t)b;
      quat_to_rot(pa, RA);
      quat_to_rot(pb, RB);
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
          f.R[3 * i + k] = RA[i] * RB[k] + RA[3 + i] * RB[3 + k] + RA[6 + i] * RB[6 + k];
      const float dx = pb[4] - pa[4], dy = pb[5] - pa[5], dz = pb[6] - pa[6];
      f.t = v3(RA[0] * dx + RA[3] * dy + RA[6] * dz, RA[1] * dx + RA[4] * dy + RA[7] * dz,
               RA[2] * dx + RA[5] * dy + RA[8] * dz);
    }
    const int ea = elem_off[sa], na = elem_off[sa + 1] - ea;
    const int eb = elem_off[sb], nb = elem_off[sb + 1] - eb;
    bool hit = false;
    for (int e = lane; e < na * nb; e += 32) {
      const int i = ea + e / nb, j = eb + e % nb;
      hit |= gjk_pair(verts + vert_off[i], vert_off[i + 1] - vert_off[i], verts + vert_off[j],
                      vert_off[j + 1] - vert_off[j], f, iters);
    }
    const bool any = __any_sync(0xffffffffu, hit);
    if (lane == 0) collide[p] = any ? 1 : 0;
  }
}

}  // namespace
}  // namespace locc

using namespace locc;

struct locc_gjk {
  int n_shapes = 0, n_elems = 0, n_verts = 0, n_sm = 148;
  int32_t* d_elem_off = nullptr;
  int32_t* d_vert_off = nullptr;
  float4* d_verts = nullptr;
  int* d_err = nullptr;
};

extern "C" {

int locc_gjk_create(int32_t n_shapes, const int32_t* elem_off, const int32_t* vert_off,
                    const float* verts, locc_gjk** out) {
  if (!out) {
    set_error("out is NULL");
    return LOCC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (n_shapes < 1 || !elem_off || !vert_off || !verts || elem_off[0] != 0) {
    set_error("invalid convex decomposition");
    return LOCC_ERR_INVALID_ARG;
  }
  const int E = elem_off[n_shapes];
  for (int s = 0; s < n_shapes; ++s)
    if (elem_off[s + 1] <= elem_off[s]) {
      set_error("every shape needs at least one convex element");
      return LOCC_ERR_INVALID_ARG;
    }
  if (vert_off[0] != 0) {
    set_error("vert_off[0] must be 0");
    return LOCC_ERR_INVALID_ARG;
  }
  for (int e = 0; e < E; ++e)
    if (vert_off[e + 1] <= vert_off[e]) {
      set_error("every convex element needs at least one vertex");
      return LOCC_ERR_INVALID_ARG;
    }
  const int V = vert_off[E];
  std::vector<float4> v4(V);
  for (int i = 0; i < V; ++i) v4[i] = make_float4(verts[3 * i], verts[3 * i + 1], verts[3 * i + 2], 0.f);
  auto* h = new locc_gjk();
  h->n_shapes = n_shapes, h->n_elems = E, h->n_verts = V;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  bool ok = cudaMalloc(&h->d_elem_off, (n_shapes + 1) * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&h->d_vert_off, (E + 1) * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&h->d_verts, V * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&h->d_err, sizeof(int)) == cudaSuccess;
  ok = ok &&
       cudaMemcpy(h->d_elem_off, elem_off, (n_shapes + 1) * sizeof(int32_t), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(h->d_vert_off, vert_off, (E + 1) * sizeof(int32_t), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(h->d_verts, v4.data(), V * sizeof(float4), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->d_err, 0, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    locc_gjk_destroy(h);
    set_error("GJK handle: device allocation or copy failed");
    return LOCC_ERR_OOM;
  }
  *out = h;
  return LOCC_OK;
}

int locc_gjk_detect(locc_gjk* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                    const int32_t* pairs, int32_t n_pairs, int32_t iterations, uint8_t* collide,
                    void* stream) {
  if (!h || n_pairs < 0 || n_obj < 0 || iterations < 1 || iterations > 1024) {
    set_error("invalid GJK arguments");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !collide) {
    set_error("NULL array argument");
    return LOCC_ERR_INVALID_ARG;
  }
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  const int grid = std::min((n_pairs + 7) / 8, 8 * h->n_sm);
  gjk_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      in, h->n_shapes, h->d_elem_off, h->d_vert_off, h->d_verts, iterations, collide, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("gjk_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

int locc_gjk_status(locc_gjk* h, void* stream) {
  if (!h) {
    set_error("handle is NULL");
    return LOCC_ERR_INVALID_ARG;
  }
  int err = 0;
  auto st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    set_error("GJK status: CUDA error");
    return LOCC_ERR_CUDA;
  }
  if (err) {
    cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    set_error("a pair had an out-of-range object index or shape id");
    return LOCC_ERR_BAD_INDEX;
  }
  return LOCC_OK;
}

void locc_gjk_destroy(locc_gjk* h) {
  if (!h) return;
  cudaFree(h->d_elem_off);
  cudaFree(h->d_vert_off);
  cudaFree(h->d_verts);
  cudaFree(h->d_err);
  delete h;
}

}  // extern "C"

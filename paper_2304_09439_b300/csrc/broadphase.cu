// AABB broadphase: candidate pairs of every environment.
//
// Paper: Sec. II, footnote 1 -- far-apart objects are ruled out in the broad
// phase before the narrow phase runs.  Each object's posed body box is
// enclosed in a world axis-aligned box (centre R c + t, half extents |R| h);
// every pair (i, j), i < j, of one environment whose world boxes overlap on all
// three axes (|c_i - c_j| <= h_i + h_j) becomes a candidate.  The float32
// arithmetic uses round-to-nearest intrinsics in a fixed order, so the pair
// list is reproducible bit for bit.
//
// Three launches keep the output in (environment, i, j) order without
// atomics: count per environment (one warp each), exclusive scan of the
// counts (one CTA), write (one warp each, ballot + popc compaction).
#include "common.cuh"
#include "handle.cuh"

namespace locc {
namespace {

constexpr int BP_WARPS = 4;
constexpr int BP_CACHE = 128;  // objects per environment kept in shared memory

__device__ __forceinline__ void world_box(const DevLibrary& lib, const float* poses,
                                          const int32_t* obj_shape, int o, float4* c4,
                                          float4* h4, int* err) {
  int s = obj_shape[o];
  if (s < 0 || s >= lib.n_shapes) {
    atomicOr(err, 1);
    const float nan = __int_as_float(0x7fc00000);
    *c4 = make_float4(nan, nan, nan, 0.f);
    *h4 = make_float4(nan, nan, nan, 0.f);
    return;
  }
  const float* q = poses + 7 * (size_t)o;
  float R[9];
  quat_to_rot(q, R);
  const float4 lo = lib.aabb[2 * s], hi = lib.aabb[2 * s + 1];
  const float cl[3] = {fmul(fadd(lo.x, hi.x), 0.5f), fmul(fadd(lo.y, hi.y), 0.5f),
                       fmul(fadd(lo.z, hi.z), 0.5f)};
  const float hl[3] = {fmul(fsub(hi.x, lo.x), 0.5f), fmul(fsub(hi.y, lo.y), 0.5f),
                       fmul(fsub(hi.z, lo.z), 0.5f)};
  float c[3], h[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c[i] = fadd(dot3_rn(R[3 * i], R[3 * i + 1], R[3 * i + 2], cl[0], cl[1], cl[2]), q[4 + i]);
    h[i] = dot3_rn(fabsf(R[3 * i]), fabsf(R[3 * i + 1]), fabsf(R[3 * i + 2]), hl[0], hl[1], hl[2]);
  }
  *c4 = make_float4(c[0], c[1], c[2], 0.f);
  *h4 = make_float4(h[0], h[1], h[2], 0.f);
}

__device__ __forceinline__ bool overlap(float4 ca, float4 ha, float4 cb, float4 hb) {
  return fabsf(fsub(ca.x, cb.x)) <= fadd(ha.x, hb.x) &&
         fabsf(fsub(ca.y, cb.y)) <= fadd(ha.y, hb.y) &&
         fabsf(fsub(ca.z, cb.z)) <= fadd(ha.z, hb.z);
}

// MODE 0: count pairs of each environment into counts[e].
// MODE 1: write pairs at offsets[e].
template <int MODE>
__global__ void __launch_bounds__(32 * BP_WARPS) bp_kernel(DevLibrary lib, const float* poses,
                                                           const int32_t* obj_shape,
                                                           const int32_t* env_offsets, int n_env,
                                                           int32_t* counts, int32_t* pairs_out,
                                                           int max_pairs, int* err) {
  __shared__ float4 cache[BP_WARPS][BP_CACHE][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * BP_WARPS + warp;
  if (e >= n_env) return;
  const int o0 = env_offsets[e], o1 = env_offsets[e + 1];
  const int n = o1 - o0;
  if (n <= 1) {
    if (MODE == 0 && lane == 0) counts[e] = 0;
    return;
  }
  const bool cached = n <= BP_CACHE;
  if (cached) {
    for (int i = lane; i < n; i += 32)
      world_box(lib, poses, obj_shape, o0 + i, &cache[warp][i][0], &cache[warp][i][1], err);
  }
  __syncwarp();
  int base = MODE == 1 ? counts[e] : 0;  // in MODE 1 counts holds the offsets
  for (int i = 0; i < n - 1; ++i) {
    float4 ci, hi;
    if (cached) ci = cache[warp][i][0], hi = cache[warp][i][1];
    else world_box(lib, poses, obj_shape, o0 + i, &ci, &hi, err);
    for (int j0 = i + 1; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      bool hit = false;
      if (j < n) {
        float4 cj, hj;
        if (cached) cj = cache[warp][j][0], hj = cache[warp][j][1];
        else world_box(lib, poses, obj_shape, o0 + j, &cj, &hj, err);
        hit = overlap(ci, hi, cj, hj);
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (MODE == 1 && hit) {
        const int slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < max_pairs) {
          pairs_out[2 * (size_t)slot] = o0 + i;
          pairs_out[2 * (size_t)slot + 1] = o0 + j;
        }
      }
      base += __popc(m);
    }
  }
  if (MODE == 0 && lane == 0) counts[e] = base;
}

// Exclusive scan of counts[0..n) in place; total -> *total.  One CTA.
__global__ void __launch_bounds__(1024) bp_scan_kernel(int32_t* counts, int n, int32_t* total) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;  // exclusive prefix of this thread's chunk
  for (int i = lo; i < hi; ++i) {
    const int c = counts[i];
    counts[i] = run;
    run += c;
  }
  if (t == 1023) *total = part[1023];
}

}  // namespace

int broadphase_run(locc_handle* h, const float* poses, const int32_t* obj_shape,
                   const int32_t* env_offsets, int n_env, int32_t* pairs_out,
                   int32_t* n_pairs_out, int max_pairs, cudaStream_t stream) {
  if (n_env <= 0) {
    return cudaMemsetAsync(n_pairs_out, 0, sizeof(int32_t), stream) == cudaSuccess ? LOCC_OK
                                                                                   : LOCC_ERR_CUDA;
  }
  const int st = ensure_env_capacity(h, n_env, stream);
  if (st) return st;
  const DevLibrary lib = dev_library(h);
  const int grid = (n_env + BP_WARPS - 1) / BP_WARPS;
  bp_kernel<0><<<grid, 32 * BP_WARPS, 0, stream>>>(lib, poses, obj_shape, env_offsets, n_env,
                                                   h->d_env_counts, pairs_out, max_pairs, h->d_err);
  bp_scan_kernel<<<1, 1024, 0, stream>>>(h->d_env_counts, n_env, n_pairs_out);
  bp_kernel<1><<<grid, 32 * BP_WARPS, 0, stream>>>(lib, poses, obj_shape, env_offsets, n_env,
                                                   h->d_env_counts, pairs_out, max_pairs, h->d_err);
  return cudaGetLastError() == cudaSuccess ? LOCC_OK : LOCC_ERR_CUDA;
}

}  // namespace locc

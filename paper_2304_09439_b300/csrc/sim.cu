// Contact resolution driven by the detector's outputs: one rigid-body step of
// every object (gravity, an analytic ground plane z = 0, and pair contacts
// from a contact array in the detector's output format), for simulations
// whose object-object contacts come from the contact network (Sec. IV-C: the
// network is integrated into a GPU simulator with a contact-resolution step;
// Table 2 measures how far apart or interpenetrating objects are whenever a
// contact arises).
//
// The resolution is a penalty method (the paper names its contact solver only
// by reference): a contact of penetration depth d >= 0 along the unit normal n
// (from A towards B) at the world point p pushes B by
//   F = max(0, k_contact d - c_contact v_n) n,  v_n = (v_B(p) - v_A(p)) . n,
// and A by -F, both at p (so they also turn); a body-box corner below the
// plane pushes its object up by max(0, k_plane pen - c_plane v_z) with a
// viscous tangential term -mu_plane (v_x, v_y).  Objects have unit mass and
// the inertia of a solid box filling their body AABB.  Semi-implicit Euler
// with linear and angular damping; the quaternion is renormalised.
#include <algorithm>

#include "common.cuh"
#include "handle.cuh"

namespace locc {
namespace {

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Pair contacts: out[p] = {logit, point xyz, normal xyz, depth} (world).
// acc [n_obj][6] = force, torque (world, about the object's centre).
__global__ void sim_pair_kernel(const float* __restrict__ out, const int32_t* __restrict__ pairs,
                                const int32_t* __restrict__ n_dev, int n_cap, int n_obj,
                                const float* __restrict__ poses, const float* __restrict__ vel,
                                locc_sim_params prm, float* __restrict__ acc) {
  int n = n_cap;
  if (n_dev) n = min(*n_dev, n_cap);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const float* o = out + 8 * (size_t)p;
    const int a = pairs[2 * p], b = pairs[2 * p + 1];
    if (!(o[0] > 0.f) || a < 0 || b < 0 || a >= n_obj || b >= n_obj) continue;  // no contact / NaN
    const float d = fmaxf(o[7], 0.f);
    const float pt[3] = {o[1], o[2], o[3]}, nn[3] = {o[4], o[5], o[6]};
    float rA[3], rB[3], vA[3], vB[3], t[3];
    for (int k = 0; k < 3; ++k) {
      rA[k] = pt[k] - poses[7 * a + 4 + k];
      rB[k] = pt[k] - poses[7 * b + 4 + k];
    }
    cross3(vel + 6 * a + 3, rA, t);
    for (int k = 0; k < 3; ++k) vA[k] = vel[6 * a + k] + t[k];
    cross3(vel + 6 * b + 3, rB, t);
    for (int k = 0; k < 3; ++k) vB[k] = vel[6 * b + k] + t[k];
    const float vn = (vB[0] - vA[0]) * nn[0] + (vB[1] - vA[1]) * nn[1] + (vB[2] - vA[2]) * nn[2];
    const float f = fmaxf(prm.k_contact * d - prm.c_contact * vn, 0.f);
    if (f == 0.f) continue;
    const float F[3] = {f * nn[0], f * nn[1], f * nn[2]};
    float tA[3], tB[3];
    cross3(rB, F, tB);
    cross3(rA, F, tA);
    for (int k = 0; k < 3; ++k) {
      atomicAdd(acc + 6 * b + k, F[k]);
      atomicAdd(acc + 6 * b + 3 + k, tB[k]);
      atomicAdd(acc + 6 * a + k, -F[k]);
      atomicAdd(acc + 6 * a + 3 + k, -tA[k]);
    }
  }
}

// Gravity, ground plane and integration of every object; clears acc.
__global__ void sim_integrate_kernel(float* __restrict__ poses, float* __restrict__ vel,
                                     const int32_t* __restrict__ obj_shape, int n_obj,
                                     const float4* __restrict__ aabb, int n_shapes,
                                     locc_sim_params prm, float* __restrict__ acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_obj) return;
  float* P = poses + 7 * (size_t)i;
  float* V = vel + 6 * (size_t)i;
  float F[3], T[3];
  for (int k = 0; k < 3; ++k) {
    F[k] = acc[6 * i + k];
    T[k] = acc[6 * i + 3 + k];
    acc[6 * i + k] = 0.f;
    acc[6 * i + 3 + k] = 0.f;
  }
  const int s = obj_shape[i];
  if (s < 0 || s >= n_shapes) return;
  const float4 lo = aabb[2 * s], hi = aabb[2 * s + 1];
  float R[9];
  quat_to_rot(P, R);
  // ground plane: the eight corners of the body box
  for (int c = 0; c < 8; ++c) {
    const float b[3] = {(c & 1) ? hi.x : lo.x, (c & 2) ? hi.y : lo.y, (c & 4) ? hi.z : lo.z};
    float r[3];
    for (int k = 0; k < 3; ++k) r[k] = R[3 * k] * b[0] + R[3 * k + 1] * b[1] + R[3 * k + 2] * b[2];
    const float z = r[2] + P[6];
    if (z >= 0.f) continue;
    float wr[3];
    cross3(V + 3, r, wr);
    const float vc[3] = {V[0] + wr[0], V[1] + wr[1], V[2] + wr[2]};
    const float fz = fmaxf(prm.k_plane * (-z) - prm.c_plane * vc[2], 0.f);
    const float fc[3] = {-prm.mu_plane * vc[0], -prm.mu_plane * vc[1], fz};
    float tc[3];
    cross3(r, fc, tc);
    for (int k = 0; k < 3; ++k) {
      F[k] += fc[k];
      T[k] += tc[k];
    }
  }
  F[2] -= prm.gravity;  // unit mass
  // inverse inertia of a solid box of unit mass: 12 / (e_j^2 + e_k^2)
  const float ex = hi.x - lo.x, ey = hi.y - lo.y, ez = hi.z - lo.z;
  const float inv[3] = {12.f / fmaxf(ey * ey + ez * ez, 1e-12f), 12.f / fmaxf(ex * ex + ez * ez, 1e-12f),
                        12.f / fmaxf(ex * ex + ey * ey, 1e-12f)};
  // world angular acceleration R diag(inv) R^T T
  float tb[3], alpha[3];
  for (int k = 0; k < 3; ++k) tb[k] = (R[k] * T[0] + R[3 + k] * T[1] + R[6 + k] * T[2]) * inv[k];
  for (int k = 0; k < 3; ++k) alpha[k] = R[3 * k] * tb[0] + R[3 * k + 1] * tb[1] + R[3 * k + 2] * tb[2];
  const float dt = prm.dt;
  const float ld = fmaxf(1.f - prm.lin_damp * dt, 0.f), ad = fmaxf(1.f - prm.ang_damp * dt, 0.f);
  for (int k = 0; k < 3; ++k) {
    V[k] = (V[k] + dt * F[k]) * ld;
    V[3 + k] = (V[3 + k] + dt * alpha[k]) * ad;
    P[4 + k] += dt * V[k];
  }
  // q += dt / 2 (0, w) q, renormalised
  const float w = P[0], x = P[1], y = P[2], z = P[3];
  const float ox = V[3], oy = V[4], oz = V[5];
  float q[4] = {w + 0.5f * dt * (-ox * x - oy * y - oz * z), x + 0.5f * dt * (ox * w + oy * z - oz * y),
                y + 0.5f * dt * (oy * w + oz * x - ox * z), z + 0.5f * dt * (oz * w + ox * y - oy * x)};
  const float nq = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) P[k] = q[k] * nq;
}

// Bounding-sphere contacts in the detector's output format (a proxy-geometry
// contact source to compare the network against): pair touches when
// |x_B - x_A| < r_A + r_B; depth = r_A + r_B - |x_B - x_A|, normal along
// x_B - x_A, point halfway between the sphere surfaces.
__global__ void sim_sphere_contacts_kernel(const int32_t* __restrict__ pairs,
                                           const int32_t* __restrict__ n_dev, int n_cap,
                                           const float* __restrict__ poses,
                                           const int32_t* __restrict__ obj_shape, int n_obj,
                                           const float* __restrict__ radius, int n_shapes,
                                           float* __restrict__ out) {
  int n = n_cap;
  if (n_dev) n = min(*n_dev, n_cap);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    float* o = out + 8 * (size_t)p;
    const int a = pairs[2 * p], b = pairs[2 * p + 1];
    if (a < 0 || b < 0 || a >= n_obj || b >= n_obj || obj_shape[a] < 0 || obj_shape[b] < 0 ||
        obj_shape[a] >= n_shapes || obj_shape[b] >= n_shapes) {
      for (int k = 0; k < 8; ++k) o[k] = __int_as_float(0x7fc00000);
      continue;
    }
    const float ra = radius[obj_shape[a]], rb = radius[obj_shape[b]];
    float d[3], len2 = 0.f;
    for (int k = 0; k < 3; ++k) {
      d[k] = poses[7 * b + 4 + k] - poses[7 * a + 4 + k];
      len2 += d[k] * d[k];
    }
    const float len = sqrtf(len2), pen = ra + rb - len;
    const float inv = len > 1e-12f ? 1.f / len : 0.f;
    o[0] = pen;
    for (int k = 0; k < 3; ++k) {
      const float nk = len > 1e-12f ? d[k] * inv : (k == 2 ? 1.f : 0.f);
      o[4 + k] = nk;
      o[1 + k] = poses[7 * a + 4 + k] + nk * (ra - 0.5f * pen);
    }
    o[7] = pen;
  }
}

}  // namespace
}  // namespace locc

using namespace locc;

extern "C" {

int locc_sim_step(locc_handle* h, const locc_sim_params* prm, float* poses, float* vel,
                  const int32_t* obj_shape, int32_t n_obj, const int32_t* pairs,
                  const int32_t* n_pairs_dev, int32_t max_pairs, const float* contacts,
                  float* acc, void* stream) {
  if (!h || !prm || !poses || !vel || !obj_shape || !acc) {
    set_error("NULL argument");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_obj < 0 || max_pairs < 0 || (max_pairs > 0 && (!pairs || !contacts))) {
    set_error("invalid size or NULL pair arrays");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_obj == 0) return LOCC_OK;
  auto st = static_cast<cudaStream_t>(stream);
  if (max_pairs > 0) {
    const int grid = std::min((max_pairs + 255) / 256, 4 * h->n_sm);
    sim_pair_kernel<<<grid, 256, 0, st>>>(contacts, pairs, n_pairs_dev, max_pairs, n_obj, poses,
                                          vel, *prm, acc);
  }
  const DevLibrary lib = dev_library(h);
  sim_integrate_kernel<<<(n_obj + 127) / 128, 128, 0, st>>>(poses, vel, obj_shape, n_obj, lib.aabb,
                                                            lib.n_shapes, *prm, acc);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("simulation kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

int locc_sphere_contacts(locc_handle* h, const float* poses, const int32_t* obj_shape,
                         int32_t n_obj, const int32_t* pairs, const int32_t* n_pairs_dev,
                         int32_t max_pairs, const float* radius, float* out, void* stream) {
  if (!h || !poses || !obj_shape || !radius || (max_pairs > 0 && (!pairs || !out))) {
    set_error("NULL argument");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_obj < 0 || max_pairs < 0) {
    set_error("negative size");
    return LOCC_ERR_INVALID_ARG;
  }
  if (max_pairs == 0) return LOCC_OK;
  const int grid = std::min((max_pairs + 255) / 256, 4 * h->n_sm);
  sim_sphere_contacts_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      pairs, n_pairs_dev, max_pairs, poses, obj_shape, n_obj, radius, dev_library(h).n_shapes, out);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("sphere contact kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

}  // extern "C"

// Shared definitions of the sm_103a contact-detection library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/locc.h"

namespace locc {

constexpr int KMAX = LOCC_CROP_POINTS;   // points per object crop
constexpr int ROWS = 2 * KMAX;           // crop rows per pair (A then B)
constexpr int FEAT = 256;                // pooled feature per object
constexpr int OUTD = LOCC_OUT_DIM;
constexpr int BLOCK_PTS = 32;            // library points per culling block

// Layer dimensions (in, out): encoder 3-64-128-256, head 512-256-256-8.
constexpr int L_IN[6] = {3, 64, 128, 512, 256, 256};
constexpr int L_OUT[6] = {64, 128, 256, 256, 256, 8};

// Device copy of the shape library.
//   points: [S][n_pad] float4 (x, y, z, bits = (orig_index)), blocks of 32
//           points in Morton order, tail padded with NaN points;
//   blocks: [S][n_blocks][2] float4 (lo, hi) bounding box of each block;
//   aabb:   [S][2] float4 (lo, hi) body box of each shape.
struct DevLibrary {
  const float4* points;
  const float4* blocks;
  const float4* aabb;
  const int32_t* inv;  // [S][n_points]: storage position of sample index i
  int n_shapes;
  int n_points;
  int n_pad;
  int n_blocks;
};

// Pair-level inputs shared by every kernel of the path.
struct PairInputs {
  const float* poses;       // [n_obj][7]
  const int32_t* obj_shape; // [n_obj]
  const int32_t* pairs;     // [n_pairs][2]
  int n_obj;
  int n_pairs;
};

// The pairs a launch works on: chunk `chunk` of `n_chunks` equal parts of
// [0, n), where n = min(*n_dev, n_cap) when the count lives on the device
// (n_dev != NULL) and n_cap otherwise.  Chunks let the crop gather of one part
// run on one stream while the network runs on the previous part on another.
struct PairRange {
  int n_cap;
  const int* n_dev;
  int chunk;
  int n_chunks;
};

__host__ __device__ inline PairRange whole_range(int n, const int* n_dev) {
  return PairRange{n, n_dev, 0, 1};
}

__device__ __forceinline__ void range_bounds(const PairRange& r, int* lo, int* hi) {
  int n = r.n_cap;
  if (r.n_dev) n = min(*r.n_dev, r.n_cap);
  if (n < 0) n = 0;
  *lo = (int)(((long long)n * r.chunk) / r.n_chunks);
  *hi = (int)(((long long)n * (r.chunk + 1)) / r.n_chunks);
}

// Pooled-feature operand tiles of the tensor-core heads, per 128 pairs:
// BF16: 32 K-chunks of 16 features, each a [128 x 16] bf16 hi tile and a lo
// tile FT_SUB bytes further (K-major, no swizzle); FP8: 8 K-chunks of 64
// e4m3 features of 8 KB each.
constexpr int FT_K = 16;                         // features per BF16 chunk
constexpr int FT_SUB = 128 * FT_K * 2;           // one [128 x 16] bf16 tile
constexpr int FT_CHUNK = 2 * FT_SUB;             // hi + lo
constexpr int FT_TILE = (512 / FT_K) * FT_CHUNK; // BF16 tile of 128 pairs
constexpr int FT8_TILE = 128 * 512;              // e4m3 tile of 128 pairs

// Zero pooled feature of object `side` of pair row rel (relative to the
// launch's first pair), written by one warp: an empty crop pools to exactly
// 0.  BF16: 64 pieces of 16 bytes (chunk side 16 + i / 4, hi / lo tile, K
// columns 0..7 / 8..15), two per lane; FP8: 16 pieces (chunk side 4 + i / 4,
// a row's 64 bytes as four pieces 128 bytes apart), lanes 0..15.
__device__ __forceinline__ void zero_feat_warp(unsigned char* ftile, int rel, int side, int lane,
                                               bool e4m3) {
  const int r = rel & 127;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  if (e4m3) {
    if (lane < 16)
      *reinterpret_cast<uint4*>(ftile + (size_t)(rel >> 7) * FT8_TILE +
                                (size_t)(side * 4 + (lane >> 2)) * 8192 + (r >> 3) * 512 +
                                (lane & 3) * 128 + (r & 7) * 16) = z;
    return;
  }
  unsigned char* t = ftile + (size_t)(rel >> 7) * FT_TILE + (r >> 3) * 256 + (r & 7) * 16;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    *reinterpret_cast<uint4*>(t + (size_t)(side * 16 + (i >> 2)) * FT_CHUNK +
                              ((i >> 1) & 1) * FT_SUB + (i & 1) * 128) = z;
  }
}

// One warp zeroes the pooled features of the objects with crop count 0 among
// its CTA's slice of the launch's objects [2 lo, 2 hi): every CTA of the
// grid takes a contiguous, 32-aligned slice, so that all objects are covered
// whatever the number of CTAs that have encoder tiles.
__device__ __forceinline__ void zero_empty_objects(const int32_t* cnt, unsigned char* ftile, int lo,
                                                   int hi, int lane, bool e4m3) {
  const int n_obj = 2 * (hi - lo);
  const int per = ((n_obj + (int)gridDim.x - 1) / (int)gridDim.x + 31) & ~31;
  const int o0 = (int)blockIdx.x * per, o1 = min(o0 + per, n_obj);
  for (int b = o0; b < o1; b += 32) {
    const int i = b + lane;
    unsigned em = __ballot_sync(0xffffffffu, i < o1 && cnt[2 * (size_t)lo + i] == 0);
    while (em) {
      const int j = b + __ffs(em) - 1;
      em &= em - 1;
      zero_feat_warp(ftile, j >> 1, j & 1, lane, e4m3);
    }
  }
}

// Float32 parameters for the CUDA-core kernels: per layer W^T [in][out]
// followed by b [out].
struct Fp32Params {
  const float* wt[6];
  const float* b[6];
};

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }

// (a0 b0 + a1 b1) + a2 b2, every operation rounded separately (no FMA).
__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0,
                                         float b1, float b2) {
  float s = fmul(a0, b0);
  s = fadd(s, fmul(a1, b1));
  return fadd(s, fmul(a2, b2));
}

// Rotation of the unit quaternion (w, x, y, z), row-major R[9], body -> world.
__device__ __forceinline__ void quat_to_rot(const float* q, float* R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  const float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
  const float xy = fmul(x, y), xz = fmul(x, z), yz = fmul(y, z);
  const float wx = fmul(w, x), wy = fmul(w, y), wz = fmul(w, z);
  R[0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
  R[1] = fmul(2.0f, fsub(xy, wz));
  R[2] = fmul(2.0f, fadd(xz, wy));
  R[3] = fmul(2.0f, fadd(xy, wz));
  R[4] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
  R[5] = fmul(2.0f, fsub(yz, wx));
  R[6] = fmul(2.0f, fsub(xz, wy));
  R[7] = fmul(2.0f, fadd(yz, wx));
  R[8] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
}

// Validated indices of pair p; returns false (and raises the error flag) if
// an object index or shape id is out of range.
__device__ __forceinline__ bool load_pair(const PairInputs& in, int n_shapes,
                                          int p, int* a, int* b, int* sa,
                                          int* sb, int* err) {
  const int ia = in.pairs[2 * p], ib = in.pairs[2 * p + 1];
  bool ok = ia >= 0 && ib >= 0 && ia < in.n_obj && ib < in.n_obj;
  int s0 = -1, s1 = -1;
  if (ok) {
    s0 = in.obj_shape[ia];
    s1 = in.obj_shape[ib];
    ok = s0 >= 0 && s1 >= 0 && s0 < n_shapes && s1 < n_shapes;
  }
  if (!ok && err) atomicOr(err, 1);
  *a = ia, *b = ib, *sa = s0, *sb = s1;
  return ok;
}

// Epilogue (shared with the tensor-core head): raw crop-frame outputs y[8] ->
// world frame.  Point: R_A (y[1:4] + c) + t_A; normal: R_A n / max(|n|, 1e-12).
__device__ __forceinline__ void epilogue_world(const float* y, const float* poseA, float4 c, float* o) {
  float R[9];
  quat_to_rot(poseA, R);
  const float px = y[1] + c.x, py = y[2] + c.y, pz = y[3] + c.z;
  float nx = y[4], ny = y[5], nz = y[6];
  const float nn = fmaxf(sqrtf(nx * nx + ny * ny + nz * nz), 1e-12f);
  nx /= nn, ny /= nn, nz /= nn;
  o[0] = y[0];
  o[1] = R[0] * px + R[1] * py + R[2] * pz + poseA[4];
  o[2] = R[3] * px + R[4] * py + R[5] * pz + poseA[5];
  o[3] = R[6] * px + R[7] * py + R[8] * pz + poseA[6];
  o[4] = R[0] * nx + R[1] * ny + R[2] * nz;
  o[5] = R[3] * nx + R[4] * ny + R[5] * nz;
  o[6] = R[6] * nx + R[7] * ny + R[8] * nz;
  o[7] = y[7];
}

}  // namespace locc

// Launchers (defined in the .cu files), all asynchronous on `stream`.
namespace locc {
// n_dev (nullable): device count of pairs actually present (<= n_pairs), read
// by the kernels so that a fixed launch serves a count produced on the device.
// grid_cap (crop): at most this many resident CTAs per SM (0 = occupancy limit).
// defer (crop): device int [2 + 2 * (pairs of one launch)], scratch: defer[0]
// counts the objects left to the exact fallback kernel, defer[1] hands out
// objects to the crop warps, defer[2..] lists the deferred objects.
// mode: LOCC_CROP_LOCAL (nearest-first within the ball) or LOCC_CROP_GLOBAL
// (the first KMAX samples of each shape, same canonical frame).
// list / list_n (local mode, nullable): the object list of the tensor-core
// encoders -- every object with a non-empty crop (2 p + side) is appended to
// list + 2 lo (lo = the chunk's first pair), counted in list_n[chunk] (zeroed
// here before the crop).
cudaError_t launch_crop(const DevLibrary& lib, const PairInputs& in, const PairRange& rg,
                        float r, float4* xyz, int32_t* idx, int32_t* cnt, float4* centre,
                        int* err, int* defer, int n_sm, int grid_cap, cudaStream_t stream,
                        int mode = LOCC_CROP_LOCAL, int* list = nullptr, int* list_n = nullptr);
// Per-device set-up of the kernels above, run by locc_create with the
// handle's device current: loads their modules (so that no later launch
// loads one) and records the crop kernel's occupancy for that device.
cudaError_t prepare_crop_kernels(int device);
// Exact crop of the objects listed in defer (defer[0] = count, defer[2 + i] =
// 2 p + object) into xyz / cnt; a fixed grid that reads the count on the
// device (does nothing when no object was deferred).
cudaError_t launch_crop_fallback(const DevLibrary& lib, const PairInputs& in, float r, float4* xyz,
                                 int32_t* cnt, int* defer, int defer_cap, int n_sm,
                                 cudaStream_t stream);
// Sets the dynamic shared-memory limits of the float32 network kernels.
cudaError_t prepare_fp32_kernels();
cudaError_t launch_encoder_fp32(const float4* xyz, const PairRange& rg,
                                const Fp32Params& prm, float* feat, int n_sm,
                                cudaStream_t stream);
cudaError_t launch_head_fp32(const float* feat, const PairRange& rg,
                             const Fp32Params& prm, const PairInputs* in,
                             const float4* centre, float* out, float* y_raw, int n_sm,
                             cudaStream_t stream);
}  // namespace locc

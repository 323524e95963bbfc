// Plain float32 crop network on CUDA cores (the LOCC_FP32 path).
//
// Paper: Sec. III and appendix -- a point-wise MLP encodes every crop point,
// features are pooled per object, and an MLP head predicts the contact; ReLU on
// all layers.  Here: encoder 3 -> 64 -> 128 -> 256 with ReLU, max-pool over the
// valid points of each object (an empty crop pools to 0), head
// [f_A, f_B] 512 -> 256 -> 256 (ReLU) -> 8, then the epilogue that maps the
// crop-frame point and normal back to the world frame.
//
// encoder_fp32_kernel: one CTA of 256 threads per pair; activations of the
// 128 crop rows stay in shared memory, every thread owns an 8 x 8 register
// tile (8 points x 8 channels); the max-pool runs in registers and warp
// shuffles, so the 128 x 256 layer-3 output is never stored.
// head_fp32_kernel: one CTA of 256 threads per 32 pairs; thread c owns output
// channel c of all 32 pairs; weights are read as W^T so each k step is one
// coalesced row.
#include <algorithm>

#include "common.cuh"

namespace locc {
namespace {

constexpr int ENC_THREADS = 256;
// shared memory: X [128] float4, H1^T [64][128], H2^T [128][128]
constexpr size_t ENC_SMEM = (size_t)ROWS * 16 + (size_t)64 * ROWS * 4 + (size_t)128 * ROWS * 4;

// acc[i][j] += A^T[k][p0 + i] * W^T[k][c0 + j] for k < K.
template <int K>
__device__ __forceinline__ void tile_8x8(const float* __restrict__ AT, const float* __restrict__ WT,
                                         int ldw, int p0, int c0, float (&acc)[8][8]) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(AT + k * ROWS + p0);
    const float4 a1 = *reinterpret_cast<const float4*>(AT + k * ROWS + p0 + 4);
    const float4 b0 = __ldg(reinterpret_cast<const float4*>(WT + (size_t)k * ldw + c0));
    const float4 b1 = __ldg(reinterpret_cast<const float4*>(WT + (size_t)k * ldw + c0 + 4));
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

__device__ __forceinline__ void encode_pair(const float4* __restrict__ xyz, int p, const Fp32Params& prm,
                                            float* __restrict__ feat, unsigned char* smem) {
  float4* X = reinterpret_cast<float4*>(smem);
  float* H1T = reinterpret_cast<float*>(smem + ROWS * 16);
  float* H2T = H1T + 64 * ROWS;
  const int t = threadIdx.x;
  if (t < ROWS) X[t] = xyz[(size_t)p * ROWS + t];
  __syncthreads();
  // layer 1: 3 -> 64
  {
    const int row = t & (ROWS - 1), half = t >> 7;
    const float4 x = X[row];
    const float* W = prm.wt[0];
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int c = half * 32 + j;
      float h = prm.b[0][c];
      h = fmaf(W[0 * 64 + c], x.x, h);
      h = fmaf(W[1 * 64 + c], x.y, h);
      h = fmaf(W[2 * 64 + c], x.z, h);
      H1T[c * ROWS + row] = fmaxf(h, 0.0f);
    }
  }
  __syncthreads();
  const int tp = t & 15, tc = t >> 4;
  const int p0 = tp * 8, c0 = tc * 8;
  // layer 2: 64 -> 128
  {
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    tile_8x8<64>(H1T, prm.wt[1], 128, p0, c0, acc);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float bj = prm.b[1][c0 + j];
      float4 v0 = make_float4(fmaxf(acc[0][j] + bj, 0.f), fmaxf(acc[1][j] + bj, 0.f),
                              fmaxf(acc[2][j] + bj, 0.f), fmaxf(acc[3][j] + bj, 0.f));
      float4 v1 = make_float4(fmaxf(acc[4][j] + bj, 0.f), fmaxf(acc[5][j] + bj, 0.f),
                              fmaxf(acc[6][j] + bj, 0.f), fmaxf(acc[7][j] + bj, 0.f));
      *reinterpret_cast<float4*>(H2T + (c0 + j) * ROWS + p0) = v0;
      *reinterpret_cast<float4*>(H2T + (c0 + j) * ROWS + p0 + 4) = v1;
    }
  }
  __syncthreads();
  // validity of this thread's 8 rows
  bool valid[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) valid[i] = X[p0 + i].w > 0.0f;
  const int obj = tp >> 3;  // rows 0..63 -> A, 64..127 -> B
  // layer 3: 128 -> 256 in two halves of 128 channels, fused max-pool
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int cc = half * 128 + c0;
    tile_8x8<128>(H2T, prm.wt[2], 256, p0, cc, acc);
    float m[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float bj = prm.b[2][cc + j];
      float v = 0.0f;  // ReLU outputs are >= 0, so 0 is the empty-crop value
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (valid[i]) v = fmaxf(v, acc[i][j] + bj);
      m[j] = v;
    }
    // reduce over the 8 row groups of the same object (lane bits 0..2)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      m[j] = fmaxf(m[j], __shfl_xor_sync(0xffffffffu, m[j], 1));
      m[j] = fmaxf(m[j], __shfl_xor_sync(0xffffffffu, m[j], 2));
      m[j] = fmaxf(m[j], __shfl_xor_sync(0xffffffffu, m[j], 4));
    }
    if ((tp & 7) == 0) {
      float* dst = feat + (size_t)p * 512 + obj * 256 + cc;
      *reinterpret_cast<float4*>(dst) = make_float4(m[0], m[1], m[2], m[3]);
      *reinterpret_cast<float4*>(dst + 4) = make_float4(m[4], m[5], m[6], m[7]);
    }
  }
}

__global__ void __launch_bounds__(ENC_THREADS, 2) encoder_fp32_kernel(const float4* __restrict__ xyz,
                                                                      PairRange rg, Fp32Params prm,
                                                                      float* __restrict__ feat) {
  extern __shared__ __align__(16) unsigned char smem[];
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  for (int p = lo + blockIdx.x; p < hi; p += gridDim.x) {
    encode_pair(xyz, p, prm, feat, smem);
    __syncthreads();
  }
}


constexpr int HEAD_PAIRS = 32;

// out[q][c] = relu(b[c] + sum_k in[q][k] W^T[k][c]) for the CTA's pairs,
// thread c = threadIdx.x (256 output channels).
template <int K>
__device__ __forceinline__ void head_layer(const float* __restrict__ in, const float* __restrict__ WT,
                                           const float* __restrict__ b, float* __restrict__ out) {
  const int c = threadIdx.x;
  float acc[HEAD_PAIRS];
#pragma unroll
  for (int q = 0; q < HEAD_PAIRS; ++q) acc[q] = 0.f;
#pragma unroll 1
  for (int k = 0; k < K; k += 4) {
    const float w0 = __ldg(WT + (size_t)(k + 0) * 256 + c);
    const float w1 = __ldg(WT + (size_t)(k + 1) * 256 + c);
    const float w2 = __ldg(WT + (size_t)(k + 2) * 256 + c);
    const float w3 = __ldg(WT + (size_t)(k + 3) * 256 + c);
#pragma unroll
    for (int q = 0; q < HEAD_PAIRS; ++q) {
      const float4 x = *reinterpret_cast<const float4*>(in + q * K + k);
      acc[q] = fmaf(x.x, w0, acc[q]);
      acc[q] = fmaf(x.y, w1, acc[q]);
      acc[q] = fmaf(x.z, w2, acc[q]);
      acc[q] = fmaf(x.w, w3, acc[q]);
    }
  }
  const float bc = b[c];
#pragma unroll
  for (int q = 0; q < HEAD_PAIRS; ++q) out[q * 256 + c] = fmaxf(acc[q] + bc, 0.f);
}

// shared memory: f [32][512], g1 [32][256], g2 [32][256], y [32][8]
constexpr size_t HEAD_SMEM = (size_t)HEAD_PAIRS * (512 + 256 + 256 + 8) * 4;

}  // namespace

namespace {

__device__ __forceinline__ void head_tile(const float* __restrict__ feat, int n_pairs, int q0,
                                          const Fp32Params& prm, const PairInputs& in, int have_in,
                                          const float4* __restrict__ centre, float* __restrict__ out,
                                          float* __restrict__ y_raw, float* hsm);

__global__ void __launch_bounds__(256) head_fp32_kernel(const float* __restrict__ feat, PairRange rg,
                                                        Fp32Params prm, PairInputs in, int have_in,
                                                        const float4* __restrict__ centre,
                                                        float* __restrict__ out,
                                                        float* __restrict__ y_raw) {
  extern __shared__ __align__(16) float hsm[];
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  for (int q0 = lo + blockIdx.x * HEAD_PAIRS; q0 < hi; q0 += gridDim.x * HEAD_PAIRS) {
    head_tile(feat, hi, q0, prm, in, have_in, centre, out, y_raw, hsm);
    __syncthreads();
  }
}

__device__ __forceinline__ void head_tile(const float* __restrict__ feat, int n_pairs, int q0,
                                          const Fp32Params& prm, const PairInputs& in, int have_in,
                                          const float4* __restrict__ centre, float* __restrict__ out,
                                          float* __restrict__ y_raw, float* hsm) {
  float* F = hsm;
  float* G1 = F + HEAD_PAIRS * 512;
  float* G2 = G1 + HEAD_PAIRS * 256;
  float* Y = G2 + HEAD_PAIRS * 256;
  const int t = threadIdx.x;
  const int nq = min(HEAD_PAIRS, n_pairs - q0);
  for (int i = t; i < HEAD_PAIRS * 512 / 4; i += 256) {
    const int q = i / 128;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < nq) v = reinterpret_cast<const float4*>(feat + (size_t)q0 * 512)[i];
    reinterpret_cast<float4*>(F)[i] = v;
  }
  __syncthreads();
  head_layer<512>(F, prm.wt[3], prm.b[3], G1);
  __syncthreads();
  head_layer<256>(G1, prm.wt[4], prm.b[4], G2);
  __syncthreads();
  {
    // layer 3: 256 -> 8, thread = (pair q, output o)
    const int q = t >> 3, o = t & 7;
    const float* W = prm.wt[5];
    float acc = prm.b[5][o];
    for (int k = 0; k < 256; ++k) acc = fmaf(G2[q * 256 + k], __ldg(W + k * 8 + o), acc);
    Y[q * 8 + o] = acc;
  }
  __syncthreads();
  if (t < nq) {
    const int p = q0 + t;
    const float* y = Y + t * 8;
    if (y_raw) {
#pragma unroll
      for (int o = 0; o < 8; ++o) y_raw[(size_t)p * 8 + o] = y[o];
    }
    if (out) {
      float o8[8];
      const int a = have_in ? in.pairs[2 * p] : -1;
      const float4 c = centre[p];
      if (a >= 0 && a < in.n_obj && !isnan(c.x)) {
        epilogue_world(y, in.poses + 7 * (size_t)a, c, o8);
      } else {
#pragma unroll
        for (int o = 0; o < 8; ++o) o8[o] = __int_as_float(0x7fc00000);
      }
#pragma unroll
      for (int o = 0; o < 8; ++o) out[(size_t)p * 8 + o] = o8[o];
    }
  }
}

}  // namespace

cudaError_t prepare_fp32_kernels() {
  cudaError_t e = cudaFuncSetAttribute(encoder_fp32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ENC_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(head_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HEAD_SMEM);
  return e;
}

cudaError_t launch_encoder_fp32(const float4* xyz, const PairRange& rg, const Fp32Params& prm,
                                float* feat, int n_sm, cudaStream_t stream) {
  const int n_pairs = (rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1;
  if (rg.n_cap <= 0) return cudaSuccess;
  const int grid = std::min(n_pairs, 2 * n_sm);
  encoder_fp32_kernel<<<grid, ENC_THREADS, ENC_SMEM, stream>>>(xyz, rg, prm, feat);
  return cudaGetLastError();
}

cudaError_t launch_head_fp32(const float* feat, const PairRange& rg, const Fp32Params& prm,
                             const PairInputs* in, const float4* centre, float* out, float* y_raw,
                             int n_sm, cudaStream_t stream) {
  const int n_pairs = (rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1;
  if (rg.n_cap <= 0) return cudaSuccess;
  PairInputs pin{};
  if (in) pin = *in;
  const int grid = std::min((n_pairs + HEAD_PAIRS - 1) / HEAD_PAIRS, n_sm);
  head_fp32_kernel<<<grid, 256, HEAD_SMEM, stream>>>(feat, rg, prm, pin, in != nullptr, centre,
                                                     out, y_raw);
  return cudaGetLastError();
}

}  // namespace locc

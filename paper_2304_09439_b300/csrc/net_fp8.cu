// FP8 (e4m3) crop network on tcgen05 (LOCC_FP8).
//
// Same network and kernel structure as the BF16 path (net_tc.cu); the matrix
// products of encoder layers 2-3 and of all head layers use tcgen05.mma
// kind::f8f6f4 with e4m3 operands and float32 accumulation in TMEM:
//   * weights: one scale per output channel, s_w[c] = max_k |W[c][k]| / 448,
//     quantised once on the GPU (quant_e4m3_kernel);
//   * activations: one scale per row (crop point, or pair in the head),
//     s_a[r] = max_k a[r][k] / 448, chosen by the epilogue that produces the
//     row (ReLU outputs are >= 0);
//   * the accumulator is dequantised in the epilogue: z = D s_a[r] s_w[c] + b.
// Layer 1 (K = 3) keeps the bf16 hi/lo split of the BF16 path.  In the
// transposed layer 3 each thread owns a channel, so the per-point scales s_h2
// of the columns come from shared memory and the channel scale is applied
// after the max (a positive factor commutes with max).
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

using namespace tc;

constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz
constexpr float E4M3_MAX = 448.f;

__device__ __forceinline__ uint4 ldg_v4(const void* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}

// ------------------------------------------------------ weight quantisation
// Row r of W [rows][K] (float32, row-major) -> e4m3 bytes in K-chunks of
// chunkK columns, each chunk a K-major no-swizzle tile [rows][chunkK] stored
// one after the other; scales[r] = max |W[r][:]| / 448 (1 for an all-zero row).
__global__ void quant_e4m3_kernel(const float* __restrict__ W, int rows, int K, int chunkK,
                                  unsigned char* __restrict__ img, float* __restrict__ scales) {
  __shared__ float red[128];
  const int r = blockIdx.x, t = threadIdx.x;
  float m = 0.f;
  for (int k = t; k < K; k += 128) m = fmaxf(m, fabsf(W[(size_t)r * K + k]));
  red[t] = m;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (t < s) red[t] = fmaxf(red[t], red[t + s]);
    __syncthreads();
  }
  const float amax = red[0];
  const float sc = amax > 0.f ? amax / E4M3_MAX : 1.f;
  const float inv = amax > 0.f ? E4M3_MAX / amax : 0.f;
  for (int k = t; k < K; k += 128) {
    const uint32_t q = pack_e4m3x4(W[(size_t)r * K + k] * inv, 0.f, 0.f, 0.f);
    const int c = k / chunkK, kk = k % chunkK;
    img[(size_t)c * rows * chunkK + kmajor_off8(r, kk, chunkK)] = (unsigned char)(q & 0xffu);
  }
  if (t == 0) scales[r] = sc;
}

// ------------------------------------------------------------- encoder
constexpr int F_W1 = 0;                        // [64 x 16] bf16 (hi/lo)   2 KB
constexpr int F_W2 = F_W1 + 64 * 16 * 2;       // [128 x 64] e4m3          8 KB
constexpr int F_W3 = F_W2 + 128 * 64;          // [256 x 128] e4m3        32 KB
constexpr int F_SC = F_W3 + 256 * 128;         // sw2 128, sw3 256 (f32)
constexpr int F_BIAS = F_SC + (128 + 256) * 4; // b1 64, b2 128, b3 256 (f32)
constexpr int F_IMG_BYTES = F_BIAS + (64 + 128 + 256) * 4;
static_assert(F_IMG_BYTES % 16 == 0, "encoder fp8 image must be 16-byte chunks");
constexpr int F_SLOT0 = (F_IMG_BYTES + 1023) / 1024 * 1024;
constexpr int FS_STG = 0;                   // [128] float4        2 KB
constexpr int FS_X = FS_STG + ROWS * 16;    // [128 x 16] bf16     4 KB
constexpr int FS_H1 = FS_X + 128 * 16 * 2;  // [128 x 64] e4m3     8 KB
constexpr int FS_H2 = FS_H1 + 128 * 64;     // [128 x 128] e4m3   16 KB
constexpr int FS_SH2 = FS_H2 + 128 * 128;   // s_h2 [128] f32
constexpr int F_SLOT_BYTES = FS_SH2 + 128 * 4;
constexpr int F_CTRL = F_SLOT0 + 2 * F_SLOT_BYTES;
constexpr int C_BAR = 0, C_TMEM = 128, C_ABORT = 132, C_CNT = 136;
constexpr int F_SMEM = F_CTRL + 256;
static_assert(F_SMEM <= 227 * 1024, "fp8 encoder shared memory");
constexpr int F_THREADS = 288;
constexpr int SLOT_COLS = 256;
constexpr int B_FULLX = 0, B_XRDY = 2, B_H1RDY = 4, B_H2RDY = 6, B_D1 = 8, B_D2 = 10, B_D3 = 12,
              B_W = 14, B_DRAIN = 15;

__global__ void __launch_bounds__(F_THREADS, 1)
    encoder_fp8_kernel(const float4* __restrict__ xyz, int n_pairs, const int* n_dev,
                       const unsigned char* __restrict__ img, float* __restrict__ feat,
                       int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = n_dev ? min(*n_dev, n_pairs) : n_pairs;
  if ((int)blockIdx.x >= n) return;
  const int my_pairs = (n - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  unsigned char* ctrl = smem + F_CTRL;
  const uint32_t bar0 = smem_u32(ctrl + C_BAR);
  auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + C_TMEM);
  volatile int* abort = reinterpret_cast<volatile int*>(ctrl + C_ABORT);
  int* s_cnt = reinterpret_cast<int*>(ctrl + C_CNT);

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(BAR(B_FULLX + s), 1);
      mbar_init(BAR(B_XRDY + s), 128);
      mbar_init(BAR(B_H1RDY + s), 128);
      mbar_init(BAR(B_H2RDY + s), 128);
      mbar_init(BAR(B_D1 + s), 1);
      mbar_init(BAR(B_D2 + s), 1);
      mbar_init(BAR(B_D3 + s), 1);
    }
    mbar_init(BAR(B_W), 1);
    mbar_init(BAR(B_DRAIN), 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const float* sw2 = reinterpret_cast<const float*>(smem + F_SC);
  const float* sw3 = sw2 + 128;
  const float* b1 = reinterpret_cast<const float*>(smem + F_BIAS);
  const float* b2 = b1 + 64;
  const float* b3 = b2 + 128;

  if (warp == 8) {
    if (lane == 0) {
      const uint32_t sW1 = smem_u32(smem + F_W1), sW2 = smem_u32(smem + F_W2);
      const uint32_t sW3 = smem_u32(smem + F_W3);
      mbar_expect_tx(BAR(B_W), F_IMG_BYTES);
      for (int off = 0; off < F_IMG_BYTES; off += 32768)
        bulk_g2s(smem_u32(smem + off), img + off, min(32768, F_IMG_BYTES - off), BAR(B_W));
      int issued[2] = {0, 0};
      auto load_pair = [&](int i) {
        const int s = i & 1;
        const int p = blockIdx.x + i * gridDim.x;
        mbar_expect_tx(BAR(B_FULLX + s), ROWS * 16);
        bulk_g2s(smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_STG), xyz + (size_t)p * ROWS,
                 ROWS * 16, BAR(B_FULLX + s));
        ++issued[s];
      };
      load_pair(0);
      if (my_pairs > 1) load_pair(1);
      bool ok = mbar_wait_or_abort(BAR(B_W), 0, abort, WAIT_CYCLES);
      tc_fence_after();
      const uint32_t id64 = idesc_bf16(128, 64), id128 = idesc_e4m3(128, 128);
      for (int r = 0; ok && 2 * r < my_pairs; ++r) {
        const uint32_t ph = r & 1;
        for (int s = 0; s < 2 && ok; ++s) {
          const int i = 2 * r + s;
          if (i >= my_pairs) break;
          if (!(ok = mbar_wait_or_abort(BAR(B_XRDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (i + 2 < my_pairs) load_pair(i + 2);
          const uint32_t sX = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_X);
          mma_bf16(tbase + s * SLOT_COLS, sdesc(sX, 128, 256), sdesc(sW1, 128, 256), id64, 0);
          mma_commit(BAR(B_D1 + s));
        }
        for (int s = 0; s < 2 && ok; ++s) {
          if (2 * r + s >= my_pairs) break;
          if (!(ok = mbar_wait_or_abort(BAR(B_H1RDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          const uint32_t sH1 = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_H1);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            mma_e4m3(tbase + s * SLOT_COLS + 64, sdesc(sH1 + 256 * kk, 128, 512),
                     sdesc(sW2 + 256 * kk, 128, 512), id128, kk > 0);
          mma_commit(BAR(B_D2 + s));
        }
        for (int s = 0; s < 2 && ok; ++s) {
          if (2 * r + s >= my_pairs) break;
          if (!(ok = mbar_wait_or_abort(BAR(B_H2RDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          const uint32_t sH2 = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_H2);
#pragma unroll
          for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_e4m3(tbase + s * SLOT_COLS + 128 * half,
                       sdesc(sW3 + half * 16384 + 256 * kk, 128, 1024),
                       sdesc(sH2 + 256 * kk, 128, 1024), id128, kk > 0);
          mma_commit(BAR(B_D3 + s));
        }
      }
      if (*abort) {
        mma_commit(BAR(B_DRAIN));
        mbar_wait(BAR(B_DRAIN), 0, WAIT_CYCLES);
        for (int s = 0; s < 2; ++s)
          if (issued[s] > 0) mbar_wait(BAR(B_FULLX + s), (issued[s] - 1) & 1, WAIT_CYCLES);
      }
    }
    __syncwarp();
  } else {
    const int s = warp >> 2, row = tid & 127, wq = warp & 3;
    unsigned char* slot = smem + F_SLOT0 + s * F_SLOT_BYTES;
    float* s_h2 = reinterpret_cast<float*>(slot + FS_SH2);
    const uint32_t tslot = tbase + s * SLOT_COLS + ((uint32_t)(32 * wq) << 16);
    int* cnt_s = s_cnt + 4 * s;
    bool ok = mbar_wait_or_abort(BAR(B_W), 0, abort, WAIT_CYCLES);
    for (int j = 0; ok; ++j) {
      const int i = 2 * j + s;
      if (i >= my_pairs) break;
      const int p = blockIdx.x + i * gridDim.x;
      const uint32_t ph = j & 1;
      if (!(ok = mbar_wait_or_abort(BAR(B_FULLX + s), ph, abort, WAIT_CYCLES))) break;
      {
        const float4 q = reinterpret_cast<const float4*>(slot + FS_STG)[row];
        const unsigned m = __ballot_sync(0xffffffffu, q.w > 0.5f);
        if (lane == 0) cnt_s[wq] = __popc(m);
        const float fx = __bfloat162float(__float2bfloat16_rn(q.x));
        const float fy = __bfloat162float(__float2bfloat16_rn(q.y));
        const float fz = __bfloat162float(__float2bfloat16_rn(q.z));
        uint4 c0, c1;
        c0.x = pack_bf16(fx, fy);
        c0.y = pack_bf16(fz, q.x - fx);
        c0.z = pack_bf16(q.y - fy, q.z - fz);
        c0.w = pack_bf16(fx, fy);
        c1.x = pack_bf16(fz, 0.f);
        c1.y = c1.z = c1.w = 0u;
        *reinterpret_cast<uint4*>(slot + FS_X + kmajor_off(row, 0, 16)) = c0;
        *reinterpret_cast<uint4*>(slot + FS_X + kmajor_off(row, 8, 16)) = c1;
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_XRDY + s));
      // ---- layer 1 epilogue: relu(D1 + b1), per-row e4m3 scale
      if (!(ok = mbar_wait_or_abort(BAR(B_D1 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      float sa;  // this row's H1 scale
      {
        float v0[32], v1[32];
        tmem_ld32(tslot + 0, v0);
        tmem_ld32(tslot + 32, v1);
        float amax = 0.f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          v0[jj] = fmaxf(v0[jj] + b1[jj], 0.f);
          v1[jj] = fmaxf(v1[jj] + b1[32 + jj], 0.f);
          amax = fmaxf(amax, fmaxf(v0[jj], v1[jj]));
        }
        sa = amax > 0.f ? amax / E4M3_MAX : 1.f;
        const float inv = amax > 0.f ? E4M3_MAX / amax : 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          uint4 w;
          w.x = pack_e4m3x4(v0[16 * c + 0] * inv, v0[16 * c + 1] * inv, v0[16 * c + 2] * inv, v0[16 * c + 3] * inv);
          w.y = pack_e4m3x4(v0[16 * c + 4] * inv, v0[16 * c + 5] * inv, v0[16 * c + 6] * inv, v0[16 * c + 7] * inv);
          w.z = pack_e4m3x4(v0[16 * c + 8] * inv, v0[16 * c + 9] * inv, v0[16 * c + 10] * inv, v0[16 * c + 11] * inv);
          w.w = pack_e4m3x4(v0[16 * c + 12] * inv, v0[16 * c + 13] * inv, v0[16 * c + 14] * inv, v0[16 * c + 15] * inv);
          *reinterpret_cast<uint4*>(slot + FS_H1 + kmajor_off8(row, 16 * c, 64)) = w;
          w.x = pack_e4m3x4(v1[16 * c + 0] * inv, v1[16 * c + 1] * inv, v1[16 * c + 2] * inv, v1[16 * c + 3] * inv);
          w.y = pack_e4m3x4(v1[16 * c + 4] * inv, v1[16 * c + 5] * inv, v1[16 * c + 6] * inv, v1[16 * c + 7] * inv);
          w.z = pack_e4m3x4(v1[16 * c + 8] * inv, v1[16 * c + 9] * inv, v1[16 * c + 10] * inv, v1[16 * c + 11] * inv);
          w.w = pack_e4m3x4(v1[16 * c + 12] * inv, v1[16 * c + 13] * inv, v1[16 * c + 14] * inv, v1[16 * c + 15] * inv);
          *reinterpret_cast<uint4*>(slot + FS_H1 + kmajor_off8(row, 32 + 16 * c, 64)) = w;
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H1RDY + s));
      // ---- layer 2 epilogue: z = D2 sa sw2 + b2, relu; two passes over TMEM
      if (!(ok = mbar_wait_or_abort(BAR(B_D2 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      {
        float v[32];
        float amax = 0.f;
#pragma unroll 1
        for (int h = 0; h < 4; ++h) {
          tmem_ld32(tslot + 64 + 32 * h, v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj)
            amax = fmaxf(amax, fmaf(v[jj], sa * sw2[32 * h + jj], b2[32 * h + jj]));
        }
        const float sh = amax > 0.f ? amax / E4M3_MAX : 1.f;
        const float inv = amax > 0.f ? E4M3_MAX / amax : 0.f;
#pragma unroll 1
        for (int h = 0; h < 4; ++h) {
          tmem_ld32(tslot + 64 + 32 * h, v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj)
            v[jj] = fmaxf(fmaf(v[jj], sa * sw2[32 * h + jj], b2[32 * h + jj]), 0.f) * inv;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint4 w;
            w.x = pack_e4m3x4(v[16 * c + 0], v[16 * c + 1], v[16 * c + 2], v[16 * c + 3]);
            w.y = pack_e4m3x4(v[16 * c + 4], v[16 * c + 5], v[16 * c + 6], v[16 * c + 7]);
            w.z = pack_e4m3x4(v[16 * c + 8], v[16 * c + 9], v[16 * c + 10], v[16 * c + 11]);
            w.w = pack_e4m3x4(v[16 * c + 12], v[16 * c + 13], v[16 * c + 14], v[16 * c + 15]);
            *reinterpret_cast<uint4*>(slot + FS_H2 + kmajor_off8(row, 32 * h + 16 * c, 128)) = w;
          }
        }
        s_h2[row] = sh;
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H2RDY + s));
      // ---- layer 3 epilogue: max over valid points of D3^T s_h2[pt], then * sw3 + b3
      if (!(ok = mbar_wait_or_abort(BAR(B_D3 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      // crop counts (and row scales) written by other threads of this warpgroup
      asm volatile("bar.sync %0, 128;" ::"r"(1 + s) : "memory");
      const int cntA = cnt_s[0] + cnt_s[1], cntB = cnt_s[2] + cnt_s[3];
      float v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float mA = -INFINITY, mB = -INFINITY;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cnt = q < 2 ? cntA : cntB;
          const int c0 = 32 * (q & 1);
          if (c0 < cnt) {
            tmem_ld32(tslot + 128 * half + 32 * q, v);
            float m = -INFINITY;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              m = fmaxf(m, (c0 + jj < cnt) ? v[jj] * s_h2[32 * q + jj] : -INFINITY);
            if (q < 2) mA = fmaxf(mA, m);
            else mB = fmaxf(mB, m);
          }
        }
        const int ch = 128 * half + row;
        const float sc = sw3[ch], bias = b3[ch];
        feat[(size_t)p * 512 + ch] = cntA > 0 ? fmaxf(fmaf(mA, sc, bias), 0.f) : 0.f;
        feat[(size_t)p * 512 + 256 + ch] = cntB > 0 ? fmaxf(fmaf(mB, sc, bias), 0.f) : 0.f;
      }
      tc_fence_before();
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(err, 2);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ----------------------------------------------------------------- head
constexpr int HT = 128;
constexpr int G_W3 = 0;                          // Wh3 [16 x 256] e4m3 (rows 8.. zero) 4 KB
constexpr int G_SC = G_W3 + 16 * 256;            // swh1 256, swh2 256, swh3 16 (f32)
constexpr int G_BIAS = G_SC + (256 + 256 + 16) * 4;  // hb1 256, hb2 256, hb3 16
constexpr int G_RES_BYTES = G_BIAS + (256 + 256 + 16) * 4;
static_assert(G_RES_BYTES % 128 == 0, "fp8 head resident image");
constexpr int G_CHUNK = 256 * 128;               // one B chunk [256 x 128] e4m3, 32 KB
constexpr int G_IMG_W1 = G_RES_BYTES;            // 4 chunks
constexpr int G_IMG_W2 = G_IMG_W1 + 4 * G_CHUNK; // 2 chunks
constexpr int G_IMG_BYTES = G_IMG_W2 + 2 * G_CHUNK;
constexpr int G_A = G_RES_BYTES;                 // A chunk [128 x 128] e4m3, 16 KB
constexpr int G_B = G_A + 128 * 128;             // B chunk 32 KB
constexpr int G_G = G_B + G_CHUNK;               // G [128 x 256] e4m3, 32 KB
constexpr int G_CTRL = G_G + 128 * 256;
constexpr int G_SMEM = G_CTRL + 64;

__device__ __forceinline__ void copy_chunk(unsigned char* dst, const unsigned char* src, int bytes) {
  for (int i = threadIdx.x; i < bytes / 16; i += 128)
    reinterpret_cast<uint4*>(dst)[i] = ldg_v4(src + 16 * (size_t)i);
}

// Head epilogue of a 256-wide layer in e4m3: z = relu(D sa sw + b), per-row
// scale; writes G (K = 256) and returns the row scale.
__device__ __forceinline__ float head_epi_fp8(uint32_t taddr, float sa, const float* sw,
                                              const float* b, unsigned char* G, int row) {
  float v[32];
  float amax = 0.f;
#pragma unroll 1
  for (int h = 0; h < 8; ++h) {
    tmem_ld32(taddr + 32 * h, v);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) amax = fmaxf(amax, fmaf(v[jj], sa * sw[32 * h + jj], b[32 * h + jj]));
  }
  const float inv = amax > 0.f ? E4M3_MAX / amax : 0.f;
#pragma unroll 1
  for (int h = 0; h < 8; ++h) {
    tmem_ld32(taddr + 32 * h, v);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      v[jj] = fmaxf(fmaf(v[jj], sa * sw[32 * h + jj], b[32 * h + jj]), 0.f) * inv;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint4 w;
      w.x = pack_e4m3x4(v[16 * c + 0], v[16 * c + 1], v[16 * c + 2], v[16 * c + 3]);
      w.y = pack_e4m3x4(v[16 * c + 4], v[16 * c + 5], v[16 * c + 6], v[16 * c + 7]);
      w.z = pack_e4m3x4(v[16 * c + 8], v[16 * c + 9], v[16 * c + 10], v[16 * c + 11]);
      w.w = pack_e4m3x4(v[16 * c + 12], v[16 * c + 13], v[16 * c + 14], v[16 * c + 15]);
      *reinterpret_cast<uint4*>(G + kmajor_off8(row, 32 * h + 16 * c, 256)) = w;
    }
  }
  return amax > 0.f ? amax / E4M3_MAX : 1.f;
}

__global__ void __launch_bounds__(128, 1)
    head_fp8_kernel(const float* __restrict__ feat, int n_pairs, const int* n_dev,
                    const unsigned char* __restrict__ img, PairInputs in, int have_in,
                    const float4* __restrict__ centre, float* __restrict__ out,
                    float* __restrict__ y_raw, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n = n_dev ? min(*n_dev, n_pairs) : n_pairs;
  const int n_tiles = (n + HT - 1) / HT;
  if ((int)blockIdx.x >= n_tiles) return;
  for (int i = tid; i < G_RES_BYTES / 16; i += 128)
    reinterpret_cast<uint4*>(smem)[i] = ldg_v4(img + 16 * (size_t)i);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + G_CTRL);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G_CTRL + 8);
  const uint32_t bar = smem_u32(mbar);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
  const float* swh1 = reinterpret_cast<const float*>(smem + G_SC);
  const float* swh2 = swh1 + 256;
  const float* swh3 = swh2 + 256;
  const float* hb1 = reinterpret_cast<const float*>(smem + G_BIAS);
  const float* hb2 = hb1 + 256;
  const float* hb3 = hb2 + 256;
  unsigned char* A = smem + G_A;
  unsigned char* B = smem + G_B;
  unsigned char* G = smem + G_G;
  const uint32_t sA = smem_u32(A), sB = smem_u32(B), sG = smem_u32(G), sW3 = smem_u32(smem + G_W3);
  const uint32_t id256 = idesc_e4m3(128, 256), id16 = idesc_e4m3(128, 16);
  uint32_t phase = 0;
  bool ok = true;

  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int pr = tile * HT + tid;
    const bool row_ok = pr < n;
    const float* src = feat + (size_t)pr * 512;
    // per-pair scale of the pooled features
    float amax = 0.f;
    if (row_ok) {
      for (int k = 0; k < 512; k += 4) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(src + k));
        amax = fmaxf(amax, fmaxf(fmaxf(f.x, f.y), fmaxf(f.z, f.w)));
      }
    }
    const float sf = amax > 0.f ? amax / E4M3_MAX : 1.f;
    const float inv = amax > 0.f ? E4M3_MAX / amax : 0.f;
#pragma unroll 1
    for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
        if (row_ok) {
          const float* sp = src + 128 * kc + 16 * c;
          a0 = __ldg(reinterpret_cast<const float4*>(sp));
          a1 = __ldg(reinterpret_cast<const float4*>(sp + 4));
          a2 = __ldg(reinterpret_cast<const float4*>(sp + 8));
          a3 = __ldg(reinterpret_cast<const float4*>(sp + 12));
        }
        uint4 w;
        w.x = pack_e4m3x4(a0.x * inv, a0.y * inv, a0.z * inv, a0.w * inv);
        w.y = pack_e4m3x4(a1.x * inv, a1.y * inv, a1.z * inv, a1.w * inv);
        w.z = pack_e4m3x4(a2.x * inv, a2.y * inv, a2.z * inv, a2.w * inv);
        w.w = pack_e4m3x4(a3.x * inv, a3.y * inv, a3.z * inv, a3.w * inv);
        *reinterpret_cast<uint4*>(A + kmajor_off8(tid, 16 * c, 128)) = w;
      }
      copy_chunk(B, img + G_IMG_W1 + (size_t)kc * G_CHUNK, G_CHUNK);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_e4m3(tbase + 0, sdesc(sA + 256 * kk, 128, 1024), sdesc(sB + 256 * kk, 128, 1024), id256,
                   (kc > 0 || kk > 0) ? 1u : 0u);
        mma_commit(bar);
      }
      ok = mbar_wait(bar, phase, WAIT_CYCLES);
      phase ^= 1;
      if (!__syncthreads_and(ok)) { ok = false; break; }
      tc_fence_after();
    }
    if (!ok) break;
    const float sg1 = head_epi_fp8(tbase + lane_off + 0, sf, swh1, hb1, G, tid);
#pragma unroll 1
    for (int kc = 0; kc < 2; ++kc) {
      copy_chunk(B, img + G_IMG_W2 + (size_t)kc * G_CHUNK, G_CHUNK);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_e4m3(tbase + 256, sdesc(sG + 1024 * kc + 256 * kk, 128, 2048),
                   sdesc(sB + 256 * kk, 128, 1024), id256, (kc > 0 || kk > 0) ? 1u : 0u);
        mma_commit(bar);
      }
      ok = mbar_wait(bar, phase, WAIT_CYCLES);
      phase ^= 1;
      if (!__syncthreads_and(ok)) { ok = false; break; }
      tc_fence_after();
    }
    if (!ok) break;
    const float sg2 = head_epi_fp8(tbase + lane_off + 256, sg1, swh2, hb2, G, tid);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma_e4m3(tbase + 0, sdesc(sG + 256 * kk, 128, 2048), sdesc(sW3 + 256 * kk, 128, 2048), id16,
                 kk > 0);
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase, WAIT_CYCLES);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc_fence_after();
    {
      float v[16];
      tmem_ld16(tbase + lane_off + 0, v);
      if (row_ok) {
        float y[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) y[o] = fmaf(v[o], sg2 * swh3[o], hb3[o]);
        if (y_raw) {
#pragma unroll
          for (int o = 0; o < 8; ++o) y_raw[(size_t)pr * 8 + o] = y[o];
        }
        if (out) {
          float o8[8];
          const int a = have_in ? in.pairs[2 * pr] : -1;
          const float4 c = centre[pr];
          if (a >= 0 && a < in.n_obj && !isnan(c.x)) {
            epilogue_world(y, in.poses + 7 * (size_t)a, c, o8);
          } else {
#pragma unroll
            for (int o = 0; o < 8; ++o) o8[o] = __int_as_float(0x7fc00000);
          }
#pragma unroll
          for (int o = 0; o < 8; ++o) out[(size_t)pr * 8 + o] = o8[o];
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(err, 2);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

uint16_t bf16_bits_h(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value_h(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

int upload_fp8_params(locc_handle* h, const std::vector<float>& params) {
  size_t off[6], offb[6], o = 0;
  for (int l = 0; l < 6; ++l) {
    off[l] = o;
    o += (size_t)L_IN[l] * L_OUT[l];
    offb[l] = o;
    o += L_OUT[l];
  }
  const size_t enc_bytes = (F_IMG_BYTES + 255) / 256 * 256;
  const size_t total = enc_bytes + G_IMG_BYTES;
  std::vector<unsigned char> img(total, 0);
  unsigned char* e = img.data();
  for (int c = 0; c < 64; ++c)
    for (int k = 0; k < 16; ++k) {
      float val = 0.f;
      if (k < 9) {
        const float w = params[off[0] + (size_t)c * 3 + (k % 3)];
        const float hi = bf16_value_h(bf16_bits_h(w));
        val = k < 6 ? hi : w - hi;
      }
      const uint16_t b = bf16_bits_h(val);
      std::memcpy(e + F_W1 + kmajor_off(c, k, 16), &b, 2);
    }
  std::memcpy(e + F_BIAS, &params[offb[0]], 64 * 4);
  std::memcpy(e + F_BIAS + 64 * 4, &params[offb[1]], 128 * 4);
  std::memcpy(e + F_BIAS + 192 * 4, &params[offb[2]], 256 * 4);
  unsigned char* hd = img.data() + enc_bytes;
  std::memcpy(hd + G_BIAS, &params[offb[3]], 256 * 4);
  std::memcpy(hd + G_BIAS + 256 * 4, &params[offb[4]], 256 * 4);
  std::memcpy(hd + G_BIAS + 512 * 4, &params[offb[5]], 8 * 4);
  float* d_params = nullptr;
  bool ok = cudaMalloc(&h->d_wf8, total) == cudaSuccess &&
            cudaMemcpy(h->d_wf8, img.data(), total, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMalloc(&d_params, params.size() * 4) == cudaSuccess &&
            cudaMemcpy(d_params, params.data(), params.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    unsigned char* de = static_cast<unsigned char*>(h->d_wf8);
    unsigned char* dh = de + enc_bytes;
    float* esc = reinterpret_cast<float*>(de + F_SC);
    float* hsc = reinterpret_cast<float*>(dh + G_SC);
    quant_e4m3_kernel<<<128, 128>>>(d_params + off[1], 128, 64, 64, de + F_W2, esc);
    quant_e4m3_kernel<<<256, 128>>>(d_params + off[2], 256, 128, 128, de + F_W3, esc + 128);
    quant_e4m3_kernel<<<256, 128>>>(d_params + off[3], 256, 512, 128, dh + G_IMG_W1, hsc);
    quant_e4m3_kernel<<<256, 128>>>(d_params + off[4], 256, 256, 128, dh + G_IMG_W2, hsc + 256);
    quant_e4m3_kernel<<<8, 128>>>(d_params + off[5], 8, 256, 256, dh + G_W3, hsc + 512);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    h->wf8_enc = de;
    h->wf8_head = dh;
  }
  cudaFree(d_params);
  if (!ok) {
    cudaGetLastError();
    set_error("cannot build the e4m3 parameter images");
    return LOCC_ERR_OOM;
  }
  return LOCC_OK;
}

int run_network_fp8(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                    const PairInputs* in, const float4* centre, float* out, float* y_raw,
                    float* feat_out, cudaStream_t stream, cudaEvent_t mid) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(encoder_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             F_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(head_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G_SMEM) != cudaSuccess) {
      set_error("cudaFuncSetAttribute failed for the fp8 kernels");
      return LOCC_ERR_CUDA;
    }
    attr = true;
  }
  float* feat = feat_out ? feat_out : h->d_feat;
  encoder_fp8_kernel<<<std::min(n_pairs, h->n_sm), F_THREADS, F_SMEM, stream>>>(
      xyz, n_pairs, n_dev, h->wf8_enc, feat, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("encoder_fp8_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  if (mid && cudaEventRecord(mid, stream) != cudaSuccess) return LOCC_ERR_CUDA;
  PairInputs pin{};
  if (in) pin = *in;
  head_fp8_kernel<<<std::min((n_pairs + HT - 1) / HT, h->n_sm), 128, G_SMEM, stream>>>(
      feat, n_pairs, n_dev, h->wf8_head, pin, in != nullptr, centre, out, y_raw, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("head_fp8_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

}  // namespace locc

// Tensor-core crop network (LOCC_BF16): tcgen05.mma with bf16 operands in
// shared memory and float32 accumulators in TMEM.
//
// Paper: Sec. III and appendix -- point-wise MLP encoder, pooling per object,
// MLP head, ReLU everywhere.  Same network as net_fp32.cu: encoder
// 3 -> 64 -> 128 -> 256, max-pool over the valid crop points of each object,
// head 512 -> 256 -> 256 -> 8, world-frame epilogue.
//
// encoder_tc_kernel (persistent, one CTA of 128 threads per SM, one pair at a
// time):
//   * the bf16 images of W1, W2, W3 (82 KB) and the biases are copied into
//     shared memory once and stay there for the life of the CTA;
//   * the 128 crop rows of a pair (64 of A, 64 of B) form the M = 128 tile;
//   * layer 1 packs K = 16: coordinates and weights are split into bf16 hi/lo
//     parts, x.W ~ x_hi W_hi + x_lo W_hi + x_hi W_lo (9 of the 16 columns);
//   * layers 1 and 2: D[128 x N] in TMEM, thread r owns row r (point r); the
//     epilogue adds the bias, applies ReLU and writes the bf16 row as the next
//     layer's A operand;
//   * layer 3 is computed transposed, D^T = W3 . H2^T (M = 128 channels per
//     half, N = 128 points): thread r owns channel r, so the max-pool over the
//     valid points of each object is a register reduction over TMEM columns.
// head_tc_kernel (persistent over tiles of 128 pairs): layer 1 streams W_h1 in
// K-chunks of 64 through shared memory, layers 2 and 3 likewise; activations
// stay on chip (TMEM -> bf16 in shared memory); the epilogue maps outputs to
// the world frame.
//
// Every mbarrier wait is bounded; on a timeout the CTA raises bit 2 of the
// error flag, stops, releases its TMEM and returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

using namespace tc;

constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

// ----------------------------------------------------------------- encoder
constexpr int E_W1 = 0;                       // [64 x 16]   2 KB
constexpr int E_W2 = E_W1 + 64 * 16 * 2;      // [128 x 64] 16 KB
constexpr int E_W3 = E_W2 + 128 * 64 * 2;     // [256 x 128] 64 KB
constexpr int E_BIAS = E_W3 + 256 * 128 * 2;  // b1 64, b2 128, b3 256 (f32)
constexpr int E_IMG_BYTES = E_BIAS + (64 + 128 + 256) * 4;
constexpr int E_X = (E_IMG_BYTES + 127) / 128 * 128;  // [128 x 16]  4 KB
constexpr int E_H1 = E_X + 128 * 16 * 2;              // [128 x 64] 16 KB
constexpr int E_H2 = E_H1 + 128 * 64 * 2;             // [128 x 128] 32 KB
constexpr int E_CTRL = E_H2 + 128 * 128 * 2;          // mbar, tmem base, counts
constexpr int E_SMEM = E_CTRL + 64;
static_assert(E_IMG_BYTES % 16 == 0, "image must be a whole number of 16-byte chunks");

// TMEM columns: D1 [0, 64), D2 [64, 192), D3 halves [256, 384), [384, 512)
constexpr uint32_t T_D1 = 0, T_D2 = 64, T_D3 = 256;

__device__ __forceinline__ uint4 ld_global_v4(const void* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}

__global__ void __launch_bounds__(128, 1)
    encoder_tc_kernel(const float4* __restrict__ xyz, int n_pairs, const int* n_dev,
                      const unsigned char* __restrict__ img, float* __restrict__ feat,
                      int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = n_dev ? min(*n_dev, n_pairs) : n_pairs;
  if ((int)blockIdx.x >= n) return;

  // resident weights and biases
  for (int i = tid; i < E_IMG_BYTES / 16; i += 128)
    reinterpret_cast<uint4*>(smem)[i] = ld_global_v4(img + 16 * (size_t)i);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + E_CTRL);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + E_CTRL + 8);
  int* s_cnt = reinterpret_cast<int*>(smem + E_CTRL + 16);
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
  const float* b1 = reinterpret_cast<const float*>(smem + E_BIAS);
  const float* b2 = b1 + 64;
  const float* b3 = b2 + 128;
  const uint32_t sW1 = smem_u32(smem + E_W1), sW2 = smem_u32(smem + E_W2);
  const uint32_t sW3 = smem_u32(smem + E_W3), sX = smem_u32(smem + E_X);
  const uint32_t sH1 = smem_u32(smem + E_H1), sH2 = smem_u32(smem + E_H2);
  uint32_t phase = 0;
  bool ok = true;

  for (int p = blockIdx.x; p < n && ok; p += gridDim.x) {
    // ---- stage the crop rows (row = tid) as bf16 hi/lo, K = 16
    {
      const float4 q = xyz[(size_t)p * ROWS + tid];
      const bool valid = q.w > 0.5f;
      const unsigned m = __ballot_sync(0xffffffffu, valid);
      if (lane == 0) s_cnt[warp] = __popc(m);
      const __nv_bfloat16 xh = __float2bfloat16_rn(q.x), yh = __float2bfloat16_rn(q.y),
                          zh = __float2bfloat16_rn(q.z);
      const float xl = q.x - __bfloat162float(xh), yl = q.y - __bfloat162float(yh),
                  zl = q.z - __bfloat162float(zh);
      uint4 c0, c1;
      c0.x = pack_bf16(__bfloat162float(xh), __bfloat162float(yh));
      c0.y = pack_bf16(__bfloat162float(zh), xl);
      c0.z = pack_bf16(yl, zl);
      c0.w = pack_bf16(__bfloat162float(xh), __bfloat162float(yh));
      c1.x = pack_bf16(__bfloat162float(zh), 0.f);
      c1.y = c1.z = c1.w = 0u;
      *reinterpret_cast<uint4*>(smem + E_X + kmajor_off(tid, 0, 16)) = c0;
      *reinterpret_cast<uint4*>(smem + E_X + kmajor_off(tid, 8, 16)) = c1;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    const int cntA = s_cnt[0] + s_cnt[1], cntB = s_cnt[2] + s_cnt[3];
    // ---- layer 1: D1[128 x 64] = X[128 x 16] . W1img^T
    if (tid == 0) {
      tc_fence_after();
      mma_bf16(tbase + T_D1, sdesc(sX, 128, 256), sdesc(sW1, 128, 256), idesc_bf16(128, 64), 0);
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase, WAIT_CYCLES);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc_fence_after();
    {
      float v[32];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tmem_ld32(tbase + lane_off + T_D1 + 32 * h, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint4 w;
          const int j = 8 * c;
          w.x = pack_bf16(fmaxf(v[j + 0] + b1[32 * h + j + 0], 0.f), fmaxf(v[j + 1] + b1[32 * h + j + 1], 0.f));
          w.y = pack_bf16(fmaxf(v[j + 2] + b1[32 * h + j + 2], 0.f), fmaxf(v[j + 3] + b1[32 * h + j + 3], 0.f));
          w.z = pack_bf16(fmaxf(v[j + 4] + b1[32 * h + j + 4], 0.f), fmaxf(v[j + 5] + b1[32 * h + j + 5], 0.f));
          w.w = pack_bf16(fmaxf(v[j + 6] + b1[32 * h + j + 6], 0.f), fmaxf(v[j + 7] + b1[32 * h + j + 7], 0.f));
          *reinterpret_cast<uint4*>(smem + E_H1 + kmajor_off(tid, 32 * h + j, 64)) = w;
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 2: D2[128 x 128] = H1[128 x 64] . W2img^T
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(tbase + T_D2, sdesc(sH1 + 256 * kk, 128, 1024), sdesc(sW2 + 256 * kk, 128, 1024),
                 idesc_bf16(128, 128), kk > 0);
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase, WAIT_CYCLES);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc_fence_after();
    {
      float v[32];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        tmem_ld32(tbase + lane_off + T_D2 + 32 * h, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint4 w;
          const int j = 8 * c, o = 32 * h + j;
          w.x = pack_bf16(fmaxf(v[j + 0] + b2[o + 0], 0.f), fmaxf(v[j + 1] + b2[o + 1], 0.f));
          w.y = pack_bf16(fmaxf(v[j + 2] + b2[o + 2], 0.f), fmaxf(v[j + 3] + b2[o + 3], 0.f));
          w.z = pack_bf16(fmaxf(v[j + 4] + b2[o + 4], 0.f), fmaxf(v[j + 5] + b2[o + 5], 0.f));
          w.w = pack_bf16(fmaxf(v[j + 6] + b2[o + 6], 0.f), fmaxf(v[j + 7] + b2[o + 7], 0.f));
          *reinterpret_cast<uint4*>(smem + E_H2 + kmajor_off(tid, o, 128)) = w;
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 3 (transposed): D3^T[128 ch x 128 pts] = W3img[half] . H2^T
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int half = 0; half < 2; ++half)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma_bf16(tbase + T_D3 + 128 * half, sdesc(sW3 + half * 32768 + 256 * kk, 128, 2048),
                   sdesc(sH2 + 256 * kk, 128, 2048), idesc_bf16(128, 128), kk > 0);
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase, WAIT_CYCLES);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc_fence_after();
    {
      float v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float mA = -INFINITY, mB = -INFINITY;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cnt = q < 2 ? cntA : cntB;
          const int c0 = 32 * (q & 1);  // first point slot of this chunk within its object
          if (c0 < cnt) {
            tmem_ld32(tbase + lane_off + T_D3 + 128 * half + 32 * q, v);
            float m = -INFINITY;
#pragma unroll
            for (int j = 0; j < 32; ++j) m = fmaxf(m, (c0 + j < cnt) ? v[j] : -INFINITY);
            if (q < 2) mA = fmaxf(mA, m);
            else mB = fmaxf(mB, m);
          }
        }
        const int ch = 128 * half + tid;
        const float bias = b3[ch];
        feat[(size_t)p * 512 + ch] = cntA > 0 ? fmaxf(mA + bias, 0.f) : 0.f;
        feat[(size_t)p * 512 + 256 + ch] = cntB > 0 ? fmaxf(mB + bias, 0.f) : 0.f;
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

// -------------------------------------------------------------------- head
constexpr int HT = 128;                                   // pairs per tile
constexpr int H_W3 = 0;                                    // [16 x 256] 8 KB
constexpr int H_BIAS = H_W3 + 16 * 256 * 2;                // hb1 256, hb2 256, hb3 16
constexpr int H_RES_BYTES = H_BIAS + (256 + 256 + 16) * 4; // resident part of the image
constexpr int H_A = (H_RES_BYTES + 127) / 128 * 128;       // A chunk [128 x 64] 16 KB
constexpr int H_B = H_A + 128 * 64 * 2;                    // B chunk [256 x 64] 32 KB
constexpr int H_G = H_B + 256 * 64 * 2;                    // G [128 x 256] 64 KB
constexpr int H_CTRL = H_G + 128 * 256 * 2;
constexpr int H_SMEM = H_CTRL + 64;
constexpr int H_CHUNK = 256 * 64 * 2;                      // bytes of one B chunk
// global image: [resident][W_h1 chunks x 8][W_h2 chunks x 4]
constexpr int H_IMG_W1 = (H_RES_BYTES + 127) / 128 * 128;
constexpr int H_IMG_W2 = H_IMG_W1 + 8 * H_CHUNK;
constexpr int H_IMG_BYTES = H_IMG_W2 + 4 * H_CHUNK;
static_assert(H_RES_BYTES % 16 == 0, "resident image must be 16-byte chunks");

__device__ __forceinline__ void copy_chunk(unsigned char* dst, const unsigned char* src, int bytes) {
  for (int i = threadIdx.x; i < bytes / 16; i += 128)
    reinterpret_cast<uint4*>(dst)[i] = ld_global_v4(src + 16 * (size_t)i);
}

// Epilogue of a 256-wide layer: TMEM row tid, columns [col0, col0 + 256) ->
// relu(x + b) as bf16 into G (K = 256).
__device__ __forceinline__ void head_epi_256(uint32_t taddr, const float* b, unsigned char* G, int row) {
  float v[32];
#pragma unroll 1
  for (int h = 0; h < 8; ++h) {
    tmem_ld32(taddr + 32 * h, v);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 w;
      const int j = 8 * c, o = 32 * h + j;
      w.x = pack_bf16(fmaxf(v[j + 0] + b[o + 0], 0.f), fmaxf(v[j + 1] + b[o + 1], 0.f));
      w.y = pack_bf16(fmaxf(v[j + 2] + b[o + 2], 0.f), fmaxf(v[j + 3] + b[o + 3], 0.f));
      w.z = pack_bf16(fmaxf(v[j + 4] + b[o + 4], 0.f), fmaxf(v[j + 5] + b[o + 5], 0.f));
      w.w = pack_bf16(fmaxf(v[j + 6] + b[o + 6], 0.f), fmaxf(v[j + 7] + b[o + 7], 0.f));
      *reinterpret_cast<uint4*>(G + kmajor_off(row, o, 256)) = w;
    }
  }
}

__global__ void __launch_bounds__(128, 1)
    head_tc_kernel(const float* __restrict__ feat, int n_pairs, const int* n_dev,
                   const unsigned char* __restrict__ img, PairInputs in, int have_in,
                   const float4* __restrict__ centre, float* __restrict__ out,
                   float* __restrict__ y_raw, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n = n_dev ? min(*n_dev, n_pairs) : n_pairs;
  const int n_tiles = (n + HT - 1) / HT;
  if ((int)blockIdx.x >= n_tiles) return;
  for (int i = tid; i < H_RES_BYTES / 16; i += 128)
    reinterpret_cast<uint4*>(smem)[i] = ld_global_v4(img + 16 * (size_t)i);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + H_CTRL);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + H_CTRL + 8);
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
  const float* hb1 = reinterpret_cast<const float*>(smem + H_BIAS);
  const float* hb2 = hb1 + 256;
  const float* hb3 = hb2 + 256;
  unsigned char* A = smem + H_A;
  unsigned char* B = smem + H_B;
  unsigned char* G = smem + H_G;
  const uint32_t sA = smem_u32(A), sB = smem_u32(B), sG = smem_u32(G), sW3 = smem_u32(smem + H_W3);
  uint32_t phase = 0;
  bool ok = true;

  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int q0 = tile * HT;
    const int pr = q0 + tid;  // this thread's pair (row)
    const bool row_ok = pr < n;
    // ---- layer 1: D1[128 x 256] = F[128 x 512] . Wh1^T, K in chunks of 64
#pragma unroll 1
    for (int kc = 0; kc < 8; ++kc) {
      const float* src = feat + (size_t)pr * 512 + 64 * kc;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        if (row_ok) {
          a0 = __ldg(reinterpret_cast<const float4*>(src + 8 * c));
          a1 = __ldg(reinterpret_cast<const float4*>(src + 8 * c + 4));
        }
        uint4 w;
        w.x = pack_bf16(a0.x, a0.y);
        w.y = pack_bf16(a0.z, a0.w);
        w.z = pack_bf16(a1.x, a1.y);
        w.w = pack_bf16(a1.z, a1.w);
        *reinterpret_cast<uint4*>(A + kmajor_off(tid, 8 * c, 64)) = w;
      }
      copy_chunk(B, img + H_IMG_W1 + (size_t)kc * H_CHUNK, H_CHUNK);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tbase + 0, sdesc(sA + 256 * kk, 128, 1024), sdesc(sB + 256 * kk, 128, 1024),
                   idesc_bf16(128, 256), (kc > 0 || kk > 0) ? 1u : 0u);
        mma_commit(bar);
      }
      ok = mbar_wait(bar, phase, WAIT_CYCLES);
      phase ^= 1;
      if (!__syncthreads_and(ok)) { ok = false; break; }
      tc_fence_after();
    }
    if (!ok) break;
    head_epi_256(tbase + lane_off + 0, hb1, G, tid);
    // ---- layer 2: D2[128 x 256] = G[128 x 256] . Wh2^T
#pragma unroll 1
    for (int kc = 0; kc < 4; ++kc) {
      copy_chunk(B, img + H_IMG_W2 + (size_t)kc * H_CHUNK, H_CHUNK);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tbase + 256, sdesc(sG + 1024 * kc + 256 * kk, 128, 4096),
                   sdesc(sB + 256 * kk, 128, 1024), idesc_bf16(128, 256),
                   (kc > 0 || kk > 0) ? 1u : 0u);
        mma_commit(bar);
      }
      ok = mbar_wait(bar, phase, WAIT_CYCLES);
      phase ^= 1;
      if (!__syncthreads_and(ok)) { ok = false; break; }
      tc_fence_after();
    }
    if (!ok) break;
    head_epi_256(tbase + lane_off + 256, hb2, G, tid);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 3: D3[128 x 16] = G[128 x 256] . Wh3img^T (rows 8..15 zero)
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk)
        mma_bf16(tbase + 0, sdesc(sG + 256 * kk, 128, 4096), sdesc(sW3 + 256 * kk, 128, 4096),
                 idesc_bf16(128, 16), kk > 0);
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
        for (int o = 0; o < 8; ++o) y[o] = v[o] + hb3[o];
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

// ------------------------------------------------------------- host images
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even (finite inputs)
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Write rows x K values (val(r, k)) as a K-major no-swizzle bf16 tile.
template <typename F>
void put_tile(unsigned char* dst, int rows, int K, F val) {
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < K; ++k) {
      const uint16_t b = bf16_bits(val(r, k));
      std::memcpy(dst + kmajor_off(r, k, K), &b, 2);
    }
}

}  // namespace

int upload_tc_params(locc_handle* h, const std::vector<float>& params) {
  // flat parameter offsets (W then b per layer)
  size_t off[6], offb[6], o = 0;
  for (int l = 0; l < 6; ++l) {
    off[l] = o;
    o += (size_t)L_IN[l] * L_OUT[l];
    offb[l] = o;
    o += L_OUT[l];
  }
  auto W = [&](int l, int out_c, int in_k) {
    return params[off[l] + (size_t)out_c * L_IN[l] + in_k];
  };
  const size_t enc_bytes = (E_IMG_BYTES + 255) / 256 * 256;
  const size_t total = enc_bytes + H_IMG_BYTES;
  std::vector<unsigned char> img(total, 0);
  unsigned char* e = img.data();
  // layer 1 B operand: row c = [W_hi(3), W_hi(3), W_lo(3), 0 x 7]
  put_tile(e + E_W1, 64, 16, [&](int c, int k) -> float {
    if (k >= 9) return 0.f;
    const float w = W(0, c, k % 3);
    const float hi = bf16_value(bf16_bits(w));
    return k < 6 ? hi : w - hi;
  });
  put_tile(e + E_W2, 128, 64, [&](int c, int k) { return W(1, c, k); });
  put_tile(e + E_W3, 256, 128, [&](int c, int k) { return W(2, c, k); });
  std::memcpy(e + E_BIAS, &params[offb[0]], 64 * 4);
  std::memcpy(e + E_BIAS + 64 * 4, &params[offb[1]], 128 * 4);
  std::memcpy(e + E_BIAS + 192 * 4, &params[offb[2]], 256 * 4);
  unsigned char* hd = img.data() + enc_bytes;
  put_tile(hd + H_W3, 16, 256, [&](int c, int k) { return c < 8 ? W(5, c, k) : 0.f; });
  std::memcpy(hd + H_BIAS, &params[offb[3]], 256 * 4);
  std::memcpy(hd + H_BIAS + 256 * 4, &params[offb[4]], 256 * 4);
  std::memcpy(hd + H_BIAS + 512 * 4, &params[offb[5]], 8 * 4);
  for (int kc = 0; kc < 8; ++kc)
    put_tile(hd + H_IMG_W1 + (size_t)kc * H_CHUNK, 256, 64,
             [&](int c, int k) { return W(3, c, 64 * kc + k); });
  for (int kc = 0; kc < 4; ++kc)
    put_tile(hd + H_IMG_W2 + (size_t)kc * H_CHUNK, 256, 64,
             [&](int c, int k) { return W(4, c, 64 * kc + k); });
  if (cudaMalloc(&h->d_wtc, total) != cudaSuccess ||
      cudaMemcpy(h->d_wtc, img.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot upload tensor-core parameter images");
    return LOCC_ERR_OOM;
  }
  h->wtc_bytes = total;
  h->wtc_enc = static_cast<unsigned char*>(h->d_wtc);
  h->wtc_head = static_cast<unsigned char*>(h->d_wtc) + enc_bytes;
  return LOCC_OK;
}

int run_network_tc(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                   const PairInputs* in, const float4* centre, float* out, float* y_raw,
                   float* feat_out, cudaStream_t stream, cudaEvent_t mid) {
  if (h->prec != LOCC_BF16) {
    set_error("FP8 tensor-core path not available in this build");
    return LOCC_ERR_INVALID_ARG;
  }
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(encoder_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             E_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(head_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             H_SMEM) != cudaSuccess) {
      set_error("cudaFuncSetAttribute failed for the tensor-core kernels");
      return LOCC_ERR_CUDA;
    }
    attr = true;
  }
  float* feat = feat_out ? feat_out : h->d_feat;
  const int grid_e = std::min(n_pairs, h->n_sm);
  encoder_tc_kernel<<<grid_e, 128, E_SMEM, stream>>>(xyz, n_pairs, n_dev, h->wtc_enc, feat,
                                                     h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("encoder_tc_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  if (mid && cudaEventRecord(mid, stream) != cudaSuccess) return LOCC_ERR_CUDA;
  PairInputs pin{};
  if (in) pin = *in;
  const int grid_h = std::min((n_pairs + HT - 1) / HT, h->n_sm);
  head_tc_kernel<<<grid_h, 128, H_SMEM, stream>>>(feat, n_pairs, n_dev, h->wtc_head, pin,
                                                  in != nullptr, centre, out, y_raw, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("head_tc_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

}  // namespace locc

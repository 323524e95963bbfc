// Tensor-core kernels of the BF16 trainer (locc_trainer_set_precision(t,
// LOCC_BF16)): the dense products of the forward and backward passes run as
// tcgen05.mma with bf16 operands and float32 accumulation in TMEM; parameters,
// Adam and every stored activation and gradient stay float32.
//
// tg_kernel: C[M x N] (+)= op(A)[M x K] op(B)[K x N] on tiles of 128 x BN.
//   op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k]
//   op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n]
//   Four warps load float32 tiles of 128 x 32 (A) and BN x 32 (B) from global
//   memory into registers (the next tile while the current one is multiplied),
//   round them to bf16 and store them in the K-major no-swizzle layout of the
//   MMA operands (three stages); one elected lane issues two K = 16 MMAs
//   per stage and commits them to the stage's mbarrier, which the loaders wait
//   on (bounded) before refilling the stage.  Split-K runs over gridDim.z;
//   BN = 64 where 128-column tiles would leave SMs idle.
//   Epilogues (TMEM lane = tile row):
//   STORE  + bias, ReLU-mask (mask > 0), ReLU, accumulate, atomic split-K;
//          rows staged through shared memory so that each warp reads and
//          writes C and the mask in whole 128-byte segments;
//   POOL   layer 3 of the encoder computed transposed (M = 256 channels,
//          N = the 128 crop rows of one pair, A = W3, B = H2): relu(z + b3)
//          max-pooled over each object's valid rows with the argmax slot
//          (ties to the lower slot), Z3 never stored;
//   L1GRAD dH1 = dH2 W2 masked by the recomputed layer-1 ReLU, reduced in the
//          CTA into dL/dW1 = dH1^T X and dL/db1 = sum dH1 (dH1 never stored).
//   H1 (layer 1's output) is never stored either: the A operand of layer 2 and
//   the B operand of dL/dW2 recompute it from the crop rows while staging.
//
// Layer 3's backward is sparse (Sec. III-A max-pooling: dL/dZ3 is non-zero
// only at each channel's argmax row, at most 256 of 64 x 256 entries per
// object), so it runs on the CUDA cores in float32 without forming dZ3:
//   sparse_dh2_kernel: dH2 = [H2 > 0] * sum_c dF[c] W3[c, :] at row amax[c],
//                      plus dL/db2 = column sums of dH2;
//   sparse_gw3_kernel: dL/dW3[c, :] = sum over objects of dF[c] H2[amax[c], :],
//                      dL/db3[c] = sum of dF[c].
#include <algorithm>

#include <cuda_bf16.h>

#include "handle.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

using namespace tc;

constexpr long long TG_WAIT = 2000000000LL;  // ~1 s at 2 GHz
constexpr int TG_BM = 128, TG_BK = 32, TG_NS = 3;
constexpr int TG_A_BYTES = TG_BM * TG_BK * 2;  // 8 KB per stage
enum { TG_STORE = 0, TG_POOL = 1, TG_L1GRAD = 2 };
enum { TG_MEM = 0, TG_A_H1 = 1, TG_B_H1 = 2 };  // operand recomputed from X

__host__ __device__ constexpr int tg_stage_bytes(int bn) { return TG_A_BYTES + bn * TG_BK * 2; }
// Dynamic shared memory: the stages, also reused by the epilogues (STORE:
// 128 x 36 floats; L1GRAD: 128 x 65 floats + crop rows).  Padded so
// that at most four CTAs of BN = 128 (five of BN = 64, by registers) share an
// SM: their TMEM columns (BN each) then always fit the SM's 512.
__host__ __device__ constexpr int tg_smem_bytes(int bn) { return bn == 128 ? 54 * 1024 : 40 * 1024; }
static_assert(TG_NS * (TG_A_BYTES + 128 * TG_BK * 2) <= 54 * 1024, "stages of BN = 128");
static_assert(TG_NS * (TG_A_BYTES + 64 * TG_BK * 2) <= 40 * 1024, "stages of BN = 64");
static_assert(128 * 65 * 4 + 128 * 16 + 256 * 4 <= 40 * 1024, "L1GRAD scratch");

struct TgArgs {
  int M, N, K;
  const float* A;
  int lda;
  const float* B;
  int ldb;
  float* C;
  int ldc;
  const float* bias;
  const float* mask;
  int ldm;
  int relu, accumulate, k_split;
  int vec_a, vec_b;  // 16-byte aligned rows: float4 loads
  // POOL: crop rows (float4, w = valid), pooled features [P][512], argmax
  const float* X;
  float* F;
  int32_t* amax;
  // L1GRAD: layer-1 weights and biases, their gradients
  const float* W1;
  const float* b1;
  float* gW1;
  float* gB1;
  int* err;
};

// Operand tiles of R rows x 32 K columns, staged through registers: each
// thread holds R / 32 items of 8 consecutive K values of one row.  All loads
// of a tile are issued before any of them is stored, and the next tile's
// loads are in flight while the current one is multiplied.
//   RC = false: K index contiguous in memory, src(r, k) = P[r ld + k]
//               (float4 loads when vec, 4 threads per row);
//   RC = true:  row index contiguous, src(r, k) = P[k ld + r] (consecutive
//               threads take consecutive rows: each load coalesced).
// Entries outside r < rlim, k < klim are zero.
template <int R, bool RC>
__device__ __forceinline__ void tile_item(int u, int* r, int* kg) {
  const int it = threadIdx.x + 128 * u;
  if (RC) *r = it % R, *kg = it / R;
  else *r = it >> 2, *kg = it & 3;
}

template <int R, bool RC>
__device__ __forceinline__ void tile_load(float (&v)[R / 32][8], const float* __restrict__ P,
                                          int ld, int r0, int rlim, int k0, int klim, int vec) {
#pragma unroll
  for (int u = 0; u < R / 32; ++u) {
    int r, kg;
    tile_item<R, RC>(u, &r, &kg);
    const int gr = r0 + r, gk = k0 + kg * 8;
    if (RC) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[u][j] = (gr < rlim && gk + j < klim) ? __ldg(P + (size_t)(gk + j) * ld + gr) : 0.f;
    } else {
      const float* src = P + (size_t)gr * ld + gk;
      if (vec && gr < rlim && gk + 8 <= klim) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(src));
        const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
        v[u][0] = a.x, v[u][1] = a.y, v[u][2] = a.z, v[u][3] = a.w;
        v[u][4] = b.x, v[u][5] = b.y, v[u][6] = b.z, v[u][7] = b.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[u][j] = (gr < rlim && gk + j < klim) ? __ldg(src + j) : 0.f;
      }
    }
  }
}

// Layer 1 of the encoder recomputed while staging (H1 is never stored):
// relu(W1 x + b1) with the float32 operation order of the forward pass
// (b1, then W1[c] x, y, z by fused multiply-adds), so that every consumer
// sees the same H1 bits.  w = {W1[c][0..2], b1[c]} per channel c, in shared
// memory; X rows are float4 (x, y, z, valid).
__device__ __forceinline__ float layer1_value(const float4* w, int c, float4 x) {
  const float4 q = w[c];
  float h = q.w;
  h = fmaf(q.x, x.x, h);
  h = fmaf(q.y, x.y, h);
  h = fmaf(q.z, x.z, h);
  return fmaxf(h, 0.f);
}

// RC = false: rows are crop rows, K = the 64 layer-1 channels (the A operand
// of layer 2); RC = true: rows are channels, K = crop rows (the B operand of
// dL/dW2 = dH2^T H1).  The load keeps the raw crop rows in registers (one per
// item for RC = false, eight for RC = true) and the layer-1 arithmetic runs
// when the tile is stored, so that the loads stay in flight meanwhile.
template <int R, bool RC>
struct H1Regs {
  float4 x[R / 32][RC ? 8 : 1];
};

template <int R, bool RC>
__device__ __forceinline__ void tile_load_h1(H1Regs<R, RC>& v, const float4* __restrict__ X, int r0,
                                             int rlim, int k0, int klim) {
#pragma unroll
  for (int u = 0; u < R / 32; ++u) {
    int r, kg;
    tile_item<R, RC>(u, &r, &kg);
    const int gr = r0 + r, gk = k0 + kg * 8;
    if (RC) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v.x[u][j] = (gr < rlim && gk + j < klim) ? __ldg(X + gk + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      v.x[u][0] = gr < rlim ? __ldg(X + gr) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

template <int R, bool RC>
__device__ __forceinline__ void tile_store_h1(unsigned char* dst, const H1Regs<R, RC>& v,
                                              const float4* w, int r0, int rlim, int k0, int klim) {
#pragma unroll
  for (int u = 0; u < R / 32; ++u) {
    int r, kg;
    tile_item<R, RC>(u, &r, &kg);
    const int gr = r0 + r, gk = k0 + kg * 8;
    float h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool e = gr < rlim && gk + j < klim;
      h[j] = e ? (RC ? layer1_value(w, gr, v.x[u][j]) : layer1_value(w, gk + j, v.x[u][0])) : 0.f;
    }
    uint4 q;
    q.x = pack_bf16(h[0], h[1]);
    q.y = pack_bf16(h[2], h[3]);
    q.z = pack_bf16(h[4], h[5]);
    q.w = pack_bf16(h[6], h[7]);
    *reinterpret_cast<uint4*>(dst + kmajor_off(r, kg * 8, TG_BK)) = q;
  }
}

// Registers -> bf16 K-major no-swizzle tile (lbo 128, sbo 32 * 16).
template <int R, bool RC>
__device__ __forceinline__ void tile_store(unsigned char* dst, const float (&v)[R / 32][8]) {
#pragma unroll
  for (int u = 0; u < R / 32; ++u) {
    int r, kg;
    tile_item<R, RC>(u, &r, &kg);
    uint4 w;
    w.x = pack_bf16(v[u][0], v[u][1]);
    w.y = pack_bf16(v[u][2], v[u][3]);
    w.z = pack_bf16(v[u][4], v[u][5]);
    w.w = pack_bf16(v[u][6], v[u][7]);
    *reinterpret_cast<uint4*>(dst + kmajor_off(r, kg * 8, TG_BK)) = w;
  }
}

template <bool TA, bool TB, int BN, int EPI, int XS>
__global__ void __launch_bounds__(128, (BN == 128 || XS == TG_B_H1) ? 4 : 5) tg_kernel(TgArgs g) {
  static_assert(BN == 64 || BN == 128, "tile width");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[TG_NS];
  __shared__ uint32_t tslot;
  constexpr bool W1S = XS != TG_MEM || EPI == TG_L1GRAD;
  __shared__ float4 s_w1[W1S ? 64 : 1];  // {W1[c][0..2], b1[c]}
  constexpr int ST = tg_stage_bytes(BN);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * TG_BM;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  const int nk = ke > kb ? (ke - kb + TG_BK - 1) / TG_BK : 0;
  if (tid == 0) {
    for (int s = 0; s < TG_NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  if (W1S && tid < 64)
    s_w1[tid] = make_float4(g.W1[3 * tid], g.W1[3 * tid + 1], g.W1[3 * tid + 2], g.b1[tid]);
  // L1GRAD: this thread's crop row, loaded before the K loop
  float4 x_row = make_float4(0.f, 0.f, 0.f, 0.f);
  if (EPI == TG_L1GRAD && (int)blockIdx.y * TG_BM + tid < g.M)
    x_row = __ldg(reinterpret_cast<const float4*>(g.X) + (size_t)blockIdx.y * TG_BM + tid);
  if (warp == 0) {
    tmem_alloc(smem_u32(&tslot), BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  constexpr uint32_t idesc = idesc_bf16(TG_BM, BN);
  bool ok = true;
  float ra[XS == TG_A_H1 ? 1 : TG_BM / 32][8], rb[XS == TG_B_H1 ? 1 : BN / 32][8];
  H1Regs<XS == TG_A_H1 ? TG_BM : 32, false> xa;
  H1Regs<XS == TG_B_H1 ? BN : 32, true> xb;
  const float4* X4 = reinterpret_cast<const float4*>(g.X);
  auto load_tiles = [&](int k0) {
    if constexpr (XS == TG_A_H1) tile_load_h1<TG_BM, false>(xa, X4, m0, g.M, k0, ke);
    else tile_load<TG_BM, TA>(ra, g.A, g.lda, m0, g.M, k0, ke, g.vec_a);
    if constexpr (XS == TG_B_H1) tile_load_h1<BN, true>(xb, X4, n0, g.N, k0, ke);
    else tile_load<BN, !TB>(rb, g.B, g.ldb, n0, g.N, k0, ke, g.vec_b);
  };
  if (nk > 0) load_tiles(kb);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % TG_NS;
    unsigned char* sA = smem + s * ST;
    unsigned char* sB = sA + TG_A_BYTES;
    // the MMAs that read this stage TG_NS steps ago must be done
    if (kt >= TG_NS) ok = mbar_wait(smem_u32(&bars[s]), ((kt / TG_NS) - 1) & 1, TG_WAIT);
    if (ok) {
      const int k0 = kb + kt * TG_BK;
      if constexpr (XS == TG_A_H1) tile_store_h1<TG_BM, false>(sA, xa, s_w1, m0, g.M, k0, ke);
      else tile_store<TG_BM, TA>(sA, ra);
      if constexpr (XS == TG_B_H1) tile_store_h1<BN, true>(sB, xb, s_w1, n0, g.N, k0, ke);
      else tile_store<BN, !TB>(sB, rb);
    }
    fence_async_smem();
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (warp == 0) {
      tc_fence_after();
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < TG_BK / 16; ++kk)
          mma_bf16(tbase, sdesc(smem_u32(sA) + 256 * kk, 128, TG_BK * 16),
                   sdesc(smem_u32(sB) + 256 * kk, 128, TG_BK * 16), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
        mma_commit(smem_u32(&bars[s]));
      }
      __syncwarp();
    }
    if (kt + 1 < nk) load_tiles(kb + (kt + 1) * TG_BK);  // overlaps this tile's MMAs
  }
  if (ok && nk > 0) ok = mbar_wait(smem_u32(&bars[(nk - 1) % TG_NS]), ((nk - 1) / TG_NS) & 1, TG_WAIT);
  ok = __syncthreads_and(ok);
  tc_fence_after();
  const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
  if (ok && nk > 0) {
    if (EPI == TG_STORE) {
      // TMEM rows -> shared memory (thread = row), then each warp writes its
      // 32 rows four at a time: eight lanes per row, a float4 each, so that
      // every access of C and of the mask is a whole 128-byte segment
      float* T = reinterpret_cast<float*>(smem);  // [128][36]
      const bool split = gridDim.z > 1, first = blockIdx.z == 0;
      const int lr = lane >> 3, lc = (lane & 7) * 4;
#pragma unroll 1
      for (int cc = 0; cc < BN; cc += 32) {
        float v[32];
        tmem_ld32(trow + cc, v);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(T + tid * 36 + 4 * q) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncthreads();
        const int n = n0 + cc + lc;
        const bool nv = n < g.N;  // N is a multiple of 4
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g.bias && first && nv) b = *reinterpret_cast<const float4*>(g.bias + n);
        float4 cur[8], msk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // all loads first
          const int m = m0 + warp * 32 + 4 * q + lr;
          const bool e = nv && m < g.M;
          cur[q] = (e && g.accumulate && !split)
                       ? *reinterpret_cast<const float4*>(g.C + (size_t)m * g.ldc + n)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
          msk[q] = (e && g.mask) ? *reinterpret_cast<const float4*>(g.mask + (size_t)m * g.ldm + n)
                                 : make_float4(1.f, 1.f, 1.f, 1.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int r = warp * 32 + 4 * q + lr, m = m0 + r;
          if (!nv || m >= g.M) continue;
          const float4 t = *reinterpret_cast<const float4*>(T + r * 36 + lc);
          float o[4] = {t.x + b.x, t.y + b.y, t.z + b.z, t.w + b.w};
          const float mk[4] = {msk[q].x, msk[q].y, msk[q].z, msk[q].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (!(mk[e] > 0.f)) o[e] = 0.f;
            if (g.relu) o[e] = fmaxf(o[e], 0.f);
          }
          float* c = g.C + (size_t)m * g.ldc + n;
          if (split) {
#pragma unroll
            for (int e = 0; e < 4; ++e) atomicAdd(c + e, o[e]);
          } else {
            *reinterpret_cast<float4*>(c) =
                make_float4(o[0] + cur[q].x, o[1] + cur[q].y, o[2] + cur[q].z, o[3] + cur[q].w);
          }
        }
        __syncthreads();
      }
    } else if (EPI == TG_POOL) {
      // n0 = first crop row of pair p; thread = channel c
      int* s_cnt = reinterpret_cast<int*>(smem);
      unsigned char* s_flag = smem + 16;
      const int p = blockIdx.x;
      s_flag[tid] = reinterpret_cast<const float4*>(g.X)[(size_t)n0 + tid].w > 0.5f ? 1 : 0;
      __syncthreads();
      if (tid < 2) {
        int c = 0;
        while (c < KMAX && s_flag[tid * KMAX + c]) ++c;
        s_cnt[tid] = c;
      }
      __syncthreads();
      const int c = m0 + warp * 32 + lane;
      const float b = g.bias[c];
#pragma unroll 1
      for (int o = 0; o < 2; ++o) {
        const int cnt = s_cnt[o];
        float best = 0.f;
        int arg = -1;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(trow + o * KMAX + 32 * h, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int k = 32 * h + i;
            const float z = fmaxf(v[i] + b, 0.f);
            if (k < cnt && (arg < 0 || z > best)) best = z, arg = k;
          }
        }
        g.F[(size_t)p * 512 + o * FEAT + c] = best;
        g.amax[(size_t)p * 512 + o * FEAT + c] = arg;
      }
    } else {  // TG_L1GRAD, BN = 64: thread = crop row
      float* s_g = reinterpret_cast<float*>(smem);         // [128][65]
      float4* s_x = reinterpret_cast<float4*>(smem + 128 * 65 * 4);
      const int m = m0 + tid;
      const float4 x = x_row;
      s_x[tid] = x;
      __syncthreads();
      float v[64];
      tmem_ld32x2(trow, v);
#pragma unroll
      for (int i = 0; i < 64; ++i) {
        // the forward's layer 1, same operation order: the same ReLU decision
        const float4 q = s_w1[i];
        float h = q.w;
        h = fmaf(q.x, x.x, h);
        h = fmaf(q.y, x.y, h);
        h = fmaf(q.z, x.z, h);
        s_g[tid * 65 + i] = (m < g.M && h > 0.f) ? v[i] : 0.f;
      }
      __syncthreads();
      const int i = tid & 63, r0 = (tid >> 6) * 64;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, sb = 0.f;
#pragma unroll 4
      for (int r = r0; r < r0 + 64; ++r) {
        const float gv = s_g[r * 65 + i];
        const float4 xr = s_x[r];
        s0 = fmaf(gv, xr.x, s0);
        s1 = fmaf(gv, xr.y, s1);
        s2 = fmaf(gv, xr.z, s2);
        sb += gv;
      }
      atomicAdd(g.gW1 + 3 * i, s0);
      atomicAdd(g.gW1 + 3 * i + 1, s1);
      atomicAdd(g.gW1 + 3 * i + 2, s2);
      atomicAdd(g.gB1 + i, sb);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && !ok) atomicOr(g.err, 2);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, BN);
  }
}

// dH2 of one object (blockIdx.x = 2 p + o), thread = column j: the column's
// 64 row sums accumulate in shared memory over the object's 256 channels
// (each adds dF[c] W3[c, j] to its argmax row; a channel without gradient
// adds 0 to row 0), then are masked by H2 > 0.  One object per CTA (34 KB of
// shared memory) lets about six CTAs share an SM, which hides the latency of
// the W3 loads and of the read-modify-write chain.
__global__ void __launch_bounds__(128) sparse_dh2_kernel(const float* __restrict__ dF,
                                                         const float* __restrict__ F,
                                                         const int32_t* __restrict__ amax,
                                                         const float* __restrict__ W3,
                                                         const float* __restrict__ H2,
                                                         float* __restrict__ dH2,
                                                         float* __restrict__ gB2, int n_obj) {
  __shared__ float acc[KMAX][128];
  __shared__ int s_k[FEAT];
  __shared__ float s_g[FEAT];
  const int ob = blockIdx.x, j = threadIdx.x;
  if (ob >= n_obj) return;
  const int p = ob >> 1, o = ob & 1;
  const size_t row0 = (size_t)p * ROWS + o * KMAX;
  for (int c = j; c < FEAT; c += 128) {
    const size_t f = (size_t)p * 512 + o * FEAT + c;
    const int k = amax[f];
    const bool on = k >= 0 && F[f] > 0.f;
    s_k[c] = on ? k : 0;
    s_g[c] = on ? dF[f] : 0.f;
  }
  for (int k = 0; k < KMAX; ++k) acc[k][j] = 0.f;
  __syncthreads();
#pragma unroll 16
  for (int c = 0; c < FEAT; ++c)
    acc[s_k[c]][j] = fmaf(s_g[c], __ldg(W3 + (size_t)c * 128 + j), acc[s_k[c]][j]);
  float col = 0.f;
#pragma unroll 16
  for (int k = 0; k < KMAX; ++k) {
    const size_t e = (row0 + k) * 128 + j;
    const float v = H2[e] > 0.f ? acc[k][j] : 0.f;
    dH2[e] = v;
    col += v;
  }
  atomicAdd(gB2 + j, col);
}

// dL/dW3 rows [c0, c0 + 16) (blockIdx.x) over the objects of blockIdx.y's
// range, thread = column j; dL/db3 from the same sums.  The range is taken in
// chunks of 16 objects whose argmax rows and gradients are first gathered
// into shared memory, so that the row loads of four objects (64 rows) are in
// flight together.
constexpr int GW3_CB = 16, GW3_OB = 16;
__global__ void __launch_bounds__(128) sparse_gw3_kernel(const float* __restrict__ dF,
                                                         const float* __restrict__ F,
                                                         const int32_t* __restrict__ amax,
                                                         const float* __restrict__ H2,
                                                         float* __restrict__ gW3,
                                                         float* __restrict__ gB3, int n_obj,
                                                         int obj_per_block) {
  __shared__ int s_row[GW3_OB][GW3_CB];  // H2 row of the channel's argmax, -1 if none
  __shared__ float s_g[GW3_OB][GW3_CB];
  const int c0 = blockIdx.x * GW3_CB, j = threadIdx.x;
  const int ob = blockIdx.y * obj_per_block, oe = min(n_obj, ob + obj_per_block);
  float acc[GW3_CB], bs = 0.f;
#pragma unroll
  for (int i = 0; i < GW3_CB; ++i) acc[i] = 0.f;
  for (int o0 = ob; o0 < oe; o0 += GW3_OB) {
    __syncthreads();
    for (int e = j; e < GW3_OB * GW3_CB; e += 128) {
      const int oi = e / GW3_CB, ci = e % GW3_CB, obj = o0 + oi;
      int row = -1;
      float gv = 0.f;
      if (obj < oe) {
        const int p = obj >> 1, o = obj & 1;
        const size_t f = (size_t)p * 512 + o * FEAT + c0 + ci;
        const int k = amax[f];
        if (k >= 0 && F[f] > 0.f) {
          row = p * ROWS + o * KMAX + k;
          gv = dF[f];
        }
      }
      s_row[oi][ci] = row;
      s_g[oi][ci] = gv;
    }
    __syncthreads();
    if (j < GW3_CB)
      for (int oi = 0; oi < GW3_OB; ++oi) bs += s_g[oi][j];
#pragma unroll 1
    for (int oi = 0; oi < GW3_OB; oi += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int ci = 0; ci < GW3_CB; ++ci) {
          const int row = s_row[oi + u][ci];
          const float h = row >= 0 ? __ldg(H2 + (size_t)row * 128 + j) : 0.f;
          acc[ci] = fmaf(s_g[oi + u][ci], h, acc[ci]);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < GW3_CB; ++i) atomicAdd(gW3 + (size_t)(c0 + i) * 128 + j, acc[i]);
  if (j < GW3_CB) atomicAdd(gB3 + c0 + j, bs);
}

template <bool TA, bool TB, int BN, int EPI, int XS = TG_MEM>
cudaError_t tg_launch(TgArgs g, int splits, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  splits = std::max(1, std::min(splits, (g.K + TG_BK - 1) / TG_BK));
  int ks = (g.K + splits - 1) / splits;
  ks = (ks + TG_BK - 1) / TG_BK * TG_BK;
  splits = (g.K + ks - 1) / ks;
  g.k_split = ks;
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  g.vec_a = (!TA && g.lda % 4 == 0 && al16(g.A)) ? 1 : 0;
  g.vec_b = (TB && g.ldb % 4 == 0 && al16(g.B)) ? 1 : 0;
  dim3 grid((g.N + BN - 1) / BN, (g.M + TG_BM - 1) / TG_BM, splits);
  tg_kernel<TA, TB, BN, EPI, XS><<<grid, 128, tg_smem_bytes(BN), s>>>(g);
  return cudaGetLastError();
}

// The STORE epilogue accesses C, the mask and the bias as float4: N, ldc and
// ldm multiples of 4, the three 16-byte aligned.
bool tg_store_aligned(const TgArgs& g) {
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return g.N % 4 == 0 && g.ldc % 4 == 0 && al16(g.C) && (!g.bias || al16(g.bias)) &&
         (!g.mask || (g.ldm % 4 == 0 && al16(g.mask)));
}

TgArgs tg_args(int M, int N, int K, const float* A, int lda, const float* B, int ldb, int* err) {
  TgArgs g{};
  g.M = M, g.N = N, g.K = K, g.A = A, g.lda = lda, g.B = B, g.ldb = ldb, g.err = err;
  return g;
}

}  // namespace

cudaError_t tg_gemm(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B,
                    int ldb, float* C, int ldc, const float* bias, const float* mask, int ldm,
                    bool relu, bool accumulate, int splits, int* err, cudaStream_t s) {
  TgArgs g = tg_args(M, N, K, A, lda, B, ldb, err);
  g.C = C, g.ldc = ldc, g.bias = bias, g.mask = mask, g.ldm = ldm;
  g.relu = relu ? 1 : 0, g.accumulate = accumulate ? 1 : 0;
  if (!tg_store_aligned(g)) return cudaErrorInvalidValue;
  // tiles of 64 columns where 128-column tiles would leave most SMs idle (the
  // head's products on small batches: 16-32 tiles with long K loops)
  int n_sm = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 148;
  const long long tiles128 = (long long)((N + 127) / 128) * ((M + TG_BM - 1) / TG_BM) * std::max(splits, 1);
  const bool narrow = N <= 64 || tiles128 < n_sm;
  if (!ta && tb) {
    if (narrow) return tg_launch<false, true, 64, TG_STORE>(g, splits, s);
    return tg_launch<false, true, 128, TG_STORE>(g, splits, s);
  }
  if (ta && !tb) {
    if (narrow) return tg_launch<true, false, 64, TG_STORE>(g, splits, s);
    return tg_launch<true, false, 128, TG_STORE>(g, splits, s);
  }
  if (!ta && !tb) {
    if (narrow) return tg_launch<false, false, 64, TG_STORE>(g, splits, s);
    return tg_launch<false, false, 128, TG_STORE>(g, splits, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tg_layer2_forward(const float* X, const float* W1, const float* b1, const float* W2,
                              const float* b2, int M, float* H2, int* err, cudaStream_t s) {
  TgArgs g = tg_args(M, 128, 64, nullptr, 0, W2, 64, err);
  g.X = X, g.W1 = W1, g.b1 = b1;
  g.C = H2, g.ldc = 128, g.bias = b2, g.relu = 1;
  if (!tg_store_aligned(g)) return cudaErrorInvalidValue;
  return tg_launch<false, true, 128, TG_STORE, TG_A_H1>(g, 1, s);
}

cudaError_t tg_layer2_wgrad(const float* dH2, const float* X, const float* W1, const float* b1, int M,
                            float* gW2, int splits, int* err, cudaStream_t s) {
  TgArgs g = tg_args(128, 64, M, dH2, 128, nullptr, 0, err);
  g.X = X, g.W1 = W1, g.b1 = b1;
  g.C = gW2, g.ldc = 64, g.accumulate = 1;
  if (!tg_store_aligned(g)) return cudaErrorInvalidValue;
  return tg_launch<true, false, 64, TG_STORE, TG_B_H1>(g, splits, s);
}

cudaError_t tg_layer3_pool(const float* W3, const float* b3, const float* H2, const float* X, int P,
                           float* F, int32_t* amax, int* err, cudaStream_t s) {
  TgArgs g = tg_args(FEAT, P * ROWS, 128, W3, 128, H2, 128, err);
  g.bias = b3, g.X = X, g.F = F, g.amax = amax;
  return tg_launch<false, true, 128, TG_POOL>(g, 1, s);
}

cudaError_t tg_layer1_grad(const float* dH2, const float* W2, const float* X, const float* W1,
                           const float* b1, int M, float* gW1, float* gB1, int* err, cudaStream_t s) {
  TgArgs g = tg_args(M, 64, 128, dH2, 128, W2, 64, err);
  g.X = X, g.W1 = W1, g.b1 = b1, g.gW1 = gW1, g.gB1 = gB1;
  return tg_launch<false, false, 64, TG_L1GRAD>(g, 1, s);
}

cudaError_t sparse_layer3_backward(const float* dF, const float* F, const int32_t* amax,
                                   const float* W3, const float* H2, int P, float* dH2, float* gW3,
                                   float* gB3, float* gB2, int n_sm, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  sparse_dh2_kernel<<<2 * P, 128, 0, s>>>(dF, F, amax, W3, H2, dH2, gB2, 2 * P);
  const int n_obj = 2 * P;
  // about 8 x n_sm CTAs over 16 channel blocks; whole 16-object chunks
  const int want = std::max(1, (8 * n_sm) / (FEAT / GW3_CB));
  int per = (n_obj + want - 1) / want;
  per = std::max(GW3_OB, (per + GW3_OB - 1) / GW3_OB * GW3_OB);
  dim3 grid(FEAT / GW3_CB, (n_obj + per - 1) / per);
  sparse_gw3_kernel<<<grid, 128, 0, s>>>(dF, F, amax, H2, gW3, gB3, n_obj, per);
  return cudaGetLastError();
}

cudaError_t prepare_train_tc_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)tg_kernel<false, true, 128, TG_STORE, TG_MEM>, tg_smem_bytes(128));
  set((const void*)tg_kernel<false, true, 64, TG_STORE, TG_MEM>, tg_smem_bytes(64));
  set((const void*)tg_kernel<false, false, 64, TG_STORE, TG_MEM>, tg_smem_bytes(64));
  set((const void*)tg_kernel<true, false, 64, TG_STORE, TG_MEM>, tg_smem_bytes(64));
  set((const void*)tg_kernel<true, false, 128, TG_STORE, TG_MEM>, tg_smem_bytes(128));
  set((const void*)tg_kernel<false, false, 128, TG_STORE, TG_MEM>, tg_smem_bytes(128));
  set((const void*)tg_kernel<false, true, 128, TG_POOL, TG_MEM>, tg_smem_bytes(128));
  set((const void*)tg_kernel<false, false, 64, TG_L1GRAD, TG_MEM>, tg_smem_bytes(64));
  set((const void*)tg_kernel<false, true, 128, TG_STORE, TG_A_H1>, tg_smem_bytes(128));
  set((const void*)tg_kernel<true, false, 64, TG_STORE, TG_B_H1>, tg_smem_bytes(64));
  return e;
}

}  // namespace locc

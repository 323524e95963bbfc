// FP8 (e4m3) crop network on tcgen05 (LOCC_FP8).
//
// Same network and kernel structure as the BF16 path (net_tc.cu); encoder
// layers 2-3 and all head layers use tcgen05.mma kind::f8f6f4 (e4m3 operands,
// float32 accumulation in TMEM).  Layer 1 (K = 3) keeps the bf16 hi/lo split.
//
// Scales.  Crop coordinates lie in the crop ball (|x| <= r), so every
// activation channel has a bound that follows from the weights alone:
//   B1_c = r |W1_c|_2 + b1_c,  B_{l+1,c} = sum_k |W_{l+1}[c][k]| B_{l,k} + b_{l+1,c}
// (ReLU outputs lie in [0, B]).  Channel k of a layer's output is stored as
// e4m3 of a / s_k with the static scale s_k = 1.1 B_k / 448, and s_k is folded
// into the next layer's weights: W'[c][k] = W[c][k] s_k, quantised with one
// scale per output channel, w_c = max_k |W'[c][k]| / 448.  The accumulator D of
// channel c then equals sum_k a_k W[c][k] / w_c, so each epilogue is one FMA
// and one saturating cvt:  next = cvt_relu(D alpha_c + beta_c) with
// alpha_c = w_c / s_c, beta_c = b_c / s_c.  e4m3 is a floating-point format
// (2^14.8 of range), so a loose bound costs little precision.  The
// coefficients are computed on the host in float64 at create time.  Layer 1
// (bf16 hi/lo) has 1 / s_c folded into W1 and its bias b1 / s_c accumulated
// by the MMA through two constant-one columns of X, so its epilogue is the
// cvt alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

using namespace tc;

constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

// ------------------------------------------------------ weight quantisation
// Row r of W [rows][K] (float32, row-major) times inv[r] -> e4m3 bytes in
// K-chunks of chunkK columns, each chunk a K-major no-swizzle tile
// [rows][chunkK] stored one after the other.
__global__ void quant_e4m3_kernel(const float* __restrict__ W, const float* __restrict__ inv,
                                  int rows, int K, int chunkK, unsigned char* __restrict__ img) {
  const int r = blockIdx.x;
  const float s = inv[r];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const uint32_t q = pack_e4m3x4(W[(size_t)r * K + k] * s, 0.f, 0.f, 0.f);
    const int c = k / chunkK, kk = k % chunkK;
    img[(size_t)c * rows * chunkK + kmajor_off8(r, kk, chunkK)] = (unsigned char)(q & 0xffu);
  }
}

// ------------------------------------------------------------- encoder
constexpr int F_W1 = 0;                        // [64 x 16] bf16 (hi/lo, b1)  2 KB
constexpr int F_W2 = F_W1 + 64 * 16 * 2;       // [128 x 64] e4m3          8 KB
constexpr int F_W3 = F_W2 + 128 * 64;          // [256 x 128] e4m3        32 KB
constexpr int F_EP = F_W3 + 256 * 128;         // a1 c1 [64], a2 c2 [128], w3 b3 finv [256] (f32)
constexpr int F_IMG_BYTES = F_EP + (2 * 64 + 2 * 128 + 3 * 256) * 4;
static_assert(F_IMG_BYTES % 16 == 0, "encoder fp8 image must be 16-byte chunks");
// NSLOT pair slots; each: raw crop rows (2 KB) and a 16 KB operand region
// holding in turn X (bf16, 4 KB), H1 (e4m3, 8 KB) and H2 (e4m3, 16 KB).
constexpr int NSLOT = 4;
constexpr int F_SLOT0 = (F_IMG_BYTES + 1023) / 1024 * 1024;
constexpr int FS_STG = 0;
constexpr int FS_OPD = FS_STG + ROWS * 16;
constexpr int F_SLOT_BYTES = FS_OPD + 128 * 128;
constexpr int F_CTRL = F_SLOT0 + NSLOT * F_SLOT_BYTES;
constexpr int NBAR = 9 * NSLOT + 2;
constexpr int C_BAR = 0, C_TMEM = 8 * NBAR, C_ABORT = C_TMEM + 4, C_CNT = C_ABORT + 4;
constexpr int C_OBJ = C_CNT + 16 * NSLOT;  // [slot][tile parity][u, v] object ids
constexpr int F_SMEM = F_CTRL + C_OBJ + 16 * NSLOT;
static_assert(F_SMEM <= 227 * 1024, "fp8 encoder shared memory");
constexpr int F_THREADS = 32 * (4 * NSLOT + 2);
constexpr int MMA_WARP = 4 * NSLOT;
// zeroes the pooled features of the empty objects (zero_empty_objects)
constexpr int ZERO_WARP = 4 * NSLOT + 1;
constexpr int SLOT_COLS = 512 / NSLOT;
constexpr int B_FULLX = 0, B_XRDY = NSLOT, B_H1RDY = 2 * NSLOT, B_H2RDY = 3 * NSLOT,
              B_E3A = 4 * NSLOT, B_D1 = 5 * NSLOT, B_D2 = 6 * NSLOT, B_D3A = 7 * NSLOT,
              B_D3B = 8 * NSLOT, B_W = 9 * NSLOT, B_DRAIN = 9 * NSLOT + 1;

// relu(D alpha + beta) for 32 TMEM columns -> 32 e4m3 bytes at row `row`,
// columns [k0, k0 + 32) of a K-wide tile.
template <int K>
__device__ __forceinline__ void epi_e4m3_32(const float (&v)[32], const float* alpha,
                                            const float* beta, unsigned char* dst, int row, int k0) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    float t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) t[j] = fmaf(v[16 * c + j], alpha[16 * c + j], beta[16 * c + j]);
    uint4 w;
    w.x = pack_e4m3x4_relu(t[0], t[1], t[2], t[3]);
    w.y = pack_e4m3x4_relu(t[4], t[5], t[6], t[7]);
    w.z = pack_e4m3x4_relu(t[8], t[9], t[10], t[11]);
    w.w = pack_e4m3x4_relu(t[12], t[13], t[14], t[15]);
    *reinterpret_cast<uint4*>(dst + kmajor_off8(row, k0 + 16 * c, K)) = w;
  }
}

// relu(D) for 32 TMEM columns (scale and bias already in D) -> 32 e4m3
// bytes at row `row`, columns [k0, k0 + 32) of a K-wide tile.
template <int K>
__device__ __forceinline__ void epi_e4m3_relu_32(const float (&v)[32], unsigned char* dst, int row,
                                                 int k0) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const float* t = v + 16 * c;
    uint4 w;
    w.x = pack_e4m3x4_relu(t[0], t[1], t[2], t[3]);
    w.y = pack_e4m3x4_relu(t[4], t[5], t[6], t[7]);
    w.z = pack_e4m3x4_relu(t[8], t[9], t[10], t[11]);
    w.w = pack_e4m3x4_relu(t[12], t[13], t[14], t[15]);
    *reinterpret_cast<uint4*>(dst + kmajor_off8(row, k0 + 16 * c, K)) = w;
  }
}

// Masked max over the valid points of each object (thread = channel);
// columns [0, 64) are A's points, [64, 128) B's.  Whole valid 32-column
// chunks are loads with max reduction (tcgen05.ld.red).
__device__ __forceinline__ void pool8(uint32_t taddr, int cntA, int cntB, float* mA, float* mB) {
  float v[32];
  float a = -INFINITY, b = -INFINITY;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cnt = q < 2 ? cntA : cntB;
    const int q0 = 32 * (q & 1);
    if (q0 < cnt) {
      float m = -INFINITY;
      if (q0 + 32 <= cnt) {
        m = tmem_ldmax32(taddr + 32 * q);
      } else {
        tmem_ld32(taddr + 32 * q, v);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) m = fmaxf(m, (q0 + jj < cnt) ? v[jj] : -INFINITY);
      }
      if (q < 2) a = fmaxf(a, m);
      else b = fmaxf(b, m);
    }
  }
  *mA = a;
  *mB = b;
}

// Pooled feature k of pair p (rel = p - first pair of the launch): float32
// [P][512] when feat is given, and always e4m3 of v / s_k (the head's input
// scale) in the head's operand layout -- tiles of 128 pairs, each 8 K-chunks
// of 64 features, K-major (8 KB per chunk) -- for bulk copies into the head.
__device__ __forceinline__ void put_feat8(float* feat, unsigned char* ftile, int p, int rel, int k,
                                          float v, float inv_s) {
  if (feat) feat[(size_t)p * 512 + k] = v;
  unsigned char* t = ftile + (size_t)(rel >> 7) * (128 * 512) + (size_t)(k >> 6) * (128 * 64);
  t[kmajor_off8(rel & 127, k & 63, 64)] = (unsigned char)(pack_e4m3x4(v * inv_s, 0.f, 0.f, 0.f) & 0xffu);
}

// Tiles of two listed objects with non-empty crops, as in the BF16 encoder
// (object u in rows 0..63, v in 64..127; CTA b takes tiles b, b + G, ...).
__global__ void __launch_bounds__(F_THREADS, 1)
    encoder_fp8_kernel(const float4* __restrict__ xyz, PairRange rg,
                       const int* __restrict__ list, const int* __restrict__ list_n,
                       const int32_t* __restrict__ cnt,
                       const unsigned char* __restrict__ img, float* __restrict__ feat,
                       unsigned char* __restrict__ ftile, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  const int n_objs = min(list_n[rg.chunk], 2 * (hi - lo));
  const int* lst = list + 2 * (size_t)lo;
  const int n = (n_objs + 1) >> 1;  // tiles
  if ((int)blockIdx.x >= n) {  // no tile here: only this CTA's share of the zero features
    if (warp == ZERO_WARP && cnt) zero_empty_objects(cnt, ftile, lo, hi, lane, true);
    return;
  }
  const int my_pairs = (n - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles

  unsigned char* ctrl = smem + F_CTRL;
  const uint32_t bar0 = smem_u32(ctrl + C_BAR);
  auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + C_TMEM);
  volatile int* abort = reinterpret_cast<volatile int*>(ctrl + C_ABORT);
  int* s_cnt = reinterpret_cast<int*>(ctrl + C_CNT);

  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(BAR(B_FULLX + s), 1);
      mbar_init(BAR(B_XRDY + s), 128);
      mbar_init(BAR(B_H1RDY + s), 128);
      mbar_init(BAR(B_H2RDY + s), 128);
      mbar_init(BAR(B_E3A + s), 128);
      mbar_init(BAR(B_D1 + s), 1);
      mbar_init(BAR(B_D2 + s), 1);
      mbar_init(BAR(B_D3A + s), 1);
      mbar_init(BAR(B_D3B + s), 1);
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
  // (a1, c1 stay in the image for reference; layer 1 has them folded into W1)
  const float* a2 = reinterpret_cast<const float*>(smem + F_EP) + 128;
  const float* c2 = a2 + 128;
  const float* w3 = c2 + 128;
  const float* b3 = w3 + 256;
  const float* fin = b3 + 256;

  if (warp == MMA_WARP) {
    // MMA issuer warp: warp-uniform control flow, weight copies by lane 0,
    // MMAs by an elected lane
    const uint32_t sW1 = smem_u32(smem + F_W1), sW2 = smem_u32(smem + F_W2);
    const uint32_t sW3 = smem_u32(smem + F_W3);
    if (lane == 0) {
      mbar_expect_tx(BAR(B_W), F_IMG_BYTES);
      for (int off = 0; off < F_IMG_BYTES; off += 32768)
        bulk_g2s(smem_u32(smem + off), img + off, min(32768, F_IMG_BYTES - off), BAR(B_W));
    }
    bool ok = mbar_wait_warp(BAR(B_W), 0, abort, WAIT_CYCLES);
    tc_fence_after();
    const uint32_t id64 = idesc_bf16(128, 64), id128 = idesc_e4m3(128, 128);
    for (int r = 0; ok && NSLOT * r < my_pairs; ++r) {
      const uint32_t ph = r & 1;
      const int ns = min(NSLOT, my_pairs - NSLOT * r);
      // layers 1 and 2 in the order L1 0, L1 1, L1 2, L2 0, L1 3, L2 1, L2 2,
      // L2 3 (nibble t of kOrder: slot | layer << 2): slot 0's layer 2 goes
      // out while slot 3 is still building its X, instead of waiting behind it
      constexpr uint32_t kOrder = 0x76534210u;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = (int)((kOrder >> (4 * t)) & 0xfu), s = e & 3;
        if (!ok || s >= ns) continue;
        const uint32_t sO = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_OPD);
        if ((e >> 2) == 0) {
          if (!(ok = mbar_wait_warp(BAR(B_XRDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (elect_one()) {
            mma_bf16(tbase + s * SLOT_COLS, sdesc(sO, 128, 256), sdesc(sW1, 128, 256), id64, 0);
            mma_commit(BAR(B_D1 + s));
          }
        } else {
          if (!(ok = mbar_wait_warp(BAR(B_H1RDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (elect_one()) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
              mma_e4m3(tbase + s * SLOT_COLS, sdesc(sO + 256 * kk, 128, 512),
                       sdesc(sW2 + 256 * kk, 128, 512), id128, kk > 0);
            mma_commit(BAR(B_D2 + s));
          }
        }
        __syncwarp();
      }
      for (int s = 0; s < ns && ok; ++s) {
        if (!(ok = mbar_wait_warp(BAR(B_H2RDY + s), ph, abort, WAIT_CYCLES))) break;
        tc_fence_after();
        const uint32_t sH = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_OPD);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_e4m3(tbase + s * SLOT_COLS, sdesc(sW3 + 256 * kk, 128, 1024),
                     sdesc(sH + 256 * kk, 128, 1024), id128, kk > 0);
          mma_commit(BAR(B_D3A + s));
        }
        __syncwarp();
      }
      for (int s = 0; s < ns && ok; ++s) {
        if (!(ok = mbar_wait_warp(BAR(B_E3A + s), ph, abort, WAIT_CYCLES))) break;
        tc_fence_after();
        const uint32_t sH = smem_u32(smem + F_SLOT0 + s * F_SLOT_BYTES + FS_OPD);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_e4m3(tbase + s * SLOT_COLS, sdesc(sW3 + 16384 + 256 * kk, 128, 1024),
                     sdesc(sH + 256 * kk, 128, 1024), id128, kk > 0);
          mma_commit(BAR(B_D3B + s));
        }
        __syncwarp();
      }
    }
    if (__any_sync(0xffffffffu, *abort) && elect_one()) {
      mma_commit(BAR(B_DRAIN));
      mbar_wait(BAR(B_DRAIN), 0, WAIT_CYCLES);
    }
    __syncwarp();
  } else if (warp == ZERO_WARP) {
    // the empty objects' pooled features (exactly 0, e4m3) for the head
    if (cnt) zero_empty_objects(cnt, ftile, lo, hi, lane, true);
  } else {
    const int s = warp >> 2, row = tid & 127, wq = warp & 3;
    unsigned char* slot = smem + F_SLOT0 + s * F_SLOT_BYTES;
    unsigned char* opd = slot + FS_OPD;
    const uint32_t tslot = tbase + s * SLOT_COLS + ((uint32_t)(32 * wq) << 16);
    int* cnt_s = s_cnt + 4 * s;
    int* obj_s = reinterpret_cast<int*>(ctrl + C_OBJ) + 4 * s;  // [parity][u, v]
    int tu0 = -1, tv0 = -1, tu1 = -1, tv1 = -1;  // objects of the slot's tiles, by parity
    // crop rows of the slot's tile jn -> bf16 hi/lo X tile (over the previous
    // tile's H2, dead once its layer 3 has completed), crop counts, XRDY
    auto build_x = [&](int jn) {
      if (!mbar_wait_or_abort(BAR(B_FULLX + s), jn & 1, abort, WAIT_CYCLES)) return false;
      const int nu = obj_s[2 * (jn & 1)], nv = obj_s[2 * (jn & 1) + 1];
      if (jn & 1) tu1 = nu, tv1 = nv;
      else tu0 = nu, tv0 = nv;
      float4 q = reinterpret_cast<const float4*>(slot + FS_STG)[row];
      if (row >= KMAX && nv < 0) q = make_float4(0.f, 0.f, 0.f, 0.f);
      const unsigned m = __ballot_sync(0xffffffffu, q.w > 0.5f);
      if (lane == 0) cnt_s[wq] = __popc(m);
      const float fx = __bfloat162float(__float2bfloat16_rn(q.x));
      const float fy = __bfloat162float(__float2bfloat16_rn(q.y));
      const float fz = __bfloat162float(__float2bfloat16_rn(q.z));
      uint4 c0, cc1;
      c0.x = pack_bf16(fx, fy);
      c0.y = pack_bf16(fz, q.x - fx);
      c0.z = pack_bf16(q.y - fy, q.z - fz);
      c0.w = pack_bf16(fx, fy);
      cc1.x = pack_bf16(fz, 1.f);  // K columns 9, 10: ones against b1 / s1 (hi, lo)
      cc1.y = pack_bf16(1.f, 0.f);
      cc1.z = cc1.w = 0u;
      *reinterpret_cast<uint4*>(opd + kmajor_off(row, 0, 16)) = c0;
      *reinterpret_cast<uint4*>(opd + kmajor_off(row, 8, 16)) = cc1;
      fence_async_smem();
      return true;
    };
    // X of the pair is in place and this thread's TMEM reads of the slot are
    // done: the slot's layer 1 may run
    auto x_ready = [&]() {
      tc_fence_before();
      mbar_arrive(BAR(B_XRDY + s));
    };
    // the slot's crop rows by bulk copy, issued by one lane of the
    // warpgroup: pair 0 at the start, pair j + 1 once layer 1 of pair j has
    // completed (every read of the staging rows is done by then)
    const bool copier = wq == 0 && lane == 0;
    int n_loads = 0;
    auto load_rows = [&](int jn) {
      const int tg = blockIdx.x + (NSLOT * jn + s) * gridDim.x;
      const int u = lst[2 * tg], v = 2 * tg + 1 < n_objs ? lst[2 * tg + 1] : -1;
      obj_s[2 * (jn & 1)] = u;
      obj_s[2 * (jn & 1) + 1] = v;
      mbar_expect_tx(BAR(B_FULLX + s), (v >= 0 ? 2 : 1) * KMAX * 16);
      bulk_g2s(smem_u32(slot + FS_STG), xyz + (size_t)u * KMAX, KMAX * 16, BAR(B_FULLX + s));
      if (v >= 0)
        bulk_g2s(smem_u32(slot + FS_STG + KMAX * 16), xyz + (size_t)v * KMAX, KMAX * 16,
                 BAR(B_FULLX + s));
      ++n_loads;
    };
    if (copier && s < my_pairs) load_rows(0);
    bool ok = mbar_wait_or_abort(BAR(B_W), 0, abort, WAIT_CYCLES);
    if (ok && s < my_pairs) {
      ok = build_x(0);
      if (ok) x_ready();
    }
    for (int j = 0; ok; ++j) {
      const int i = NSLOT * j + s;
      if (i >= my_pairs) break;
      const uint32_t ph = j & 1;
      // layer 1 epilogue -> e4m3 H1 (scale and bias already in D1), over X
      if (!(ok = mbar_wait_or_abort(BAR(B_D1 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      if (copier && i + NSLOT < my_pairs) load_rows(j + 1);
      {
        float v[32];
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          tmem_ld32(tslot + 32 * h, v);
          epi_e4m3_relu_32<64>(v, opd, row, 32 * h);
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H1RDY + s));
      // layer 2 epilogue -> e4m3 H2, over H1
      if (!(ok = mbar_wait_or_abort(BAR(B_D2 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      {
        float v[32];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          tmem_ld32(tslot + 32 * h, v);
          epi_e4m3_32<128>(v, a2 + 32 * h, c2 + 32 * h, opd, row, 32 * h);
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H2RDY + s));
      // layer 3 epilogues: max over valid points, then * w3 + b3, relu
      if (!(ok = mbar_wait_or_abort(BAR(B_D3A + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      asm volatile("bar.sync %0, 128;" ::"r"(1 + s) : "memory");  // counts of other warps
      const int cntA = cnt_s[0] + cnt_s[1], cntB = cnt_s[2] + cnt_s[3];
      float mA, mB;
      pool8(tslot, cntA, cntB, &mA, &mB);
      tc_fence_before();
      mbar_arrive(BAR(B_E3A + s));
      const int u = ph ? tu1 : tu0, v = ph ? tv1 : tv0;
      const int pu = u >> 1, ku = (u & 1) * 256, pv = v >> 1, kv = (v & 1) * 256;
      {
        const float sc = w3[row], bias = b3[row], fi = fin[row];
        put_feat8(feat, ftile, pu, pu - lo, ku + row,
                  cntA > 0 ? fmaxf(fmaf(mA, sc, bias), 0.f) : 0.f, fi);
        if (v >= 0)
          put_feat8(feat, ftile, pv, pv - lo, kv + row,
                    cntB > 0 ? fmaxf(fmaf(mB, sc, bias), 0.f) : 0.f, fi);
      }
      if (!(ok = mbar_wait_or_abort(BAR(B_D3B + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      // the next pair's X (H2 is dead once layer 3 has completed), the second
      // pooling, then XRDY (the slot's TMEM columns are free only after it)
      const bool nx = i + NSLOT < my_pairs;
      if (nx) ok = build_x(j + 1);
      pool8(tslot, cntA, cntB, &mA, &mB);
      if (nx && ok) x_ready();
      {
        const float sc = w3[128 + row], bias = b3[128 + row], fi = fin[128 + row];
        put_feat8(feat, ftile, pu, pu - lo, ku + 128 + row,
                  cntA > 0 ? fmaxf(fmaf(mA, sc, bias), 0.f) : 0.f, fi);
        if (v >= 0)
          put_feat8(feat, ftile, pv, pv - lo, kv + 128 + row,
                    cntB > 0 ? fmaxf(fmaf(mB, sc, bias), 0.f) : 0.f, fi);
      }
      tc_fence_before();
    }
    // on an abort: wait (bounded) for this lane's copy still in flight
    if (copier && n_loads > 0 && *abort) mbar_wait(BAR(B_FULLX + s), (n_loads - 1) & 1, WAIT_CYCLES);
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
constexpr int G_W3 = 0;                  // Wh3' [16 x 256] e4m3 (rows 8.. zero) 4 KB
constexpr int G_EP = G_W3 + 16 * 256;    // f_inv [256], a4 c4 [256], a5 c5 [256], w6 hb3 [16]
constexpr int G_RES_BYTES = G_EP + (5 * 256 + 2 * 16) * 4;
static_assert(G_RES_BYTES % 128 == 0, "fp8 head resident image");
constexpr int GK = 64;                    // K of one streamed chunk (bytes per row)
constexpr int G_CHUNK = 256 * GK;        // one B chunk [256 x 64] e4m3, 16 KB
constexpr int G_L1C = 512 / GK, G_NCH = G_L1C + 256 / GK;  // chunks per tile: 8 + 4
constexpr int G_IMG_W1 = G_RES_BYTES;    // 8 chunks
constexpr int G_IMG_W2 = G_IMG_W1 + G_L1C * G_CHUNK;  // 4 chunks
constexpr int G_IMG_BYTES = G_IMG_W2 + (G_NCH - G_L1C) * G_CHUNK;
constexpr int G_ACHUNK = 128 * GK;                        // one A (feature) chunk, e4m3, 8 KB
constexpr int G_NST = 6;                                   // operand stages
constexpr int G_A0 = (G_RES_BYTES + 1023) / 1024 * 1024;  // A stages [128 x 64] e4m3
constexpr int G_B0 = G_A0 + G_NST * G_ACHUNK;              // B stages [256 x 64] e4m3
constexpr int G_G = G_B0 + G_NST * G_CHUNK;                // G [128 x 256] e4m3, 32 KB
constexpr int G_CTRL = G_G + 128 * 256;                    // mbarriers, TMEM address, abort
constexpr int G_SMEM = G_CTRL + 256;
constexpr int G_THREADS = 320;  // 8 epilogue warps, the copy warp, the MMA warp
constexpr int G_COPY = 256, G_MMA_WARP = 9;
static_assert(G_RES_BYTES % 16 == 0 && G_IMG_W1 % 16 == 0, "bulk copies need 16-byte chunks");
static_assert(G_SMEM <= 227 * 1024, "fp8 head shared memory");

// Half of a 256-wide layer: 128 columns from taddr -> e4m3 G columns
// [k0, k0 + 128).
__device__ __forceinline__ void head_epi_fp8(uint32_t taddr, const float* alpha, const float* beta,
                                             unsigned char* G, int row, int k0) {
  float v[32];
#pragma unroll 2
  for (int h = 0; h < 4; ++h) {
    tmem_ld32(taddr + 32 * h, v);
    epi_e4m3_32<256>(v, alpha + 32 * h, beta + 32 * h, G, row, k0 + 32 * h);
  }
}

// Same schedule as the BF16 head (a copy thread in warp 8 streaming operand
// chunks through G_NST stages by bulk copy, an MMA thread in warp 9, layer 3
// of tile t deferred behind the layer-1 MMAs of tile t + 1; epilogue warps
// 0-7) over 12 K-chunks of 64 per tile: 8 of W_h1 against the e4m3 features
// the encoder wrote in operand layout, 4 of W_h2 against G.  The layer-1
// epilogue fills G in four 64-column chunks (mbarriers GC0-GC3); layer-2 chunk
// j starts once G chunk j is ready.
__global__ void __launch_bounds__(G_THREADS, 1)
    head_fp8_kernel(const unsigned char* __restrict__ ftile, PairRange rg,
                    const unsigned char* __restrict__ img, PairInputs in, int have_in,
                    const float4* __restrict__ centre, float* __restrict__ out,
                    float* __restrict__ y_raw, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  int lo, n;
  range_bounds(rg, &lo, &n);  // this launch's pairs: [lo, n)
  const int n_tiles = (n - lo + HT - 1) / HT;
  if ((int)blockIdx.x >= n_tiles) return;
  const int my_tiles = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  // mbarriers: [0, 6) operands of stage s landed; [6, 12) MMAs of stage s
  // done; 12 layer 3 done; 13 EPI (two per tile: G holds layer 2; outputs
  // left TMEM); 14 resident image; 15 drain; 16 / 17 layer 1 / layer 2 of the
  // tile done; [18, 22) G chunk k holds layer 1
  const uint32_t bar0 = smem_u32(smem + G_CTRL);
  const uint32_t B_FULL = bar0, B_DONE = bar0 + 48;
  const uint32_t B_L3 = bar0 + 96, B_EPI = bar0 + 104, B_RES = bar0 + 112, B_DRAIN = bar0 + 120;
  const uint32_t B_L1D = bar0 + 128, B_L2D = bar0 + 136, B_GC = bar0 + 144;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G_CTRL + 192);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G_CTRL + 196);
  int* s_issued = reinterpret_cast<int*>(smem + G_CTRL + 200);
  if (tid == 0) {
    for (int i = 0; i < 22; ++i) mbar_init(bar0 + 8 * i, (i == 13 || i >= 18) ? 256 : 1);
    *abort = 0;
    *s_issued = 0;
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
  // epilogue warps w and w + 4 share TMEM lane quarter w % 4 and split the
  // columns between them
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  const int row = tid & 127, half = (tid >> 7) & 1;
  const float* finv = reinterpret_cast<const float*>(smem + G_EP);
  const float* a4 = finv + 256;
  const float* c4 = a4 + 256;
  const float* a5 = c4 + 256;
  const float* c5 = a5 + 256;
  const float* w6 = c5 + 256;
  const float* hb3 = w6 + 16;
  unsigned char* G = smem + G_G;
  const uint32_t sG = smem_u32(G), sW3 = smem_u32(smem + G_W3);
  const uint32_t id256 = idesc_e4m3(128, 256), id16 = idesc_e4m3(128, 16);
  const int n_chunks = G_NCH * my_tiles;  // this CTA's chunk stream
  bool ok = true;

  if (tid == G_COPY) {
    mbar_expect_tx(B_RES, G_RES_BYTES);
    bulk_g2s(smem_u32(smem), img, G_RES_BYTES, B_RES);
    for (int g = 0; g < n_chunks; ++g) {
      const int st = g % G_NST, c = g % G_NCH;
      if (g >= G_NST &&
          !(ok = mbar_wait_or_abort(B_DONE + 8 * st, (g / G_NST - 1) & 1, abort, WAIT_CYCLES)))
        break;
      const int tile = (int)blockIdx.x + (g / G_NCH) * (int)gridDim.x;
      const uint32_t bf = B_FULL + 8 * st;
      if (c < G_L1C) {
        mbar_expect_tx(bf, G_ACHUNK + G_CHUNK);
        bulk_g2s(smem_u32(smem + G_A0 + st * G_ACHUNK),
                 ftile + (size_t)tile * (128 * 512) + (size_t)c * G_ACHUNK, G_ACHUNK, bf);
        bulk_g2s(smem_u32(smem + G_B0 + st * G_CHUNK), img + G_IMG_W1 + (size_t)c * G_CHUNK,
                 G_CHUNK, bf);
      } else {
        mbar_expect_tx(bf, G_CHUNK);
        bulk_g2s(smem_u32(smem + G_B0 + st * G_CHUNK),
                 img + G_IMG_W2 + (size_t)(c - G_L1C) * G_CHUNK, G_CHUNK, bf);
      }
      *s_issued = g + 1;
    }
    if (!ok) *abort = 1;
  } else if (warp == G_MMA_WARP) {
    // layer 3: D3[128 x 16] = G . Wh3'^T (rows 8..15 zero), in the layer-2 columns
    auto layer3 = [&]() {
      tc_fence_after();
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma_e4m3(tbase + 256, sdesc(sG + 256 * kk, 128, 2048), sdesc(sW3 + 256 * kk, 128, 2048),
                   id16, kk > 0);
        mma_commit(B_L3);
      }
      __syncwarp();
    };
    ok = mbar_wait_warp(B_RES, 0, abort, WAIT_CYCLES);
    int l3 = -1;  // tile whose layer 3 waits for its layer-2 epilogue
    // two chunks (four MMAs) per step, so that the per-step waits cost less
    // than the tensor work they gate
    for (int g = 0; g < n_chunks && ok; g += 2) {
      const int st0 = g % G_NST, st1 = (g + 1) % G_NST, c = g % G_NCH, t = g / G_NCH;
      if (l3 >= 0) {
        // EPI phase 2 l3: G holds layer 2 of tile l3.  Layer 2 of the next
        // tile needs its outputs out of TMEM, so by then it is waited for.
        if (c == G_L1C) {
          ok = mbar_wait_warp(B_EPI, (2 * l3) & 1, abort, WAIT_CYCLES);
          if (!ok) break;
        }
        if (c == G_L1C || __all_sync(0xffffffffu, mbar_test_wait(B_EPI, (2 * l3) & 1))) {
          layer3();
          l3 = -1;
        }
      }
      const bool l1 = c < G_L1C;
      const int j = c - G_L1C;  // layer-2 chunk (even)
      if (!l1) {
        // the previous tile's outputs have left the layer-2 columns (EPI
        // phase 2 t - 1), and G chunks j and j + 1 (64 columns each) hold
        // layer 1
        if (j == 0 && t > 0) ok = mbar_wait_warp(B_EPI, (2 * t - 1) & 1, abort, WAIT_CYCLES);
        ok = ok && mbar_wait_warp(B_GC + 8 * j, t & 1, abort, WAIT_CYCLES);
        ok = ok && mbar_wait_warp(B_GC + 8 * (j + 1), t & 1, abort, WAIT_CYCLES);
      }
      ok = ok && mbar_wait_warp(B_FULL + 8 * st0, (g / G_NST) & 1, abort, WAIT_CYCLES);
      ok = ok && mbar_wait_warp(B_FULL + 8 * st1, ((g + 1) / G_NST) & 1, abort, WAIT_CYCLES);
      if (!ok) break;
      tc_fence_after();
      // descriptors from warp-uniform values; one elected lane issues
      const uint32_t sB0 = smem_u32(smem + G_B0 + st0 * G_CHUNK);
      const uint32_t sB1 = smem_u32(smem + G_B0 + st1 * G_CHUNK);
      const uint32_t sA0 = l1 ? smem_u32(smem + G_A0 + st0 * G_ACHUNK) : sG + 512 * j;
      const uint32_t sA1 = l1 ? smem_u32(smem + G_A0 + st1 * G_ACHUNK) : sG + 512 * (j + 1);
      const uint32_t dcol = l1 ? 0u : 256u, sbo = l1 ? 512u : 2048u;
      const uint32_t acc0 = (l1 ? c : j) > 0 ? 1u : 0u;
      if (elect_one()) {
        mma_e4m3(tbase + dcol, sdesc(sA0, 128, sbo), sdesc(sB0, 128, 512), id256, acc0);
        mma_e4m3(tbase + dcol, sdesc(sA0 + 256, 128, sbo), sdesc(sB0 + 256, 128, 512), id256, 1u);
        mma_commit(B_DONE + 8 * st0);
        mma_e4m3(tbase + dcol, sdesc(sA1, 128, sbo), sdesc(sB1, 128, 512), id256, 1u);
        mma_e4m3(tbase + dcol, sdesc(sA1 + 256, 128, sbo), sdesc(sB1 + 256, 128, 512), id256, 1u);
        mma_commit(B_DONE + 8 * st1);
        if (c + 1 == G_L1C - 1) mma_commit(B_L1D);
        if (c + 1 == G_NCH - 1) mma_commit(B_L2D);
      }
      __syncwarp();
      if (c + 1 == G_NCH - 1) l3 = t;
    }
    if (ok && l3 >= 0) {
      ok = mbar_wait_warp(B_EPI, (2 * l3) & 1, abort, WAIT_CYCLES);
      if (ok) layer3();
    }
    if (!ok) *abort = 1;
  }
  if (tid < 256) ok = mbar_wait_or_abort(B_RES, 0, abort, WAIT_CYCLES);
  for (int t = 0; tid < 256 && t < my_tiles && ok; ++t) {
    const int pr = lo + ((int)blockIdx.x + t * (int)gridDim.x) * HT + row;
    const bool row_ok = pr < n;
    bool geo = false;
    float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
    float pose[7];
    if (half == 0 && row_ok && out) {
      const int a = have_in ? in.pairs[2 * pr] : -1;
      cc = centre[pr];
      geo = a >= 0 && a < in.n_obj && !isnan(cc.x);
#pragma unroll
      for (int i = 0; i < 7; ++i) pose[i] = geo ? in.poses[7 * (size_t)a + i] : 0.f;
    }
    ok = mbar_wait_or_abort(B_L1D, t & 1, abort, WAIT_CYCLES);
    if (!ok) break;
    tc_fence_after();
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const int col = 64 * k + 32 * half;
      float v[32];
      tmem_ld32(tbase + lane_off + col, v);
      epi_e4m3_32<256>(v, a4 + col, c4 + col, G, row, col);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(B_GC + 8 * k);
    }
    ok = mbar_wait_or_abort(B_L2D, t & 1, abort, WAIT_CYCLES);
    if (!ok) break;
    tc_fence_after();
    head_epi_fp8(tbase + lane_off + 256 + 128 * half, a5 + 128 * half, c5 + 128 * half, G, row,
                 128 * half);
    fence_async_smem();
    tc_fence_before();
    mbar_arrive(B_EPI);
    ok = mbar_wait_or_abort(B_L3, t & 1, abort, WAIT_CYCLES);
    if (!ok) break;
    tc_fence_after();
    if (half == 0) {
      float v[16];
      tmem_ld16(tbase + lane_off + 256, v);  // layer 3 sits in the layer-2 columns
      if (row_ok) {
        float y[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) y[o] = fmaf(v[o], w6[o], hb3[o]);
        if (y_raw) {
#pragma unroll
          for (int o = 0; o < 8; ++o) y_raw[(size_t)pr * 8 + o] = y[o];
        }
        if (out) {
          float o8[8];
          if (geo) {
            epilogue_world(y, pose, cc, o8);
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
    mbar_arrive(B_EPI);
  }
  __syncthreads();
  if (*abort) {
    // drain (bounded): the MMA thread waits for its MMAs, the copy thread for
    // the copies it issued
    if (tid == 0) atomicOr(err, 2);
    if (warp == G_MMA_WARP && (tid & 31) == 0) {
      mma_commit(B_DRAIN);
      mbar_wait(B_DRAIN, 0, WAIT_CYCLES);
    }
    if (tid == G_COPY) {
      const int issued = *s_issued;
      for (int g = issued - G_NST; g < issued; ++g)
        if (g >= 0) mbar_wait(B_FULL + 8 * (g % G_NST), (g / G_NST) & 1, WAIT_CYCLES);
    }
  }
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

// Scales of one folded layer: for W [out][in] with input channel scales
// s_in[in], returns the folded weights W' = W s_in (float32 [out][in]), the
// per-output-channel weight scales w = max|W'| / 448 and their inverses, and
// the output bound B_out[c] = max(0, sum_k |W[c][k]| B_in[k] + b[c]).
struct Folded {
  std::vector<float> Wf, inv;
  std::vector<double> w, bound;
};

Folded fold(const float* W, const float* b, int out, int in, const std::vector<double>& s_in,
            const std::vector<double>& B_in) {
  Folded f;
  f.Wf.resize((size_t)out * in);
  f.inv.resize(out);
  f.w.resize(out);
  f.bound.resize(out);
  for (int c = 0; c < out; ++c) {
    double amax = 0.0, acc = b[c];
    for (int k = 0; k < in; ++k) {
      const double wf = (double)W[(size_t)c * in + k] * s_in[k % s_in.size()];
      f.Wf[(size_t)c * in + k] = (float)wf;
      amax = std::max(amax, std::fabs(wf));
      acc += std::fabs((double)W[(size_t)c * in + k]) * B_in[k % B_in.size()];
    }
    f.w[c] = amax > 0 ? amax / 448.0 : 1.0;
    f.inv[c] = (float)(1.0 / f.w[c]);
    f.bound[c] = std::max(0.0, acc);
  }
  return f;
}

// activation scale of a channel with bound B: 1.1 B / 448 (1 for B == 0)
std::vector<double> act_scale(const std::vector<double>& B) {
  std::vector<double> s(B.size());
  for (size_t i = 0; i < B.size(); ++i) s[i] = B[i] > 0 ? 1.1 * B[i] / 448.0 : 1.0;
  return s;
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
  const float* P = params.data();
  // layer-1 output bound from the crop ball |x| <= r
  std::vector<double> B1(64);
  for (int c = 0; c < 64; ++c) {
    const float* w = P + off[0] + 3 * c;
    const double nrm = std::sqrt((double)w[0] * w[0] + (double)w[1] * w[1] + (double)w[2] * w[2]);
    B1[c] = std::max(0.0, (double)h->radius * nrm + P[offb[0] + c]);
  }
  const std::vector<double> s1 = act_scale(B1);
  const Folded L2 = fold(P + off[1], P + offb[1], 128, 64, s1, B1);
  const std::vector<double> s2 = act_scale(L2.bound);
  const Folded L3 = fold(P + off[2], P + offb[2], 256, 128, s2, L2.bound);
  const std::vector<double> s3 = act_scale(L3.bound);
  const Folded H1 = fold(P + off[3], P + offb[3], 256, 512, s3, L3.bound);
  const std::vector<double> s4 = act_scale(H1.bound);
  const Folded H2 = fold(P + off[4], P + offb[4], 256, 256, s4, H1.bound);
  const std::vector<double> s5 = act_scale(H2.bound);
  const Folded H3 = fold(P + off[5], P + offb[5], 8, 256, s5, H2.bound);

  const size_t enc_bytes = (F_IMG_BYTES + 255) / 256 * 256;
  const size_t total = enc_bytes + G_IMG_BYTES;
  std::vector<unsigned char> img(total, 0);
  unsigned char* e = img.data();
  // layer 1 B operand, scaled by 1 / s1: row c = [W_hi(3), W_hi(3), W_lo(3),
  // (b1 / s1)_hi, (b1 / s1)_lo, 0 x 5]
  for (int c = 0; c < 64; ++c)
    for (int k = 0; k < 16; ++k) {
      float val = 0.f;
      if (k < 9 || k == 9 || k == 10) {
        const float w = k < 9 ? (float)(P[off[0] + (size_t)c * 3 + (k % 3)] / s1[c])
                              : (float)(P[offb[0] + c] / s1[c]);
        const float hi = bf16_value_h(bf16_bits_h(w));
        val = (k < 6 || k == 9) ? hi : w - hi;
      }
      const uint16_t b = bf16_bits_h(val);
      std::memcpy(e + F_W1 + kmajor_off(c, k, 16), &b, 2);
    }
  float* ep = reinterpret_cast<float*>(e + F_EP);
  for (int c = 0; c < 64; ++c) {
    ep[c] = (float)(1.0 / s1[c]);                     // a1
    ep[64 + c] = (float)(P[offb[0] + c] / s1[c]);     // c1
  }
  for (int c = 0; c < 128; ++c) {
    ep[128 + c] = (float)(L2.w[c] / s2[c]);           // a2
    ep[256 + c] = (float)(P[offb[1] + c] / s2[c]);    // c2
  }
  for (int c = 0; c < 256; ++c) {
    ep[384 + c] = (float)L3.w[c];                     // w3
    ep[640 + c] = P[offb[2] + c];                     // b3
    ep[896 + c] = (float)(1.0 / s3[c]);               // feature inverse scale (head input)
  }
  unsigned char* hd = img.data() + enc_bytes;
  float* hp = reinterpret_cast<float*>(hd + G_EP);
  for (int c = 0; c < 256; ++c) {
    hp[c] = (float)(1.0 / s3[c]);                     // feature inverse scale
    hp[256 + c] = (float)(H1.w[c] / s4[c]);           // a4
    hp[512 + c] = (float)(P[offb[3] + c] / s4[c]);    // c4
    hp[768 + c] = (float)(H2.w[c] / s5[c]);           // a5
    hp[1024 + c] = (float)(P[offb[4] + c] / s5[c]);   // c5
  }
  for (int c = 0; c < 8; ++c) {
    hp[1280 + c] = (float)H3.w[c];                    // w6
    hp[1296 + c] = P[offb[5] + c];                    // hb3
  }
  // folded weights and their inverse scales, quantised on the GPU
  std::vector<float> fw;
  auto put = [&](const Folded& f) {
    const size_t at = fw.size();
    fw.insert(fw.end(), f.Wf.begin(), f.Wf.end());
    fw.insert(fw.end(), f.inv.begin(), f.inv.end());
    return at;
  };
  const size_t o2 = put(L2), o3 = put(L3), o4 = put(H1), o5 = put(H2), o6 = put(H3);
  float* d_fw = nullptr;
  bool ok = cudaMalloc(&h->d_wf8, total) == cudaSuccess &&
            cudaMemcpy(h->d_wf8, img.data(), total, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMalloc(&d_fw, fw.size() * 4) == cudaSuccess &&
            cudaMemcpy(d_fw, fw.data(), fw.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    unsigned char* de = static_cast<unsigned char*>(h->d_wf8);
    unsigned char* dh = de + enc_bytes;
    quant_e4m3_kernel<<<128, 128>>>(d_fw + o2, d_fw + o2 + 128 * 64, 128, 64, 64, de + F_W2);
    quant_e4m3_kernel<<<256, 128>>>(d_fw + o3, d_fw + o3 + 256 * 128, 256, 128, 128, de + F_W3);
    quant_e4m3_kernel<<<256, 128>>>(d_fw + o4, d_fw + o4 + 256 * 512, 256, 512, GK, dh + G_IMG_W1);
    quant_e4m3_kernel<<<256, 128>>>(d_fw + o5, d_fw + o5 + 256 * 256, 256, 256, GK, dh + G_IMG_W2);
    quant_e4m3_kernel<<<8, 128>>>(d_fw + o6, d_fw + o6 + 8 * 256, 8, 256, 256, dh + G_W3);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    h->wf8_enc = de;
    h->wf8_head = dh;
  }
  cudaFree(d_fw);
  if (!ok) {
    cudaGetLastError();
    set_error("cannot build the e4m3 parameter images");
    return LOCC_ERR_OOM;
  }
  return LOCC_OK;
}

cudaError_t prepare_fp8_kernels() {
  cudaError_t e = cudaFuncSetAttribute(encoder_fp8_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(head_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  return e;
}

int run_network_fp8(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                    const float4* centre, float* out, float* y_raw, float* feat_out,
                    cudaStream_t stream, cudaEvent_t mid, int list_mode) {
  const int n_pairs = (rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1;  // pairs of one chunk, at most
  unsigned char* ftile = static_cast<unsigned char*>(h->d_feat_tc);
  if (list_mode != LIST_FROM_CROP &&
      launch_enc_list(h, xyz, rg, feat_out, list_mode == LIST_AND_COUNTS_FROM_ROWS, nullptr, 1,
                      stream) != cudaSuccess) {
    set_error("enc_list_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  encoder_fp8_kernel<<<std::min(n_pairs, h->n_sm), F_THREADS, F_SMEM, stream>>>(
      xyz, rg, h->d_list, h->d_list_n, h->d_cnt, h->wf8_enc, feat_out, ftile, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("encoder_fp8_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  if (mid && cudaEventRecord(mid, stream) != cudaSuccess) return LOCC_ERR_CUDA;
  PairInputs pin{};
  if (in) pin = *in;
  head_fp8_kernel<<<std::min((n_pairs + HT - 1) / HT, h->n_sm), G_THREADS, G_SMEM, stream>>>(
      ftile, rg, h->wf8_head, pin, in != nullptr, centre, out, y_raw, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("head_fp8_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

}  // namespace locc

// Tensor-core crop network (LOCC_BF16): tcgen05.mma with bf16 operands in
// shared memory and float32 accumulators in TMEM.
//
// Paper: Sec. III and appendix -- point-wise MLP encoder, pooling per object,
// MLP head, ReLU everywhere.  Same network as net_fp32.cu: encoder
// 3 -> 64 -> 128 -> 256, max-pool over the valid crop points of each object,
// head 512 -> 256 -> 256 -> 8, world-frame epilogue.
//
// encoder_tc_kernel (persistent, one CTA of 544 threads per SM, warp
// specialised, NSLOT = 4 pairs in flight per CTA):
//   * warp 16 copies the bf16 weight images (90 KB) into shared memory once
//     (cp.async.bulk) and issues every tcgen05.mma (one elected lane);
//     warps 4s..4s+3 are the epilogue warpgroup of slot s (one thread per
//     TMEM lane / crop row), and one of its lanes streams the 128 crop rows
//     of the slot's pairs into its staging buffer (bulk copies on an
//     mbarrier);
//   * each slot owns 128 TMEM columns and one 32 KB shared operand region that
//     holds X (layer-1 A operand), then H1, then H2 as the pair moves through
//     the layers, so four pairs overlap: while one slot's epilogue converts a
//     layer's accumulators, the tensor pipe works on the other slots;
//   * the 128 crop rows of a pair (64 of A, 64 of B) form the M = 128 tile;
//   * layer 1 packs K = 16: coordinates and weights are split into bf16 hi/lo
//     parts, x.W ~ x_hi W_hi + x_lo W_hi + x_hi W_lo (9 of the 16 columns);
//   * layers 1 and 2: D[128 x N] in TMEM, thread r owns row r (point r); the
//     MMAs accumulate the bias as well, the epilogue applies ReLU and writes
//     the bf16 row as the next layer's A operand;
//   * layer 3 is computed transposed, D^T = W3 . H2^T (M = 128 channels per
//     half, N = 128 points) in two halves that reuse the slot's 128 columns:
//     thread r owns channel r, so the max-pool over the valid points of each
//     object is a reduction over TMEM columns (tcgen05.ld.red max); the
//     second half is issued once the first has been pooled.
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

#include "enc_tc.cuh"
#include "handle.cuh"

namespace locc {
namespace {

using namespace tc;

// ----------------------------------------------------------------- encoder
// NSLOT pair slots.  Each slot: raw crop rows (f32, 2 KB) and one 32 KB
// operand region that holds, in turn, the X tile (4 KB), H1 (16 KB) and H2
// (32 KB): each is dead once the MMA that reads it has completed, which the
// epilogue that writes the next one has already waited for.  The operand
// regions of all slots are contiguous, so the H2 tiles of slots s and s + 1
// form one [256 points x 128] operand: layer 3 of a slot pair is one N = 256
// MMA chain (W3 read once for two pairs).
constexpr int NSLOT = 4;
constexpr int E_STG0 = (E_IMG_BYTES + 1023) / 1024 * 1024;  // [NSLOT][128] float4
constexpr int E_OPD0 = E_STG0 + NSLOT * ROWS * 16;           // [NSLOT][128 x 128] bf16
constexpr int STG_BYTES = ROWS * 16, OPD_BYTES = 128 * 128 * 2;
constexpr int E_CTRL = E_OPD0 + NSLOT * OPD_BYTES;
static_assert(E_OPD0 % 1024 == 0, "operand regions must stay 1 KB aligned");
// control block: mbarriers (8 B each), tmem slot, abort flag, counts [slot][4 warps]
constexpr int NBAR = 9 * NSLOT + 2;
constexpr int C_BAR = 0, C_TMEM = 8 * NBAR, C_ABORT = C_TMEM + 4, C_CNT = C_ABORT + 4;
constexpr int C_OBJ = C_CNT + 16 * NSLOT;  // [slot][tile parity][u, v] object ids
constexpr int E_SMEM = E_CTRL + C_OBJ + 16 * NSLOT;
static_assert(E_SMEM <= 227 * 1024, "encoder shared memory");
constexpr int E_THREADS = 32 * (4 * NSLOT + 2);  // 4 epilogue warps per slot + the MMA/TMA warp
constexpr int MMA_WARP = 4 * NSLOT;
// zeroes the pooled features of the empty objects (zero_empty_objects)
constexpr int ZERO_WARP = 4 * NSLOT + 1;
constexpr int SLOT_COLS = 512 / NSLOT;  // TMEM columns per slot: D1 [0,64), D2 / D3a / D3b [0,128)

// barrier indices (per slot s: index + s)
constexpr int B_FULLX = 0, B_XRDY = NSLOT, B_H1RDY = 2 * NSLOT, B_H2RDY = 3 * NSLOT,
              B_E3A = 4 * NSLOT, B_D1 = 5 * NSLOT, B_D2 = 6 * NSLOT, B_D3A = 7 * NSLOT,
              B_D3B = 8 * NSLOT, B_W = 9 * NSLOT, B_DRAIN = 9 * NSLOT + 1;

// ------------------------------------------------------------- object list
// The tensor-core encoders work on the objects whose crop is not empty, two
// objects (2 x 64 crop rows) per M = 128 tile.  An empty crop pools to
// exactly 0 (the max-pool runs over no point and ReLU outputs are >= 0), so
// those objects need no MMA; their pooled features (zeros) are written by the
// crop kernel, or here (ftile).  The crop kernel lists the objects as it goes;
// for crops given by the caller (or global crops) this kernel lists the
// objects of the launch's pairs [lo, hi) with a valid row 0 (the valid
// points of an object come first in its 64 rows) into list[2 lo ..] (object
// id 2 p + side, in no particular order: each object's features depend on its
// own rows only), counted in list_n[chunk], which the caller has zeroed.
// cnt_out (nullable): 1 / 0 per object (non-empty or not); feat (nullable):
// float32 zero features of the empty objects; ftile (nullable): their zero
// features in the head's operand tiles (bf16 hi / lo, or e4m3), one warp per
// empty object (zero_feat_warp).
__global__ void __launch_bounds__(256)
    enc_list_kernel(const float4* __restrict__ xyz, PairRange rg, int* __restrict__ list,
                    int* __restrict__ list_n, int32_t* __restrict__ cnt_out,
                    float* __restrict__ feat, unsigned char* __restrict__ ftile, int e4m3) {
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  const int n_obj = 2 * (hi - lo), lane = threadIdx.x & 31;
  int* lst = list + 2 * (size_t)lo;
  for (int base = blockIdx.x * blockDim.x; base < n_obj; base += gridDim.x * blockDim.x) {
    const int i = base + (int)threadIdx.x;
    bool live = false;
    if (i < n_obj) live = xyz[(size_t)(2 * lo + i) * KMAX].w > 0.5f;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    int b0 = 0;
    if (lane == 0 && m) b0 = atomicAdd(list_n + rg.chunk, __popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (live) lst[b0 + __popc(m & ((1u << lane) - 1u))] = 2 * lo + i;
    if (i < n_obj && cnt_out) cnt_out[2 * lo + i] = live ? 1 : 0;
    if (ftile) {
      unsigned em = __ballot_sync(0xffffffffu, i < n_obj && !live);
      while (em) {
        const int j = base + (int)(threadIdx.x & ~31u) + __ffs(em) - 1;
        em &= em - 1;
        zero_feat_warp(ftile, j >> 1, j & 1, lane, e4m3 != 0);
      }
    }
    if (i < n_obj && !live && feat) {
      float4* f = reinterpret_cast<float4*>(feat + (size_t)(lo + (i >> 1)) * 512 + (i & 1) * 256);
#pragma unroll 4
      for (int k = 0; k < 64; ++k) f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Tiles: the launch's list of objects with non-empty crops (enc_list_kernel),
// two per tile -- object u in rows / points 0..63, object v in 64..127 (a
// last odd object runs alone, its second half counting as empty).  CTA b
// takes tiles b, b + G, b + 2G, ...
__global__ void __launch_bounds__(E_THREADS, 1)
    encoder_tc_kernel(const float4* __restrict__ xyz, PairRange rg,
                      const int* __restrict__ list, const int* __restrict__ list_n,
                      const int32_t* __restrict__ cnt,
                      const unsigned char* __restrict__ img, float* __restrict__ feat,
                      __nv_bfloat16* __restrict__ ftile, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  const int n_objs = min(list_n[rg.chunk], 2 * (hi - lo));
  const int* lst = list + 2 * (size_t)lo;
  const int n = (n_objs + 1) >> 1;  // tiles
  if ((int)blockIdx.x >= n) {  // no tile here: only this CTA's share of the zero features
    if (warp == ZERO_WARP && cnt) zero_empty_objects(cnt, reinterpret_cast<unsigned char*>(ftile), lo, hi, lane, false);
    return;
  }
  const int my_pairs = (n - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles

  unsigned char* ctrl = smem + E_CTRL;
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
  const float* b3 = reinterpret_cast<const float*>(smem + E_BIAS) + 64 + 128;

  if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer warp
    // (warp-uniform control flow; weight copies by lane 0, MMAs by an elected lane)
    const uint32_t sW1 = smem_u32(smem + E_W1), sW2 = smem_u32(smem + E_W2);
    const uint32_t sW3 = smem_u32(smem + E_W3);
    const uint32_t sB2T = smem_u32(smem + E_B2T), sOne = smem_u32(smem + E_ONE);
    // resident weights, in bulk copies of at most 32 KB
    if (lane == 0) {
      mbar_expect_tx(BAR(B_W), E_IMG_BYTES);
      for (int off = 0; off < E_IMG_BYTES; off += 32768) {
        const int bytes = min(32768, E_IMG_BYTES - off);
        bulk_g2s(smem_u32(smem + off), img + off, bytes, BAR(B_W));
      }
    }
    bool ok = mbar_wait_warp(BAR(B_W), 0, abort, WAIT_CYCLES);
    tc_fence_after();
    const uint32_t id64 = idesc_bf16(128, 64), id128 = idesc_bf16(128, 128);
    const uint32_t id256 = idesc_bf16(128, 256);
    for (int r = 0; ok && NSLOT * r < my_pairs; ++r) {
      const uint32_t ph = r & 1;
      const int ns = min(NSLOT, my_pairs - NSLOT * r);  // slots in use this round
      // layers 1 and 2 in the order L1 0, L1 1, L1 2, L2 0, L1 3, L2 1, L2 2,
      // L2 3 (nibble t of kOrder: slot | layer << 2): slot 0's layer 2 goes
      // out while slot 3 is still building its X (slots 2 and 3 finish the
      // previous round's layer 3 last), instead of waiting behind it
      constexpr uint32_t kOrder = 0x76534210u;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = (int)((kOrder >> (4 * t)) & 0xfu), s = e & 3;
        if (!ok || s >= ns) continue;
        const uint32_t sO = smem_u32(smem + E_OPD0 + s * OPD_BYTES);
        if ((e >> 2) == 0) {
          // layer 1: D1[128 x 64] = X[128 x 16] . W1img^T (+ b1 via the ones columns)
          if (!(ok = mbar_wait_warp(BAR(B_XRDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (elect_one()) {
            mma_bf16(tbase + s * SLOT_COLS, sdesc(sO, 128, 256), sdesc(sW1, 128, 256), id64, 0);
            mma_commit(BAR(B_D1 + s));
          }
        } else {
          // layer 2: D2[128 x 128] = ones . b2img^T + H1[128 x 64] . W2img^T
          if (!(ok = mbar_wait_warp(BAR(B_H1RDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (elect_one()) {
            mma_bf16(tbase + s * SLOT_COLS, sdesc(sOne, 128, 256), sdesc(sB2T, 2048, 128), id128,
                     0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(tbase + s * SLOT_COLS, sdesc(sO + 256 * kk, 128, 1024),
                       sdesc(sW2 + 256 * kk, 128, 1024), id128, 1);
            mma_commit(BAR(B_D2 + s));
          }
        }
        __syncwarp();
      }
      // layer 3, transposed: D3^T = W3img[half] . H2^T, two slots per chain
      // (N = 256: slot s's points in its columns, slot s + 1's in the next
      // 128); half 0 (channels 0..127) after both slots' H2, half 1
      // (channels 128..255) once both have pooled half 0.  A last odd slot
      // runs alone with N = 128.
      for (int half = 0; half < 2 && ok; ++half) {
        const int bwait = half ? B_E3A : B_H2RDY, bdone = half ? B_D3B : B_D3A;
        const uint32_t sW = sW3 + 32768 * half;
        for (int s = 0; s < ns && ok; s += 2) {
          const bool two = s + 1 < ns;
          ok = mbar_wait_warp(BAR(bwait + s), ph, abort, WAIT_CYCLES);
          if (two) ok = ok && mbar_wait_warp(BAR(bwait + s + 1), ph, abort, WAIT_CYCLES);
          if (!ok) break;
          tc_fence_after();
          const uint32_t sH = smem_u32(smem + E_OPD0 + s * OPD_BYTES);
          if (elect_one()) {
            const uint32_t idn = two ? id256 : id128;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              mma_bf16(tbase + s * SLOT_COLS, sdesc(sW + 256 * kk, 128, 2048),
                       sdesc(sH + 256 * kk, 128, 2048), idn, kk > 0);
            mma_commit(BAR(bdone + s));
            if (two) mma_commit(BAR(bdone + s + 1));
          }
          __syncwarp();
        }
      }
    }
    if (__any_sync(0xffffffffu, *abort) && elect_one()) {
      // drain: wait (bounded) for every MMA this warp issued
      mma_commit(BAR(B_DRAIN));
      mbar_wait(BAR(B_DRAIN), 0, WAIT_CYCLES);
    }
    __syncwarp();
  } else if (warp == ZERO_WARP) {
    // the empty objects' pooled features (exactly 0) for the head
    if (cnt) zero_empty_objects(cnt, reinterpret_cast<unsigned char*>(ftile), lo, hi, lane, false);
  } else {
    // ------------------------------------------------ epilogue warpgroup of slot s
    const int s = warp >> 2, row = tid & 127, wq = warp & 3;
    unsigned char* stg = smem + E_STG0 + s * STG_BYTES;
    unsigned char* opd = smem + E_OPD0 + s * OPD_BYTES;
    const uint32_t tslot = tbase + s * SLOT_COLS + ((uint32_t)(32 * wq) << 16);
    int* cnt_s = s_cnt + 4 * s;
    int* obj_s = reinterpret_cast<int*>(ctrl + C_OBJ) + 4 * s;  // [parity][u, v]
    int tu0 = -1, tv0 = -1, tu1 = -1, tv1 = -1;  // objects of the slot's tiles, by parity
    // crop rows of the slot's tile jn -> bf16 hi/lo X tile (over the previous
    // tile's H2, dead once its layer 3 has completed), crop counts, XRDY
    auto build_x = [&](int jn) {
      if (!mbar_wait_or_abort(BAR(B_FULLX + s), jn & 1, abort, WAIT_CYCLES)) return false;
      // the copier wrote the tile's objects before its expect_tx arrival
      const int nu = obj_s[2 * (jn & 1)], nv = obj_s[2 * (jn & 1) + 1];
      if (jn & 1) tu1 = nu, tv1 = nv;
      else tu0 = nu, tv0 = nv;
      float4 q = reinterpret_cast<const float4*>(stg)[row];
      if (row >= KMAX && nv < 0) q = make_float4(0.f, 0.f, 0.f, 0.f);
      const unsigned m = __ballot_sync(0xffffffffu, q.w > 0.5f);
      if (lane == 0) cnt_s[wq] = __popc(m);
      x_tile_row(q, opd, row);
      fence_async_smem();
      return true;
    };
    // X of the pair is in place and this thread's TMEM reads of the slot are
    // done: the slot's layer 1 may run
    auto x_ready = [&]() {
      tc_fence_before();
      mbar_arrive(BAR(B_XRDY + s));
    };
    // The slot's crop rows arrive by bulk copy into its staging buffer, issued
    // by one lane of the warpgroup: tile 0 at the start, tile j + 1 once
    // layer 1 of tile j has completed (all of X_j, hence every read of the
    // staging rows and of the tile's object ids, is done).  Keeps the copies
    // off the MMA warp's path.
    const bool copier = wq == 0 && lane == 0;
    int n_loads = 0;
    auto load_rows = [&](int jn) {
      const int tg = blockIdx.x + (NSLOT * jn + s) * gridDim.x;
      const int u = lst[2 * tg], v = 2 * tg + 1 < n_objs ? lst[2 * tg + 1] : -1;
      obj_s[2 * (jn & 1)] = u;
      obj_s[2 * (jn & 1) + 1] = v;
      mbar_expect_tx(BAR(B_FULLX + s), (v >= 0 ? 2 : 1) * KMAX * 16);
      bulk_g2s(smem_u32(stg), xyz + (size_t)u * KMAX, KMAX * 16, BAR(B_FULLX + s));
      if (v >= 0)
        bulk_g2s(smem_u32(stg + KMAX * 16), xyz + (size_t)v * KMAX, KMAX * 16, BAR(B_FULLX + s));
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
      // layer 1 epilogue -> H1 (over X: MMA1 has completed)
      if (!(ok = mbar_wait_or_abort(BAR(B_D1 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      if (copier && i + NSLOT < my_pairs) load_rows(j + 1);
      enc_epi_rows<64>(tslot, opd, row);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H1RDY + s));
      // layer 2 epilogue -> H2 (over H1: MMA2 has completed)
      if (!(ok = mbar_wait_or_abort(BAR(B_D2 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      enc_epi_rows<128>(tslot, opd, row);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(B_H2RDY + s));
      // layer 3 epilogues: masked max over the valid points of each object
      if (!(ok = mbar_wait_or_abort(BAR(B_D3A + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      // crop counts written by other threads of this warpgroup (the next
      // pair's counts overwrite them only after every thread has passed
      // E3A below, which layer 3's second half waits for)
      asm volatile("bar.sync %0, 128;" ::"r"(1 + s) : "memory");
      const int cntA = cnt_s[0] + cnt_s[1], cntB = cnt_s[2] + cnt_s[3];
      float mA, mB;
      enc_pool(tslot, cntA, cntB, &mA, &mB);
      tc_fence_before();
      mbar_arrive(BAR(B_E3A + s));
      // the tile's objects (before build_x of the next tile reuses the other
      // parity's registers; this parity's stay until tile j + 2)
      const int u = ph ? tu1 : tu0, v = ph ? tv1 : tv0;
      const int pu = u >> 1, ku = (u & 1) * 256, pv = v >> 1, kv = (v & 1) * 256;
      {
        const float bias = b3[row];
        put_feat(feat, ftile, pu, pu - lo, ku + row, cntA > 0 ? fmaxf(mA + bias, 0.f) : 0.f);
        if (v >= 0)
          put_feat(feat, ftile, pv, pv - lo, kv + row, cntB > 0 ? fmaxf(mB + bias, 0.f) : 0.f);
      }
      if (!(ok = mbar_wait_or_abort(BAR(B_D3B + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      // the next pair's X first (H2 is dead once layer 3 has completed), then
      // the second pooling, then XRDY (the slot's TMEM columns are free only
      // after that pooling), then the feature stores: layer 1 of the next pair
      // waits for neither the X build nor the stores
      const bool nx = i + NSLOT < my_pairs;
      if (nx) ok = build_x(j + 1);
      enc_pool(tslot, cntA, cntB, &mA, &mB);
      if (nx && ok) x_ready();
      {
        const float bias = b3[128 + row];
        put_feat(feat, ftile, pu, pu - lo, ku + 128 + row, cntA > 0 ? fmaxf(mA + bias, 0.f) : 0.f);
        if (v >= 0)
          put_feat(feat, ftile, pv, pv - lo, kv + 128 + row,
                   cntB > 0 ? fmaxf(mB + bias, 0.f) : 0.f);
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

// -------------------------------------------------------------------- head
// Layer 1 and layer 3 run in split precision: the features arrive as bf16
// hi / lo pairs (FT_*), W_h1 and W_h3 are stored as bf16 hi / lo pairs, and
// D = A_hi W_hi + A_lo W_hi + A_hi W_lo (layer 3: G W_hi + G W_lo); the
// dropped A_lo W_lo term is ~2^-16 relative.  Layer 2 keeps plain bf16.
constexpr int HT = 128;                                    // pairs per tile
constexpr int H_W3 = 0;                                    // [16 x 256] hi 8 KB, lo 8 KB
constexpr int H_W3LO = 16 * 256 * 2;
constexpr int H_BIAS = H_W3 + 2 * 16 * 256 * 2;            // hb1 256, hb2 256, hb3 16
constexpr int H_RES_BYTES = H_BIAS + (256 + 256 + 16) * 4; // resident part of the image
constexpr int HK1 = FT_K;                                  // K of one layer-1 chunk (hi + lo)
constexpr int HK2 = 32;                                    // K of one layer-2 chunk
constexpr int H_CHUNK = 16384;                             // one B chunk: [256 x 16] hi + lo,
                                                           // or [256 x 32]
constexpr int H_BSUB = 256 * HK1 * 2;                      // offset of the lo B tile
constexpr int H_ACHUNK = FT_CHUNK;                         // one A chunk: [128 x 16] hi + lo
static_assert(2 * H_BSUB == H_CHUNK && 256 * HK2 * 2 == H_CHUNK, "chunk sizes");
constexpr int H_NST = 6;                                   // operand stages
constexpr int H_L1C = 512 / HK1, H_NCH = H_L1C + 256 / HK2;  // chunks per tile: 32 + 8
constexpr int H_A0 = (H_RES_BYTES + 127) / 128 * 128;      // A stages 8 KB each
constexpr int H_B0 = H_A0 + H_NST * H_ACHUNK;              // B stages [256 x 32] 16 KB each
constexpr int H_G = H_B0 + H_NST * H_CHUNK;                // G [128 x 256] 64 KB
constexpr int H_CTRL = H_G + 128 * 256 * 2;                // mbarriers, TMEM address, abort
constexpr int H_SMEM = H_CTRL + 256;
// global image: [resident][W_h1 chunks x 16][W_h2 chunks x 8]
constexpr int H_IMG_W1 = (H_RES_BYTES + 127) / 128 * 128;
constexpr int H_IMG_W2 = H_IMG_W1 + H_L1C * H_CHUNK;
constexpr int H_IMG_BYTES = H_IMG_W2 + (H_NCH - H_L1C) * H_CHUNK;
static_assert(H_RES_BYTES % 16 == 0, "resident image must be 16-byte chunks");
static_assert(H_IMG_W1 % 16 == 0 && H_CHUNK % 16 == 0, "bulk copies need 16-byte chunks");
static_assert(H_SMEM <= 227 * 1024, "head shared memory");

// One 32-column group of a 256-wide layer: TMEM row `row` at taddr ->
// relu(x + b) as bf16 into G columns [k0, k0 + 32) (K = 256).
__device__ __forceinline__ void head_epi_32(uint32_t taddr, const float* b, unsigned char* G, int row,
                                            int k0) {
  float v[32];
  tmem_ld32(taddr, v);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint4 w;
    const int j = 8 * c;
    w.x = pack_relu_bf16(v[j + 0] + b[j + 0], v[j + 1] + b[j + 1]);
    w.y = pack_relu_bf16(v[j + 2] + b[j + 2], v[j + 3] + b[j + 3]);
    w.z = pack_relu_bf16(v[j + 4] + b[j + 4], v[j + 5] + b[j + 5]);
    w.w = pack_relu_bf16(v[j + 6] + b[j + 6], v[j + 7] + b[j + 7]);
    *reinterpret_cast<uint4*>(G + kmajor_off(row, k0 + j, 256)) = w;
  }
}

// Epilogue of half of a 256-wide layer: TMEM row `row`, 128 columns from
// taddr -> relu(x + b) as bf16 into G columns [k0, k0 + 128) (K = 256).
__device__ __forceinline__ void head_epi_256(uint32_t taddr, const float* b, unsigned char* G, int row,
                                             int k0) {
  float v[32];
#pragma unroll 1
  for (int h = 0; h < 4; ++h) {
    tmem_ld32(taddr + 32 * h, v);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 w;
      const int j = 8 * c, o = 32 * h + j;
      w.x = pack_relu_bf16(v[j + 0] + b[o + 0], v[j + 1] + b[o + 1]);
      w.y = pack_relu_bf16(v[j + 2] + b[o + 2], v[j + 3] + b[o + 3]);
      w.z = pack_relu_bf16(v[j + 4] + b[o + 4], v[j + 5] + b[o + 5]);
      w.w = pack_relu_bf16(v[j + 6] + b[o + 6], v[j + 7] + b[o + 7]);
      *reinterpret_cast<uint4*>(G + kmajor_off(row, k0 + o, 256)) = w;
    }
  }
}

// Head over tiles of HT = 128 pairs (one pair per TMEM lane).  Warps 0-7 are
// the epilogue (warps w and w + 4 read lane quarter w % 4 and split the
// columns); one lane of warp 8 streams operands, one lane of warp 9 issues the
// MMAs.  Layers 1 and 2 are 24 K-chunks of 32 per tile (16 of W_h1 against the
// bf16 features the encoder wrote in operand layout, 8 of W_h2 against G);
// every operand chunk arrives by bulk copy through H_NST stages.  The stream
// is bound by the rate at which operands arrive (the weights are streamed
// again for every tile), so the copy thread keeps H_NST - 1 chunks in flight
// and refills a stage as soon as the MMAs that read it have completed,
// independently of the MMA thread.  TMEM: layer 1 accumulates in columns
// [0, 256), layer 2 and layer 3 in [256, 512).  The layer-1 epilogue fills G
// in four 64-column chunks, each announced on its own mbarrier (GC0-GC3);
// layer-2 chunk j starts once G chunk j / 2 is ready.  Layer 3 of tile t waits
// for the layer-2 epilogue without blocking the stream: the MMA thread polls
// for it between the layer-1 chunks of tile t + 1 (whose accumulator columns
// are already free), so the layer-2 and output epilogues of tile t overlap
// the layer-1 MMAs of tile t + 1.
// mbarrier phases (one waiter each, never more than one phase behind):
//   full[s] / done[s]: one per chunk in stage s; L1D, L2D, L3: one per tile;
//   GC0-GC3: one per tile (G chunk k holds layer 1); EPI: two per tile (G
//   holds layer 2; outputs have left TMEM).
constexpr int H_THREADS = 320;  // 8 epilogue warps, the copy warp, the MMA warp
constexpr int H_COPY = 256, H_MMA_WARP = 9;
__global__ void __launch_bounds__(H_THREADS, 1)
    head_tc_kernel(const __nv_bfloat16* __restrict__ ftile, PairRange rg,
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
  // done; 12 layer 3 done; 13 EPI; 14 resident image; 15 drain; 16 / 17 layer
  // 1 / layer 2 of the tile done; [18, 22) G chunk k holds layer 1
  const uint32_t bar0 = smem_u32(smem + H_CTRL);
  const uint32_t B_FULL = bar0, B_DONE = bar0 + 48;
  const uint32_t B_L3 = bar0 + 96, B_EPI = bar0 + 104, B_RES = bar0 + 112, B_DRAIN = bar0 + 120;
  const uint32_t B_L1D = bar0 + 128, B_L2D = bar0 + 136, B_GC = bar0 + 144;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + H_CTRL + 192);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + H_CTRL + 196);
  int* s_issued = reinterpret_cast<int*>(smem + H_CTRL + 200);
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
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  const int row = tid & 127, half = (tid >> 7) & 1;
  const float* hb1 = reinterpret_cast<const float*>(smem + H_BIAS);
  const float* hb2 = hb1 + 256;
  const float* hb3 = hb2 + 256;
  unsigned char* G = smem + H_G;
  const uint32_t sG = smem_u32(G), sW3 = smem_u32(smem + H_W3);
  const int n_chunks = H_NCH * my_tiles;  // this CTA's chunk stream
  bool ok = true;

  if (tid == H_COPY) {
    // ---------------------------------------------------------- copy thread
    mbar_expect_tx(B_RES, H_RES_BYTES);
    bulk_g2s(smem_u32(smem), img, H_RES_BYTES, B_RES);
    for (int g = 0; g < n_chunks; ++g) {
      const int st = g % H_NST, c = g % H_NCH;
      // the stage was last read by the MMAs of chunk g - H_NST
      if (g >= H_NST &&
          !(ok = mbar_wait_or_abort(B_DONE + 8 * st, (g / H_NST - 1) & 1, abort, WAIT_CYCLES)))
        break;
      const int tile = (int)blockIdx.x + (g / H_NCH) * (int)gridDim.x;
      const uint32_t bf = B_FULL + 8 * st;
      if (c < H_L1C) {
        mbar_expect_tx(bf, H_ACHUNK + H_CHUNK);
        bulk_g2s(smem_u32(smem + H_A0 + st * H_ACHUNK),
                 reinterpret_cast<const unsigned char*>(ftile) + (size_t)tile * FT_TILE +
                     (size_t)c * H_ACHUNK,
                 H_ACHUNK, bf);
        bulk_g2s(smem_u32(smem + H_B0 + st * H_CHUNK), img + H_IMG_W1 + (size_t)c * H_CHUNK,
                 H_CHUNK, bf);
      } else {
        mbar_expect_tx(bf, H_CHUNK);
        bulk_g2s(smem_u32(smem + H_B0 + st * H_CHUNK),
                 img + H_IMG_W2 + (size_t)(c - H_L1C) * H_CHUNK, H_CHUNK, bf);
      }
      *s_issued = g + 1;
    }
    if (!ok) *abort = 1;
  } else if (warp == H_MMA_WARP) {
    // ------------------------------------------------------------- MMA warp
    // layer 3 of a tile: D3[128 x 16] = G . Wh3img^T (rows 8..15 zero), in
    // the layer-2 columns
    auto layer3 = [&]() {
      tc_fence_after();
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
          mma_bf16(tbase + 256, sdesc(sG + 256 * kk, 128, 4096), sdesc(sW3 + 256 * kk, 128, 4096),
                   idesc_bf16(128, 16), kk > 0);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
          mma_bf16(tbase + 256, sdesc(sG + 256 * kk, 128, 4096),
                   sdesc(sW3 + H_W3LO + 256 * kk, 128, 4096), idesc_bf16(128, 16), 1u);
        mma_commit(B_L3);
      }
      __syncwarp();
    };
    ok = mbar_wait_warp(B_RES, 0, abort, WAIT_CYCLES);
    int l3 = -1;  // tile whose layer 3 waits for its layer-2 epilogue
    // two chunks (four MMAs) per step, so that the per-step waits cost less
    // than the tensor work they gate
    for (int g = 0; g < n_chunks && ok; g += 2) {
      const int st0 = g % H_NST, st1 = (g + 1) % H_NST, c = g % H_NCH, t = g / H_NCH;
      if (l3 >= 0) {
        // EPI phase 2 l3: G holds layer 2 of tile l3.  Layer 2 of the next
        // tile needs its outputs out of TMEM, so by then it is waited for.
        if (c == H_L1C) {
          ok = mbar_wait_warp(B_EPI, (2 * l3) & 1, abort, WAIT_CYCLES);
          if (!ok) break;
        }
        if (c == H_L1C || __all_sync(0xffffffffu, mbar_test_wait(B_EPI, (2 * l3) & 1))) {
          layer3();
          l3 = -1;
        }
      }
      const bool l1 = c < H_L1C;
      const int j = c - H_L1C;  // layer-2 chunk (even)
      if (!l1) {
        // the previous tile's outputs have left the layer-2 columns (EPI
        // phase 2 t - 1), and G chunk j / 2 (64 columns: K-chunks j and
        // j + 1) holds layer 1
        if (j == 0 && t > 0) ok = mbar_wait_warp(B_EPI, (2 * t - 1) & 1, abort, WAIT_CYCLES);
        ok = ok && mbar_wait_warp(B_GC + 8 * (j >> 1), t & 1, abort, WAIT_CYCLES);
      }
      ok = ok && mbar_wait_warp(B_FULL + 8 * st0, (g / H_NST) & 1, abort, WAIT_CYCLES);
      ok = ok && mbar_wait_warp(B_FULL + 8 * st1, ((g + 1) / H_NST) & 1, abort, WAIT_CYCLES);
      if (!ok) break;
      tc_fence_after();
      // descriptors from warp-uniform values; one elected lane issues
      const uint32_t sB0 = smem_u32(smem + H_B0 + st0 * H_CHUNK);
      const uint32_t sB1 = smem_u32(smem + H_B0 + st1 * H_CHUNK);
      const uint32_t sA0 = l1 ? smem_u32(smem + H_A0 + st0 * H_ACHUNK) : sG + 512 * j;
      const uint32_t sA1 = l1 ? smem_u32(smem + H_A0 + st1 * H_ACHUNK) : sG + 512 * (j + 1);
      // (layer 2: chunk j of G is K columns [32 j, 32 j + 32), 512 bytes per K = 32 step)
      const uint32_t acc0 = (l1 ? c : j) > 0 ? 1u : 0u;
      const uint32_t id = idesc_bf16(128, 256);
      if (elect_one()) {
        if (l1) {
          // [128 x 16] A and [256 x 16] B tiles (sbo 256): A_hi B_hi, A_lo B_hi, A_hi B_lo
          mma_bf16(tbase, sdesc(sA0, 128, 256), sdesc(sB0, 128, 256), id, acc0);
          mma_bf16(tbase, sdesc(sA0 + FT_SUB, 128, 256), sdesc(sB0, 128, 256), id, 1u);
          mma_bf16(tbase, sdesc(sA0, 128, 256), sdesc(sB0 + H_BSUB, 128, 256), id, 1u);
          mma_commit(B_DONE + 8 * st0);
          mma_bf16(tbase, sdesc(sA1, 128, 256), sdesc(sB1, 128, 256), id, 1u);
          mma_bf16(tbase, sdesc(sA1 + FT_SUB, 128, 256), sdesc(sB1, 128, 256), id, 1u);
          mma_bf16(tbase, sdesc(sA1, 128, 256), sdesc(sB1 + H_BSUB, 128, 256), id, 1u);
          mma_commit(B_DONE + 8 * st1);
        } else {
          // G (K = 256, sbo 4096) against [256 x 32] B chunks (sbo 512), two K = 16 steps each
          mma_bf16(tbase + 256, sdesc(sA0, 128, 4096), sdesc(sB0, 128, 512), id, acc0);
          mma_bf16(tbase + 256, sdesc(sA0 + 256, 128, 4096), sdesc(sB0 + 256, 128, 512), id, 1u);
          mma_commit(B_DONE + 8 * st0);
          mma_bf16(tbase + 256, sdesc(sA1, 128, 4096), sdesc(sB1, 128, 512), id, 1u);
          mma_bf16(tbase + 256, sdesc(sA1 + 256, 128, 4096), sdesc(sB1 + 256, 128, 512), id, 1u);
          mma_commit(B_DONE + 8 * st1);
        }
        if (c + 1 == H_L1C - 1) mma_commit(B_L1D);
        if (c + 1 == H_NCH - 1) mma_commit(B_L2D);
      }
      __syncwarp();
      if (c + 1 == H_NCH - 1) l3 = t;
    }
    if (ok && l3 >= 0) {
      ok = mbar_wait_warp(B_EPI, (2 * l3) & 1, abort, WAIT_CYCLES);
      if (ok) layer3();
    }
    if (!ok) *abort = 1;
  }
  // epilogue warps
  if (tid < 256) ok = mbar_wait_or_abort(B_RES, 0, abort, WAIT_CYCLES);
  for (int t = 0; tid < 256 && t < my_tiles && ok; ++t) {
    const int pr = lo + ((int)blockIdx.x + t * (int)gridDim.x) * HT + row;
    const bool row_ok = pr < n;
    // operands of the world-frame epilogue, loaded while the MMAs run
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
      head_epi_32(tbase + lane_off + col, hb1 + col, G, row, col);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(B_GC + 8 * k);
    }
    ok = mbar_wait_or_abort(B_L2D, t & 1, abort, WAIT_CYCLES);
    if (!ok) break;
    tc_fence_after();
    head_epi_256(tbase + lane_off + 256 + 128 * half, hb2 + 128 * half, G, row, 128 * half);
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
        for (int o = 0; o < 8; ++o) y[o] = v[o] + hb3[o];
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
    if (warp == H_MMA_WARP && (tid & 31) == 0) {
      mma_commit(B_DRAIN);
      mbar_wait(B_DRAIN, 0, WAIT_CYCLES);
    }
    if (tid == H_COPY) {
      const int issued = *s_issued;
      for (int g = issued - H_NST; g < issued; ++g)
        if (g >= 0) mbar_wait(B_FULL + 8 * (g % H_NST), (g / H_NST) & 1, WAIT_CYCLES);
    }
  }
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

// One CTA waits, bounded, on an mbarrier nothing completes (the test entry
// locc_selftest_wait_timeout): same primitives and same abort path as the
// encoder and head kernels -- bounded wait, error bit 2, TMEM released.
__global__ void __launch_bounds__(128) wait_timeout_kernel(long long max_cycles, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  volatile int* abort = &abort_flag;
  if (tid == 0) {
    mbar_init(smem_u32(&bar), 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&tslot), 32);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  const bool ok = mbar_wait_or_abort(smem_u32(&bar), 0, abort, max_cycles);
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && (!ok || *abort)) atomicOr(err, 2);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 32);
  }
}

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
  // bias (hi, lo): two bf16 values whose float32 sum is b to ~2^-17 relative
  auto bias_split = [&](int l, int c, int part) -> float {
    const float b = params[offb[l] + c];
    const float hi = bf16_value(bf16_bits(b));
    return part == 0 ? hi : b - hi;
  };
  // layer 1 B operand: row c = [W_hi(3), W_hi(3), W_lo(3), b1_hi, b1_lo, 0 x 5]
  put_tile(e + E_W1, 64, 16, [&](int c, int k) -> float {
    if (k == 9 || k == 10) return bias_split(0, c, k - 9);
    if (k >= 9) return 0.f;
    const float w = W(0, c, k % 3);
    const float hi = bf16_value(bf16_bits(w));
    return k < 6 ? hi : w - hi;
  });
  // layer 2 bias tile (first core matrix of each row group: K columns 0..7)
  // and the ones tile it is multiplied with
  put_tile(e + E_B2T, 128, 8, [&](int c, int k) { return k < 2 ? bias_split(1, c, k) : 0.f; });
  put_tile(e + E_ONE, 128, 16, [&](int, int k) { return k < 2 ? 1.f : 0.f; });
  put_tile(e + E_W2, 128, 64, [&](int c, int k) { return W(1, c, k); });
  put_tile(e + E_W3, 256, 128, [&](int c, int k) { return W(2, c, k); });
  std::memcpy(e + E_BIAS, &params[offb[0]], 64 * 4);
  std::memcpy(e + E_BIAS + 64 * 4, &params[offb[1]], 128 * 4);
  std::memcpy(e + E_BIAS + 192 * 4, &params[offb[2]], 256 * 4);
  unsigned char* hd = img.data() + enc_bytes;
  auto hi_of = [&](float w) { return bf16_value(bf16_bits(w)); };
  put_tile(hd + H_W3, 16, 256, [&](int c, int k) { return c < 8 ? W(5, c, k) : 0.f; });
  put_tile(hd + H_W3LO, 16, 256,
           [&](int c, int k) { return c < 8 ? W(5, c, k) - hi_of(W(5, c, k)) : 0.f; });
  std::memcpy(hd + H_BIAS, &params[offb[3]], 256 * 4);
  std::memcpy(hd + H_BIAS + 256 * 4, &params[offb[4]], 256 * 4);
  std::memcpy(hd + H_BIAS + 512 * 4, &params[offb[5]], 8 * 4);
  for (int kc = 0; kc < H_L1C; ++kc) {
    put_tile(hd + H_IMG_W1 + (size_t)kc * H_CHUNK, 256, HK1,
             [&](int c, int k) { return W(3, c, HK1 * kc + k); });
    put_tile(hd + H_IMG_W1 + (size_t)kc * H_CHUNK + H_BSUB, 256, HK1, [&](int c, int k) {
      const float w = W(3, c, HK1 * kc + k);
      return w - hi_of(w);
    });
  }
  for (int kc = 0; kc < H_NCH - H_L1C; ++kc)
    put_tile(hd + H_IMG_W2 + (size_t)kc * H_CHUNK, 256, HK2,
             [&](int c, int k) { return W(4, c, HK2 * kc + k); });
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

cudaError_t launch_enc_list(locc_handle* h, const float4* xyz, const PairRange& rg, float* feat,
                            bool counts, void* ftile, int e4m3, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(h->d_list_n + rg.chunk, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const int n_obj = 2 * ((rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1);
  const int grid = std::max(1, std::min((n_obj + 255) / 256, 8 * h->n_sm));
  enc_list_kernel<<<grid, 256, 0, stream>>>(xyz, rg, h->d_list, h->d_list_n,
                                            counts ? h->d_cnt : nullptr, feat,
                                            static_cast<unsigned char*>(ftile), e4m3);
  return cudaGetLastError();
}

cudaError_t prepare_tc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(encoder_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(head_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, H_SMEM);
  return e;
}

int run_network_tc(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                   const float4* centre, float* out, float* y_raw, float* feat_out,
                   cudaStream_t stream, cudaEvent_t mid, int list_mode) {
  if (h->prec == LOCC_FP8)
    return run_network_fp8(h, xyz, rg, in, centre, out, y_raw, feat_out, stream, mid, list_mode);
  const int n_pairs = (rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1;  // pairs of one chunk, at most
  __nv_bfloat16* ftile = static_cast<__nv_bfloat16*>(h->d_feat_tc);
  if (list_mode != LIST_FROM_CROP &&
      launch_enc_list(h, xyz, rg, feat_out, list_mode == LIST_AND_COUNTS_FROM_ROWS, nullptr, 0,
                      stream) != cudaSuccess) {
    set_error("enc_list_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  const int grid_e = std::min(n_pairs, h->n_sm);
  encoder_tc_kernel<<<grid_e, E_THREADS, E_SMEM, stream>>>(xyz, rg, h->d_list, h->d_list_n,
                                                           h->d_cnt, h->wtc_enc, feat_out, ftile,
                                                           h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("encoder_tc_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  if (mid && cudaEventRecord(mid, stream) != cudaSuccess) return LOCC_ERR_CUDA;
  return launch_head_tc(h, rg, in, centre, out, y_raw, stream);
}

int launch_head_tc(locc_handle* h, const PairRange& rg, const PairInputs* in, const float4* centre,
                   float* out, float* y_raw, cudaStream_t stream) {
  const int n_pairs = (rg.n_cap + rg.n_chunks - 1) / rg.n_chunks + 1;  // pairs of one chunk, at most
  PairInputs pin{};
  if (in) pin = *in;
  const int grid_h = std::min((n_pairs + HT - 1) / HT, h->n_sm);
  head_tc_kernel<<<grid_h, H_THREADS, H_SMEM, stream>>>(static_cast<__nv_bfloat16*>(h->d_feat_tc),
                                                        rg, h->wtc_head, pin, in != nullptr, centre,
                                                        out, y_raw, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("head_tc_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

int launch_encoder_list(locc_handle* h, const float4* xyz, const PairRange& rg, const int* list,
                        const int* list_n, int grid, cudaStream_t stream) {
  encoder_tc_kernel<<<grid, E_THREADS, E_SMEM, stream>>>(
      xyz, rg, list, list_n, nullptr, h->wtc_enc, nullptr,
      static_cast<__nv_bfloat16*>(h->d_feat_tc), h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("encoder_tc_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

}  // namespace locc

extern "C" int locc_selftest_wait_timeout(locc_handle* h, int64_t max_cycles, void* stream) {
  if (!h) {
    locc::set_error("handle is NULL");
    return LOCC_ERR_INVALID_ARG;
  }
  if (max_cycles < 1 || max_cycles > 2000000000LL) {
    locc::set_error("max_cycles must be in [1, 2e9]");
    return LOCC_ERR_INVALID_ARG;
  }
  locc::wait_timeout_kernel<<<1, 128, 0, (cudaStream_t)stream>>>((long long)max_cycles, h->d_err);
  if (cudaGetLastError() != cudaSuccess) {
    locc::set_error("wait_timeout_kernel launch failed");
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

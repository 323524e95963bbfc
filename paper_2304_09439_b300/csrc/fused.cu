// Fused crop gather + BF16 tensor-core encoder: one persistent launch per
// step in which warps on the CUDA cores crop object pairs and hand each
// object's crop rows, through shared memory, to the encoder slots whose MMAs
// run on the tensor cores (Sec. III: the collision predictor selects the
// parts of both shapes inside the intersection region and encodes them with a
// point-wise MLP and pooling; Sec. I / IV: one uniform flow for many pairs).
//
// The crop (CUDA cores, L2 loads, ballots) and the encoder (tensor pipe,
// TMEM) use different units of the SM, so running them side by side on the
// same SM overlaps them; the crop rows no longer go through HBM.
//
// CTA layout (one CTA per SM, persistent):
//   * warps 0 .. 4 FS - 1: the epilogue warpgroups of FS = 3 encoder slots
//     (one thread per crop row / TMEM lane, as in encoder_tc_kernel);
//   * warp 4 FS: loads the weight image and issues every tcgen05.mma;
//   * FC crop warps: each takes whole pairs from the device counter (the
//     first statically), computes the pair frame and crop centre and selects
//     both objects' crops exactly as crop_kernel does (crop_dev.cuh).  An
//     object with an empty crop gets its pooled feature (exactly 0) written
//     directly; a deferred one (one d^2 bin overflows the list) is left to
//     crop_fallback_kernel and a list-driven encoder pass after this kernel;
//     every other object's 64 rows go into the next entry of a ring of
//     F_RING one-object entries in shared memory.
//   * Hand-off: a producer claims ring tickets in order (shared counter),
//     waits for the entry's previous use to be consumed (REMPTY), writes the
//     rows and object id and arrives on REMPTY's partner RFULL (all 32 lanes).
//     Encoder tile k of the CTA (slot k % FS) takes tickets 2k (rows 0..63)
//     and 2k + 1 (rows 64..127), converts them into its X tile and releases
//     the entries.  When the last crop warp of the CTA runs out of pairs it
//     publishes the number of tickets; a slot whose tile would need a ticket
//     beyond it stops (a last odd object runs alone, its second half empty)
//     and tells the MMA warp through its XRDY arrival and an end flag.
// A slot waits for tickets that were claimed at most F_RING tickets after
// the last ones consumed, so the full/empty parities are never ambiguous.
//
// Every wait is bounded; on a timeout the CTA raises the abort flag, every
// role stops, TMEM is released and bit 2 of the error flag is set.
#include <algorithm>

#include "crop_dev.cuh"
#include "enc_tc.cuh"
#include "handle.cuh"

namespace locc {
namespace {

constexpr int FS = 3;                              // encoder slots
constexpr int F_RING = 8;                          // ring entries, one object crop each
constexpr int F_ENTRY = KMAX * 16;                 // 64 rows x float4
constexpr int F_OPD = 128 * 128 * 2;               // slot operand region (X / H1 / H2)
constexpr int F_COLS = 128;                        // TMEM columns per slot
constexpr int F_RING0 = (E_IMG_BYTES + 1023) / 1024 * 1024;
constexpr int F_OPD0 = F_RING0 + F_RING * F_ENTRY;
static_assert(F_OPD0 % 1024 == 0, "operand regions must stay 1 KB aligned");
constexpr int F_CROP0 = F_OPD0 + FS * F_OPD;
// per crop warp: key list, rank buffer, histogram, pair frame
constexpr int F_CW = CAND_CAP * 8 + EBUF * 8 + NBINS * 4 + 16 * 4;
static_assert(F_CW % 16 == 0, "crop warp scratch alignment");
// barriers: per slot XRDY H1RDY H2RDY E3A D1 D2 D3A D3B, per entry RFULL
// REMPTY, then W and DRAIN
constexpr int FB_XRDY = 0, FB_H1RDY = FS, FB_H2RDY = 2 * FS, FB_E3A = 3 * FS, FB_D1 = 4 * FS,
              FB_D2 = 5 * FS, FB_D3A = 6 * FS, FB_D3B = 7 * FS, FB_RFULL = 8 * FS,
              FB_REMPTY = 8 * FS + F_RING, FB_W = 8 * FS + 2 * F_RING, FB_DRAIN = FB_W + 1;
constexpr int F_NBAR = FB_DRAIN + 1;
// control words after the barriers
constexpr int FC_TMEM = 8 * F_NBAR, FC_ABORT = FC_TMEM + 4, FC_TICKET = FC_ABORT + 4,
              FC_DONE = FC_TICKET + 4, FC_FINAL = FC_DONE + 4, FC_END = FC_FINAL + 4,
              FC_OBJ = FC_END + 4 * FS, FC_OCNT = FC_OBJ + 4 * F_RING,
              FC_BYTES = FC_OCNT + 4 * F_RING;

template <int FC>
struct Fused {
  static constexpr int THREADS = 32 * (4 * FS + 1 + FC);
  static constexpr int MMA_WARP = 4 * FS;
  static constexpr int CTRL = F_CROP0 + FC * F_CW;
  static constexpr int SMEM = CTRL + FC_BYTES;
  static_assert(SMEM <= 227 * 1024, "fused kernel shared memory");
};

enum { TK_GOT = 0, TK_END = 1, TK_ABORT = 2 };

template <int FC>
__global__ void __launch_bounds__(Fused<FC>::THREADS, 1)
    fused_crop_encoder_kernel(DevLibrary lib, PairInputs in, PairRange rg, float radius,
                              int32_t* __restrict__ cnt_out, float4* __restrict__ centre_out,
                              int* __restrict__ err, int* __restrict__ defer, int defer_cap,
                              const unsigned char* __restrict__ img,
                              __nv_bfloat16* __restrict__ ftile) {
  using K = Fused<FC>;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  const int n_pairs = hi - lo;

  unsigned char* ctrl = smem + K::CTRL;
  const uint32_t bar0 = smem_u32(ctrl);
  auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + FC_TMEM);
  volatile int* abort = reinterpret_cast<volatile int*>(ctrl + FC_ABORT);
  int* s_ticket = reinterpret_cast<int*>(ctrl + FC_TICKET);
  int* s_done = reinterpret_cast<int*>(ctrl + FC_DONE);
  volatile int* s_final = reinterpret_cast<volatile int*>(ctrl + FC_FINAL);
  volatile int* s_end = reinterpret_cast<volatile int*>(ctrl + FC_END);
  int* s_obj = reinterpret_cast<int*>(ctrl + FC_OBJ);    // object id of each ring entry
  int* s_ocnt = reinterpret_cast<int*>(ctrl + FC_OCNT);  // its crop count
  const float4* ring = reinterpret_cast<const float4*>(smem + F_RING0);

  if (tid == 0) {
    for (int s = 0; s < FS; ++s) {
      mbar_init(BAR(FB_XRDY + s), 128);
      mbar_init(BAR(FB_H1RDY + s), 128);
      mbar_init(BAR(FB_H2RDY + s), 128);
      mbar_init(BAR(FB_E3A + s), 128);
      mbar_init(BAR(FB_D1 + s), 1);
      mbar_init(BAR(FB_D2 + s), 1);
      mbar_init(BAR(FB_D3A + s), 1);
      mbar_init(BAR(FB_D3B + s), 1);
      s_end[s] = 0;
    }
    for (int e = 0; e < F_RING; ++e) {
      mbar_init(BAR(FB_RFULL + e), 32);   // the producing warp's 32 lanes
      mbar_init(BAR(FB_REMPTY + e), 64);  // the 64 consumer threads of its rows
    }
    mbar_init(BAR(FB_W), 1);
    mbar_init(BAR(FB_DRAIN), 1);
    *abort = 0;
    *s_ticket = 0;
    *s_done = 0;
    *s_final = -1;
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

  if (warp > K::MMA_WARP) {
    // ------------------------------------------------------------ crop warps
    const int cw = warp - K::MMA_WARP - 1;
    unsigned char* scratch = smem + F_CROP0 + cw * F_CW;
    unsigned long long* buf = reinterpret_cast<unsigned long long*>(scratch);
    unsigned long long* ebuf = buf + CAND_CAP;
    int* hist = reinterpret_cast<int*>(ebuf + EBUF);
    float* rsh = reinterpret_cast<float*>(hist + NBINS);
    const int first = FC * (int)gridDim.x;
    int pr = (int)blockIdx.x * FC + cw;
    bool ok = true;
    while (ok && pr < n_pairs) {
      int nxt = 0;
      if (lane == 0) nxt = first + atomicAdd(&defer[1], 1);
      const int p = lo + pr;
      int a, b, sa, sb;
      if (!load_pair(in, lib.n_shapes, p, &a, &b, &sa, &sb, lane == 0 ? err : nullptr)) {
        // invalid indices: zero features, count 0, NaN centre (the head
        // writes the NaN row)
        zero_feat_warp(reinterpret_cast<unsigned char*>(ftile), p - lo, 0, lane, false);
        zero_feat_warp(reinterpret_cast<unsigned char*>(ftile), p - lo, 1, lane, false);
        if (lane == 0) {
          const float nan = __int_as_float(0x7fc00000);
          cnt_out[2 * p] = cnt_out[2 * p + 1] = 0;
          centre_out[p] = make_float4(nan, nan, nan, nan);
        }
        pr = __shfl_sync(FULL, nxt, 0);
        continue;
      }
      {
        Frame f;
        pair_frame(in.poses + 7 * (size_t)a, in.poses + 7 * (size_t)b, lib.aabb[2 * sa],
                   lib.aabb[2 * sa + 1], lib.aabb[2 * sb], lib.aabb[2 * sb + 1], f);
        if (lane == 0) {
          centre_out[p] = make_float4(f.c[0], f.c[1], f.c[2], 0.f);
#pragma unroll
          for (int i = 0; i < 9; ++i) rsh[i] = f.rrel[i];
          rsh[9] = f.c[0], rsh[10] = f.c[1], rsh[11] = f.c[2];
          rsh[12] = f.cb[0], rsh[13] = f.cb[1], rsh[14] = f.cb[2];
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int obj = 0; obj < 2 && ok; ++obj) {
        const float* c = rsh + 9 + 3 * obj;
        const int shape = obj ? sb : sa;
        const int cnt = select_object(lib, p, obj, shape, c[0], c[1], c[2], lane, radius, buf,
                                      hist, ebuf, defer, defer_cap);
        if (cnt < 0) continue;  // deferred: fallback crop + list-driven encoder
        if (lane == 0) cnt_out[2 * p + obj] = cnt;
        if (cnt == 0) {  // the pooled feature is exactly 0
          zero_feat_warp(reinterpret_cast<unsigned char*>(ftile), p - lo, obj, lane, false);
          continue;
        }
        int t = 0;
        if (lane == 0) t = atomicAdd(s_ticket, 1);
        t = __shfl_sync(FULL, t, 0);
        const int e = t % F_RING, use = t / F_RING;
        if (use > 0 && !(ok = mbar_wait_warp(BAR(FB_REMPTY + e), (use - 1) & 1, abort,
                                             WAIT_CYCLES)))
          break;
        write_crop(buf, cnt, lib.points + (size_t)shape * lib.n_pad, c[0], c[1], c[2],
                   obj ? rsh : nullptr, const_cast<float4*>(ring) + e * KMAX, nullptr, lane);
        if (lane == 0) s_obj[e] = 2 * p + obj, s_ocnt[e] = cnt;
        __syncwarp();
        mbar_arrive(BAR(FB_RFULL + e));
      }
      pr = __shfl_sync(FULL, nxt, 0);
    }
    // the last crop warp of the CTA to finish publishes the ticket count
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(s_done, 1) == FC - 1) {
        __threadfence_block();
        *s_final = atomicAdd(s_ticket, 0);
      }
    }
  } else if (warp == K::MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer warp
    const uint32_t sW1 = smem_u32(smem + E_W1), sW2 = smem_u32(smem + E_W2);
    const uint32_t sW3 = smem_u32(smem + E_W3);
    const uint32_t sB2T = smem_u32(smem + E_B2T), sOne = smem_u32(smem + E_ONE);
    if (lane == 0) {
      mbar_expect_tx(BAR(FB_W), E_IMG_BYTES);
      for (int off = 0; off < E_IMG_BYTES; off += 32768)
        bulk_g2s(smem_u32(smem + off), img + off, min(32768, E_IMG_BYTES - off), BAR(FB_W));
    }
    bool ok = mbar_wait_warp(BAR(FB_W), 0, abort, WAIT_CYCLES);
    tc_fence_after();
    const uint32_t id64 = idesc_bf16(128, 64), id128 = idesc_bf16(128, 128);
    const uint32_t id256 = idesc_bf16(128, 256);
    bool more = true;
    for (int r = 0; ok && more; ++r) {
      const uint32_t ph = r & 1;
      bool act[FS];
#pragma unroll
      for (int s = 0; s < FS; ++s) act[s] = false;
      // layers 1 and 2 in the order L1 0, L1 1, L2 0, L1 2, L2 1, L2 2
      // (nibble t of kOrder: slot | layer << 2); a slot without a tile this
      // round (end of the CTA's work) skips its layers
      constexpr uint32_t kOrder = 0x652410u;
#pragma unroll
      for (int t = 0; t < 2 * FS; ++t) {
        const int e = (int)((kOrder >> (4 * t)) & 0xfu), s = e & 3;
        if (!ok) break;
        const uint32_t sO = smem_u32(smem + F_OPD0 + s * F_OPD);
        if ((e >> 2) == 0) {
          if (!(ok = mbar_wait_warp(BAR(FB_XRDY + s), ph, abort, WAIT_CYCLES))) break;
          act[s] = s_end[s] == 0;
          if (!act[s]) continue;
          tc_fence_after();
          if (elect_one()) {
            mma_bf16(tbase + s * F_COLS, sdesc(sO, 128, 256), sdesc(sW1, 128, 256), id64, 0);
            mma_commit(BAR(FB_D1 + s));
          }
        } else {
          if (!act[s]) continue;
          if (!(ok = mbar_wait_warp(BAR(FB_H1RDY + s), ph, abort, WAIT_CYCLES))) break;
          tc_fence_after();
          if (elect_one()) {
            mma_bf16(tbase + s * F_COLS, sdesc(sOne, 128, 256), sdesc(sB2T, 2048, 128), id128, 0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(tbase + s * F_COLS, sdesc(sO + 256 * kk, 128, 1024),
                       sdesc(sW2 + 256 * kk, 128, 1024), id128, 1);
            mma_commit(BAR(FB_D2 + s));
          }
        }
        __syncwarp();
      }
      // layer 3 (transposed), slots 0 and 1 as one N = 256 chain, slot 2 alone
      for (int half = 0; half < 2 && ok; ++half) {
        const int bwait = half ? FB_E3A : FB_H2RDY, bdone = half ? FB_D3B : FB_D3A;
        const uint32_t sW = sW3 + 32768 * half;
        for (int s = 0; s < FS && ok; s += 2) {
          if (!act[s]) break;
          const bool two = s + 1 < FS && act[s + 1];
          ok = mbar_wait_warp(BAR(bwait + s), ph, abort, WAIT_CYCLES);
          if (two) ok = ok && mbar_wait_warp(BAR(bwait + s + 1), ph, abort, WAIT_CYCLES);
          if (!ok) break;
          tc_fence_after();
          const uint32_t sH = smem_u32(smem + F_OPD0 + s * F_OPD);
          if (elect_one()) {
            const uint32_t idn = two ? id256 : id128;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              mma_bf16(tbase + s * F_COLS, sdesc(sW + 256 * kk, 128, 2048),
                       sdesc(sH + 256 * kk, 128, 2048), idn, kk > 0);
            mma_commit(BAR(bdone + s));
            if (two) mma_commit(BAR(bdone + s + 1));
          }
          __syncwarp();
        }
      }
#pragma unroll
      for (int s = 0; s < FS; ++s) more = more && act[s];
    }
    if (__any_sync(0xffffffffu, *abort) && elect_one()) {
      mma_commit(BAR(FB_DRAIN));
      mbar_wait(BAR(FB_DRAIN), 0, WAIT_CYCLES);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue warpgroup of slot s
    const int s = warp >> 2, row = tid & 127, wq = warp & 3;
    unsigned char* opd = smem + F_OPD0 + s * F_OPD;
    const uint32_t tslot = tbase + s * F_COLS + ((uint32_t)(32 * wq) << 16);
    const float* b3 = reinterpret_cast<const float*>(smem + E_BIAS) + 64 + 128;
    // Wait for ticket t: TK_GOT once its entry is full, TK_END once the
    // CTA's ticket count is known and t is beyond it (every lane reaches the
    // same answer); warp-uniform: TK_ABORT on all lanes if any lane gave up.
    auto wait_ticket = [&](int t) {
      const uint32_t bar = BAR(FB_RFULL + t % F_RING), par = (t / F_RING) & 1;
      int st = TK_GOT;
      if (!mbar_test_wait(bar, par)) {
        const long long t0 = clock64();
        for (;;) {
          const int fin = *s_final;
          if (fin >= 0 && t >= fin) {
            st = TK_END;
            break;
          }
          if (mbar_try_wait(bar, par)) break;
          if (*abort) {
            st = TK_ABORT;
            break;
          }
          if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            st = TK_ABORT;
            break;
          }
        }
      }
      if (__any_sync(0xffffffffu, st == TK_ABORT)) return (int)TK_ABORT;
      return st;
    };
    // objects (2 p + side) and crop counts of the slot's tiles, by parity
    int tu0 = -1, tv0 = -1, tu1 = -1, tv1 = -1, cu0 = 0, cv0 = 0, cu1 = 0, cv1 = 0;
    // tile jn of this slot (CTA tile k = FS jn + s): tickets 2k, 2k + 1 ->
    // X tile; releases the ring entries.  Returns TK_* (warp-uniform).
    auto build_x = [&](int jn) {
      const int k = FS * jn + s;
      const int st0 = wait_ticket(2 * k);
      if (st0 != TK_GOT) return st0;
      const int st1 = wait_ticket(2 * k + 1);
      if (st1 == TK_ABORT) return st1;
      const int e0 = (2 * k) % F_RING, e1 = (2 * k + 1) % F_RING;
      const int nu = s_obj[e0], nv = st1 == TK_GOT ? s_obj[e1] : -1;
      const int cu = s_ocnt[e0], cv = nv >= 0 ? s_ocnt[e1] : 0;
      if (jn & 1) tu1 = nu, tv1 = nv, cu1 = cu, cv1 = cv;
      else tu0 = nu, tv0 = nv, cu0 = cu, cv0 = cv;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < KMAX) q = ring[e0 * KMAX + row];
      else if (nv >= 0) q = ring[e1 * KMAX + row - KMAX];
      // rows and metadata read: the entries may be refilled
      if (row < KMAX) mbar_arrive(BAR(FB_REMPTY + e0));
      else if (nv >= 0) mbar_arrive(BAR(FB_REMPTY + e1));
      x_tile_row(q, opd, row);
      fence_async_smem();
      return (int)TK_GOT;
    };
    // X in place (or no tile: the end flag is set first) and this thread's
    // TMEM reads of the slot done: the MMA warp may go on with the slot
    auto x_ready = [&](bool end) {
      if (end) s_end[s] = 1;
      tc_fence_before();
      mbar_arrive(BAR(FB_XRDY + s));
    };
    bool ok = mbar_wait_warp(BAR(FB_W), 0, abort, WAIT_CYCLES);
    int st = TK_ABORT;
    if (ok) {
      st = build_x(0);
      if (st != TK_ABORT) x_ready(st == TK_END);
    }
    ok = ok && st == TK_GOT;
    for (int j = 0; ok; ++j) {
      const uint32_t ph = j & 1;
      // layer 1 epilogue -> H1 (over X: MMA1 has completed)
      if (!(ok = mbar_wait_warp(BAR(FB_D1 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      enc_epi_rows<64>(tslot, opd, row);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(FB_H1RDY + s));
      // layer 2 epilogue -> H2 (over H1: MMA2 has completed)
      if (!(ok = mbar_wait_warp(BAR(FB_D2 + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      enc_epi_rows<128>(tslot, opd, row);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(FB_H2RDY + s));
      // layer 3 epilogues: masked max over the valid points of each object
      if (!(ok = mbar_wait_warp(BAR(FB_D3A + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      const int cntA = ph ? cu1 : cu0, cntB = ph ? cv1 : cv0;
      float mA, mB;
      enc_pool(tslot, cntA, cntB, &mA, &mB);
      tc_fence_before();
      mbar_arrive(BAR(FB_E3A + s));
      const int u = ph ? tu1 : tu0, v = ph ? tv1 : tv0;
      const int pu = u >> 1, ku = (u & 1) * 256, pv = v >> 1, kv = (v & 1) * 256;
      {
        const float bias = b3[row];
        put_feat(nullptr, ftile, pu, pu - lo, ku + row, cntA > 0 ? fmaxf(mA + bias, 0.f) : 0.f);
        if (v >= 0)
          put_feat(nullptr, ftile, pv, pv - lo, kv + row, cntB > 0 ? fmaxf(mB + bias, 0.f) : 0.f);
      }
      if (!(ok = mbar_wait_warp(BAR(FB_D3B + s), ph, abort, WAIT_CYCLES))) break;
      tc_fence_after();
      // the next tile's X first (H2 is dead once layer 3 has completed),
      // then the second pooling, then XRDY (the slot's TMEM columns are free
      // only after it), then the feature stores
      st = build_x(j + 1);
      enc_pool(tslot, cntA, cntB, &mA, &mB);
      if (st != TK_ABORT) x_ready(st == TK_END);
      {
        const float bias = b3[128 + row];
        put_feat(nullptr, ftile, pu, pu - lo, ku + 128 + row,
                 cntA > 0 ? fmaxf(mA + bias, 0.f) : 0.f);
        if (v >= 0)
          put_feat(nullptr, ftile, pv, pv - lo, kv + 128 + row,
                   cntB > 0 ? fmaxf(mB + bias, 0.f) : 0.f);
      }
      tc_fence_before();
      ok = st == TK_GOT;
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(err, 2);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

template <int FC>
cudaError_t launch_fused_fc(const DevLibrary& lib, const PairInputs& in, const PairRange& rg,
                            float r, int32_t* cnt, float4* centre, int* err, int* defer,
                            int defer_cap, const unsigned char* img, __nv_bfloat16* ftile,
                            int n_sm, cudaStream_t s) {
  fused_crop_encoder_kernel<FC><<<n_sm, Fused<FC>::THREADS, Fused<FC>::SMEM, s>>>(
      lib, in, rg, r, cnt, centre, err, defer, defer_cap, img, ftile);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_fused_kernels() {
  cudaError_t e = cudaFuncSetAttribute(fused_crop_encoder_kernel<6>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Fused<6>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_crop_encoder_kernel<8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Fused<8>::SMEM);
  return e;
}

cudaError_t launch_fused(const DevLibrary& lib, const PairInputs& in, const PairRange& rg, float r,
                         int32_t* cnt, float4* centre, int* err, int* defer, int defer_cap,
                         const unsigned char* img, __nv_bfloat16* ftile, int n_sm, int crop_warps,
                         cudaStream_t s) {
  // defer[0]: deferred objects, defer[1]: pair counter of the crop warps
  cudaError_t e = cudaMemsetAsync(defer, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (crop_warps == 6)
    return launch_fused_fc<6>(lib, in, rg, r, cnt, centre, err, defer, defer_cap, img, ftile, n_sm,
                              s);
  return launch_fused_fc<8>(lib, in, rg, r, cnt, centre, err, defer, defer_cap, img, ftile, n_sm, s);
}

}  // namespace locc

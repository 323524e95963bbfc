// Device code of the crop gather shared by the crop kernels (crop.cu) and
// the fused crop + encoder kernel (fused.cu): pose composition and crop
// centre (pair_frame), block culling, in-ball key compaction and the exact
// top-64 selection (select_object), and the rows of one object crop in the
// canonical frame (write_crop).  What the selection computes and why it is
// reproducible bit for bit is described in crop.cu.
#pragma once

#include "common.cuh"

namespace locc {
namespace {

constexpr int CAND_CAP = 256;
constexpr int NBINS = 64;  // d^2 histogram bins of the exact top-64 selection
constexpr int EBUF = 64;   // keys of the cut bin resolved by rank
constexpr unsigned FULL = 0xffffffffu;

// One compare-exchange stage between lanes (partner lane ^ lj) for all R
// registers; element e = lane * R + r sorts ascending where (e & k) == 0.
template <int R>
__device__ __forceinline__ void lane_stage(unsigned long long (&v)[R], int lane, int lj, int k) {
  const bool lower = (lane & lj) == 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const unsigned long long w = __shfl_xor_sync(FULL, v[r], lj);
    const bool asc = ((lane * R + r) & k) == 0;
    const unsigned long long lo = v[r] < w ? v[r] : w;
    const unsigned long long hi = v[r] < w ? w : v[r];
    v[r] = (lower == asc) ? lo : hi;
  }
}

// One compare-exchange stage inside a lane between registers r and r | J.
template <int R, int J>
__device__ __forceinline__ void reg_stage(unsigned long long (&v)[R], int lane, int k) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if ((r & J) == 0) {
      const int r2 = r | J;
      const bool asc = ((lane * R + r) & k) == 0;
      const unsigned long long a = v[r], b = v[r2];
      const bool sw = asc ? (a > b) : (a < b);
      v[r] = sw ? b : a;
      v[r2] = sw ? a : b;
    }
  }
}

// Sort the first n keys of buf ascending in place (n <= 32 R; slots n.. become
// ~0): bitonic network over N = 32 R keys, R per lane (element
// e = lane * R + r).  Stage loops stay rolled and the function is not inlined,
// so each size exists once in the binary (instruction-cache footprint).
template <int R>
__device__ __noinline__ void sort_list(unsigned long long* buf, int n, int lane) {
  constexpr int N = 32 * R;
  unsigned long long v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = lane * R + r;
    v[r] = e < n ? buf[e] : ~0ull;
  }
#pragma unroll 1
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= R) {
        lane_stage<R>(v, lane, j / R, k);
      } else if (j == 4) {
        if constexpr (R > 4) reg_stage<R, 4>(v, lane, k);
      } else if (j == 2) {
        if constexpr (R > 2) reg_stage<R, 2>(v, lane, k);
      } else {
        reg_stage<R, 1>(v, lane, k);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r) buf[lane * R + r] = v[r];
  __syncwarp();
}

__device__ __forceinline__ void sort_any(unsigned long long* buf, int n, int lane) {
  if (n <= 64) sort_list<2>(buf, n, lane);
  else if (n <= 128) sort_list<4>(buf, n, lane);
  else sort_list<8>(buf, n, lane);
}

struct Frame {
  float rrel[9];
  float c[3];   // crop centre, A frame
  float cb[3];  // crop centre, B frame
};

__device__ __forceinline__ void pair_frame(const float* pa, const float* pb,
                                           float4 alo, float4 ahi, float4 blo,
                                           float4 bhi, Frame& f) {
  float RA[9], RB[9];
  quat_to_rot(pa, RA);
  quat_to_rot(pb, RB);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      f.rrel[3 * i + j] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], RB[j], RB[3 + j], RB[6 + j]);
  const float dt0 = fsub(pb[4], pa[4]), dt1 = fsub(pb[5], pa[5]), dt2 = fsub(pb[6], pa[6]);
  float trel[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) trel[i] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], dt0, dt1, dt2);
  const float bl[3] = {blo.x, blo.y, blo.z}, bh[3] = {bhi.x, bhi.y, bhi.z};
  const float al[3] = {alo.x, alo.y, alo.z}, ah[3] = {ahi.x, ahi.y, ahi.z};
  float cbx[3], hbx[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    cbx[j] = fmul(fadd(bl[j], bh[j]), 0.5f);
    hbx[j] = fmul(fsub(bh[j], bl[j]), 0.5f);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float* r = f.rrel + 3 * i;
    const float c = fadd(dot3_rn(r[0], r[1], r[2], cbx[0], cbx[1], cbx[2]), trel[i]);
    const float h = dot3_rn(fabsf(r[0]), fabsf(r[1]), fabsf(r[2]), hbx[0], hbx[1], hbx[2]);
    const float lo = fsub(c, h), hi = fadd(c, h);
    const float a = fmaxf(al[i], lo);
    const float b = fminf(ah[i], hi);
    f.c[i] = fmul(fadd(a, b), 0.5f);
  }
  const float e0 = fsub(f.c[0], trel[0]), e1 = fsub(f.c[1], trel[1]), e2 = fsub(f.c[2], trel[2]);
#pragma unroll
  for (int j = 0; j < 3; ++j)
    f.cb[j] = dot3_rn(f.rrel[j], f.rrel[3 + j], f.rrel[6 + j], e0, e1, e2);
}

__device__ __forceinline__ float box_dist2(float4 lo, float4 hi, float cx, float cy, float cz) {
  const float dx = fmaxf(fmaxf(lo.x - cx, cx - hi.x), 0.0f);
  const float dy = fmaxf(fmaxf(lo.y - cy, cy - hi.y), 0.0f);
  const float dz = fmaxf(fmaxf(lo.z - cz, cz - hi.z), 0.0f);
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ float point_d2(float4 q, float cx, float cy, float cz) {
  const float d0 = fsub(q.x, cx), d1 = fsub(q.y, cy), d2 = fsub(q.z, cz);
  float s = fmul(d0, d0);
  s = fadd(s, fmul(d1, d1));
  return fadd(s, fmul(d2, d2));
}

// Selection key: d^2 bits (non-negative floats order as their bit patterns),
// then the sample's library index (ties go to the lower index), then its
// storage position (to find the point again).
__device__ __forceinline__ unsigned long long make_key(float s, float4 q, int pos) {
  return ((unsigned long long)__float_as_uint(s) << 32) |
         ((unsigned long long)(__float_as_uint(q.w) & 0xffffu) << 16) | (unsigned)pos;
}

__device__ __forceinline__ int d2_bin(float s, float inv_w) {
  return min(NBINS - 1, (int)fmul(s, inv_w));
}

__device__ __forceinline__ int key_bin(unsigned long long key, float inv_w) {
  return d2_bin(__uint_as_float((unsigned)(key >> 32)), inv_w);
}

// The first bin b* at which the cumulative histogram count reaches KMAX
// (requires a total above KMAX) and the count of the bins below it.
__device__ __forceinline__ void cut_bin(const int* hist, int lane, int* bstar, int* below) {
  const int h0 = hist[2 * lane], h1 = hist[2 * lane + 1];
  int c = h0 + h1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, c, o);
    if (lane >= o) c += t;
  }
  const int L = __ffs(__ballot_sync(FULL, c >= KMAX)) - 1;
  const int cL = __shfl_sync(FULL, c, L), h0L = __shfl_sync(FULL, h0, L),
            h1L = __shfl_sync(FULL, h1, L);
  const int excl = cL - h0L - h1L;
  if (excl + h0L >= KMAX) {
    *bstar = 2 * L;
    *below = excl;
  } else {
    *bstar = 2 * L + 1;
    *below = excl + h0L;
  }
}

// Histogram of the d^2 bins of buf[0, n) (NBINS counters in shared memory).
__device__ __forceinline__ void bin_histogram(const unsigned long long* buf, int n, float inv_w,
                                              int* hist, int lane) {
  hist[lane] = 0;
  hist[lane + 32] = 0;
  __syncwarp();
  for (int j = lane; j < n; j += 32) atomicAdd(&hist[key_bin(buf[j], inv_w)], 1);
  __syncwarp();
}

// Keep the keys of buf[0, n) whose bin is below `lim`, in order; returns
// their number.
__device__ __forceinline__ int keep_bins_below(unsigned long long* buf, int n, float inv_w, int lim,
                                               int lane) {
  const unsigned lt = (1u << lane) - 1u;
  int w = 0;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const unsigned long long key = j < n ? buf[j] : ~0ull;
    const bool keep = j < n && key_bin(key, inv_w) < lim;
    const unsigned km = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) buf[w + __popc(km & lt)] = key;
    w += __popc(km);
    __syncwarp();
  }
  return w;
}

// Keep the keys of buf[0, n) that are among the KMAX smallest: every key of
// a bin below b* (compacted in place, in list order) and then the `need`
// smallest keys of bin b* (rank selection over that bin's keys, which are
// unique).  buf must hold every in-ball key of bins <= b*.  Returns false when
// bin b* holds more than EBUF keys; buf is then partly overwritten and the
// caller defers the object.
__device__ __forceinline__ bool select_cut(unsigned long long* buf, int n, float inv_w, int bstar,
                                           int need, int lane, unsigned long long* ebuf) {
  const unsigned lt = (1u << lane) - 1u;
  int w = 0, m = 0;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const unsigned long long key = j < n ? buf[j] : ~0ull;
    const int bin = j < n ? key_bin(key, inv_w) : NBINS;
    const unsigned bm = __ballot_sync(FULL, bin < bstar);
    const unsigned am = __ballot_sync(FULL, bin == bstar);
    if (m + __popc(am) > EBUF) return false;
    __syncwarp();  // every lane has read its key before any is overwritten
    if (bin < bstar) buf[w + __popc(bm & lt)] = key;
    if (bin == bstar) ebuf[m + __popc(am & lt)] = key;
    w += __popc(bm);
    m += __popc(am);
    __syncwarp();
  }
  for (int e = lane; e < m; e += 32) {
    const unsigned long long k = ebuf[e];
    int rank = 0;
    for (int i = 0; i < m; ++i) rank += ebuf[i] < k;
    if (rank < need) buf[w + rank] = k;
  }
  __syncwarp();
  return true;
}

// Rows of one object crop: the points of the first cnt keys of buf in the
// canonical frame (A: p - c; B: R_rel (p - c_B)), w = 1; zeros beyond.
__device__ __forceinline__ void write_crop(const unsigned long long* buf, int cnt,
                                           const float4* pts, float cx, float cy, float cz,
                                           const float* R, float4* xo, int32_t* io, int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    int oi = -1;
    if (s < cnt) {
      const unsigned long long key = buf[s];
      const int pos = (int)(key & 0xffffu);
      oi = (int)((key >> 16) & 0xffffu);
      const float4 q = pts[pos];
      const float d0 = fsub(q.x, cx), d1 = fsub(q.y, cy), d2 = fsub(q.z, cz);
      if (!R) {
        o = make_float4(d0, d1, d2, 1.0f);
      } else {
        o = make_float4(dot3_rn(R[0], R[1], R[2], d0, d1, d2),
                        dot3_rn(R[3], R[4], R[5], d0, d1, d2),
                        dot3_rn(R[6], R[7], R[8], d0, d1, d2), 1.0f);
      }
    }
    xo[s] = o;
    if (io) io[s] = oi;
  }
}

// Selection for one object of pair p (obj 0 = A, 1 = B) about the crop
// centre (cx, cy, cz) in its body frame: on return buf[0, cnt) holds the keys
// of the chosen samples (in list order) and the count is returned; -1 when
// the object was deferred to the exact fallback (its code 2 p + obj is then
// in the defer list).
__device__ __forceinline__ int select_object(const DevLibrary& lib, int p, int obj, int shape,
                                             float cx, float cy, float cz, int lane, float r,
                                             unsigned long long* buf, int* hist,
                                             unsigned long long* ebuf, int* defer,
                                             int defer_cap) {
  const float r2 = fmul(r, r);
  const float r2_cull = r2 * 1.001f + 1e-30f;  // conservative block test
  const float4* pts = lib.points + (size_t)shape * lib.n_pad;
  const float4* blk = lib.blocks + (size_t)shape * lib.n_blocks * 2;
  const unsigned lt = (1u << lane) - 1u;  // lanes below this one
  int n = 0;      // keys in buf
  int n_in = 0;   // in-ball points seen
  const float inv_w = (float)NBINS / r2;
  // Keys of bins >= bcut cannot be among the KMAX smallest any more (the
  // bound only tightens while the pass runs).
  int bcut = NBINS;
  bool deferred = false;  // left to the exact fallback kernel
  // One pass over the culled blocks: the keys of in-ball points are appended
  // to buf in visiting order.  When buf fills up, its histogram of d^2 over
  // NBINS equal bins of [0, r^2] gives the first bin b' at which its
  // cumulative count reaches KMAX; bins are a monotone function of d^2, so no
  // key of a higher bin can be among the KMAX smallest: buf keeps the keys of
  // bins <= b' (in order), later keys of higher bins are skipped and blocks
  // whose box lies beyond bin b' are no longer loaded.  If even that leaves no
  // room (one bin holding most keys), the object is deferred.
  float lim2 = r2_cull;  // blocks farther than this hold no key that can still matter
  for (int bg = 0; bg < lib.n_blocks && !deferred; bg += 32) {
    const int bi = bg + lane;
    const float bd2 =
        bi < lib.n_blocks ? box_dist2(blk[2 * bi], blk[2 * bi + 1], cx, cy, cz) : INFINITY;
    unsigned mask = __ballot_sync(FULL, bd2 <= lim2);
    while (mask && !deferred) {
      // four blocks per round: all four loads are in flight together (two
      // per round at 20 CTAs/SM was 2 % slower than four at 16)
      int posu[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        posu[u] = mask ? (bg + __ffs(mask) - 1) * BLOCK_PTS + lane : -1;
        if (mask) mask &= mask - 1;
      }
      float4 qu[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) qu[u] = pts[posu[u] >= 0 ? posu[u] : posu[0]];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int pos = posu[u];
        if (pos < 0 || deferred) break;
        const float4 q = qu[u];
        const float s = point_d2(q, cx, cy, cz);
        const bool in = s <= r2;
        const unsigned im = __ballot_sync(FULL, in);
        n_in += __popc(im);
        // the bins matter only once the list has overflowed (bcut < NBINS,
        // warp-uniform): until then every in-ball key is taken
        unsigned tm = im;
        if (bcut < NBINS) tm = __ballot_sync(FULL, in && d2_bin(s, inv_w) < bcut);
        if (tm == 0) continue;
        bool take = (tm >> lane) & 1u;
        if (n + __popc(tm) > CAND_CAP) {
          int below;
          bin_histogram(buf, n, inv_w, hist, lane);
          cut_bin(hist, lane, &bcut, &below);
          n = keep_bins_below(buf, n, inv_w, bcut + 1, lane);
          bcut += 1;
          // a key of bin >= bcut has d^2 >= bcut / inv_w (up to rounding):
          // skip the blocks whose box lies farther (with a safety margin)
          lim2 = fminf(lim2, (float)bcut / inv_w * 1.001f + 1e-30f);
          mask &= __ballot_sync(FULL, bd2 <= lim2);
          take = take && d2_bin(s, inv_w) < bcut;
          tm = __ballot_sync(FULL, take);
          if (n + __popc(tm) > CAND_CAP) {
            deferred = true;
            break;
          }
        }
        if (take) buf[n + __popc(tm & lt)] = make_key(s, q, pos);
        n += __popc(tm);
      }
    }
  }
  __syncwarp();
  int cnt = n_in;  // n_in <= KMAX: every in-ball point is in buf, nothing to choose
  if (!deferred && n_in > KMAX) {
    cnt = KMAX;
    // buf holds every in-ball key of the bins that can still matter; the
    // histogram of buf gives the bin b* that holds the KMAX-th smallest key:
    // every key of a lower bin is kept, and rank selection among the few
    // keys of bin b* picks the rest
    int bstar, below;
    bin_histogram(buf, n, inv_w, hist, lane);
    cut_bin(hist, lane, &bstar, &below);
    deferred = !select_cut(buf, n, inv_w, bstar, KMAX - below, lane, ebuf);
  }
  if (deferred) {
    // rare: one d^2 bin holds more keys than the list or the rank buffer;
    // crop_fallback_kernel redoes this object with an exact streaming sort
    if (lane == 0) {
      const int slot = atomicAdd(defer, 1);
      if (slot < defer_cap) defer[2 + slot] = 2 * p + obj;
    }
    return -1;
  }
  __syncwarp();
  return cnt;
}

}  // namespace
}  // namespace locc

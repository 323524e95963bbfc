// Crop gather: pose composition, crop centre and nearest-first selection of
// each object's surface points inside the crop ball (steps 1-3 of the path).
//
// Paper: Sec. III (collision predictor: "create the OBB of shape embeddings of
// two objects by using their poses ... select the features in colliding
// cells"), appendix ("identify the intersection region of two AABB").  The
// crop centre is the centre of A's body box intersected with B's posed box
// seen as an axis-aligned box of A's frame; each object keeps at most 64 of
// its surface samples inside the ball of radius r about that centre, nearest
// first, ties to the lower sample index, expressed in the canonical crop frame
// (A's body axes, origin at the centre).
//
// Design (CTAs of two warps; each warp takes whole pairs from a device
// counter and crops object A, then object B):
//   * every float32 operation of the selection uses an explicit round-to-
//     nearest intrinsic in a fixed order, so index sets are reproducible bit
//     for bit on any IEEE-754 machine that performs the same operations;
//   * the library keeps each shape's samples in Morton-ordered blocks of 32
//     with a bounding box per block; a warp first tests the ball against the
//     block boxes (conservatively) and streams only the blocks that may hold
//     in-ball points, one coalesced 512-byte float4 load per block;
//   * in-ball points become 64-bit keys (d^2 bits, sample index, storage
//     position) and are appended to a per-warp shared-memory list by ballot +
//     popc compaction, in one pass over the culled blocks (four block loads in
//     flight per round);
//   * at most 64 in-ball points: all are kept, nothing is sorted;
//   * more: a 64-bin histogram of d^2 over [0, r^2] built from the list gives
//     the bin b* that holds the 64th smallest key; every key of a lower bin is
//     kept, and rank selection among the few keys of bin b* picks the rest
//     (exact: the bin is a monotone function of d^2, keys are unique);
//   * when the list fills up during the pass, the same histogram bounds the
//     bins that can still matter: the list keeps those bins and later keys of
//     higher bins are skipped; only if one bin alone overflows the list is it
//     sorted and cut to its 64 smallest keys (an exact streaming top-64);
//   * the kept keys are written in list order (storage order), the chosen
//     keys of bin b* last; the order is not part of the result: the encoder
//     max-pools over points.
#include <algorithm>

#include "crop_dev.cuh"

namespace locc {
namespace {

// Crop of one object of pair p (obj 0 = A, 1 = B) about the crop centre
// (cx, cy, cz) in its body frame; R (shared memory) = R_rel for B, null for A.
// Returns the count, -1 when the object was deferred.
__device__ __forceinline__ int crop_object(const DevLibrary& lib, int p, int obj, int shape,
                                            float cx, float cy, float cz, const float* R, int lane,
                                            float r, float4* __restrict__ xyz_out,
                                            int32_t* __restrict__ idx_out,
                                            int32_t* __restrict__ cnt_out,
                                            unsigned long long* buf, int* hist,
                                            unsigned long long* ebuf, int* defer, int defer_cap) {
  const int cnt = select_object(lib, p, obj, shape, cx, cy, cz, lane, r, buf, hist, ebuf, defer,
                                defer_cap);
  if (cnt < 0) return -1;
  write_crop(buf, cnt, lib.points + (size_t)shape * lib.n_pad, cx, cy, cz, R,
             xyz_out + ((size_t)p * 2 + obj) * KMAX,
             idx_out ? idx_out + ((size_t)p * 2 + obj) * KMAX : nullptr, lane);
  if (lane == 0) cnt_out[2 * p + obj] = cnt;
  __syncwarp();
  return cnt;
}

// Object list of the tensor-core encoders (list[0, *list_n) = 2 p + side of
// the objects with non-empty crops, any order): one atomic per call.
__device__ __forceinline__ void list_objects(int* list, int* list_n, int p, bool a, bool b) {
  const int k = (int)a + (int)b;
  if (k == 0) return;
  const int base = atomicAdd(list_n, k);
  if (a) list[base] = 2 * p;
  if (b) list[base + (int)a] = 2 * p + 1;
}

// Both objects of pair p, one after the other on one warp: the pair's frame
// (two rotations, the relative pose, the crop centre in both body frames) is
// computed once.  R_rel and both centres wait in shared memory, so that they
// hold no registers through the selections.
__device__ __forceinline__ void crop_pair(const DevLibrary& lib, const PairInputs& in, int p,
                                          int lane,
                                          float r, float4* __restrict__ xyz_out,
                                          int32_t* __restrict__ idx_out,
                                          int32_t* __restrict__ cnt_out,
                                          float4* __restrict__ centre_out, int* __restrict__ err,
                                          unsigned long long* buf, int* hist,
                                          unsigned long long* ebuf, float* rsh, int* defer,
                                          int defer_cap, int* list, int* list_n) {
  int a, b, sa, sb;
  const bool ok = load_pair(in, lib.n_shapes, p, &a, &b, &sa, &sb, lane == 0 ? err : nullptr);
  if (!ok) {
    const float nan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int obj = 0; obj < 2; ++obj) {
      float4* xo = xyz_out + ((size_t)p * 2 + obj) * KMAX;
      int32_t* io = idx_out ? idx_out + ((size_t)p * 2 + obj) * KMAX : nullptr;
      xo[lane] = xo[lane + 32] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (io) io[lane] = io[lane + 32] = -1;
      if (lane == 0) cnt_out[2 * p + obj] = 0;
    }
    if (lane == 0 && centre_out) centre_out[p] = make_float4(nan, nan, nan, nan);
    return;
  }
  {
    Frame f;
    pair_frame(in.poses + 7 * (size_t)a, in.poses + 7 * (size_t)b, lib.aabb[2 * sa],
               lib.aabb[2 * sa + 1], lib.aabb[2 * sb], lib.aabb[2 * sb + 1], f);
    if (lane == 0) {
      if (centre_out) centre_out[p] = make_float4(f.c[0], f.c[1], f.c[2], 0.f);
#pragma unroll
      for (int i = 0; i < 9; ++i) rsh[i] = f.rrel[i];
      rsh[9] = f.c[0];
      rsh[10] = f.c[1];
      rsh[11] = f.c[2];
      rsh[12] = f.cb[0];
      rsh[13] = f.cb[1];
      rsh[14] = f.cb[2];
    }
  }
  __syncwarp();
  // one call site: the selection code exists once in the binary
  int c0 = 0, c1 = 0;
#pragma unroll 1
  for (int obj = 0; obj < 2; ++obj) {
    const float* c = rsh + 9 + 3 * obj;
    const int cnt = crop_object(lib, p, obj, obj ? sb : sa, c[0], c[1], c[2], obj ? rsh : nullptr,
                                lane, r, xyz_out, idx_out, cnt_out, buf, hist, ebuf, defer,
                                defer_cap);
    if (obj) c1 = cnt;
    else c0 = cnt;
  }
  // deferred objects (-1) are listed by the fallback kernel
  if (list && lane == 0) list_objects(list, list_n, p, c0 > 0, c1 > 0);
}

// Exact fallback for the objects crop_kernel deferred: the classic streaming
// top-KMAX -- keys collected into the list, and whenever it is full it is
// sorted and cut to its KMAX smallest keys, whose largest bounds later keys.
__device__ __forceinline__ void fallback_object(const DevLibrary& lib, const PairInputs& in, int p,
                                                int obj, int lane, float r,
                                                float4* __restrict__ xyz_out,
                                                int32_t* __restrict__ idx_out,
                                                int32_t* __restrict__ cnt_out,
                                                unsigned long long* buf, int* list, int* list_n) {
  int a, b, sa, sb;
  if (!load_pair(in, lib.n_shapes, p, &a, &b, &sa, &sb, nullptr)) return;
  Frame f;
  pair_frame(in.poses + 7 * (size_t)a, in.poses + 7 * (size_t)b, lib.aabb[2 * sa],
             lib.aabb[2 * sa + 1], lib.aabb[2 * sb], lib.aabb[2 * sb + 1], f);
  const int shape = obj == 0 ? sa : sb;
  const float cx = obj == 0 ? f.c[0] : f.cb[0];
  const float cy = obj == 0 ? f.c[1] : f.cb[1];
  const float cz = obj == 0 ? f.c[2] : f.cb[2];
  const float r2 = fmul(r, r);
  const float r2_cull = r2 * 1.001f + 1e-30f;
  const float4* pts = lib.points + (size_t)shape * lib.n_pad;
  const float4* blk = lib.blocks + (size_t)shape * lib.n_blocks * 2;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long bound = ~0ull;
  int n = 0, n_in = 0;
  for (int bg = 0; bg < lib.n_blocks; bg += 32) {
    const int bi = bg + lane;
    bool hit = false;
    if (bi < lib.n_blocks) hit = box_dist2(blk[2 * bi], blk[2 * bi + 1], cx, cy, cz) <= r2_cull;
    unsigned mask = __ballot_sync(FULL, hit);
    while (mask) {
      const int pos = (bg + __ffs(mask) - 1) * BLOCK_PTS + lane;
      mask &= mask - 1;
      const float4 q = pts[pos];
      const float s = point_d2(q, cx, cy, cz);
      const bool in = s <= r2;
      n_in += __popc(__ballot_sync(FULL, in));
      const unsigned long long key = make_key(s, q, pos);
      bool take = in && key < bound;
      unsigned tm = __ballot_sync(FULL, take);
      if (tm == 0) continue;
      if (n + __popc(tm) > CAND_CAP) {
        sort_list<8>(buf, n, lane);
        n = KMAX;
        bound = buf[KMAX - 1];
        take = take && key < bound;
        tm = __ballot_sync(FULL, take);
      }
      if (take) buf[n + __popc(tm & lt)] = key;
      n += __popc(tm);
      __syncwarp();
    }
  }
  __syncwarp();
  sort_any(buf, n, lane);
  const int cnt = n_in < KMAX ? n_in : KMAX;
  write_crop(buf, cnt, pts, cx, cy, cz, obj == 1 ? f.rrel : nullptr,
             xyz_out + ((size_t)p * 2 + obj) * KMAX,
             idx_out ? idx_out + ((size_t)p * 2 + obj) * KMAX : nullptr, lane);
  if (lane == 0) cnt_out[2 * p + obj] = cnt;
  if (list && lane == 0 && cnt > 0) list[atomicAdd(list_n, 1)] = 2 * p + obj;
  __syncwarp();
}

__global__ void __launch_bounds__(64, 16) crop_kernel(DevLibrary lib, PairInputs in, PairRange rg,
                                                      float r, float4* __restrict__ xyz_out,
                                                      int32_t* __restrict__ idx_out,
                                                      int32_t* __restrict__ cnt_out,
                                                      float4* __restrict__ centre_out,
                                                      int* __restrict__ err, int* __restrict__ defer,
                                                      int defer_cap, int* __restrict__ list,
                                                      int* __restrict__ list_n) {
  __shared__ unsigned long long cand[2][CAND_CAP];
  __shared__ unsigned long long ebuf[2][EBUF];
  __shared__ int hist[2][NBINS];
  __shared__ float rsh[2][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  // Pairs are handed out one at a time: the first of every warp statically,
  // the rest from a counter (defer[1], zeroed before the launch).  Per-pair
  // costs are heavy-tailed (culled blocks and in-ball points vary with the
  // overlap), so a static split leaves most warps idle while the unluckiest
  // finish; with the counter all warps stop within about one pair of each
  // other.  The next index is fetched while the current pair runs.
  const int n_pairs = hi - lo;
  const int first = 2 * (int)gridDim.x;
  int* lbase = list ? list + 2 * (size_t)lo : nullptr;  // this chunk's part of the list
  int* lcnt = list ? list_n + rg.chunk : nullptr;
  int pr = 2 * (int)blockIdx.x + warp;
  while (pr < n_pairs) {
    int nxt = 0;
    if (lane == 0) nxt = first + atomicAdd(&defer[1], 1);
    crop_pair(lib, in, lo + pr, lane, r, xyz_out, idx_out, cnt_out, centre_out, err, cand[warp],
              hist[warp], ebuf[warp], rsh[warp], defer, defer_cap, lbase, lcnt);
    pr = __shfl_sync(FULL, nxt, 0);
  }
}

// One warp per deferred object (defer[0] = count, defer[2 + i] = 2 p + object).
__global__ void __launch_bounds__(64) crop_fallback_kernel(DevLibrary lib, PairInputs in, float r,
                                                           PairRange rg,
                                                           float4* __restrict__ xyz_out,
                                                           int32_t* __restrict__ idx_out,
                                                           int32_t* __restrict__ cnt_out,
                                                           const int* __restrict__ defer,
                                                           int defer_cap, int* __restrict__ list,
                                                           int* __restrict__ list_n) {
  __shared__ unsigned long long cand[2][CAND_CAP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = min(defer[0], defer_cap);
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  int* lbase = list ? list + 2 * (size_t)lo : nullptr;
  int* lcnt = list ? list_n + rg.chunk : nullptr;
  for (int e = 2 * blockIdx.x + warp; e < n; e += 2 * gridDim.x) {
    const int code = defer[2 + e];
    fallback_object(lib, in, code >> 1, code & 1, lane, r, xyz_out, idx_out, cnt_out, cand[warp],
                    lbase, lcnt);
  }
}

// Global crops (the ablation without locality): each object keeps its first
// KMAX surface samples -- an area-uniform subset of the whole surface -- in
// the same canonical frame as the local crop (A's body axes, origin at the
// crop centre).  One CTA of two warps (A, B) per pair.
__global__ void __launch_bounds__(64)
    crop_global_kernel(DevLibrary lib, PairInputs in, PairRange rg, float4* __restrict__ xyz_out,
                       int32_t* __restrict__ idx_out, int32_t* __restrict__ cnt_out,
                       float4* __restrict__ centre_out, int* __restrict__ err) {
  __shared__ unsigned long long keys[2][KMAX];
  __shared__ float rsh[9];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int lo, hi;
  range_bounds(rg, &lo, &hi);
  for (int p = lo + blockIdx.x; p < hi; p += gridDim.x) {
    int a, b, sa, sb;
    const bool ok =
        load_pair(in, lib.n_shapes, p, &a, &b, &sa, &sb, (warp == 0 && lane == 0) ? err : nullptr);
    float4* xo = xyz_out + ((size_t)p * 2 + warp) * KMAX;
    int32_t* io = idx_out ? idx_out + ((size_t)p * 2 + warp) * KMAX : nullptr;
    if (!ok) {
      const float nan = __int_as_float(0x7fc00000);
      xo[lane] = xo[lane + 32] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (io) io[lane] = io[lane + 32] = -1;
      if (lane == 0) cnt_out[2 * p + warp] = 0;
      if (warp == 0 && lane == 0 && centre_out) centre_out[p] = make_float4(nan, nan, nan, nan);
      __syncthreads();
      continue;
    }
    Frame f;
    pair_frame(in.poses + 7 * (size_t)a, in.poses + 7 * (size_t)b, lib.aabb[2 * sa],
               lib.aabb[2 * sa + 1], lib.aabb[2 * sb], lib.aabb[2 * sb + 1], f);
    if (warp == 0 && lane == 0 && centre_out) centre_out[p] = make_float4(f.c[0], f.c[1], f.c[2], 0.f);
    if (warp == 1 && lane == 0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) rsh[i] = f.rrel[i];
    }
    const int shape = warp == 0 ? sa : sb;
    const int cnt = min(KMAX, lib.n_points);
    for (int k = lane; k < cnt; k += 32) {
      const int pos = lib.inv[(size_t)shape * lib.n_points + k];
      keys[warp][k] = ((unsigned long long)k << 16) | (unsigned long long)pos;
    }
    __syncthreads();
    write_crop(keys[warp], cnt, lib.points + (size_t)shape * lib.n_pad, warp == 0 ? f.c[0] : f.cb[0],
               warp == 0 ? f.c[1] : f.cb[1], warp == 0 ? f.c[2] : f.cb[2], warp == 1 ? rsh : nullptr,
               xo, io, lane);
    if (lane == 0) cnt_out[2 * p + warp] = cnt;
    __syncthreads();
  }
}

constexpr int kMaxDevices = 64;
// resident crop CTAs per SM, per device (set by prepare_crop_kernels)
int g_crop_per_sm[kMaxDevices] = {};

}  // namespace

cudaError_t prepare_crop_kernels(int device) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, crop_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, crop_fallback_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, crop_global_kernel);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crop_kernel, 64, 0);
  if (e != cudaSuccess) return e;
  g_crop_per_sm[device] = per_sm < 1 ? 1 : per_sm;
  return cudaSuccess;
}

cudaError_t launch_crop_fallback(const DevLibrary& lib, const PairInputs& in, float r, float4* xyz,
                                 int32_t* cnt, int* defer, int defer_cap, int n_sm,
                                 cudaStream_t stream) {
  crop_fallback_kernel<<<n_sm, 64, 0, stream>>>(lib, in, r, whole_range(0, nullptr), xyz, nullptr,
                                                 cnt, defer, defer_cap, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_crop(const DevLibrary& lib, const PairInputs& in, const PairRange& rg, float r,
                        float4* xyz, int32_t* idx, int32_t* cnt, float4* centre, int* err,
                        int* defer, int n_sm, int grid_cap, cudaStream_t stream, int mode,
                        int* list, int* list_n) {
  if (in.n_pairs <= 0) return cudaSuccess;
  if (mode == LOCC_CROP_GLOBAL) {
    const int span = (in.n_pairs + rg.n_chunks - 1) / rg.n_chunks + 1;
    crop_global_kernel<<<std::max(1, std::min(span, 16 * n_sm)), 64, 0, stream>>>(
        lib, in, rg, xyz, idx, cnt, centre, err);
    return cudaGetLastError();
  }
  // one wave of resident CTAs (at most grid_cap per SM); each strides over its pairs
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = (dev >= 0 && dev < kMaxDevices) ? g_crop_per_sm[dev] : 0;
  if (per_sm < 1) per_sm = 1;
  const int cap = grid_cap > 0 ? std::min(grid_cap, per_sm) : per_sm;
  const int span = (in.n_pairs + rg.n_chunks - 1) / rg.n_chunks + 1;
  const int grid = std::max(1, std::min(span, n_sm * cap));
  const int defer_cap = 2 * (span - 1);  // both objects of every pair of one chunk
  cudaError_t e = cudaMemsetAsync(defer, 0, 2 * sizeof(int), stream);  // count, object counter
  if (e == cudaSuccess && list) e = cudaMemsetAsync(list_n + rg.chunk, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  crop_kernel<<<grid, 64, 0, stream>>>(lib, in, rg, r, xyz, idx, cnt, centre, err, defer,
                                       defer_cap, list, list_n);
  // a fixed grid that reads the count on the device (graph-capturable); it
  // finds nothing to do unless some object was deferred
  crop_fallback_kernel<<<n_sm, 64, 0, stream>>>(lib, in, r, rg, xyz, idx, cnt, defer, defer_cap,
                                                list, list_n);
  return cudaGetLastError();
}

}  // namespace locc

// Allocation-free contact detection (locc_detect_noalloc).
//
// Some callers may not allocate device memory at call time: a simulator that
// hands the whole of HBM to its own pool allocator at start-up, or a
// latency-critical control loop in which cudaMalloc / cudaFree (which can
// synchronise the device) are not allowed.  For them this entry point runs the
// same crop gather and float32 network kernels as locc_detect, but its
// per-call scratch lives in one file-scope __device__ array instead of
// buffers allocated by the handle.
//
// The array holds at most LOCC_NOALLOC_MAX_PAIRS pairs of scratch (about
// 4 MiB) and stays resident on every device that loads the library until the
// process exits.  locc_create looks up its device address (and so loads it)
// together with the kernels this entry point launches, so a detection call
// itself neither allocates nor loads anything.  All calls share the array, so
// two calls whose kernels overlap on a GPU (different streams, different
// handles or different host threads) corrupt each other's results; the
// caller must order them.  No scratch
// location has to start at zero: every call writes each byte it later reads.
#include <cstdio>

#include "handle.cuh"

namespace {

constexpr int kMaxPairs = LOCC_NOALLOC_MAX_PAIRS;
constexpr size_t kXyzBytes = (size_t)kMaxPairs * locc::ROWS * sizeof(float4);
constexpr size_t kFeatBytes = (size_t)kMaxPairs * 512 * sizeof(float);
constexpr size_t kCentreBytes = (size_t)kMaxPairs * sizeof(float4);
constexpr size_t kCntBytes = (size_t)kMaxPairs * 2 * sizeof(int32_t);
constexpr size_t kDeferBytes = (2 + (size_t)kMaxPairs * 2) * sizeof(int32_t);
constexpr size_t kScratchBytes = kXyzBytes + kFeatBytes + kCentreBytes + kCntBytes + kDeferBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

}  // namespace

namespace locc {

// Set-up, once per handle, from locc_create with the handle's device current.
// In host code `g_scratch` is only a host-side stand-in for the symbol, so
// the array's device address must come from cudaGetSymbolAddress with that
// device current.  Doing it here (not in the first detection call) also
// makes the runtime load this file's module -- and with it the array --
// while the caller can still allocate, so no detection call ever does.
int noalloc_prepare(locc_handle* h) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    set_error("cudaGetSymbolAddress of the allocation-free scratch array failed");
    return LOCC_ERR_CUDA;
  }
  h->noalloc_scratch = static_cast<unsigned char*>(p);
  return LOCC_OK;
}

}  // namespace locc

extern "C" int locc_detect_noalloc(locc_handle* h, const float* poses, const int32_t* obj_shape,
                                   int32_t n_obj, const int32_t* pairs, int32_t n_pairs,
                                   float* out, void* stream) {
  using namespace locc;
  if (!h) {
    set_error("locc_detect_noalloc: handle is NULL");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_pairs < 0 || n_obj < 0) {
    set_error("locc_detect_noalloc: negative size");
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_pairs > kMaxPairs) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "locc_detect_noalloc: n_pairs %d exceeds LOCC_NOALLOC_MAX_PAIRS (%d); split the "
                  "batch or use locc_detect",
                  (int)n_pairs, kMaxPairs);
    set_error(msg);
    return LOCC_ERR_INVALID_ARG;
  }
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !out) {
    set_error("locc_detect_noalloc: NULL array");
    return LOCC_ERR_INVALID_ARG;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
    cudaGetLastError();
    set_error("locc_detect_noalloc: the current device is not the handle's device");
    return LOCC_ERR_INVALID_ARG;
  }
  unsigned char* base = h->noalloc_scratch;
  if (!base) {
    set_error("locc_detect_noalloc: the handle has no scratch address (locc_create failed?)");
    return LOCC_ERR_INVALID_ARG;
  }
  float4* xyz = reinterpret_cast<float4*>(base);
  float* feat = reinterpret_cast<float*>(base + kXyzBytes);
  float4* centre = reinterpret_cast<float4*>(base + kXyzBytes + kFeatBytes);
  int32_t* cnt = reinterpret_cast<int32_t*>(base + kXyzBytes + kFeatBytes + kCentreBytes);
  int* defer = reinterpret_cast<int*>(base + kXyzBytes + kFeatBytes + kCentreBytes + kCntBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  const PairRange rg = whole_range(n_pairs, nullptr);
  cudaError_t e = launch_crop(dev_library(h), in, rg, h->radius, xyz, nullptr, cnt, centre,
                              h->d_err, defer, h->n_sm, 0, s, h->crop_mode);
  if (e == cudaSuccess) e = launch_encoder_fp32(xyz, rg, h->fp32, feat, h->n_sm, s);
  if (e == cudaSuccess)
    e = launch_head_fp32(feat, rg, h->fp32, &in, centre, out, nullptr, h->n_sm, s);
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    return LOCC_ERR_CUDA;
  }
  return LOCC_OK;
}

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
// process exits.  All calls share it, so two calls whose kernels overlap on a
// GPU (different streams, different handles or different host threads)
// corrupt each other's results; the caller must order them.  No scratch
// location has to start at zero: every call writes each byte it later reads.
#include <mutex>

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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device).
// In host code `g_scratch` is only a host-side stand-in for the symbol, so the
// address must come from cudaGetSymbolAddress with the device current.
int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    locc::set_error("locc_detect_noalloc: no usable current CUDA device");
    return LOCC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      locc::set_error("locc_detect_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return LOCC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LOCC_OK;
}

}  // namespace

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
    set_error("locc_detect_noalloc: n_pairs exceeds LOCC_NOALLOC_MAX_PAIRS (1024); split the "
              "batch or use locc_detect");
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
  unsigned char* base = nullptr;
  int st = scratch_for_current_device(&base);
  if (st) return st;
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

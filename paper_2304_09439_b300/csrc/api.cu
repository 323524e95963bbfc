// Host side of the C ABI declared in include/locc.h: handle, shape library and
// parameter upload, scratch management and the stream-ordered call sequence of
// the contact path.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "handle.cuh"

namespace {
// NVTX range for the duration of a scope: host-side markers of the entry
// points and stages for timeline profilers (no cost without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(LOCC_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Page-locked (pinned) host memory: copies can go straight between it and
// the device, without the handle's staging buffer.
bool is_pinned(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& host) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dptr), host.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

namespace locc {

void set_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

int ensure_capacity(locc_handle* h, int n_pairs, cudaStream_t stream) {
  if (n_pairs <= h->cap_pairs) return LOCC_OK;
  CUDA_TRY(cudaStreamSynchronize(stream));
  free_scratch(h);
  const size_t P = (size_t)std::max(n_pairs, 1024);
  if (cudaMalloc(&h->d_xyz, P * ROWS * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&h->d_cnt, P * 2 * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&h->d_centre, P * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&h->d_feat, P * 512 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->d_defer, (2 + 2 * P) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_feat_tc, (P + 127) / 128 * 128 * 512 * 2 * 2) != cudaSuccess ||
      cudaMalloc(&h->d_list, 2 * P * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_list_n, LOCC_MAX_CHUNKS * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_scratch(h);
    return fail(LOCC_ERR_OOM, "cannot allocate scratch for %d pairs", n_pairs);
  }
  h->cap_pairs = (int)P;
  return LOCC_OK;
}

void free_scratch(locc_handle* h) {
  cudaFree(h->d_xyz);
  cudaFree(h->d_cnt);
  cudaFree(h->d_centre);
  cudaFree(h->d_feat);
  cudaFree(h->d_defer);
  cudaFree(h->d_feat_tc);
  cudaFree(h->d_list);
  cudaFree(h->d_list_n);
  h->d_xyz = nullptr, h->d_cnt = nullptr, h->d_centre = nullptr, h->d_feat = nullptr;
  h->d_defer = nullptr, h->d_feat_tc = nullptr, h->d_list = nullptr, h->d_list_n = nullptr;
  h->cap_pairs = 0;
}

int ensure_env_capacity(locc_handle* h, int n_env, cudaStream_t stream) {
  if (n_env <= h->cap_env) return LOCC_OK;
  CUDA_TRY(cudaStreamSynchronize(stream));
  cudaFree(h->d_env_counts);
  h->d_env_counts = nullptr;
  h->cap_env = 0;
  if (cudaMalloc(&h->d_env_counts, (size_t)n_env * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return fail(LOCC_ERR_OOM, "cannot allocate broadphase scratch for %d environments", n_env);
  }
  h->cap_env = n_env;
  return LOCC_OK;
}

int ensure_stage(locc_handle* h, size_t need, cudaStream_t s) {
  if (need <= h->stage_bytes) return LOCC_OK;
  CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeHost(h->h_stage);
  cudaFree(h->d_stage);
  h->h_stage = nullptr, h->d_stage = nullptr, h->stage_bytes = 0;
  if (cudaMallocHost(&h->h_stage, need) != cudaSuccess || cudaMalloc(&h->d_stage, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(LOCC_ERR_OOM, "cannot allocate %zu staging bytes", need);
  }
  h->stage_bytes = need;
  return LOCC_OK;
}

DevLibrary dev_library(const locc_handle* h) {
  DevLibrary L;
  L.points = h->d_points;
  L.blocks = h->d_blocks;
  L.aabb = h->d_aabb;
  L.inv = h->d_inv;
  L.n_shapes = h->n_shapes;
  L.n_points = h->n_points;
  L.n_pad = h->n_pad;
  L.n_blocks = h->n_blocks;
  return L;
}

// Network on the crops in h->d_xyz (or `xyz`): feat -> y / out.
int run_network(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                const float4* centre, float* out, float* y_raw, float* feat_out,
                cudaStream_t stream, cudaEvent_t mid, int list_mode) {
  float* feat = feat_out ? feat_out : h->d_feat;
  switch (h->prec) {
    case LOCC_FP32:
      CUDA_TRY(launch_encoder_fp32(xyz, rg, h->fp32, feat, h->n_sm, stream));
      if (mid) CUDA_TRY(cudaEventRecord(mid, stream));
      CUDA_TRY(launch_head_fp32(feat, rg, h->fp32, in, centre, out, y_raw, h->n_sm, stream));
      return LOCC_OK;
    default:
      return run_network_tc(h, xyz, rg, in, centre, out, y_raw, feat_out, stream, mid, list_mode);
  }
}

int ensure_pipeline(locc_handle* h) {
  if (h->aux) return LOCC_OK;
  CUDA_TRY(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  for (int i = 0; i < LOCC_MAX_CHUNKS; ++i)
    CUDA_TRY(cudaEventCreateWithFlags(&h->ev_crop[i], cudaEventDisableTiming));
  return LOCC_OK;
}

// Crop gather and network for the pairs [0, n) (n = min(*n_dev, n_cap), or
// n_cap).  With h->n_chunks > 1 the range is cut into chunks: the crop of
// chunk i runs on `s`, the network of chunk i on h->aux after that crop, so
// the crop of chunk i + 1 overlaps the network of chunk i; the two streams
// fork from and join back into `s` (capturable in a CUDA graph).
int run_path(locc_handle* h, const PairInputs& in, int n_cap, const int* n_dev, float* out,
             cudaStream_t s) {
  int C = std::max(1, std::min(h->n_chunks, LOCC_MAX_CHUNKS));
  if (n_cap < 4096) C = 1;
  const bool prof = h->profiling;
  const DevLibrary lib = dev_library(h);
  h->prof_chunks = C;
  if (h->fused_warps > 0 && h->prec == LOCC_BF16 && h->crop_mode == LOCC_CROP_LOCAL) {
    // one launch crops and encodes; the rare deferred objects follow (exact
    // fallback crop, then the list-driven encoder), then the head
    h->prof_chunks = 1;
    const PairRange rg = whole_range(n_cap, n_dev);
    const int defer_cap = 2 * n_cap;
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_c0[0], s));
    {
      NvtxRange r("crop+encoder");
      CUDA_TRY(launch_fused(lib, in, rg, h->radius, h->d_cnt, h->d_centre, h->d_err, h->d_defer,
                            defer_cap, h->wtc_enc, static_cast<__nv_bfloat16*>(h->d_feat_tc),
                            h->n_sm, h->fused_warps, s));
    }
    if (prof) {
      CUDA_TRY(cudaEventRecord(h->ev_c1[0], s));
      CUDA_TRY(cudaEventRecord(h->ev_e0[0], s));
    }
    CUDA_TRY(launch_crop_fallback(lib, in, h->radius, h->d_xyz, h->d_cnt, h->d_defer, defer_cap,
                                  h->n_sm, s));
    int st = launch_encoder_list(h, h->d_xyz, rg, h->d_defer + 2, h->d_defer, 2, s);
    if (st) return st;
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_e1[0], s));
    NvtxRange r_net("head");
    st = launch_head_tc(h, rg, &in, h->d_centre, out, nullptr, s);
    if (st) return st;
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_h1[0], s));
    return LOCC_OK;
  }
  // the tensor-core encoders take the list of objects with non-empty crops:
  // local crops list them as they go, global crops through the list kernel.
  // The encoders zero the empty objects' features from the crop counts.
  const bool list_in_crop = h->prec != LOCC_FP32 && h->crop_mode == LOCC_CROP_LOCAL;
  int* list = list_in_crop ? h->d_list : nullptr;
  int* list_n = list_in_crop ? h->d_list_n : nullptr;
  const int list_mode = list_in_crop ? LIST_FROM_CROP : LIST_FROM_ROWS;
  if (C == 1) {
    const PairRange rg = whole_range(n_cap, n_dev);
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_c0[0], s));
    {
      NvtxRange r("crop");
      CUDA_TRY(launch_crop(lib, in, rg, h->radius, h->d_xyz, nullptr, h->d_cnt, h->d_centre,
                           h->d_err, h->d_defer, h->n_sm, h->crop_cap, s, h->crop_mode, list,
                           list_n));
    }
    if (prof) {
      CUDA_TRY(cudaEventRecord(h->ev_c1[0], s));
      CUDA_TRY(cudaEventRecord(h->ev_e0[0], s));
    }
    NvtxRange r_net("network");
    const int st = run_network(h, h->d_xyz, rg, &in, h->d_centre, out, nullptr, nullptr, s,
                               prof ? h->ev_e1[0] : nullptr, list_mode);
    if (st) return st;
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_h1[0], s));
    return LOCC_OK;
  }
  int st = ensure_pipeline(h);
  if (st) return st;
  CUDA_TRY(cudaEventRecord(h->ev_fork, s));
  CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
  for (int i = 0; i < C; ++i) {
    const PairRange rg{n_cap, n_dev, i, C};
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_c0[i], s));
    CUDA_TRY(launch_crop(lib, in, rg, h->radius, h->d_xyz, nullptr, h->d_cnt, h->d_centre, h->d_err,
                         h->d_defer, h->n_sm, h->crop_cap, s, h->crop_mode, list, list_n));
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_c1[i], s));
    CUDA_TRY(cudaEventRecord(h->ev_crop[i], s));
    CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_crop[i], 0));
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_e0[i], h->aux));
    st = run_network(h, h->d_xyz, rg, &in, h->d_centre, out, nullptr, nullptr, h->aux,
                     prof ? h->ev_e1[i] : nullptr, list_mode);
    if (st) return st;
    if (prof) CUDA_TRY(cudaEventRecord(h->ev_h1[i], h->aux));
  }
  CUDA_TRY(cudaEventRecord(h->ev_join, h->aux));
  CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
  return LOCC_OK;
}

}  // namespace locc

using namespace locc;

extern "C" {

const char* locc_last_error(void) { return g_err; }

int locc_create(const locc_shape_library* lib, const void* blob, size_t blob_bytes,
                float crop_radius, locc_precision prec, locc_handle** out) {
  if (!out) return fail(LOCC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!lib || !lib->points || !lib->aabb) return fail(LOCC_ERR_INVALID_ARG, "library is NULL");
  if (lib->n_shapes < 1 || lib->n_points < 1 || lib->n_points > 65536)
    return fail(LOCC_ERR_INVALID_ARG, "need n_shapes >= 1 and 1 <= n_points <= 65536");
  if (!(crop_radius > 0.0f) || !std::isfinite(crop_radius))
    return fail(LOCC_ERR_INVALID_ARG, "crop_radius must be finite and > 0");
  if (prec != LOCC_FP32 && prec != LOCC_BF16 && prec != LOCC_FP8)
    return fail(LOCC_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  std::vector<float> params;
  {
    int st = parse_weights(blob, blob_bytes, &params);
    if (st) return st;
  }
  locc_handle* h = new (std::nothrow) locc_handle();
  if (!h) return fail(LOCC_ERR_OOM, "host allocation failed");
  cudaGetDevice(&h->device);
  if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      h->n_sm <= 0) {
    cudaGetLastError();
    delete h;
    return fail(LOCC_ERR_CUDA, "no usable CUDA device");
  }
  h->n_shapes = lib->n_shapes;
  h->n_points = lib->n_points;
  h->n_pad = (lib->n_points + BLOCK_PTS - 1) / BLOCK_PTS * BLOCK_PTS;
  h->n_blocks = h->n_pad / BLOCK_PTS;
  h->radius = crop_radius;
  h->prec = prec;

  // shape library: Morton-ordered blocks of 32 samples with block boxes
  const size_t S = (size_t)h->n_shapes, NP = (size_t)h->n_points, NPAD = (size_t)h->n_pad;
  std::vector<float4> pts(S * NPAD), blocks(S * h->n_blocks * 2), aabb(S * 2);
  std::vector<int32_t> inv(S * NP);
  const float nanv = std::nanf("");
  std::vector<uint32_t> code(NP);
  std::vector<int> order(NP);
  for (size_t s = 0; s < S; ++s) {
    const float* P = lib->points + s * NP * 3;
    const float* B = lib->aabb + s * 6;
    aabb[2 * s] = make_float4(B[0], B[1], B[2], 0.f);
    aabb[2 * s + 1] = make_float4(B[3], B[4], B[5], 0.f);
    for (size_t i = 0; i < NP; ++i) {
      uint32_t c = 0;
      for (int a = 0; a < 3; ++a) {
        const float ext = B[3 + a] - B[a];
        float u = ext > 0 ? (P[3 * i + a] - B[a]) / ext : 0.f;
        u = std::min(std::max(u, 0.f), 1.f);
        c |= spread10((uint32_t)(u * 1023.0f)) << a;
      }
      code[i] = c;
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return code[x] < code[y]; });
    for (size_t k = 0; k < NP; ++k) inv[s * NP + order[k]] = (int32_t)k;
    for (size_t k = 0; k < NPAD; ++k) {
      float4 v;
      if (k < NP) {
        const int i = order[k];
        uint32_t bits = (uint32_t)i;
        float w;
        std::memcpy(&w, &bits, 4);
        v = make_float4(P[3 * i], P[3 * i + 1], P[3 * i + 2], w);
      } else {
        v = make_float4(nanv, nanv, nanv, 0.f);
      }
      pts[s * NPAD + k] = v;
    }
    for (int b = 0; b < h->n_blocks; ++b) {
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int k = b * BLOCK_PTS; k < (b + 1) * BLOCK_PTS && k < (int)NP; ++k) {
        const float4 v = pts[s * NPAD + k];
        const float c3[3] = {v.x, v.y, v.z};
        for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], c3[a]), hi[a] = std::max(hi[a], c3[a]);
      }
      blocks[(s * h->n_blocks + b) * 2] = make_float4(lo[0], lo[1], lo[2], 0.f);
      blocks[(s * h->n_blocks + b) * 2 + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
  int st = LOCC_OK;
  if (upload(&h->d_points, pts) != cudaSuccess || upload(&h->d_blocks, blocks) != cudaSuccess ||
      upload(&h->d_aabb, aabb) != cudaSuccess || upload(&h->d_inv, inv) != cudaSuccess) {
    st = fail(LOCC_ERR_OOM, "cannot upload the shape library: %s",
              cudaGetErrorString(cudaGetLastError()));
  }
  if (st == LOCC_OK) st = upload_params(h, params);
  if (st == LOCC_OK) {
    // per-device kernel set-up: shared-memory limits, module loads, the
    // allocation-free entry point's scratch address
    cudaError_t e = prepare_crop_kernels(h->device);
    if (e == cudaSuccess) e = prepare_fp32_kernels();
    if (e == cudaSuccess) e = prepare_tc_kernels();
    if (e == cudaSuccess) e = prepare_fp8_kernels();
    if (e == cudaSuccess) e = prepare_fused_kernels();
    if (e != cudaSuccess)
      st = fail(LOCC_ERR_CUDA, "kernel set-up failed: %s", cudaGetErrorString(e));
    if (st == LOCC_OK) st = noalloc_prepare(h);
  }
  if (st == LOCC_OK && cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess)
    st = fail(LOCC_ERR_OOM, "cannot allocate the error flag");
  if (st == LOCC_OK && cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess)
    st = fail(LOCC_ERR_CUDA, "cudaMemset failed");
  if (st != LOCC_OK) {
    locc_destroy(h);
    return st;
  }
  *out = h;
  return LOCC_OK;
}

int locc_set_precision(locc_handle* h, locc_precision prec) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (prec != LOCC_FP32 && prec != LOCC_BF16 && prec != LOCC_FP8)
    return fail(LOCC_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  h->prec = prec;
  return LOCC_OK;
}

int locc_reserve(locc_handle* h, int32_t max_pairs, int32_t max_envs) {
  if (!h || max_pairs < 0 || max_envs < 0) return fail(LOCC_ERR_INVALID_ARG, "bad handle or size");
  int st = ensure_capacity(h, max_pairs, nullptr);
  if (st) return st;
  return ensure_env_capacity(h, max_envs, nullptr);
}

int locc_step(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
              const int32_t* env_offsets, int32_t n_env, int32_t* pairs_out, int32_t* n_pairs_out,
              int32_t max_pairs, float* out, void* stream) {
  NvtxRange nvtx_range("locc_step");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_env < 0 || max_pairs < 0 || n_obj < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (!n_pairs_out) return fail(LOCC_ERR_INVALID_ARG, "n_pairs_out is NULL");
  if (n_env > 0 && (!poses || !obj_shape || !env_offsets))
    return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  if (max_pairs > 0 && (!pairs_out || !out)) return fail(LOCC_ERR_INVALID_ARG, "NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_capacity(h, max_pairs, s);
  if (st) return st;
  const bool prof = h->profiling;
  h->prof_chunks = 0;
  if (prof) CUDA_TRY(cudaEventRecord(h->ev_bp0, s));
  st = broadphase_run(h, poses, obj_shape, env_offsets, n_env, pairs_out, n_pairs_out, max_pairs, s);
  if (st) return st == LOCC_ERR_CUDA ? fail(st, "broadphase launch failed") : st;
  if (prof) CUDA_TRY(cudaEventRecord(h->ev_bp1, s));
  if (max_pairs > 0 && n_env > 0) {
    PairInputs in{poses, obj_shape, pairs_out, n_obj, max_pairs};
    st = run_path(h, in, max_pairs, n_pairs_out, out, s);
    if (st) return st;
  }
  if (prof) CUDA_TRY(cudaEventRecord(h->ev_end, s));
  return LOCC_OK;
}

int locc_profile(locc_handle* h, int enable) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (enable && !h->ev_bp0) {
    CUDA_TRY(cudaEventCreate(&h->ev_bp0));
    CUDA_TRY(cudaEventCreate(&h->ev_bp1));
    CUDA_TRY(cudaEventCreate(&h->ev_end));
    for (int i = 0; i < LOCC_MAX_CHUNKS; ++i) {
      CUDA_TRY(cudaEventCreate(&h->ev_c0[i]));
      CUDA_TRY(cudaEventCreate(&h->ev_c1[i]));
      CUDA_TRY(cudaEventCreate(&h->ev_e0[i]));
      CUDA_TRY(cudaEventCreate(&h->ev_e1[i]));
      CUDA_TRY(cudaEventCreate(&h->ev_h1[i]));
    }
  }
  h->profiling = enable != 0;
  h->prof_chunks = 0;
  return LOCC_OK;
}

int locc_stage_times(locc_handle* h, float* ms_out, int n) {
  if (!h || !ms_out || n < 0) return fail(LOCC_ERR_INVALID_ARG, "bad argument");
  if (!h->profiling || !h->ev_bp0) return fail(LOCC_ERR_INVALID_ARG, "profiling is off");
  CUDA_TRY(cudaEventSynchronize(h->ev_end));
  float t[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, x = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&t[0], h->ev_bp0, h->ev_bp1));
  for (int i = 0; i < h->prof_chunks; ++i) {
    CUDA_TRY(cudaEventElapsedTime(&x, h->ev_c0[i], h->ev_c1[i]));
    t[1] += x;
    CUDA_TRY(cudaEventElapsedTime(&x, h->ev_e0[i], h->ev_e1[i]));
    t[2] += x;
    CUDA_TRY(cudaEventElapsedTime(&x, h->ev_e1[i], h->ev_h1[i]));
    t[3] += x;
  }
  CUDA_TRY(cudaEventElapsedTime(&t[4], h->ev_bp0, h->ev_end));
  int k = 0;
  for (; k < n && k < 5; ++k) ms_out[k] = t[k];
  return k;
}

int locc_set_crop_mode(locc_handle* h, int32_t mode) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (mode != LOCC_CROP_LOCAL && mode != LOCC_CROP_GLOBAL)
    return fail(LOCC_ERR_INVALID_ARG, "crop mode must be LOCC_CROP_LOCAL or LOCC_CROP_GLOBAL");
  h->crop_mode = mode;
  return LOCC_OK;
}

int locc_set_pipeline(locc_handle* h, int32_t n_chunks, int32_t crop_ctas_per_sm) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_chunks == 0) {
    if (crop_ctas_per_sm != 6 && crop_ctas_per_sm != 8)
      return fail(LOCC_ERR_INVALID_ARG, "the fused launch takes 6 or 8 crop warps per CTA");
    h->n_chunks = 1;
    h->crop_cap = 0;
    h->fused_warps = crop_ctas_per_sm;
    return LOCC_OK;
  }
  if (n_chunks < 1 || n_chunks > LOCC_MAX_CHUNKS || crop_ctas_per_sm < 0)
    return fail(LOCC_ERR_INVALID_ARG, "n_chunks must be 0..%d, crop_ctas_per_sm >= 0",
                LOCC_MAX_CHUNKS);
  h->n_chunks = n_chunks;
  h->crop_cap = crop_ctas_per_sm;
  h->fused_warps = 0;
  return LOCC_OK;
}

int locc_autotune(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                  const int32_t* env_offsets, int32_t n_env, int32_t* pairs_out,
                  int32_t* n_pairs_out, int32_t max_pairs, float* out, int32_t reps,
                  int32_t* best_out, float* best_ms_out, void* stream) {
  if (!h || reps < 1) return fail(LOCC_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  // {0, w}: fused crop + encoder launch with w crop warps per CTA (BF16,
  // local crops); {c, cap}: separate kernels in c chunks, cap crop CTAs per SM
  static const int kChunks[] = {0, 1, 2, 4, 8};
  static const int kCaps[] = {0, 8, 6, 4};
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const bool prof = h->profiling;
  h->profiling = false;
  float best = 1e30f;
  int bc = h->fused_warps ? 0 : h->n_chunks, bp = h->fused_warps ? h->fused_warps : h->crop_cap;
  int st = LOCC_OK;
  const bool can_fuse = h->prec == LOCC_BF16 && h->crop_mode == LOCC_CROP_LOCAL;
  for (int c : kChunks) {
    for (int cap : kCaps) {
      if (c == 1 && cap != 0) continue;
      if (c == 0 && (!can_fuse || (cap != 8 && cap != 6))) continue;
      h->n_chunks = c == 0 ? 1 : c;
      h->crop_cap = c == 0 ? 0 : cap;
      h->fused_warps = c == 0 ? cap : 0;
      st = locc_step(h, poses, obj_shape, n_obj, env_offsets, n_env, pairs_out, n_pairs_out,
                     max_pairs, out, stream);  // warm-up
      if (st) break;
      float tot = 0.f;
      for (int r = 0; r < reps && st == LOCC_OK; ++r) {
        cudaEventRecord(e0, s);
        st = locc_step(h, poses, obj_shape, n_obj, env_offsets, n_env, pairs_out, n_pairs_out,
                       max_pairs, out, stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        tot += ms;
      }
      if (st) break;
      if (tot / reps < best) best = tot / reps, bc = c, bp = cap;
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->profiling = prof;
  h->n_chunks = bc == 0 ? 1 : bc;
  h->crop_cap = bc == 0 ? 0 : bp;
  h->fused_warps = bc == 0 ? bp : 0;
  if (st) return st;
  if (best_out) best_out[0] = bc, best_out[1] = bp;
  if (best_ms_out) *best_ms_out = best;
  return LOCC_OK;
}

int locc_step_host(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                   const int32_t* env_offsets, int32_t n_env, int32_t* pairs_out,
                   int32_t* n_pairs_out, int32_t max_pairs, float* out, void* stream) {
  NvtxRange nvtx_range("locc_step_host");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_env < 0 || max_pairs < 0 || n_obj < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (!n_pairs_out || (n_env > 0 && (!poses || !obj_shape || !env_offsets)) ||
      (max_pairs > 0 && (!pairs_out || !out)))
    return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_poses = (size_t)n_obj * 28, b_shape = (size_t)n_obj * 4;
  const size_t b_env = (size_t)(n_env + 1) * 4;
  const size_t b_pairs = (size_t)max_pairs * 8, b_out = (size_t)max_pairs * 32;
  const size_t o_shape = al(b_poses), o_env = o_shape + al(b_shape), in_bytes = o_env + al(b_env);
  const size_t o_cnt = in_bytes, o_pairs = o_cnt + 256, o_out = o_pairs + al(b_pairs);
  const size_t need = o_out + al(b_out);
  int st = ensure_stage(h, need, s);
  if (st) return st;
  char* hs = static_cast<char*>(h->h_stage);
  char* ds = static_cast<char*>(h->d_stage);
  if (is_pinned(poses) && is_pinned(obj_shape) && is_pinned(env_offsets)) {
    CUDA_TRY(cudaMemcpyAsync(ds, poses, b_poses, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ds + o_shape, obj_shape, b_shape, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ds + o_env, env_offsets, b_env, cudaMemcpyHostToDevice, s));
  } else {
    std::memcpy(hs, poses, b_poses);
    std::memcpy(hs + o_shape, obj_shape, b_shape);
    std::memcpy(hs + o_env, env_offsets, b_env);
    CUDA_TRY(cudaMemcpyAsync(ds, hs, in_bytes, cudaMemcpyHostToDevice, s));
  }
  st = locc_step(h, reinterpret_cast<float*>(ds), reinterpret_cast<int32_t*>(ds + o_shape), n_obj,
                 reinterpret_cast<int32_t*>(ds + o_env), n_env,
                 reinterpret_cast<int32_t*>(ds + o_pairs), reinterpret_cast<int32_t*>(ds + o_cnt),
                 max_pairs, reinterpret_cast<float*>(ds + o_out), stream);
  if (st) return st;
  CUDA_TRY(cudaMemcpyAsync(hs + o_cnt, ds + o_cnt, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int32_t n = 0;
  std::memcpy(&n, hs + o_cnt, 4);
  *n_pairs_out = n;
  const int32_t m = std::min(n, max_pairs);
  if (m > 0) {
    if (is_pinned(pairs_out) && is_pinned(out)) {
      CUDA_TRY(cudaMemcpyAsync(pairs_out, ds + o_pairs, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(out, ds + o_out, (size_t)m * 32, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    } else {
      CUDA_TRY(cudaMemcpyAsync(hs + o_pairs, ds + o_pairs, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(hs + o_out, ds + o_out, (size_t)m * 32, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      std::memcpy(pairs_out, hs + o_pairs, (size_t)m * 8);
      std::memcpy(out, hs + o_out, (size_t)m * 32);
    }
  }
  return LOCC_OK;
}

int locc_crop(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
              const int32_t* pairs, int32_t n_pairs, float* xyz_out, int32_t* idx_out,
              int32_t* cnt_out, float* centre_out, void* stream) {
  NvtxRange nvtx_range("locc_crop");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_pairs < 0 || n_obj < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !xyz_out || !cnt_out)
    return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  int st = ensure_capacity(h, n_pairs, (cudaStream_t)stream);  // fallback scratch
  if (st) return st;
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  CUDA_TRY(launch_crop(dev_library(h), in, whole_range(n_pairs, nullptr), h->radius,
                       reinterpret_cast<float4*>(xyz_out), idx_out, cnt_out,
                       reinterpret_cast<float4*>(centre_out), h->d_err, h->d_defer, h->n_sm, 0,
                       (cudaStream_t)stream, h->crop_mode));
  return LOCC_OK;
}

int locc_network(locc_handle* h, const float* xyz, int32_t n_pairs, float* y_out,
                 float* feat_out, void* stream) {
  NvtxRange nvtx_range("locc_network");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_pairs < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (n_pairs == 0) return LOCC_OK;
  if (!xyz || !y_out) return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_capacity(h, n_pairs, s);
  if (st) return st;
  return run_network(h, reinterpret_cast<const float4*>(xyz), whole_range(n_pairs, nullptr),
                     nullptr, nullptr, nullptr, y_out, feat_out, s, nullptr,
                     LIST_AND_COUNTS_FROM_ROWS);
}

int locc_detect(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                const int32_t* pairs, int32_t n_pairs, float* out, void* stream) {
  NvtxRange nvtx_range("locc_detect");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_pairs < 0 || n_obj < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !out) return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_capacity(h, n_pairs, s);
  if (st) return st;
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  const bool prof = h->profiling;
  h->prof_chunks = 0;
  if (prof) {
    CUDA_TRY(cudaEventRecord(h->ev_bp0, s));
    CUDA_TRY(cudaEventRecord(h->ev_bp1, s));
  }
  st = run_path(h, in, n_pairs, nullptr, out, s);
  if (st) return st;
  if (prof) CUDA_TRY(cudaEventRecord(h->ev_end, s));
  return LOCC_OK;
}

int locc_detect_host(locc_handle* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                     const int32_t* pairs, int32_t n_pairs, float* out, void* stream) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_pairs < 0 || n_obj < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !out) return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b_poses = (size_t)n_obj * 7 * 4, b_shape = (size_t)n_obj * 4;
  const size_t b_pairs = (size_t)n_pairs * 8, b_out = (size_t)n_pairs * 8 * 4;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t in_bytes = al(b_poses) + al(b_shape) + al(b_pairs);
  const size_t need = in_bytes + al(b_out);
  int st0 = ensure_stage(h, need, s);
  if (st0) return st0;
  char* hs = static_cast<char*>(h->h_stage);
  char* ds = static_cast<char*>(h->d_stage);
  if (is_pinned(poses) && is_pinned(obj_shape) && is_pinned(pairs)) {
    CUDA_TRY(cudaMemcpyAsync(ds, poses, b_poses, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ds + al(b_poses), obj_shape, b_shape, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ds + al(b_poses) + al(b_shape), pairs, b_pairs,
                             cudaMemcpyHostToDevice, s));
  } else {
    std::memcpy(hs, poses, b_poses);
    std::memcpy(hs + al(b_poses), obj_shape, b_shape);
    std::memcpy(hs + al(b_poses) + al(b_shape), pairs, b_pairs);
    CUDA_TRY(cudaMemcpyAsync(ds, hs, in_bytes, cudaMemcpyHostToDevice, s));
  }
  int st = locc_detect(h, reinterpret_cast<float*>(ds), reinterpret_cast<int32_t*>(ds + al(b_poses)),
                       n_obj, reinterpret_cast<int32_t*>(ds + al(b_poses) + al(b_shape)), n_pairs,
                       reinterpret_cast<float*>(ds + in_bytes), stream);
  if (st) return st;
  if (is_pinned(out)) {
    CUDA_TRY(cudaMemcpyAsync(out, ds + in_bytes, b_out, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    CUDA_TRY(cudaMemcpyAsync(hs + in_bytes, ds + in_bytes, b_out, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(out, hs + in_bytes, b_out);
  }
  return LOCC_OK;
}

int locc_broadphase(locc_handle* h, const float* poses, const int32_t* obj_shape,
                    const int32_t* env_offsets, int32_t n_env, int32_t* pairs_out,
                    int32_t* n_pairs_out, int32_t max_pairs, void* stream) {
  NvtxRange nvtx_range("locc_broadphase");
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_env < 0 || max_pairs < 0) return fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (!n_pairs_out) return fail(LOCC_ERR_INVALID_ARG, "n_pairs_out is NULL");
  if (n_env > 0 && (!poses || !obj_shape || !env_offsets || (max_pairs > 0 && !pairs_out)))
    return fail(LOCC_ERR_INVALID_ARG, "NULL array");
  const int st = broadphase_run(h, poses, obj_shape, env_offsets, n_env, pairs_out, n_pairs_out,
                                max_pairs, (cudaStream_t)stream);
  if (st == LOCC_ERR_CUDA) return fail(st, "broadphase launch failed");
  return st;
}

int locc_status(locc_handle* h, void* stream) {
  if (!h) return fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int flag = 0;
  CUDA_TRY(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
    if (flag & 2) return fail(LOCC_ERR_TIMEOUT, "a bounded device wait ran out");
    return fail(LOCC_ERR_BAD_INDEX, "a pair or shape index was out of range");
  }
  return LOCC_OK;
}

void locc_destroy(locc_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_scratch(h);
  free_params(h);
  cudaFree(h->d_points);
  cudaFree(h->d_blocks);
  cudaFree(h->d_inv);
  cudaFree(h->d_aabb);
  cudaFree(h->d_err);
  cudaFree(h->d_env_counts);
  cudaFree(h->d_stage);
  cudaFreeHost(h->h_stage);
  cudaEvent_t evs[] = {h->ev_fork, h->ev_join, h->ev_bp0, h->ev_bp1, h->ev_end};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < LOCC_MAX_CHUNKS; ++i) {
    cudaEvent_t ce[] = {h->ev_crop[i], h->ev_c0[i], h->ev_c1[i], h->ev_e0[i], h->ev_e1[i], h->ev_h1[i]};
    for (cudaEvent_t e : ce)
      if (e) cudaEventDestroy(e);
  }
  if (h->aux) cudaStreamDestroy(h->aux);
  delete h;
}

}  // extern "C"

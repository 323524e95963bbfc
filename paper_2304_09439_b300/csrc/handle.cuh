// The opaque detector handle and host-side helpers shared by the .cu files.
#pragma once

#include <vector>

#include "common.cuh"

constexpr int LOCC_MAX_CHUNKS = 16;

struct locc_handle {
  int device = 0;
  int n_sm = 1;
  int n_shapes = 0, n_points = 0, n_pad = 0, n_blocks = 0;
  float radius = 0.f;
  locc_precision prec = LOCC_FP32;
  // shape library (device)
  float4* d_points = nullptr;
  float4* d_blocks = nullptr;
  float4* d_aabb = nullptr;
  int32_t* d_inv = nullptr;  // [S][n_points]: storage position of each sample index
  int crop_mode = LOCC_CROP_LOCAL;
  // parameters (device): float32 W^T / b for the CUDA-core path
  float* d_w32 = nullptr;
  locc::Fp32Params fp32{};
  // parameters (device): tensor-core operand images and scales
  void* d_wtc = nullptr;
  size_t wtc_bytes = 0;
  const unsigned char* wtc_enc = nullptr;   // encoder image (W1 hi/lo, W2, W3, biases)
  const unsigned char* wtc_head = nullptr;  // head image (Wh3, biases, Wh1 / Wh2 K-chunks)
  void* d_wf8 = nullptr;                    // e4m3 images with per-channel scales
  const unsigned char* wf8_enc = nullptr;
  const unsigned char* wf8_head = nullptr;
  // per-call scratch (device), capacity cap_pairs
  int cap_pairs = 0;
  float4* d_xyz = nullptr;
  int32_t* d_cnt = nullptr;
  float4* d_centre = nullptr;
  float* d_feat = nullptr;
  int* d_defer = nullptr;  // crop objects left to the exact fallback kernel
  void* d_feat_tc = nullptr;  // pooled features in the head's operand tiles (bf16 hi/lo or e4m3)
  int* d_list = nullptr;      // [2 cap_pairs] objects with non-empty crops (tensor-core encoders)
  int* d_list_n = nullptr;    // [LOCC_MAX_CHUNKS] list length per pipeline chunk
  int* d_err = nullptr;
  // broadphase per-environment counts / offsets
  int32_t* d_env_counts = nullptr;
  int cap_env = 0;
  // staging for locc_detect_host
  void* h_stage = nullptr;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  // pipelining: the crop gather of chunk i + 1 (caller's stream) overlaps the
  // network of chunk i (aux stream); crop_cap limits the crop CTAs per SM so
  // that they fit beside a network CTA
  int n_chunks = 1;
  int crop_cap = 0;
  // BF16: crop gather and encoder in one fused launch with this many crop
  // warps per CTA (0 = separate kernels)
  int fused_warps = 0;
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_crop[LOCC_MAX_CHUNKS] = {};
  // stage timing (locc_profile): per chunk, crop start / end on the crop
  // stream, encoder start / end and head end on the network stream
  bool profiling = false;
  cudaEvent_t ev_bp0 = nullptr, ev_bp1 = nullptr, ev_end = nullptr;
  cudaEvent_t ev_c0[LOCC_MAX_CHUNKS] = {}, ev_c1[LOCC_MAX_CHUNKS] = {};
  cudaEvent_t ev_e0[LOCC_MAX_CHUNKS] = {}, ev_e1[LOCC_MAX_CHUNKS] = {}, ev_h1[LOCC_MAX_CHUNKS] = {};
  int prof_chunks = 0;
  // device address of the allocation-free entry point's static scratch array
  // on this handle's device (resolved by locc_create)
  unsigned char* noalloc_scratch = nullptr;
};

namespace locc {
void set_error(const char* msg);
int parse_weights(const void* blob, size_t bytes, std::vector<float>* params);
int upload_params(locc_handle* h, const std::vector<float>& params);
void free_params(locc_handle* h);
int ensure_capacity(locc_handle* h, int n_pairs, cudaStream_t stream);
void free_scratch(locc_handle* h);
int ensure_env_capacity(locc_handle* h, int n_env, cudaStream_t stream);
int ensure_stage(locc_handle* h, size_t need, cudaStream_t stream);
int broadphase_run(locc_handle* h, const float* poses, const int32_t* obj_shape,
                   const int32_t* env_offsets, int n_env, int32_t* pairs_out,
                   int32_t* n_pairs_out, int max_pairs, cudaStream_t stream);
DevLibrary dev_library(const locc_handle* h);
// Crop gather and network of the pairs [0, n) (n = min(*n_dev, n_cap), or
// n_cap when n_dev is NULL), chunked as set by locc_set_pipeline.
int run_path(locc_handle* h, const PairInputs& in, int n_cap, const int* n_dev, float* out,
             cudaStream_t s);
// Encoder then head for the pairs of `rg`; mid (nullable): event recorded
// between the encoder and the head.
int run_network(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                const float4* centre, float* out, float* y_raw, float* feat_out,
                cudaStream_t stream, cudaEvent_t mid, int list_mode);
int upload_fp8_params(locc_handle* h, const std::vector<float>& params);
// Per-device set-up of the tensor-core kernels (dynamic shared-memory limits;
// module load), run by locc_create with the handle's device current.
cudaError_t prepare_tc_kernels();
// Zeroes the pooled features of the objects of `rg` whose crop is empty and
// lists the others for the tensor-core encoders (h->d_list, h->d_list_n).
cudaError_t launch_enc_list(locc_handle* h, const float4* xyz, const PairRange& rg, float* feat,
                            bool counts, void* ftile, int e4m3, cudaStream_t stream);
// Who builds the tensor-core encoders' object list: the crop kernel, or the
// list kernel from the crop rows (which, for crops given by the caller, also
// writes 0 / 1 crop counts).  A warp of each encoder CTA zeroes the pooled
// features of the objects whose count is 0.
enum { LIST_FROM_CROP = 0, LIST_FROM_ROWS = 1, LIST_AND_COUNTS_FROM_ROWS = 2 };
cudaError_t prepare_fp8_kernels();
// BF16 head over the pairs of rg from the pooled features in h->d_feat_tc.
int launch_head_tc(locc_handle* h, const PairRange& rg, const PairInputs* in, const float4* centre,
                   float* out, float* y_raw, cudaStream_t stream);
// BF16 encoder over a device list of objects (2 p + side; list_n[rg.chunk]
// entries at list + 2 lo) on `grid` CTAs, rows from xyz.
int launch_encoder_list(locc_handle* h, const float4* xyz, const PairRange& rg, const int* list,
                        const int* list_n, int grid, cudaStream_t stream);
// Fused crop + BF16 encoder (fused.cu), crop_warps 6 or 8 per CTA.
cudaError_t prepare_fused_kernels();
cudaError_t launch_fused(const DevLibrary& lib, const PairInputs& in, const PairRange& rg, float r,
                         int32_t* cnt, float4* centre, int* err, int* defer, int defer_cap,
                         const unsigned char* img, __nv_bfloat16* ftile, int n_sm, int crop_warps,
                         cudaStream_t s);
// Resolves h->noalloc_scratch on the current device (the handle's).
int noalloc_prepare(locc_handle* h);
int run_network_fp8(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                    const float4* centre, float* out, float* y_raw, float* feat_out,
                    cudaStream_t stream, cudaEvent_t mid, int list_mode);
int run_network_tc(locc_handle* h, const float4* xyz, const PairRange& rg, const PairInputs* in,
                   const float4* centre, float* out, float* y_raw, float* feat_out,
                   cudaStream_t stream, cudaEvent_t mid, int list_mode);
// Tensor-core products of the BF16 trainer (train_tc.cu): same operand and
// epilogue conventions as the trainer's float32 GEMM; err gets bit 2 when a
// bounded wait runs out.
cudaError_t prepare_train_tc_kernels();
cudaError_t tg_gemm(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B,
                    int ldb, float* C, int ldc, const float* bias, const float* mask, int ldm,
                    bool relu, bool accumulate, int splits, int* err, cudaStream_t s);
cudaError_t tg_layer2_forward(const float* X, const float* W1, const float* b1, const float* W2,
                              const float* b2, int M, float* H2, int* err, cudaStream_t s);
cudaError_t tg_layer2_wgrad(const float* dH2, const float* X, const float* W1, const float* b1, int M,
                            float* gW2, int splits, int* err, cudaStream_t s);
cudaError_t tg_layer3_pool(const float* W3, const float* b3, const float* H2, const float* X, int P,
                           float* F, int32_t* amax, int* err, cudaStream_t s);
cudaError_t tg_layer1_grad(const float* dH2, const float* W2, const float* X, const float* W1,
                           const float* b1, int M, float* gW1, float* gB1, int* err, cudaStream_t s);
cudaError_t sparse_layer3_backward(const float* dF, const float* F, const int32_t* amax,
                                   const float* W3, const float* H2, int P, float* dH2, float* gW3,
                                   float* gB3, float* gB2, int n_sm, cudaStream_t s);
}  // namespace locc

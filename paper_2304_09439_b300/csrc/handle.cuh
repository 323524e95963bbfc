// The opaque detector handle and host-side helpers shared by the .cu files.
#pragma once

#include <vector>

#include "common.cuh"

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
  void* d_feat_tc = nullptr;
  size_t feat_tc_bytes = 0;
  int* d_err = nullptr;
  // broadphase per-environment counts / offsets
  int32_t* d_env_counts = nullptr;
  int cap_env = 0;
  // staging for locc_detect_host
  void* h_stage = nullptr;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  // stage timing (locc_profile)
  bool profiling = false;
  bool prof_valid = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
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
// mid (nullable): event recorded between the encoder and the head.
int run_network(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                const PairInputs* in, const float4* centre, float* out, float* y_raw,
                float* feat_out, cudaStream_t stream, cudaEvent_t mid);
int upload_fp8_params(locc_handle* h, const std::vector<float>& params);
int run_network_fp8(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                    const PairInputs* in, const float4* centre, float* out, float* y_raw,
                    float* feat_out, cudaStream_t stream, cudaEvent_t mid);
int run_network_tc(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                   const PairInputs* in, const float4* centre, float* out, float* y_raw,
                   float* feat_out, cudaStream_t stream, cudaEvent_t mid);
}  // namespace locc

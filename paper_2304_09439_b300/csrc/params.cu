// Parameter blob parsing and upload.
//
// Blob ("LOCCW001", little endian): 8-byte magic, uint32 version = 1,
// uint32 n_layers = 6, 6 x (uint32 in, uint32 out), then per layer float32
// W[out][in] followed by float32 b[out].
#include <cstring>
#include <vector>

#include "handle.cuh"

namespace locc {

int parse_weights(const void* blob, size_t bytes, std::vector<float>* params) {
  static const char kMagic[8] = {'L', 'O', 'C', 'C', 'W', '0', '0', '1'};
  const size_t header = 8 + 4 + 4 + 6 * 8;
  if (!blob || bytes < header) {
    set_error("weights blob is NULL or too short");
    return LOCC_ERR_BAD_WEIGHTS;
  }
  const unsigned char* p = static_cast<const unsigned char*>(blob);
  if (std::memcmp(p, kMagic, 8) != 0) {
    set_error("weights blob: bad magic");
    return LOCC_ERR_BAD_WEIGHTS;
  }
  uint32_t version, n_layers;
  std::memcpy(&version, p + 8, 4);
  std::memcpy(&n_layers, p + 12, 4);
  if (version != 1 || n_layers != 6) {
    set_error("weights blob: unsupported version or layer count");
    return LOCC_ERR_BAD_WEIGHTS;
  }
  size_t n = 0;
  for (int l = 0; l < 6; ++l) {
    uint32_t fi, fo;
    std::memcpy(&fi, p + 16 + 8 * l, 4);
    std::memcpy(&fo, p + 20 + 8 * l, 4);
    if ((int)fi != L_IN[l] || (int)fo != L_OUT[l]) {
      set_error("weights blob: layer dimensions differ from 3-64-128-256 / 512-256-256-8");
      return LOCC_ERR_BAD_WEIGHTS;
    }
    n += (size_t)fi * fo + fo;
  }
  if (n != LOCC_N_PARAMS || bytes != header + n * 4) {
    set_error("weights blob: size does not match the layer dimensions");
    return LOCC_ERR_BAD_WEIGHTS;
  }
  params->resize(n);
  std::memcpy(params->data(), p + header, n * 4);
  for (float v : *params) {
    if (!(v == v) || v > 3.0e38f || v < -3.0e38f) {
      set_error("weights blob: non-finite parameter");
      return LOCC_ERR_BAD_WEIGHTS;
    }
  }
  return LOCC_OK;
}

int upload_tc_params(locc_handle* h, const std::vector<float>& params);

int upload_params(locc_handle* h, const std::vector<float>& params) {
  // float32 path: W^T [in][out] then b [out] per layer
  std::vector<float> t(params.size());
  size_t src = 0, dst = 0;
  size_t offw[6], offb[6];
  for (int l = 0; l < 6; ++l) {
    const int fi = L_IN[l], fo = L_OUT[l];
    offw[l] = dst;
    for (int o = 0; o < fo; ++o)
      for (int i = 0; i < fi; ++i) t[dst + (size_t)i * fo + o] = params[src + (size_t)o * fi + i];
    src += (size_t)fi * fo;
    dst += (size_t)fi * fo;
    offb[l] = dst;
    for (int o = 0; o < fo; ++o) t[dst + o] = params[src + o];
    src += fo;
    dst += fo;
  }
  if (cudaMalloc(&h->d_w32, t.size() * 4) != cudaSuccess ||
      cudaMemcpy(h->d_w32, t.data(), t.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot upload float32 parameters");
    return LOCC_ERR_OOM;
  }
  for (int l = 0; l < 6; ++l) {
    h->fp32.wt[l] = h->d_w32 + offw[l];
    h->fp32.b[l] = h->d_w32 + offb[l];
  }
  const int st = upload_tc_params(h, params);
  if (st) return st;
  return upload_fp8_params(h, params);
}

void free_params(locc_handle* h) {
  cudaFree(h->d_w32);
  cudaFree(h->d_wtc);
  cudaFree(h->d_wf8);
  h->d_w32 = nullptr, h->d_wtc = nullptr, h->d_wf8 = nullptr;
}

}  // namespace locc

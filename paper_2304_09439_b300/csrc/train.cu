// Training of the crop network on the GPU: forward with saved activations,
// loss, backward and Adam, all in this library's kernels (float32).
//
// Paper: Sec. III-A -- trained end to end with binary cross-entropy plus
// alpha |f^SE|^2 on the shape embedding (alpha = 0.5), Adam (lr 1e-3,
// beta1 0.9, beta2 0.999, eps 1e-8; hyper-parameter table), rotation
// augmentation: rotating the shapes and counter-rotating the poses leaves the
// label unchanged, which for crops in a canonical frame is a random rotation
// of that frame.  The loss adds regression terms for the contact point,
// normal and depth outputs (weights in locc_train_config).
//
// One training step over a batch of P pairs (M = 128 P crop rows):
//   crop gather (the inference kernel) -> rotate crops and targets into the
//   augmented canonical frame -> H1 = relu(X W1^T + b1) -> H2 = relu(H1 W2^T + b2)
//   -> Z3 = H2 W3^T + b3 -> masked max-pool with argmax -> G1, G2, Y (head) ->
//   loss and dL/dY -> head backward -> scatter of dL/dF to the argmax rows ->
//   encoder backward -> Adam.
// Two precisions (locc_trainer_set_precision):
//   LOCC_FP32: every matrix product in one tiled SIMT kernel (64 x 64 tiles,
//     4 x 4 per thread) with optional transposes, bias, ReLU, ReLU-mask and
//     split-K accumulation; dZ3 formed densely from the argmax scatter.
//   LOCC_BF16: the dense products on the tensor cores (train_tc.cu: bf16
//     operands, float32 accumulation; H1 recomputed from the crop rows by its
//     consumers instead of stored, layer 3 pooled in its epilogue, layer 1's
//     gradient reduced in the epilogue of dH1), the sparse layer-3 backward
//     on the CUDA cores without dZ3, the tiny products (N or K = 8) in SIMT.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "handle.cuh"

struct locc_trainer {
  locc_handle* h = nullptr;
  int max_batch = 0;
  locc_train_config cfg{};
  long long step = 0;
  int precision = LOCC_FP32;
  int batch = 0;  // pairs of the current step
  float* params = nullptr;  // flat W [out][in], b [out] per layer
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  // batch buffers
  float4* xyz = nullptr;  // crops from the gather kernel [P][128]
  int32_t* cnt = nullptr;
  float4* centre = nullptr;
  int* defer = nullptr;   // crop objects left to the exact fallback kernel
  float* X = nullptr;      // augmented crop rows [M][4]
  float* T = nullptr;      // canonical targets [P][8]
  float* H1 = nullptr;     // [M][64]
  float* H2 = nullptr;     // [M][128]
  float* Z3 = nullptr;     // [M][256], reused as dZ3 in the backward pass
  float* F = nullptr;      // [P][512]
  int32_t* amax = nullptr; // [P][512]
  float* G1 = nullptr;     // [P][256]
  float* G2 = nullptr;     // [P][256]
  float* Y = nullptr;      // [P][8]
  float* dY = nullptr;     // [P][8]
  float* dG1 = nullptr;    // [P][256]
  float* dG2 = nullptr;    // [P][256]
  float* dF = nullptr;     // [P][512]
  float* dH1 = nullptr;    // [M][64]
  float* dH2 = nullptr;    // [M][128]
  float* loss = nullptr;   // [1]
};

namespace locc {
namespace {

constexpr int PARAM_OFF_W[6] = {0, 256, 8576, 41600, 172928, 238720};
constexpr int PARAM_OFF_B[6] = {192, 8448, 41344, 172672, 238464, 240768};

// ------------------------------------------------------------------ GEMM
// C[M x N] (+)= op(A)[M x K] op(B)[K x N]; op(A)(m,k) = TA ? A[k lda + m] : A[m lda + k],
// op(B)(k,n) = TB ? B[n ldb + k] : B[k ldb + n].  Epilogue: + bias[n], * (mask > 0),
// relu; with gridDim.z > 1 (split-K) or accumulate the result is added to C
// (atomically when split).
constexpr int GT = 64, GK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                    int lda, const float* __restrict__ B, int ldb,
                                                    float* __restrict__ C, int ldc,
                                                    const float* __restrict__ bias,
                                                    const float* __restrict__ mask, int ldm,
                                                    int relu, int accumulate, int k_split) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Bs[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      int mm, kk;
      if (TA) { kk = e / GT; mm = e % GT; } else { mm = e / GK; kk = e % GK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float a = 0.f;
      if (gm < M && gk < ke) a = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = a;
      int nn, kk2;
      if (TB) { nn = e / GK; kk2 = e % GK; } else { kk2 = e / GT; nn = e % GT; }
      const int gn = n0 + nn, gk2 = k0 + kk2;
      float b = 0.f;
      if (gn < N && gk2 < ke) b = TB ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn];
      Bs[kk2][nn] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[n];
      if (mask && !(mask[(size_t)m * ldm + n] > 0.f)) v = 0.f;
      if (relu) v = fmaxf(v, 0.f);
      float* c = C + (size_t)m * ldc + n;
      if (split) atomicAdd(c, v);
      else if (accumulate) *c += v;
      else *c = v;
    }
  }
}

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, const float* bias, const float* mask, int ldm, bool relu, bool accumulate,
                 int splits, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  splits = std::max(1, std::min(splits, (K + GK - 1) / GK));
  int ks = (K + splits - 1) / splits;
  ks = (ks + GK - 1) / GK * GK;
  splits = (K + ks - 1) / ks;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, splits);
  sgemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ldm,
                                            relu ? 1 : 0, accumulate ? 1 : 0, ks);
  return cudaGetLastError();
}

// --------------------------------------------------------------- kernels
// Canonical targets and augmented crops.  Per pair p (one block of 128
// threads): T = {label, Q (R_A^T (pt - t_A) - c), Q R_A^T n, depth}; row r of
// the crop: Q x (padding rows stay zero).  Q = rot[p] (row-major) or identity.
__global__ void prep_kernel(const float4* __restrict__ xyz, const float4* __restrict__ centre,
                            const float* __restrict__ poses, const int32_t* __restrict__ pairs,
                            int n_obj, const float* __restrict__ targets,
                            const float* __restrict__ rot, float* __restrict__ X,
                            float* __restrict__ T, int P) {
  const int p = blockIdx.x, r = threadIdx.x;
  if (p >= P) return;
  float Q[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  if (rot) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Q[i] = rot[9 * (size_t)p + i];
  }
  const float4 x = xyz[(size_t)p * ROWS + r];
  float4 o;
  o.x = Q[0] * x.x + Q[1] * x.y + Q[2] * x.z;
  o.y = Q[3] * x.x + Q[4] * x.y + Q[5] * x.z;
  o.z = Q[6] * x.x + Q[7] * x.y + Q[8] * x.z;
  o.w = x.w;
  reinterpret_cast<float4*>(X)[(size_t)p * ROWS + r] = o;
  if (r == 0) {
    const int a = pairs[2 * p];
    const float* tg = targets + 8 * (size_t)p;
    float* t = T + 8 * (size_t)p;
    const float4 c = centre[p];
    if (a < 0 || a >= n_obj || isnan(c.x)) {
      for (int i = 0; i < 8; ++i) t[i] = 0.f;
      return;
    }
    float R[9];
    quat_to_rot(poses + 7 * (size_t)a, R);
    const float d[3] = {tg[1] - poses[7 * (size_t)a + 4], tg[2] - poses[7 * (size_t)a + 5],
                        tg[3] - poses[7 * (size_t)a + 6]};
    float pc[3], nc[3];
    for (int i = 0; i < 3; ++i) {
      pc[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
      nc[i] = R[i] * tg[4] + R[3 + i] * tg[5] + R[6 + i] * tg[6];
    }
    pc[0] -= c.x, pc[1] -= c.y, pc[2] -= c.z;
    t[0] = tg[0];
    for (int i = 0; i < 3; ++i) {
      t[1 + i] = Q[3 * i] * pc[0] + Q[3 * i + 1] * pc[1] + Q[3 * i + 2] * pc[2];
      t[4 + i] = Q[3 * i] * nc[0] + Q[3 * i + 1] * nc[1] + Q[3 * i + 2] * nc[2];
    }
    t[7] = tg[7];
  }
}

// H1 = relu(X[:, :3] W1^T + b1), one thread per (row, channel).
__global__ void layer1_kernel(const float* __restrict__ X, const float* __restrict__ W1,
                              const float* __restrict__ b1, float* __restrict__ H1, int M) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)M * 64) return;
  const int r = (int)(i / 64), c = (int)(i % 64);
  const float4 x = reinterpret_cast<const float4*>(X)[r];
  float h = b1[c];
  h = fmaf(W1[3 * c], x.x, h);
  h = fmaf(W1[3 * c + 1], x.y, h);
  h = fmaf(W1[3 * c + 2], x.z, h);
  H1[i] = fmaxf(h, 0.f);
}

// Masked max-pool of relu(Z3) over the valid rows of each object, with the
// slot of the maximum (ties to the lower slot); empty crop -> 0, slot -1.
__global__ void pool_kernel(const float* __restrict__ Z3, const float* __restrict__ X,
                            float* __restrict__ F, int32_t* __restrict__ amax, int P) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * 512) return;
  const int p = (int)(i / 512), o = (int)(i % 512) / 256, c = (int)(i % 256);
  float best = 0.f;
  int arg = -1;
  for (int k = 0; k < KMAX; ++k) {
    const size_t row = (size_t)p * ROWS + o * KMAX + k;
    if (!(reinterpret_cast<const float4*>(X)[row].w > 0.5f)) break;
    const float z = fmaxf(Z3[row * 256 + c], 0.f);
    if (arg < 0 || z > best) best = z, arg = k;
  }
  F[i] = best;
  amax[i] = arg;
}

// Loss per pair (without the embedding regulariser, feat_reg_kernel) and
// dL/dY, both as shares of the mean over the batch.
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                            float* __restrict__ dY, float* __restrict__ loss, int P,
                            locc_train_config cfg) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float L = 0.f;
  if (p < P) {
    const float* y = Y + 8 * (size_t)p;
    const float* t = T + 8 * (size_t)p;
    float* dy = dY + 8 * (size_t)p;
    const float inv = 1.f / P;
    const float z = y[0], lab = t[0];
    L = fmaxf(z, 0.f) - z * lab + log1pf(expf(-fabsf(z)));
    const float sig = 1.f / (1.f + expf(-z));
    float g[8] = {sig - lab, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (lab > 0.f) {
      for (int i = 0; i < 3; ++i) {
        const float d = y[1 + i] - t[1 + i];
        L += lab * cfg.w_pt * d * d;
        g[1 + i] = lab * cfg.w_pt * 2.f * d;
      }
      const float nn = sqrtf(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
      const float tn = sqrtf(t[4] * t[4] + t[5] * t[5] + t[6] * t[6]);
      if (nn > 1e-12f && tn > 1e-12f) {
        const float cs = (y[4] * t[4] + y[5] * t[5] + y[6] * t[6]) / (nn * tn);
        L += lab * cfg.w_n * (1.f - cs);
        for (int i = 0; i < 3; ++i)
          g[4 + i] = -lab * cfg.w_n * (t[4 + i] / (nn * tn) - cs * y[4 + i] / (nn * nn));
      }
    }
    // length of the raw normal (every pair): w_len (|n| - 1)^2 keeps the
    // vector that the epilogue normalises away from zero, where rounding of
    // the reduced-precision paths would be amplified
    if (cfg.w_len > 0.f) {
      const float nn = sqrtf(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
      if (nn > 1e-12f) {
        const float d = nn - 1.f;
        L += cfg.w_len * d * d;
        for (int i = 0; i < 3; ++i) g[4 + i] += cfg.w_len * 2.f * d * y[4 + i] / nn;
      }
    }
    const float e = y[7] - t[7];
    if (fabsf(e) < cfg.huber_beta) {
      L += cfg.w_d * 0.5f * e * e / cfg.huber_beta;
      g[7] = cfg.w_d * e / cfg.huber_beta;
    } else {
      L += cfg.w_d * (fabsf(e) - 0.5f * cfg.huber_beta);
      g[7] = cfg.w_d * (e > 0.f ? 1.f : -1.f);
    }
    for (int i = 0; i < 8; ++i) dy[i] = g[i] * inv;
    L *= inv;
  }
  // block sum -> one atomic per block
  __shared__ float red[256];
  red[threadIdx.x] = L;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0]);
}

// The embedding regulariser alpha mean(f^2) of every pair, one thread per
// feature: its share of the mean loss and dL/dF = 2 alpha f / 512 / P.
__global__ void feat_reg_kernel(const float* __restrict__ F, float* __restrict__ dF,
                                float* __restrict__ loss, int P, float alpha) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const float inv = 1.f / P;
  float sq = 0.f;
  if (i < (size_t)P * 512) {
    const float f = F[i];
    dF[i] = alpha * 2.f * f / 512.f * inv;
    sq = f * f;
  }
  __shared__ float red[256];
  red[threadIdx.x] = sq;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, alpha * red[0] / 512.f * inv);
}

// dZ3 rows: dL/dF of channel c goes to the argmax slot of that channel (when
// the pooled value is positive, i.e. the ReLU passed it).  dZ3 is zeroed first.
__global__ void scatter_kernel(const float* __restrict__ dF, const float* __restrict__ F,
                               const int32_t* __restrict__ amax, float* __restrict__ dZ3, int P) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * 512) return;
  const int k = amax[i];
  if (k < 0 || !(F[i] > 0.f)) return;
  const int p = (int)(i / 512), o = (int)(i % 512) / 256, c = (int)(i % 256);
  dZ3[((size_t)p * ROWS + o * KMAX + k) * 256 + c] = dF[i];
}

// Column sums of A [M x N] added to out[N] (bias gradients).
__global__ void colsum_kernel(const float* __restrict__ A, int M, int N, float* __restrict__ out,
                              int rows_per_block) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int r0 = blockIdx.y * rows_per_block, r1 = min(M, r0 + rows_per_block);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s += A[(size_t)r * N + n];
  atomicAdd(out + n, s);
}

// dW1 [64 x 3] += dH1^T X[:, :3]; one block per channel, reduction over rows.
__global__ void dw1_kernel(const float* __restrict__ dH1, const float* __restrict__ X, int M,
                           float* __restrict__ gW1) {
  const int c = blockIdx.x;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int r = blockIdx.y * blockDim.x + threadIdx.x; r < M; r += gridDim.y * blockDim.x) {
    const float g = dH1[(size_t)r * 64 + c];
    const float4 x = reinterpret_cast<const float4*>(X)[r];
    s0 = fmaf(g, x.x, s0);
    s1 = fmaf(g, x.y, s1);
    s2 = fmaf(g, x.z, s2);
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(gW1 + 3 * c, s0);
    atomicAdd(gW1 + 3 * c + 1, s1);
    atomicAdd(gW1 + 3 * c + 2, s2);
  }
}

// Adam (Kingma & Ba), bias-corrected, on the flat parameter vector.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace
}  // namespace locc

using namespace locc;

namespace {
int tfail(int code, const char* msg) {
  set_error(msg);
  return code;
}
#define TCU(expr)                                                    \
  do {                                                               \
    if ((expr) != cudaSuccess) {                                     \
      cudaGetLastError();                                            \
      return tfail(LOCC_ERR_CUDA, "training: " #expr " failed");     \
    }                                                                \
  } while (0)

void trainer_free(locc_trainer* t) {
  void* ptrs[] = {t->params, t->grad, t->m, t->v, t->xyz, t->cnt, t->centre, t->defer, t->X, t->T, t->H1,
                  t->H2, t->Z3, t->F, t->amax, t->G1, t->G2, t->Y, t->dY, t->dG1, t->dG2, t->dF,
                  t->dH1, t->dH2, t->loss};
  for (void* p : ptrs) cudaFree(p);
}

// Forward, loss and backward of one batch in float32 SIMT (gradients into
// t->grad, which the caller zeroed).
int fp32_pass(locc_trainer* t, cudaStream_t s) {
  if (!t->Z3) {
    // H1, Z3 (dZ3) and dH1 only exist for this pass: allocated at its first
    // step, for max_batch pairs (the BF16 pass keeps none of them)
    const size_t Mx = (size_t)t->max_batch * ROWS;
    if (cudaMalloc(&t->H1, Mx * 64 * 4) != cudaSuccess || cudaMalloc(&t->Z3, Mx * 256 * 4) != cudaSuccess ||
        cudaMalloc(&t->dH1, Mx * 64 * 4) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(t->H1);
      cudaFree(t->Z3);
      cudaFree(t->dH1);
      t->H1 = t->Z3 = t->dH1 = nullptr;
      return tfail(LOCC_ERR_OOM, "cannot allocate the float32 training buffers");
    }
  }
  const int P = t->batch, M = P * ROWS;
  const float* prm = t->params;
  auto W = [&](int l) { return prm + PARAM_OFF_W[l]; };
  auto Bv = [&](int l) { return prm + PARAM_OFF_B[l]; };
  float* g = t->grad;
  auto gW = [&](int l) { return g + PARAM_OFF_W[l]; };
  auto gB = [&](int l) { return g + PARAM_OFF_B[l]; };
  layer1_kernel<<<(unsigned)(((size_t)M * 64 + 255) / 256), 256, 0, s>>>(t->X, W(0), Bv(0), t->H1, M);
  TCU(cudaGetLastError());
  TCU((gemm<false, true>(M, 128, 64, t->H1, 64, W(1), 64, t->H2, 128, Bv(1), nullptr, 0, true, false, 1, s)));
  TCU((gemm<false, true>(M, 256, 128, t->H2, 128, W(2), 128, t->Z3, 256, Bv(2), nullptr, 0, false, false, 1, s)));
  pool_kernel<<<(unsigned)(((size_t)P * 512 + 255) / 256), 256, 0, s>>>(t->Z3, t->X, t->F, t->amax, P);
  TCU(cudaGetLastError());
  TCU((gemm<false, true>(P, 256, 512, t->F, 512, W(3), 512, t->G1, 256, Bv(3), nullptr, 0, true, false, 1, s)));
  TCU((gemm<false, true>(P, 256, 256, t->G1, 256, W(4), 256, t->G2, 256, Bv(4), nullptr, 0, true, false, 1, s)));
  TCU((gemm<false, true>(P, 8, 256, t->G2, 256, W(5), 256, t->Y, 8, Bv(5), nullptr, 0, false, false, 1, s)));
  loss_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->Y, t->T, t->dY, t->loss, P, t->cfg);
  feat_reg_kernel<<<(unsigned)(((size_t)P * 512 + 255) / 256), 256, 0, s>>>(t->F, t->dF, t->loss, P,
                                                                           t->cfg.alpha);
  TCU(cudaGetLastError());
  // ---- head backward
  const int split_p = std::max(1, P / 64);
  TCU((gemm<true, false>(8, 256, P, t->dY, 8, t->G2, 256, gW(5), 256, nullptr, nullptr, 0, false, true, split_p, s)));
  TCU((gemm<false, false>(P, 256, 8, t->dY, 8, W(5), 256, t->dG2, 256, nullptr, t->G2, 256, false, false, 1, s)));
  TCU((gemm<true, false>(256, 256, P, t->dG2, 256, t->G1, 256, gW(4), 256, nullptr, nullptr, 0, false, true, split_p, s)));
  TCU((gemm<false, false>(P, 256, 256, t->dG2, 256, W(4), 256, t->dG1, 256, nullptr, t->G1, 256, false, false, 1, s)));
  TCU((gemm<true, false>(256, 512, P, t->dG1, 256, t->F, 512, gW(3), 512, nullptr, nullptr, 0, false, true, split_p, s)));
  TCU((gemm<false, false>(P, 512, 256, t->dG1, 256, W(3), 512, t->dF, 512, nullptr, nullptr, 0, false, true, 1, s)));
  {
    dim3 gb(1, std::max(1, (P + 63) / 64));
    colsum_kernel<<<gb, 256, 0, s>>>(t->dY, P, 8, gB(5), 64);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dG2, P, 256, gB(4), 64);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dG1, P, 256, gB(3), 64);
    TCU(cudaGetLastError());
  }
  // ---- encoder backward (dZ3 reuses the Z3 buffer)
  float* dZ3 = t->Z3;
  TCU(cudaMemsetAsync(dZ3, 0, (size_t)M * 256 * 4, s));
  scatter_kernel<<<(unsigned)(((size_t)P * 512 + 255) / 256), 256, 0, s>>>(t->dF, t->F, t->amax, dZ3, P);
  TCU(cudaGetLastError());
  const int split_m = std::max(1, M / 1024);
  TCU((gemm<true, false>(256, 128, M, dZ3, 256, t->H2, 128, gW(2), 128, nullptr, nullptr, 0, false, true, split_m, s)));
  TCU((gemm<false, false>(M, 128, 256, dZ3, 256, W(2), 128, t->dH2, 128, nullptr, t->H2, 128, false, false, 1, s)));
  TCU((gemm<true, false>(128, 64, M, t->dH2, 128, t->H1, 64, gW(1), 64, nullptr, nullptr, 0, false, true, split_m, s)));
  TCU((gemm<false, false>(M, 64, 128, t->dH2, 128, W(1), 64, t->dH1, 64, nullptr, t->H1, 64, false, false, 1, s)));
  {
    dim3 gb(1, std::max(1, (M + 255) / 256));
    colsum_kernel<<<gb, 256, 0, s>>>(dZ3, M, 256, gB(2), 256);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dH2, M, 128, gB(1), 256);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dH1, M, 64, gB(0), 256);
    dim3 gw(64, std::max(1, std::min(256, M / 256)));
    dw1_kernel<<<gw, 256, 0, s>>>(t->dH1, t->X, M, gW(0));
    TCU(cudaGetLastError());
  }
  return LOCC_OK;
}

// The same pass with the dense products on the tensor cores (bf16 operands,
// float32 accumulation) and the sparse layer-3 backward.
int bf16_pass(locc_trainer* t, cudaStream_t s) {
  locc_handle* h = t->h;
  int* err = h->d_err;
  const int P = t->batch, M = P * ROWS;
  const float* prm = t->params;
  auto W = [&](int l) { return prm + PARAM_OFF_W[l]; };
  auto Bv = [&](int l) { return prm + PARAM_OFF_B[l]; };
  float* g = t->grad;
  auto gW = [&](int l) { return g + PARAM_OFF_W[l]; };
  auto gB = [&](int l) { return g + PARAM_OFF_B[l]; };
  TCU(tg_layer2_forward(t->X, W(0), Bv(0), W(1), Bv(1), M, t->H2, err, s));
  TCU(tg_layer3_pool(W(2), Bv(2), t->H2, t->X, P, t->F, t->amax, err, s));
  TCU(tg_gemm(false, true, P, 256, 512, t->F, 512, W(3), 512, t->G1, 256, Bv(3), nullptr, 0, true, false, 1, err, s));
  TCU(tg_gemm(false, true, P, 256, 256, t->G1, 256, W(4), 256, t->G2, 256, Bv(4), nullptr, 0, true, false, 1, err, s));
  TCU((gemm<false, true>(P, 8, 256, t->G2, 256, W(5), 256, t->Y, 8, Bv(5), nullptr, 0, false, false, 1, s)));
  loss_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->Y, t->T, t->dY, t->loss, P, t->cfg);
  feat_reg_kernel<<<(unsigned)(((size_t)P * 512 + 255) / 256), 256, 0, s>>>(t->F, t->dF, t->loss, P,
                                                                           t->cfg.alpha);
  TCU(cudaGetLastError());
  // ---- head backward
  const int split_p = std::max(1, std::min(64, P / 64));
  TCU((gemm<true, false>(8, 256, P, t->dY, 8, t->G2, 256, gW(5), 256, nullptr, nullptr, 0, false, true, std::max(1, P / 64), s)));
  TCU((gemm<false, false>(P, 256, 8, t->dY, 8, W(5), 256, t->dG2, 256, nullptr, t->G2, 256, false, false, 1, s)));
  TCU(tg_gemm(true, false, 256, 256, P, t->dG2, 256, t->G1, 256, gW(4), 256, nullptr, nullptr, 0, false, true, split_p, err, s));
  TCU(tg_gemm(false, false, P, 256, 256, t->dG2, 256, W(4), 256, t->dG1, 256, nullptr, t->G1, 256, false, false, 1, err, s));
  TCU(tg_gemm(true, false, 256, 512, P, t->dG1, 256, t->F, 512, gW(3), 512, nullptr, nullptr, 0, false, true, split_p, err, s));
  TCU(tg_gemm(false, false, P, 512, 256, t->dG1, 256, W(3), 512, t->dF, 512, nullptr, nullptr, 0, false, true, 1, err, s));
  {
    dim3 gb(1, std::max(1, (P + 63) / 64));
    colsum_kernel<<<gb, 256, 0, s>>>(t->dY, P, 8, gB(5), 64);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dG2, P, 256, gB(4), 64);
    colsum_kernel<<<gb, 256, 0, s>>>(t->dG1, P, 256, gB(3), 64);
    TCU(cudaGetLastError());
  }
  // ---- encoder backward: layer 3 sparse (no dZ3), layers 2 and 1 on the tensor cores
  TCU(sparse_layer3_backward(t->dF, t->F, t->amax, W(2), t->H2, P, t->dH2, gW(2), gB(2), gB(1), h->n_sm, s));
  TCU(tg_layer2_wgrad(t->dH2, t->X, W(0), Bv(0), M, gW(1), 2 * h->n_sm, err, s));
  TCU(tg_layer1_grad(t->dH2, W(1), t->X, W(0), Bv(0), M, gW(0), gB(0), err, s));
  return LOCC_OK;
}
}  // namespace

extern "C" {

int locc_trainer_create(locc_handle* h, int32_t max_batch, const locc_train_config* cfg,
                        locc_trainer** out) {
  if (!out) return tfail(LOCC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!h || !cfg || max_batch < 1) return tfail(LOCC_ERR_INVALID_ARG, "bad trainer arguments");
  if (prepare_train_tc_kernels() != cudaSuccess) {
    cudaGetLastError();
    return tfail(LOCC_ERR_CUDA, "cannot configure the training kernels");
  }
  locc_trainer* t = new (std::nothrow) locc_trainer();
  if (!t) return tfail(LOCC_ERR_OOM, "host allocation failed");
  t->h = h;
  t->max_batch = max_batch;
  t->cfg = *cfg;
  const size_t P = (size_t)max_batch, M = P * ROWS, NP = LOCC_N_PARAMS;
  bool ok = cudaMalloc(&t->params, NP * 4) == cudaSuccess && cudaMalloc(&t->grad, NP * 4) == cudaSuccess &&
            cudaMalloc(&t->m, NP * 4) == cudaSuccess && cudaMalloc(&t->v, NP * 4) == cudaSuccess &&
            cudaMalloc(&t->xyz, M * 16) == cudaSuccess && cudaMalloc(&t->cnt, P * 8) == cudaSuccess &&
            cudaMalloc(&t->defer, (2 + 2 * P) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&t->centre, P * 16) == cudaSuccess && cudaMalloc(&t->X, M * 16) == cudaSuccess &&
            cudaMalloc(&t->T, P * 32) == cudaSuccess &&
            cudaMalloc(&t->H2, M * 128 * 4) == cudaSuccess &&
            cudaMalloc(&t->F, P * 512 * 4) == cudaSuccess &&
            cudaMalloc(&t->amax, P * 512 * 4) == cudaSuccess && cudaMalloc(&t->G1, P * 256 * 4) == cudaSuccess &&
            cudaMalloc(&t->G2, P * 256 * 4) == cudaSuccess && cudaMalloc(&t->Y, P * 32) == cudaSuccess &&
            cudaMalloc(&t->dY, P * 32) == cudaSuccess && cudaMalloc(&t->dG1, P * 256 * 4) == cudaSuccess &&
            cudaMalloc(&t->dG2, P * 256 * 4) == cudaSuccess && cudaMalloc(&t->dF, P * 512 * 4) == cudaSuccess &&
            cudaMalloc(&t->dH2, M * 128 * 4) == cudaSuccess &&
            cudaMalloc(&t->loss, 4) == cudaSuccess;
  if (ok) {
    // parameters start from the handle's float32 weights (W^T layout there)
    std::vector<float> wt(NP), flat(NP);
    ok = cudaMemcpy(wt.data(), h->d_w32, NP * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    size_t src = 0;
    for (int l = 0; l < 6 && ok; ++l) {
      const int fi = L_IN[l], fo = L_OUT[l];
      for (int o = 0; o < fo; ++o)
        for (int i = 0; i < fi; ++i) flat[PARAM_OFF_W[l] + (size_t)o * fi + i] = wt[src + (size_t)i * fo + o];
      src += (size_t)fi * fo;
      for (int o = 0; o < fo; ++o) flat[PARAM_OFF_B[l] + o] = wt[src + o];
      src += fo;
    }
    ok = ok && cudaMemcpy(t->params, flat.data(), NP * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(t->m, 0, NP * 4) == cudaSuccess && cudaMemset(t->v, 0, NP * 4) == cudaSuccess &&
         cudaMemset(t->grad, 0, NP * 4) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    trainer_free(t);
    delete t;
    return tfail(LOCC_ERR_OOM, "cannot allocate training buffers");
  }
  *out = t;
  return LOCC_OK;
}

int locc_train_step(locc_trainer* t, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                    const int32_t* pairs, int32_t n_pairs, const float* targets, const float* rot,
                    float* loss_out, int32_t update, void* stream) {
  if (!t) return tfail(LOCC_ERR_INVALID_ARG, "trainer is NULL");
  if (n_pairs < 1 || n_pairs > t->max_batch) return tfail(LOCC_ERR_INVALID_ARG, "batch size out of range");
  if (!poses || !obj_shape || !pairs || !targets) return tfail(LOCC_ERR_INVALID_ARG, "NULL array");
  locc_handle* h = t->h;
  cudaStream_t s = (cudaStream_t)stream;
  const int P = n_pairs;
  float* g = t->grad;
  t->batch = P;
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  TCU(launch_crop(dev_library(h), in, whole_range(n_pairs, nullptr), h->radius, t->xyz, nullptr,
                  t->cnt, t->centre, h->d_err, t->defer, h->n_sm, 0, s, h->crop_mode));
  TCU(cudaMemsetAsync(t->loss, 0, 4, s));
  TCU(cudaMemsetAsync(g, 0, (size_t)LOCC_N_PARAMS * 4, s));
  prep_kernel<<<P, ROWS, 0, s>>>(t->xyz, t->centre, poses, pairs, n_obj, targets, rot, t->X, t->T, P);
  TCU(cudaGetLastError());
  const int st = t->precision == LOCC_BF16 ? bf16_pass(t, s) : fp32_pass(t, s);
  if (st != LOCC_OK) return st;
  if (update) {
    t->step += 1;
    const float c1 = 1.f - powf(t->cfg.beta1, (float)t->step);
    const float c2 = 1.f - powf(t->cfg.beta2, (float)t->step);
    adam_kernel<<<(LOCC_N_PARAMS + 255) / 256, 256, 0, s>>>(t->params, g, t->m, t->v, LOCC_N_PARAMS,
                                                            t->cfg.lr, t->cfg.beta1, t->cfg.beta2,
                                                            t->cfg.eps, c1, c2);
    TCU(cudaGetLastError());
  }
  if (loss_out) TCU(cudaMemcpyAsync(loss_out, t->loss, 4, cudaMemcpyDeviceToDevice, s));
  return LOCC_OK;
}

int locc_trainer_grad(locc_trainer* t, float* grad_out, void* stream) {
  if (!t || !grad_out) return tfail(LOCC_ERR_INVALID_ARG, "bad argument");
  TCU(cudaMemcpyAsync(grad_out, t->grad, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream));
  return LOCC_OK;
}

int locc_trainer_params(locc_trainer* t, float* params_out, void* stream) {
  if (!t || !params_out) return tfail(LOCC_ERR_INVALID_ARG, "bad argument");
  TCU(cudaMemcpyAsync(params_out, t->params, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream));
  return LOCC_OK;
}

int locc_trainer_set_params(locc_trainer* t, const float* params, void* stream) {
  if (!t || !params) return tfail(LOCC_ERR_INVALID_ARG, "bad argument");
  TCU(cudaMemcpyAsync(t->params, params, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream));
  return LOCC_OK;
}

int locc_trainer_get_state(locc_trainer* t, float* m_out, float* v_out, int64_t* step_out,
                           void* stream) {
  if (!t || !m_out || !v_out || !step_out) return tfail(LOCC_ERR_INVALID_ARG, "bad argument");
  const cudaStream_t s = (cudaStream_t)stream;
  TCU(cudaMemcpyAsync(m_out, t->m, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice, s));
  TCU(cudaMemcpyAsync(v_out, t->v, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice, s));
  *step_out = (int64_t)t->step;
  return LOCC_OK;
}

int locc_trainer_set_state(locc_trainer* t, const float* m, const float* v, int64_t step,
                           void* stream) {
  if (!t || !m || !v || step < 0) return tfail(LOCC_ERR_INVALID_ARG, "bad argument");
  const cudaStream_t s = (cudaStream_t)stream;
  TCU(cudaMemcpyAsync(t->m, m, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice, s));
  TCU(cudaMemcpyAsync(t->v, v, (size_t)LOCC_N_PARAMS * 4, cudaMemcpyDeviceToDevice, s));
  t->step = (long long)step;
  return LOCC_OK;
}

int locc_trainer_commit(locc_trainer* t) {
  if (!t) return tfail(LOCC_ERR_INVALID_ARG, "trainer is NULL");
  std::vector<float> flat(LOCC_N_PARAMS);
  TCU(cudaDeviceSynchronize());
  TCU(cudaMemcpy(flat.data(), t->params, flat.size() * 4, cudaMemcpyDeviceToHost));
  for (float x : flat)
    if (!std::isfinite(x)) return tfail(LOCC_ERR_BAD_WEIGHTS, "training produced a non-finite parameter");
  free_params(t->h);
  return upload_params(t->h, flat);
}

int locc_trainer_set_lr(locc_trainer* t, float lr) {
  if (!t) return tfail(LOCC_ERR_INVALID_ARG, "trainer is NULL");
  if (!(lr >= 0.f) || !std::isfinite(lr)) return tfail(LOCC_ERR_INVALID_ARG, "lr must be finite and >= 0");
  t->cfg.lr = lr;
  return LOCC_OK;
}

int locc_trainer_set_precision(locc_trainer* t, int32_t precision) {
  if (!t) return tfail(LOCC_ERR_INVALID_ARG, "trainer is NULL");
  if (precision != LOCC_FP32 && precision != LOCC_BF16)
    return tfail(LOCC_ERR_INVALID_ARG, "training precision must be LOCC_FP32 or LOCC_BF16");
  t->precision = precision;
  return LOCC_OK;
}

void locc_trainer_destroy(locc_trainer* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  trainer_free(t);
  delete t;
}

}  // extern "C"

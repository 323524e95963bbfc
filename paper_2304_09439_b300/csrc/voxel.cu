// Voxel-latent variant of the method (the paper's own design): per-shape
// latents from a point MLP, a 6 x 6 x 6 voxel grid and a 3-D U-Net, computed
// once per library; per pair, the cells of each object inside the widened
// intersection region of the two boxes, average pooled, and a symmetric MLP
// predictor that returns the collision logit.
//
// Paper: Sec. III ("Local Crop Collision Network": shape encoder, voxel grid on
// each object's AABB, cell-wise max pooling, 3-D CNN with skip connections and
// a global feature; OBB cell selection with a margin of the cell's
// half-diagonal so that no colliding cell is missed; average pooling and the
// collision predictor), appendix "Architecture Details" (three 256-wide point
// MLP layers, voxel size 6, four 128-channel 3x3x3 convolutions the first
// without padding, deconvolutions in reverse order with concatenated skips,
// global features tiled onto the grid, a linear layer to F = 16, predictor
// MLPs of 3 + 3 layers of 128 around a max pool over the two objects).
//
// Readings where the paper is silent or inconsistent (the same as the CPU
// reference's): three point-MLP layers; a point's cell is floor((p - lo) * (6 /
// (hi - lo))) per axis in float32, clamped to [0, 5]; empty cells pool to 0;
// the global feature is [max || mean] over the last convolution's cells (256
// values); the deconvolutions are stride-1 transposed convolutions, padded
// except the last (4 -> 6), fed conv4, then [previous || conv3], [previous ||
// conv2], [previous || conv1]; the final 384 -> 16 layer is linear; the
// selection region of object X is X's box intersected with the other box
// seen as an axis-aligned box of X's frame, widened by X's own cell
// half-diagonal; an object without selected cells pools to 0; each object's
// pose input is its pose in A's body frame; the predictor is 23 -> 128 ->
// 128 -> 128 per object, max over the objects, 128 -> 128 -> 128 -> 128, 128
// -> 1.
//
// The selection geometry uses float32 operations with explicit rounding in a
// fixed order, so selected cell sets are reproducible bit for bit; the
// networks run in float32 on the CUDA cores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "handle.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

constexpr int VM = 6, VCELLS = 216, VF = 16, VH = 256, VC = 128, VPIN = 23, VPW = 128;
constexpr int VK1 = 32;   // first predictor layer: 23 inputs, padded to 32 rows
constexpr int VTILE = 32; // pairs per predictor tile
constexpr int VSTRIDE = VPW + 1;  // activation row stride in shared memory (floats)
constexpr size_t VOX_SMEM = 2 * (2 * VTILE) * VSTRIDE * sizeof(float) + 2 * VTILE * sizeof(int);

// Device parameters, every weight stored input-major (W^T), convolutions as
// [27][Cin][Cout] with the kernel offset (k0, k1, k2) at index (k0 * 3 + k1) *
// 3 + k2.
struct VoxParams {
  const float *e1w, *e1b, *e2w, *e2b, *e3w, *e3b;   // [3][256], [256][256]
  const float *cw[4], *cb[4];                       // [27][Cin][128]
  const float *dw[4], *db[4];                       // [27][Cin][128]
  const float *fw, *fb;                             // [384][16]
  const float *pw[3], *pb[3];                       // [32][128], [128][128] x 2
  const float *qw[4], *qb[4];                       // [128][128] x 3, [128][1]
};

// ------------------------------------------------------------ shape encoder
// Point MLP and cell-wise max pooling: one CTA of 256 threads (one per
// channel) per 32 points of one shape.  ReLU outputs are >= 0, so their IEEE
// bit patterns order like the values and an integer atomicMax pools them into
// a grid initialised to +0.0 (an empty cell stays 0).
__global__ void __launch_bounds__(256)
    vox_points_kernel(const float* __restrict__ pts, const float* __restrict__ aabb, int n_pts,
                      VoxParams prm, int* __restrict__ cellmax) {
  __shared__ float x[32][3];
  __shared__ float h[32][VH];
  __shared__ int cell[32];
  const int s = blockIdx.x, p0 = blockIdx.y * 32, c = threadIdx.x;
  const int n = min(32, n_pts - p0);
  if (c < 3 * n) x[c / 3][c % 3] = pts[((size_t)s * n_pts + p0) * 3 + c];
  __syncthreads();
  if (c < n) {
    int ci[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float lo = aabb[6 * s + d], hi = aabb[6 * s + 3 + d];
      const float inv = __fdiv_rn(6.0f, __fsub_rn(hi, lo));
      const float t = __fmul_rn(__fsub_rn(x[c][d], lo), inv);
      ci[d] = min(max((int)floorf(t), 0), VM - 1);
    }
    cell[c] = (ci[0] * VM + ci[1]) * VM + ci[2];
  }
  {
    const float w0 = prm.e1w[c], w1 = prm.e1w[VH + c], w2 = prm.e1w[2 * VH + c], b = prm.e1b[c];
    for (int p = 0; p < n; ++p)
      h[p][c] = fmaxf(fmaf(x[p][2], w2, fmaf(x[p][1], w1, fmaf(x[p][0], w0, b))), 0.f);
  }
  __syncthreads();
  float acc[32];
  for (int layer = 0; layer < 2; ++layer) {
    const float* wt = layer == 0 ? prm.e2w : prm.e3w;
    const float b = (layer == 0 ? prm.e2b : prm.e3b)[c];
#pragma unroll
    for (int p = 0; p < 32; ++p) acc[p] = b;
    for (int k = 0; k < VH; ++k) {
      const float w = __ldg(wt + (size_t)k * VH + c);
#pragma unroll
      for (int p = 0; p < 32; ++p) acc[p] = fmaf(h[p][k], w, acc[p]);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 32; ++p) h[p][c] = fmaxf(acc[p], 0.f);
    __syncthreads();
  }
  for (int p = 0; p < n; ++p)
    atomicMax(cellmax + ((size_t)s * VCELLS + cell[p]) * VH + c, __float_as_int(h[p][c]));
}

// One output cell of a stride-1 3-D (transposed) convolution for every shape:
// grid (S, dout^3), one thread per output channel.  Inputs [S][din^3][C]
// (channels innermost), the second input (nullable) concatenated after the
// first.  Convolution: u = z + k - pad; transposed: u = z - k + pad.
__global__ void __launch_bounds__(VC)
    vox_conv_kernel(const float* __restrict__ in1, int c1, const float* __restrict__ in2, int c2,
                    int din, int dout, int pad, int transposed, const float* __restrict__ wt,
                    const float* __restrict__ bias, float* __restrict__ out) {
  const int s = blockIdx.x, z = blockIdx.y, o = threadIdx.x;
  const int z0 = z / (dout * dout), z1 = (z / dout) % dout, z2 = z % dout;
  const int cin = c1 + c2, din3 = din * din * din;
  float acc = bias[o];
  for (int k = 0; k < 27; ++k) {
    const int k0 = k / 9, k1 = (k / 3) % 3, k2 = k % 3;
    const int u0 = transposed ? z0 - k0 + pad : z0 + k0 - pad;
    const int u1 = transposed ? z1 - k1 + pad : z1 + k1 - pad;
    const int u2 = transposed ? z2 - k2 + pad : z2 + k2 - pad;
    if (u0 < 0 || u1 < 0 || u2 < 0 || u0 >= din || u1 >= din || u2 >= din) continue;
    const int u = (u0 * din + u1) * din + u2;
    const float* w = wt + (size_t)k * cin * VC + o;
    const float* a = in1 + ((size_t)s * din3 + u) * c1;
    for (int i = 0; i < c1; ++i) acc = fmaf(a[i], __ldg(w + (size_t)i * VC), acc);
    if (in2) {
      const float* b2 = in2 + ((size_t)s * din3 + u) * c2;
      for (int i = 0; i < c2; ++i) acc = fmaf(b2[i], __ldg(w + (size_t)(c1 + i) * VC), acc);
    }
  }
  out[((size_t)s * dout * dout * dout + z) * VC + o] = fmaxf(acc, 0.f);
}

// Global feature [max || mean] over the 4^3 cells of the last convolution.
__global__ void vox_global_kernel(const float* __restrict__ s4, float* __restrict__ g) {
  const int s = blockIdx.x, c = threadIdx.x;
  float mx = 0.f, sum = 0.f;  // inputs are ReLU outputs (>= 0)
  for (int z = 0; z < 64; ++z) {
    const float v = s4[((size_t)s * 64 + z) * VC + c];
    mx = fmaxf(mx, v);
    sum += v;
  }
  g[(size_t)s * 2 * VC + c] = mx;
  g[(size_t)s * 2 * VC + VC + c] = sum * (1.0f / 64.0f);
}

// Latent of every cell: f.w [u(cell) || g] + f.b, 8 cells x 16 features per CTA.
__global__ void vox_final_kernel(const float* __restrict__ u, const float* __restrict__ g,
                                 VoxParams prm, float* __restrict__ lat) {
  const int s = blockIdx.x, cell = blockIdx.y * 8 + threadIdx.x / VF, f = threadIdx.x % VF;
  float acc = prm.fb[f];
  const float* uc = u + ((size_t)s * VCELLS + cell) * VC;
  for (int c = 0; c < VC; ++c) acc = fmaf(uc[c], prm.fw[c * VF + f], acc);
  const float* gs = g + (size_t)s * 2 * VC;
  for (int c = 0; c < 2 * VC; ++c) acc = fmaf(gs[c], prm.fw[(VC + c) * VF + f], acc);
  lat[((size_t)s * VCELLS + cell) * VF + f] = acc;
}

// ------------------------------------------------------------------ per pair
// Half-diagonal of a cell of a box: sqrt(a0^2 + a1^2 + a2^2) / 2 with a = (hi
// - lo) / 6, every operation rounded in this order.
__device__ __forceinline__ void cell_geometry(const float* box, float* a, float* eps) {
#pragma unroll
  for (int d = 0; d < 3; ++d) a[d] = __fdiv_rn(__fsub_rn(box[3 + d], box[d]), 6.0f);
  float s = fmul(a[0], a[0]);
  s = fadd(s, fmul(a[1], a[1]));
  s = fadd(s, fmul(a[2], a[2]));
  *eps = fmul(__fsqrt_rn(s), 0.5f);
}

// Cells of an object (box in its own frame) whose centre lo + (i + 0.5) a lies
// in [max(lo, olo) - eps, min(hi, ohi) + eps] per axis: an index range
// r[2 d], r[2 d + 1] per axis (r[0] > r[1] when empty).
__device__ __forceinline__ void cell_ranges(const float* box, const float* olo, const float* ohi,
                                            int* r) {
  float a[3], eps;
  cell_geometry(box, a, &eps);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float lo = fsub(fmaxf(box[d], olo[d]), eps);
    const float hi = fadd(fminf(box[3 + d], ohi[d]), eps);
    int i0 = VM, i1 = -1;
#pragma unroll
    for (int i = 0; i < VM; ++i) {
      const float c = fadd(box[d], fmul((float)i + 0.5f, a[d]));
      if (c >= lo && c <= hi) {
        i0 = min(i0, i);
        i1 = i;
      }
    }
    r[2 * d] = i0;
    r[2 * d + 1] = i1;
  }
}

__device__ __forceinline__ int range_count(const int* r) {
  const int n0 = r[1] - r[0] + 1, n1 = r[3] - r[2] + 1, n2 = r[5] - r[4] + 1;
  return (n0 > 0 && n1 > 0 && n2 > 0) ? n0 * n1 * n2 : 0;
}

// Mean latent over the cells of a range box, computed by one warp: lane l
// sums the 16 features of cells l, l + 32, ... (four 16-byte loads per cell,
// all independent), then a butterfly exchange reduces the 16 partial sums
// over the lanes in 16 shuffles, halving the features a lane keeps at each
// step; every lane returns the mean of feature lane % 16.
__device__ __forceinline__ float pool_range(const float* lat, const int* r, int lane) {
  const int n = range_count(r);
  const int n1 = r[3] - r[2] + 1, n2 = r[5] - r[4] + 1;
  float v[16];
#pragma unroll
  for (int f = 0; f < 16; ++f) v[f] = 0.f;
  for (int q = lane; q < n; q += 32) {
    const int i = r[0] + q / (n1 * n2), j = r[2] + (q / n2) % n1, k = r[4] + q % n2;
    const float4* c = reinterpret_cast<const float4*>(lat + ((i * VM + j) * VM + k) * VF);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 x = __ldg(c + u);
      v[4 * u] += x.x;
      v[4 * u + 1] += x.y;
      v[4 * u + 2] += x.z;
      v[4 * u + 3] += x.w;
    }
  }
  // after the steps of offsets 16, 8, 4, 2 a lane holds feature (lane >> 1)
#pragma unroll
  for (int off = 16, w = 8; off >= 2; off >>= 1, w >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f < w) {
        const float keep = up ? v[f + w] : v[f];
        const float send = up ? v[f] : v[f + w];
        v[f] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  const float mean = n > 0 ? __fdiv_rn(v[0], (float)n) : 0.f;
  return __shfl_sync(0xffffffffu, mean, 2 * (lane & 15));
}

// act_out[r][c] = act(W^T-major layer over act_in rows [0, R)), 256 threads:
// thread (ty, tx) owns rows ty * R/16 .. and channels 8 tx .. 8 tx + 7.
template <int R, int K>
__device__ __forceinline__ void dense_layer(const float* act_in, float* act_out, const float* wt,
                                            const float* b, bool relu) {
  constexpr int RPT = R / 16;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[RPT][8];
  const float4 b0 = __ldg(reinterpret_cast<const float4*>(b + 8 * tx));
  const float4 b1 = __ldg(reinterpret_cast<const float4*>(b + 8 * tx + 4));
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    acc[r][0] = b0.x, acc[r][1] = b0.y, acc[r][2] = b0.z, acc[r][3] = b0.w;
    acc[r][4] = b1.x, acc[r][5] = b1.y, acc[r][6] = b1.z, acc[r][7] = b1.w;
  }
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 w0 = __ldg(reinterpret_cast<const float4*>(wt + (size_t)k * VPW + 8 * tx));
    const float4 w1 = __ldg(reinterpret_cast<const float4*>(wt + (size_t)k * VPW + 8 * tx + 4));
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const float a = act_in[(ty * RPT + r) * VSTRIDE + k];
      acc[r][0] = fmaf(a, w0.x, acc[r][0]);
      acc[r][1] = fmaf(a, w0.y, acc[r][1]);
      acc[r][2] = fmaf(a, w0.z, acc[r][2]);
      acc[r][3] = fmaf(a, w0.w, acc[r][3]);
      acc[r][4] = fmaf(a, w1.x, acc[r][4]);
      acc[r][5] = fmaf(a, w1.y, acc[r][5]);
      acc[r][6] = fmaf(a, w1.z, acc[r][6]);
      acc[r][7] = fmaf(a, w1.w, acc[r][7]);
    }
  }
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c)
      act_out[(ty * RPT + r) * VSTRIDE + 8 * tx + c] = relu ? fmaxf(acc[r][c], 0.f) : acc[r][c];
}

// Per-pair path, tiles of 32 pairs per CTA of 256 threads (persistent): each
// warp selects and pools 4 pairs into the activation rows (A's rows 0..31,
// B's rows 32..63: [feature (16) || pose in A's frame (7) || 0 (9)]), then the
// CTA runs the predictor layer by layer out of shared memory.
// range_out (nullable): [P][2][6] cell ranges; feat_out (nullable): [P][2][16].
__global__ void __launch_bounds__(256, 2)
    vox_detect_kernel(PairInputs in, int n_shapes, const float* __restrict__ aabb,
                      const float* __restrict__ lat, VoxParams prm, float* __restrict__ logit,
                      int32_t* __restrict__ range_out, float* __restrict__ feat_out,
                      int* __restrict__ err) {
  extern __shared__ float vsm[];
  float* act0 = vsm;
  float* act1 = vsm + 2 * VTILE * VSTRIDE;
  int* valid = reinterpret_cast<int*>(vsm + 4 * VTILE * VSTRIDE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = in.n_pairs, n_tiles = (n + VTILE - 1) / VTILE;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    for (int j = 0; j < VTILE / 8; ++j) {
      const int tp = warp + 8 * j, p = tile * VTILE + tp;
      float* rowA = act0 + tp * VSTRIDE;
      float* rowB = act0 + (VTILE + tp) * VSTRIDE;
      int a = -1, b = -1, sa = -1, sb = -1;
      const bool ok = p < n && load_pair(in, n_shapes, p, &a, &b, &sa, &sb, lane == 0 ? err : nullptr);
      if (lane == 0) valid[tp] = ok;
      if (!ok) {
        rowA[lane] = 0.f;
        rowB[lane] = 0.f;
        continue;
      }
      const float* pa = in.poses + 7 * (size_t)a;
      const float* pb = in.poses + 7 * (size_t)b;
      float RA[9], RB[9], Rr[9], tr[3], dt[3];
      quat_to_rot(pa, RA);
      quat_to_rot(pb, RB);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          Rr[3 * i + k] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], RB[k], RB[3 + k], RB[6 + k]);
#pragma unroll
      for (int d = 0; d < 3; ++d) dt[d] = fsub(pb[4 + d], pa[4 + d]);
#pragma unroll
      for (int i = 0; i < 3; ++i) tr[i] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], dt[0], dt[1], dt[2]);
      float boxA[6], boxB[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) boxA[d] = aabb[6 * sa + d], boxB[d] = aabb[6 * sb + d];
      // B's box in A's frame, A's box in B's frame
      float loB[3], hiB[3], loA[3], hiA[3], cb[3], hb[3], ca[3], ha[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        cb[d] = fmul(fadd(boxB[d], boxB[3 + d]), 0.5f);
        hb[d] = fmul(fsub(boxB[3 + d], boxB[d]), 0.5f);
        ca[d] = fmul(fadd(boxA[d], boxA[3 + d]), 0.5f);
        ha[d] = fmul(fsub(boxA[3 + d], boxA[d]), 0.5f);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float c = fadd(dot3_rn(Rr[3 * i], Rr[3 * i + 1], Rr[3 * i + 2], cb[0], cb[1], cb[2]), tr[i]);
        const float h = dot3_rn(fabsf(Rr[3 * i]), fabsf(Rr[3 * i + 1]), fabsf(Rr[3 * i + 2]), hb[0],
                                hb[1], hb[2]);
        loB[i] = fsub(c, h);
        hiB[i] = fadd(c, h);
      }
      float e[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) e[d] = fsub(ca[d], tr[d]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float c = dot3_rn(Rr[k], Rr[3 + k], Rr[6 + k], e[0], e[1], e[2]);
        const float h = dot3_rn(fabsf(Rr[k]), fabsf(Rr[3 + k]), fabsf(Rr[6 + k]), ha[0], ha[1], ha[2]);
        loA[k] = fsub(c, h);
        hiA[k] = fadd(c, h);
      }
      int rA[6], rB[6];
      cell_ranges(boxA, loB, hiB, rA);
      cell_ranges(boxB, loA, hiA, rB);
      const float fA = pool_range(lat + (size_t)sa * VCELLS * VF, rA, lane);
      const float fB = pool_range(lat + (size_t)sb * VCELLS * VF, rB, lane);
      // B's pose in A's frame: q = conj(q_A) q_B, t = t_rel
      const float aw = pa[0], ax = pa[1], ay = pa[2], az = pa[3];
      const float bw = pb[0], bx = pb[1], by = pb[2], bz = pb[3];
      float pose[7] = {aw * bw + ax * bx + ay * by + az * bz, aw * bx - ax * bw - ay * bz + az * by,
                       aw * by + ax * bz - ay * bw - az * bx, aw * bz - ax * by + ay * bx - az * bw,
                       tr[0], tr[1], tr[2]};
      float vA = 0.f, vB = 0.f;
      if (lane < VF) {
        vA = fA;
        vB = fB;
      } else if (lane < VPIN) {
        vA = lane == VF ? 1.f : 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i)
          if (lane == VF + i) vB = pose[i];
      }
      rowA[lane] = vA;
      rowB[lane] = vB;
      if (range_out && lane < 12) range_out[12 * (size_t)p + lane] = lane < 6 ? rA[lane] : rB[lane - 6];
      if (feat_out && lane < VF) {
        feat_out[32 * (size_t)p + lane] = fA;
        feat_out[32 * (size_t)p + VF + lane] = fB;
      }
    }
    __syncthreads();
    // per-object MLP on 64 rows, max over the two objects, then 32 rows
    dense_layer<2 * VTILE, VK1>(act0, act1, prm.pw[0], prm.pb[0], true);
    __syncthreads();
    dense_layer<2 * VTILE, VPW>(act1, act0, prm.pw[1], prm.pb[1], true);
    __syncthreads();
    dense_layer<2 * VTILE, VPW>(act0, act1, prm.pw[2], prm.pb[2], true);
    __syncthreads();
    for (int i = threadIdx.x; i < VTILE * VPW; i += blockDim.x) {
      const int r = i / VPW, c = i % VPW;
      act0[r * VSTRIDE + c] = fmaxf(act1[r * VSTRIDE + c], act1[(VTILE + r) * VSTRIDE + c]);
    }
    __syncthreads();
    dense_layer<VTILE, VPW>(act0, act1, prm.qw[0], prm.qb[0], true);
    __syncthreads();
    dense_layer<VTILE, VPW>(act1, act0, prm.qw[1], prm.qb[1], true);
    __syncthreads();
    dense_layer<VTILE, VPW>(act0, act1, prm.qw[2], prm.qb[2], true);
    __syncthreads();
    if (threadIdx.x < VTILE) {
      const int p = tile * VTILE + threadIdx.x;
      if (p < n) {
        float acc = prm.qb[3][0];
        for (int c = 0; c < VPW; ++c) acc = fmaf(act1[threadIdx.x * VSTRIDE + c], prm.qw[3][c], acc);
        logit[p] = valid[threadIdx.x] ? acc : __int_as_float(0x7fc00000);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------ predictor on tcgen05 (BF16)
// Tiles of 128 pairs (one pair per TMEM lane).  Warps 0-7 select and pool the
// tile's pairs into the A operands X_A, X_B ([feature || pose || 0], K = 32,
// bf16) and run every epilogue (two warps per TMEM lane quarter, half of the
// columns each); one elected lane of warp 8 issues the MMAs (M = 128, N = 128)
// and streams the weights of q1..q3 through two 32 KB stages.  TMEM columns:
// object A [0, 128), object B [128, 256), the shared MLP [256, 384).
//   p1..p3 (both objects) -> max -> q1 -> q2 -> q3 -> q4 on the CUDA cores.
// Every mbarrier completes once per tile except the weight stages (stage 0
// carries q1 and q3 of every tile: two phases per tile); no wait is ever more
// than one phase behind.  Waits are bounded; on a timeout the CTA raises bit
// 2 of the error flag, drains and returns.
namespace vtc {
using namespace tc;
constexpr long long WAIT = 2000000000LL;
constexpr int WQ = 128 * 128 * 2;                       // one 128 x 128 bf16 weight tile
constexpr int S_WP1 = 0;                                // [128 x 32] bf16, 8 KB
constexpr int S_WP2 = S_WP1 + 128 * 32 * 2;             // resident p2, p3
constexpr int S_WP3 = S_WP2 + WQ;
constexpr int S_QST = S_WP3 + WQ;                       // two stages for q1..q3
constexpr int S_XA = S_QST + 2 * WQ;                    // [128 x 32] bf16
constexpr int S_XB = S_XA + 128 * 32 * 2;
constexpr int S_HA = S_XB + 128 * 32 * 2;               // [128 x 128] bf16 (also Z)
constexpr int S_HB = S_HA + WQ;
constexpr int S_BIAS = S_HB + WQ;                       // p1..p3, q1..q3 (128 each), q4 w (128), q4 b
constexpr int BIAS_FLOATS = 7 * 128 + 4;
constexpr int S_PART = S_BIAS + BIAS_FLOATS * 4;        // q4 partial sums [2][128]
constexpr int S_VALID = S_PART + 2 * 128 * 4;           // [128] int
constexpr int S_CTRL = S_VALID + 128 * 4;               // mbarriers, TMEM address, abort
constexpr int SMEM = S_CTRL + 256;
static_assert(SMEM <= 227 * 1024, "voxel tensor-core predictor shared memory");
// global image: [p1][p2][p3][q1][q2][q3][biases] (the resident part first)
constexpr int G_RES = S_QST;                            // p1, p2, p3 bytes
constexpr int G_Q = G_RES;                              // q1 at G_Q, q2, q3 follow
constexpr int G_BIAS = G_Q + 3 * WQ;
constexpr int G_BYTES = G_BIAS + BIAS_FLOATS * 4;
constexpr int THREADS = 288;

// TMEM row -> relu(x + b) bf16 into a K = 128 operand, this thread's 64 columns
__device__ __forceinline__ void epi64(uint32_t taddr, const float* b, unsigned char* dst, int row,
                                      int c0) {
  float v[32];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    tmem_ld32(taddr + c0 + 32 * h, v);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 8 * c, o = c0 + 32 * h + j;
      uint4 w;
      w.x = pack_relu_bf16(v[j + 0] + b[o + 0], v[j + 1] + b[o + 1]);
      w.y = pack_relu_bf16(v[j + 2] + b[o + 2], v[j + 3] + b[o + 3]);
      w.z = pack_relu_bf16(v[j + 4] + b[o + 4], v[j + 5] + b[o + 5]);
      w.w = pack_relu_bf16(v[j + 6] + b[o + 6], v[j + 7] + b[o + 7]);
      *reinterpret_cast<uint4*>(dst + kmajor_off(row, o, 128)) = w;
    }
  }
}

__global__ void __launch_bounds__(THREADS, 1)
    vox_tc_kernel(PairInputs in, int n_shapes, const float* __restrict__ aabb,
                  const float* __restrict__ lat, const unsigned char* __restrict__ img,
                  float* __restrict__ logit, int32_t* __restrict__ range_out,
                  float* __restrict__ feat_out, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = in.n_pairs, n_tiles = (n + 127) / 128;
  if ((int)blockIdx.x >= n_tiles) return;
  const int my_tiles = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  // barriers: 0 RES, 1 SF0, 2 SF1, 3 S0 (stage 0 read), 4 S1, 5 XR, 6 H1R, 7 H2R, 8 ZR0,
  // 9 ZR1, 10 ZR2, 11 P1D, 12 P2D, 13 P3D, 14 Q1D, 15 Q2D, 16 Q3D, 17 DRAIN,
  // 18 PART (both halves' partial logits written)
  const uint32_t bar0 = smem_u32(smem + S_CTRL);
  auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S_CTRL + 160);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + S_CTRL + 164);
  static_assert(19 * 8 <= 160, "mbarriers overlap the TMEM slot");
  if (tid == 0) {
    for (int i = 0; i < 19; ++i) mbar_init(BAR(i), ((i >= 5 && i <= 10) || i == 18) ? 256 : 1);
    *abort = 0;
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
  const float* bias = reinterpret_cast<const float*>(smem + S_BIAS);
  int* valid = reinterpret_cast<int*>(smem + S_VALID);
  float* part = reinterpret_cast<float*>(smem + S_PART);
  const uint32_t sWP1 = smem_u32(smem + S_WP1), sWP2 = smem_u32(smem + S_WP2),
                 sWP3 = smem_u32(smem + S_WP3), sQ0 = smem_u32(smem + S_QST),
                 sQ1 = smem_u32(smem + S_QST + WQ), sXA = smem_u32(smem + S_XA),
                 sXB = smem_u32(smem + S_XB), sHA = smem_u32(smem + S_HA),
                 sHB = smem_u32(smem + S_HB);
  bool ok = true;

  if (warp == 8) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      mbar_expect_tx(BAR(0), G_RES + BIAS_FLOATS * 4);
      for (int off = 0; off < G_RES; off += 32768)
        bulk_g2s(smem_u32(smem + off), img + off, min(32768, G_RES - off), BAR(0));
      bulk_g2s(smem_u32(smem + S_BIAS), img + G_BIAS, BIAS_FLOATS * 4, BAR(0));
      // q1 -> stage 0, q2 -> stage 1 of the first tile
      mbar_expect_tx(BAR(1), WQ);
      bulk_g2s(sQ0, img + G_Q, WQ, BAR(1));
      mbar_expect_tx(BAR(2), WQ);
      bulk_g2s(sQ1, img + G_Q + WQ, WQ, BAR(2));
    }
    __syncwarp();
    ok = mbar_wait_warp(BAR(0), 0, abort, WAIT);
    const uint32_t id = idesc_bf16(128, 128);
    auto chain = [&](uint32_t d, uint32_t a, uint32_t b, int K, uint32_t asbo) {
      // D[128 x 128] = A[128 x K] . B[128 x K]^T, K-major, K in steps of 16
      for (int kk = 0; kk < K / 16; ++kk)
        mma_bf16(d, sdesc(a + 256 * kk, 128, asbo), sdesc(b + 256 * kk, 128, asbo), id, kk > 0);
    };
    for (int t = 0; t < my_tiles && ok; ++t) {
      const uint32_t ph = t & 1;
      // p1 for both objects
      if (!(ok = mbar_wait_warp(BAR(5), ph, abort, WAIT))) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 0, sXA, sWP1, 32, 512);
        chain(tbase + 128, sXB, sWP1, 32, 512);
        mma_commit(BAR(11));
      }
      __syncwarp();
      if (!(ok = mbar_wait_warp(BAR(6), ph, abort, WAIT))) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 0, sHA, sWP2, 128, 2048);
        chain(tbase + 128, sHB, sWP2, 128, 2048);
        mma_commit(BAR(12));
      }
      __syncwarp();
      if (!(ok = mbar_wait_warp(BAR(7), ph, abort, WAIT))) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 0, sHA, sWP3, 128, 2048);
        chain(tbase + 128, sHB, sWP3, 128, 2048);
        mma_commit(BAR(13));
      }
      __syncwarp();
      // q1 (stage 0, phase 2t), q2 (stage 1, phase t), q3 (stage 0, phase 2t + 1)
      ok = mbar_wait_warp(BAR(8), ph, abort, WAIT) && mbar_wait_warp(BAR(1), 0, abort, WAIT);
      if (!ok) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 256, sHA, sQ0, 128, 2048);
        mma_commit(BAR(14));
        mma_commit(BAR(3));
      }
      __syncwarp();
      // stage 0 takes q3 once q1's MMAs are done
      if (!(ok = mbar_wait_warp(BAR(3), (2 * t) & 1, abort, WAIT))) break;
      if (lane == 0) {
        mbar_expect_tx(BAR(1), WQ);
        bulk_g2s(sQ0, img + G_Q + 2 * WQ, WQ, BAR(1));
      }
      __syncwarp();
      ok = mbar_wait_warp(BAR(9), ph, abort, WAIT) && mbar_wait_warp(BAR(2), ph, abort, WAIT);
      if (!ok) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 256, sHA, sQ1, 128, 2048);
        mma_commit(BAR(15));
        mma_commit(BAR(4));
      }
      __syncwarp();
      ok = mbar_wait_warp(BAR(10), ph, abort, WAIT) && mbar_wait_warp(BAR(1), 1, abort, WAIT);
      if (!ok) break;
      tc_fence_after();
      if (elect_one()) {
        chain(tbase + 256, sHA, sQ0, 128, 2048);
        mma_commit(BAR(16));
        mma_commit(BAR(3));
      }
      __syncwarp();
      // refill for the next tile: q1 -> stage 0 after q3's MMAs, q2 -> stage 1
      // after q2's
      if (t + 1 < my_tiles) {
        ok = mbar_wait_warp(BAR(3), (2 * t + 1) & 1, abort, WAIT) &&
             mbar_wait_warp(BAR(4), ph, abort, WAIT);
        if (!ok) break;
        if (lane == 0) {
          mbar_expect_tx(BAR(1), WQ);
          bulk_g2s(sQ0, img + G_Q, WQ, BAR(1));
          mbar_expect_tx(BAR(2), WQ);
          bulk_g2s(sQ1, img + G_Q + WQ, WQ, BAR(2));
        }
        __syncwarp();
      }
    }
    if (!ok) *abort = 1;
  } else {
    // ------------------------------------------------------ epilogue warps
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int row = tid & 127, half = tid >> 7, c0 = 64 * half;
    unsigned char* XA = smem + S_XA;
    unsigned char* XB = smem + S_XB;
    unsigned char* HA = smem + S_HA;
    unsigned char* HB = smem + S_HB;
    ok = mbar_wait_or_abort(BAR(0), 0, abort, WAIT);
    for (int t = 0; t < my_tiles && ok; ++t) {
      const uint32_t ph = t & 1;
      const int tile = (int)blockIdx.x + t * (int)gridDim.x;
      // selection and pooling: warp w takes the tile's pairs w, w + 8, ...
      for (int j = warp; j < 128; j += 8) {
        const int p = tile * 128 + j;
        int a = -1, b = -1, sa = -1, sb = -1;
        const bool good = p < n && load_pair(in, n_shapes, p, &a, &b, &sa, &sb, lane == 0 ? err : nullptr);
        float vA = 0.f, vB = 0.f;
        if (good) {
          const float* pa = in.poses + 7 * (size_t)a;
          const float* pb = in.poses + 7 * (size_t)b;
          float RA[9], RB[9], Rr[9], tr[3], dt[3];
          quat_to_rot(pa, RA);
          quat_to_rot(pb, RB);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              Rr[3 * i + k] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], RB[k], RB[3 + k], RB[6 + k]);
#pragma unroll
          for (int d = 0; d < 3; ++d) dt[d] = fsub(pb[4 + d], pa[4 + d]);
#pragma unroll
          for (int i = 0; i < 3; ++i) tr[i] = dot3_rn(RA[i], RA[3 + i], RA[6 + i], dt[0], dt[1], dt[2]);
          float boxA[6], boxB[6], loB[3], hiB[3], loA[3], hiA[3], cb[3], hb[3], ca[3], ha[3], e[3];
#pragma unroll
          for (int d = 0; d < 6; ++d) boxA[d] = aabb[6 * sa + d], boxB[d] = aabb[6 * sb + d];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            cb[d] = fmul(fadd(boxB[d], boxB[3 + d]), 0.5f);
            hb[d] = fmul(fsub(boxB[3 + d], boxB[d]), 0.5f);
            ca[d] = fmul(fadd(boxA[d], boxA[3 + d]), 0.5f);
            ha[d] = fmul(fsub(boxA[3 + d], boxA[d]), 0.5f);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float c = fadd(dot3_rn(Rr[3 * i], Rr[3 * i + 1], Rr[3 * i + 2], cb[0], cb[1], cb[2]), tr[i]);
            const float h = dot3_rn(fabsf(Rr[3 * i]), fabsf(Rr[3 * i + 1]), fabsf(Rr[3 * i + 2]), hb[0], hb[1], hb[2]);
            loB[i] = fsub(c, h);
            hiB[i] = fadd(c, h);
          }
#pragma unroll
          for (int d = 0; d < 3; ++d) e[d] = fsub(ca[d], tr[d]);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float c = dot3_rn(Rr[k], Rr[3 + k], Rr[6 + k], e[0], e[1], e[2]);
            const float h = dot3_rn(fabsf(Rr[k]), fabsf(Rr[3 + k]), fabsf(Rr[6 + k]), ha[0], ha[1], ha[2]);
            loA[k] = fsub(c, h);
            hiA[k] = fadd(c, h);
          }
          int rA[6], rB[6];
          cell_ranges(boxA, loB, hiB, rA);
          cell_ranges(boxB, loA, hiA, rB);
          const float fA = pool_range(lat + (size_t)sa * VCELLS * VF, rA, lane);
          const float fB = pool_range(lat + (size_t)sb * VCELLS * VF, rB, lane);
          const float aw = pa[0], ax = pa[1], ay = pa[2], az = pa[3];
          const float bw = pb[0], bx = pb[1], by = pb[2], bz = pb[3];
          const float pose[7] = {aw * bw + ax * bx + ay * by + az * bz, aw * bx - ax * bw - ay * bz + az * by,
                                 aw * by + ax * bz - ay * bw - az * bx, aw * bz - ax * by + ay * bx - az * bw,
                                 tr[0], tr[1], tr[2]};
          if (lane < VF) {
            vA = fA;
            vB = fB;
          } else if (lane < VPIN) {
            vA = lane == VF ? 1.f : 0.f;
#pragma unroll
            for (int i = 0; i < 7; ++i)
              if (lane == VF + i) vB = pose[i];
          }
          if (range_out && lane < 12) range_out[12 * (size_t)p + lane] = lane < 6 ? rA[lane] : rB[lane - 6];
          if (feat_out && lane < VF) {
            feat_out[32 * (size_t)p + lane] = fA;
            feat_out[32 * (size_t)p + VF + lane] = fB;
          }
        }
        const __nv_bfloat16 hA = __float2bfloat16_rn(vA), hB = __float2bfloat16_rn(vB);
        *reinterpret_cast<__nv_bfloat16*>(XA + kmajor_off(j, lane, 32)) = hA;
        *reinterpret_cast<__nv_bfloat16*>(XB + kmajor_off(j, lane, 32)) = hB;
        if (lane == 0) valid[j] = good;
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(BAR(5));
      // p1 .. p3
      for (int l = 0; l < 3 && ok; ++l) {
        if (!(ok = mbar_wait_or_abort(BAR(11 + l), ph, abort, WAIT))) break;
        tc_fence_after();
        if (l < 2) {
          epi64(tbase + lane_off, bias + 128 * l, HA, row, c0);
          epi64(tbase + lane_off + 128, bias + 128 * l, HB, row, c0);
        } else {
          // relu of both objects, max over the objects -> Z (in H_A)
          float va[32], vb[32];
          const float* b3 = bias + 256;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            tmem_ld32(tbase + lane_off + c0 + 32 * h, va);
            tmem_ld32(tbase + lane_off + 128 + c0 + 32 * h, vb);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int jj = 8 * c, o = c0 + 32 * h + jj;
              float z[8];
#pragma unroll
              for (int q = 0; q < 8; ++q)
                z[q] = fmaxf(fmaxf(va[jj + q] + b3[o + q], 0.f), fmaxf(vb[jj + q] + b3[o + q], 0.f));
              uint4 w;
              w.x = pack_bf16(z[0], z[1]);
              w.y = pack_bf16(z[2], z[3]);
              w.z = pack_bf16(z[4], z[5]);
              w.w = pack_bf16(z[6], z[7]);
              *reinterpret_cast<uint4*>(HA + kmajor_off(row, o, 128)) = w;
            }
          }
        }
        fence_async_smem();
        tc_fence_before();
        mbar_arrive(BAR(6 + l));  // H1R, H2R, ZR0
      }
      // q1, q2: Z <- relu(.) ; q3: the logit
      for (int l = 0; l < 2 && ok; ++l) {
        if (!(ok = mbar_wait_or_abort(BAR(14 + l), ph, abort, WAIT))) break;
        tc_fence_after();
        epi64(tbase + lane_off + 256, bias + 384 + 128 * l, HA, row, c0);
        fence_async_smem();
        tc_fence_before();
        mbar_arrive(BAR(9 + l));  // ZR1, ZR2
      }
      if (!ok) break;
      if (!(ok = mbar_wait_or_abort(BAR(16), ph, abort, WAIT))) break;
      tc_fence_after();
      {
        const float* b6 = bias + 640;
        const float* w4 = bias + 768;
        float v[32], acc = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld32(tbase + lane_off + 256 + c0 + 32 * h, v);
#pragma unroll
          for (int q = 0; q < 32; ++q) acc = fmaf(fmaxf(v[q] + b6[c0 + 32 * h + q], 0.f), w4[c0 + 32 * h + q], acc);
        }
        part[half * 128 + row] = acc;
      }
      tc_fence_before();
      // (a bounded mbarrier handoff rather than a named barrier: a thread that
      // gave up on a wait must not leave the others blocked.)  The next tile's
      // partial sums cannot overwrite these before they are read: writing them
      // needs that tile's MMAs, which need every thread's arrival on XR.
      mbar_arrive(BAR(18));
      if (half == 0) {
        if (!(ok = mbar_wait_or_abort(BAR(18), ph, abort, WAIT))) break;
        const int p = tile * 128 + row;
        if (p < n) logit[p] = valid[row] ? part[row] + part[128 + row] + bias[896]
                                         : __int_as_float(0x7fc00000);
      }
    }
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) atomicOr(err, 2);
    if (warp == 8 && elect_one()) {
      mma_commit(BAR(17));
      mbar_wait(BAR(17), 0, WAIT);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}
}  // namespace vtc

}  // namespace
}  // namespace locc

using namespace locc;

struct locc_voxel {
  int n_shapes = 0, n_points = 0, n_sm = 148;
  int prec = LOCC_FP32;
  unsigned char* d_img16 = nullptr;  // bf16 predictor image of the tensor-core kernel
  float* d_points = nullptr;  // [S][N][3]
  float* d_aabb = nullptr;    // [S][6]
  float* d_params = nullptr;  // device parameter images
  float* d_lat = nullptr;     // [S][216][16]
  float* d_work = nullptr;    // encoder scratch
  int* d_err = nullptr;
  VoxParams prm{};
  // scratch views
  int* cellmax = nullptr;
  float *s[4] = {}, *u[4] = {}, *g = nullptr;
};

namespace {

constexpr char VOX_MAGIC[8] = {'L', 'O', 'C', 'C', 'V', '0', '0', '1'};

// Host layout conversion of the blob's tensors into the device images.
struct VoxHostImage {
  std::vector<float> data;
  std::vector<size_t> off;  // offsets of the images, in the order they are added
  size_t add(const std::vector<float>& v) {
    const size_t o = data.size();
    data.insert(data.end(), v.begin(), v.end());
    while (data.size() % 4) data.push_back(0.f);  // 16-byte alignment of every image
    off.push_back(o);
    return o;
  }
};

// W [out][in] -> W^T [in_pad][out] (rows in..in_pad-1 zero)
std::vector<float> transpose_linear(const float* w, int out, int in, int in_pad) {
  std::vector<float> t((size_t)in_pad * out, 0.f);
  for (int o = 0; o < out; ++o)
    for (int i = 0; i < in; ++i) t[(size_t)i * out + o] = w[(size_t)o * in + i];
  return t;
}
// conv W [out][in][27] -> [27][in][out]; transposed conv W [in][out][27] -> [27][in][out]
std::vector<float> conv_image(const float* w, int cin, int cout, bool transposed) {
  std::vector<float> t((size_t)27 * cin * cout);
  for (int i = 0; i < cin; ++i)
    for (int o = 0; o < cout; ++o)
      for (int k = 0; k < 27; ++k) {
        const float v = transposed ? w[((size_t)i * cout + o) * 27 + k] : w[((size_t)o * cin + i) * 27 + k];
        t[((size_t)k * cin + i) * cout + o] = v;
      }
  return t;
}

uint16_t bf16_of(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even (finite values)
  return (uint16_t)(u >> 16);
}

// Predictor image of vox_tc_kernel: W [out][in] of p1 (K padded to 32), p2,
// p3, q1, q2, q3 as K-major bf16 tiles [128][K], then float32 biases p1..q3,
// q4's weights and bias.
std::vector<unsigned char> tc_image(const float* p1w, const float* p1b, const float* const* w,
                                    const float* const* b, const float* q4w, const float* q4b) {
  std::vector<unsigned char> img(vtc::G_BYTES, 0);
  auto put = [&](size_t off, const float* W, int K, int Kin) {
    for (int n = 0; n < 128; ++n)
      for (int k = 0; k < K; ++k) {
        const uint16_t v = bf16_of(k < Kin ? W[(size_t)n * Kin + k] : 0.f);
        std::memcpy(img.data() + off + tc::kmajor_off(n, k, K), &v, 2);
      }
  };
  put(0, p1w, 32, VPIN);
  put(vtc::S_WP2, w[0], 128, 128);
  put(vtc::S_WP3, w[1], 128, 128);
  for (int l = 0; l < 3; ++l) put(vtc::G_Q + (size_t)l * vtc::WQ, w[2 + l], 128, 128);
  float* bias = reinterpret_cast<float*>(img.data() + vtc::G_BIAS);
  std::memcpy(bias, p1b, 128 * 4);
  for (int l = 0; l < 5; ++l) std::memcpy(bias + 128 * (l + 1), b[l], 128 * 4);
  std::memcpy(bias + 768, q4w, 128 * 4);
  bias[896] = q4b[0];
  return img;
}

int vox_fail(int code, const char* msg) {
  set_error(msg);
  return code;
}

int vox_encode(locc_voxel* h, cudaStream_t st) {
  const int S = h->n_shapes;
  cudaMemsetAsync(h->cellmax, 0, (size_t)S * VCELLS * VH * sizeof(int), st);
  vox_points_kernel<<<dim3(S, (h->n_points + 31) / 32), 256, 0, st>>>(h->d_points, h->d_aabb,
                                                                     h->n_points, h->prm, h->cellmax);
  const float* x = reinterpret_cast<const float*>(h->cellmax);
  vox_conv_kernel<<<dim3(S, 64), VC, 0, st>>>(x, VH, nullptr, 0, 6, 4, 0, 0, h->prm.cw[0], h->prm.cb[0], h->s[0]);
  for (int l = 1; l < 4; ++l)
    vox_conv_kernel<<<dim3(S, 64), VC, 0, st>>>(h->s[l - 1], VC, nullptr, 0, 4, 4, 1, 0, h->prm.cw[l],
                                                h->prm.cb[l], h->s[l]);
  vox_global_kernel<<<S, VC, 0, st>>>(h->s[3], h->g);
  vox_conv_kernel<<<dim3(S, 64), VC, 0, st>>>(h->s[3], VC, nullptr, 0, 4, 4, 1, 1, h->prm.dw[0], h->prm.db[0], h->u[0]);
  vox_conv_kernel<<<dim3(S, 64), VC, 0, st>>>(h->u[0], VC, h->s[2], VC, 4, 4, 1, 1, h->prm.dw[1], h->prm.db[1], h->u[1]);
  vox_conv_kernel<<<dim3(S, 64), VC, 0, st>>>(h->u[1], VC, h->s[1], VC, 4, 4, 1, 1, h->prm.dw[2], h->prm.db[2], h->u[2]);
  vox_conv_kernel<<<dim3(S, 216), VC, 0, st>>>(h->u[2], VC, h->s[0], VC, 4, 6, 0, 1, h->prm.dw[3], h->prm.db[3], h->u[3]);
  vox_final_kernel<<<dim3(S, VCELLS / 8), 128, 0, st>>>(h->u[3], h->g, h->prm, h->d_lat);
  if (cudaGetLastError() != cudaSuccess) return vox_fail(LOCC_ERR_CUDA, "voxel encoder launch failed");
  return LOCC_OK;
}

}  // namespace

extern "C" {

int locc_voxel_create(const locc_shape_library* lib, const void* blob, size_t blob_bytes,
                      locc_voxel** out) {
  if (!out) return vox_fail(LOCC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!lib || !lib->points || !lib->aabb || lib->n_shapes < 1 || lib->n_points < 1 ||
      lib->n_points > 65536)
    return vox_fail(LOCC_ERR_INVALID_ARG, "invalid shape library");
  if (!blob || blob_bytes < 16 || std::memcmp(blob, VOX_MAGIC, 8) != 0)
    return vox_fail(LOCC_ERR_BAD_WEIGHTS, "voxel weights: bad magic");
  uint32_t version, count;
  std::memcpy(&version, static_cast<const char*>(blob) + 8, 4);
  std::memcpy(&count, static_cast<const char*>(blob) + 12, 4);
  if (version != 1 || count != (uint32_t)LOCC_VOXEL_N_PARAMS ||
      blob_bytes != 16 + (size_t)count * 4)
    return vox_fail(LOCC_ERR_BAD_WEIGHTS, "voxel weights: wrong version or size");
  std::vector<float> P(count);
  std::memcpy(P.data(), static_cast<const char*>(blob) + 16, (size_t)count * 4);
  for (float v : P)
    if (!std::isfinite(v)) return vox_fail(LOCC_ERR_BAD_WEIGHTS, "voxel weights: non-finite value");

  // walk the blob in its fixed order
  size_t o = 0;
  auto take = [&](size_t n) {
    const float* p = P.data() + o;
    o += n;
    return p;
  };
  VoxHostImage img;
  std::vector<size_t> at;
  auto lin = [&](int out_, int in_, int in_pad) {
    const float* w = take((size_t)out_ * in_);
    const float* b = take(out_);
    at.push_back(img.add(transpose_linear(w, out_, in_, in_pad)));
    at.push_back(img.add(std::vector<float>(b, b + out_)));
  };
  auto conv = [&](int cin, int cout, bool tr) {
    const float* w = take((size_t)cin * cout * 27);
    const float* b = take(cout);
    at.push_back(img.add(conv_image(w, cin, cout, tr)));
    at.push_back(img.add(std::vector<float>(b, b + cout)));
  };
  lin(VH, 3, 3);                    // e1
  lin(VH, VH, VH);                  // e2
  lin(VH, VH, VH);                  // e3
  conv(VH, VC, false);              // c1
  for (int l = 0; l < 3; ++l) conv(VC, VC, false);  // c2..c4
  conv(VC, VC, true);               // d1
  for (int l = 0; l < 3; ++l) conv(2 * VC, VC, true);  // d2..d4
  lin(VF, 3 * VC, 3 * VC);          // f
  lin(VPW, VPIN, VK1);              // p1
  lin(VPW, VPW, VPW);               // p2
  lin(VPW, VPW, VPW);               // p3
  for (int l = 0; l < 3; ++l) lin(VPW, VPW, VPW);  // q1..q3
  lin(1, VPW, VPW);                 // q4
  if (o != P.size()) return vox_fail(LOCC_ERR_BAD_WEIGHTS, "voxel weights: layout mismatch");
  // predictor tensors in the blob (they close it): p1 w b, p2, p3, q1, q2, q3, q4
  const size_t pred = P.size() - ((size_t)VPW * VPIN + VPW + 5 * ((size_t)VPW * VPW + VPW) + VPW + 1);
  const float* pp = P.data() + pred;
  const float* p1w = pp;
  const float* p1b = p1w + VPW * VPIN;
  const float* ws[5];
  const float* bs[5];
  const float* cur = p1b + VPW;
  for (int l = 0; l < 5; ++l) {
    ws[l] = cur;
    bs[l] = cur + VPW * VPW;
    cur = bs[l] + VPW;
  }
  const std::vector<unsigned char> img16 = tc_image(p1w, p1b, ws, bs, cur, cur + VPW);

  auto* h = new locc_voxel();
  h->n_shapes = lib->n_shapes;
  h->n_points = lib->n_points;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int S = h->n_shapes;
  const size_t pts_bytes = (size_t)S * h->n_points * 3 * sizeof(float);
  const size_t work_floats = (size_t)S * VCELLS * VH          // cellmax
                             + 4 * (size_t)S * 64 * VC        // s1..s4
                             + 3 * (size_t)S * 64 * VC        // u1..u3
                             + (size_t)S * VCELLS * VC        // u4
                             + (size_t)S * 2 * VC;            // g
  bool ok = cudaMalloc(&h->d_points, pts_bytes) == cudaSuccess &&
            cudaMalloc(&h->d_aabb, (size_t)S * 6 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->d_params, img.data.size() * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->d_lat, (size_t)S * VCELLS * VF * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->d_work, work_floats * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->d_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_img16, img16.size()) == cudaSuccess;
  ok = ok && cudaMemcpy(h->d_points, lib->points, pts_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_aabb, lib->aabb, (size_t)S * 6 * sizeof(float), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(h->d_params, img.data.data(), img.data.size() * sizeof(float),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->d_err, 0, sizeof(int)) == cudaSuccess &&
       cudaMemcpy(h->d_img16, img16.data(), img16.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    locc_voxel_destroy(h);
    return vox_fail(LOCC_ERR_OOM, "voxel handle: device allocation or copy failed");
  }
  const float* dp = h->d_params;
  int q = 0;
  auto nxt = [&]() { return dp + at[q++]; };
  VoxParams& m = h->prm;
  m.e1w = nxt(), m.e1b = nxt(), m.e2w = nxt(), m.e2b = nxt(), m.e3w = nxt(), m.e3b = nxt();
  for (int l = 0; l < 4; ++l) m.cw[l] = nxt(), m.cb[l] = nxt();
  for (int l = 0; l < 4; ++l) m.dw[l] = nxt(), m.db[l] = nxt();
  m.fw = nxt(), m.fb = nxt();
  for (int l = 0; l < 3; ++l) m.pw[l] = nxt(), m.pb[l] = nxt();
  for (int l = 0; l < 4; ++l) m.qw[l] = nxt(), m.qb[l] = nxt();
  float* w = h->d_work;
  h->cellmax = reinterpret_cast<int*>(w);
  w += (size_t)S * VCELLS * VH;
  for (int l = 0; l < 4; ++l) h->s[l] = w, w += (size_t)S * 64 * VC;
  for (int l = 0; l < 3; ++l) h->u[l] = w, w += (size_t)S * 64 * VC;
  h->u[3] = w, w += (size_t)S * VCELLS * VC;
  h->g = w;
  if (cudaFuncSetAttribute(vox_detect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)VOX_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(vtc::vox_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           vtc::SMEM) != cudaSuccess) {
    cudaGetLastError();
    locc_voxel_destroy(h);
    return vox_fail(LOCC_ERR_CUDA, "cudaFuncSetAttribute failed for vox_detect_kernel");
  }
  int rc = vox_encode(h, nullptr);
  if (rc == LOCC_OK && cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    rc = vox_fail(LOCC_ERR_CUDA, "voxel encoder failed");
  }
  if (rc != LOCC_OK) {
    locc_voxel_destroy(h);
    return rc;
  }
  *out = h;
  return LOCC_OK;
}

int locc_voxel_encode(locc_voxel* h, void* stream) {
  if (!h) return vox_fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  return vox_encode(h, static_cast<cudaStream_t>(stream));
}

int locc_voxel_latents(locc_voxel* h, float* out, void* stream) {
  if (!h || !out) return vox_fail(LOCC_ERR_INVALID_ARG, "handle or out is NULL");
  if (cudaMemcpyAsync(out, h->d_lat, (size_t)h->n_shapes * VCELLS * VF * sizeof(float),
                      cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return vox_fail(LOCC_ERR_CUDA, "latent copy failed");
  return LOCC_OK;
}

static int vox_launch(locc_voxel* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                      const int32_t* pairs, int32_t n_pairs, float* logit, int32_t* ranges,
                      float* feat, void* stream) {
  if (!h) return vox_fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (n_pairs < 0 || n_obj < 0) return vox_fail(LOCC_ERR_INVALID_ARG, "negative size");
  if (n_pairs == 0) return LOCC_OK;
  if (!poses || !obj_shape || !pairs || !logit)
    return vox_fail(LOCC_ERR_INVALID_ARG, "NULL array argument");
  PairInputs in{poses, obj_shape, pairs, n_obj, n_pairs};
  if (h->prec == LOCC_BF16) {
    const int tiles128 = (n_pairs + 127) / 128;
    vtc::vox_tc_kernel<<<std::min(tiles128, h->n_sm), vtc::THREADS, vtc::SMEM,
                         static_cast<cudaStream_t>(stream)>>>(in, h->n_shapes, h->d_aabb, h->d_lat,
                                                              h->d_img16, logit, ranges, feat, h->d_err);
    if (cudaGetLastError() != cudaSuccess) return vox_fail(LOCC_ERR_CUDA, "vox_tc_kernel launch failed");
    return LOCC_OK;
  }
  const int tiles = (n_pairs + VTILE - 1) / VTILE;
  const int grid = std::min(tiles, 2 * h->n_sm);
  vox_detect_kernel<<<grid, 256, VOX_SMEM, static_cast<cudaStream_t>(stream)>>>(
      in, h->n_shapes, h->d_aabb, h->d_lat, h->prm, logit, ranges, feat, h->d_err);
  if (cudaGetLastError() != cudaSuccess) return vox_fail(LOCC_ERR_CUDA, "vox_detect_kernel launch failed");
  return LOCC_OK;
}

int locc_voxel_detect(locc_voxel* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                      const int32_t* pairs, int32_t n_pairs, float* logit, void* stream) {
  return vox_launch(h, poses, obj_shape, n_obj, pairs, n_pairs, logit, nullptr, nullptr, stream);
}

int locc_voxel_detect_ex(locc_voxel* h, const float* poses, const int32_t* obj_shape, int32_t n_obj,
                         const int32_t* pairs, int32_t n_pairs, float* logit, int32_t* cell_ranges,
                         float* pooled, void* stream) {
  return vox_launch(h, poses, obj_shape, n_obj, pairs, n_pairs, logit, cell_ranges, pooled, stream);
}

int locc_voxel_set_precision(locc_voxel* h, int32_t precision) {
  if (!h) return vox_fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  if (precision != LOCC_FP32 && precision != LOCC_BF16)
    return vox_fail(LOCC_ERR_INVALID_ARG, "voxel predictor precision must be LOCC_FP32 or LOCC_BF16");
  h->prec = precision;
  return LOCC_OK;
}

int locc_voxel_status(locc_voxel* h, void* stream) {
  if (!h) return vox_fail(LOCC_ERR_INVALID_ARG, "handle is NULL");
  int err = 0;
  if (cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                      static_cast<cudaStream_t>(stream)) != cudaSuccess ||
      cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return vox_fail(LOCC_ERR_CUDA, "voxel status: CUDA error");
  }
  if (err) {
    cudaMemsetAsync(h->d_err, 0, sizeof(int), static_cast<cudaStream_t>(stream));
    return vox_fail(LOCC_ERR_BAD_INDEX, "a pair had an out-of-range object index or shape id");
  }
  return LOCC_OK;
}

void locc_voxel_destroy(locc_voxel* h) {
  if (!h) return;
  cudaFree(h->d_points);
  cudaFree(h->d_aabb);
  cudaFree(h->d_params);
  cudaFree(h->d_lat);
  cudaFree(h->d_work);
  cudaFree(h->d_err);
  cudaFree(h->d_img16);
  delete h;
}

}  // extern "C"

// Device code shared by the BF16 tensor-core encoder (net_tc.cu) and the
// fused crop + encoder kernel (fused.cu): the layout of the encoder's bf16
// weight image, the layer-1 X tile of one crop row, the layer-1/2 epilogue
// (TMEM row -> ReLU -> bf16 A operand), the masked max-pool of layer 3 over
// TMEM columns, and the pooled-feature store in the head's operand layout.
#pragma once

#include "common.cuh"
#include "tc_ptx.cuh"

namespace locc {
namespace {

using namespace tc;

constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

// The biases of layers 1 and 2 are added by the MMAs themselves (the
// epilogues then only apply ReLU, round and store, which more than halves
// their instruction count): layer 1 through two constant-one columns of the X
// tile against b1 (hi, lo) in W1's spare K columns; layer 2 through one extra
// K = 16 step, issued first so that it also initialises the accumulator: a
// tile of ones (columns 0, 1) against a tile holding b2 (hi, lo) in its K
// columns 0, 1.  The bias tile stores only the first core matrix of each
// 8-row group (K columns 0..7, SBO 128); its second core matrix (K 8..15)
// reads the ones tile through LBO = 2048, finite values that meet the ones
// tile's zero columns.
constexpr int E_W1 = 0;                       // [64 x 16]   2 KB
constexpr int E_W2 = E_W1 + 64 * 16 * 2;      // [128 x 64] 16 KB
constexpr int E_W3 = E_W2 + 128 * 64 * 2;     // [256 x 128] 64 KB
constexpr int E_B2T = E_W3 + 256 * 128 * 2;   // [128 x 8] b2 (hi, lo), 2 KB
constexpr int E_ONE = E_B2T + 128 * 8 * 2;    // [128 x 16] ones in columns 0, 1, 4 KB
constexpr int E_BIAS = E_ONE + 128 * 16 * 2;  // b1 64, b2 128, b3 256 (f32)
constexpr int E_IMG_BYTES = E_BIAS + (64 + 128 + 256) * 4;
static_assert(E_IMG_BYTES % 16 == 0, "image must be a whole number of 16-byte chunks");

// One crop row (x, y, z, valid) -> row `row` of the layer-1 A operand X
// [128 x 16] (K-major, no swizzle): K columns 0..8 hold x_hi, y_hi, z_hi,
// x_lo, y_lo, z_lo, x_hi, y_hi, z_hi (bf16 hi/lo split against W1img's
// W_hi, W_hi, W_lo columns), 9 and 10 the ones that meet b1 (hi, lo).
__device__ __forceinline__ void x_tile_row(float4 q, unsigned char* opd, int row) {
  const __nv_bfloat16 xh = __float2bfloat16_rn(q.x), yh = __float2bfloat16_rn(q.y),
                      zh = __float2bfloat16_rn(q.z);
  const float fx = __bfloat162float(xh), fy = __bfloat162float(yh), fz = __bfloat162float(zh);
  uint4 c0, c1;
  c0.x = pack_bf16(fx, fy);
  c0.y = pack_bf16(fz, q.x - fx);
  c0.z = pack_bf16(q.y - fy, q.z - fz);
  c0.w = pack_bf16(fx, fy);
  c1.x = pack_bf16(fz, 1.f);  // K columns 9, 10: ones against b1 (hi, lo)
  c1.y = pack_bf16(1.f, 0.f);
  c1.z = c1.w = 0u;
  *reinterpret_cast<uint4*>(opd + kmajor_off(row, 0, 16)) = c0;
  *reinterpret_cast<uint4*>(opd + kmajor_off(row, 8, 16)) = c1;
}

// Epilogue of layers 1 and 2: TMEM row (bias already accumulated) -> relu ->
// bf16 row of the next A operand (K = NCOL).
template <int NCOL>
__device__ __forceinline__ void enc_epi_rows(uint32_t taddr, unsigned char* dst, int row) {
  float v[64];
#pragma unroll 1
  for (int h = 0; h < NCOL / 64; ++h) {
    tmem_ld32x2(taddr + 64 * h, v);  // 64 columns, two loads in flight
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint4 w;
      const int j = 8 * c, o = 64 * h + j;
      w.x = pack_relu_bf16(v[j + 0], v[j + 1]);
      w.y = pack_relu_bf16(v[j + 2], v[j + 3]);
      w.z = pack_relu_bf16(v[j + 4], v[j + 5]);
      w.w = pack_relu_bf16(v[j + 6], v[j + 7]);
      *reinterpret_cast<uint4*>(dst + kmajor_off(row, o, NCOL)) = w;
    }
  }
}

// Masked max over the valid points of each object of one layer-3 half
// (thread = channel): TMEM columns [0, 64) are A's points, [64, 128) B's.
__device__ __forceinline__ void enc_pool(uint32_t taddr, int cntA, int cntB, float* mA, float* mB) {
  float v[32];
  float a = -INFINITY, b = -INFINITY;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cnt = q < 2 ? cntA : cntB;
    const int c0 = 32 * (q & 1);  // first point slot of this chunk within its object
    if (c0 < cnt) {
      float m = -INFINITY;
      if (c0 + 32 <= cnt) {
        m = tmem_ldmax32(taddr + 32 * q);  // whole chunk valid: max in the load
      } else {
        tmem_ld32(taddr + 32 * q, v);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) m = fmaxf(m, (c0 + jj < cnt) ? v[jj] : -INFINITY);
      }
      if (q < 2) a = fmaxf(a, m);
      else b = fmaxf(b, m);
    }
  }
  *mA = a;
  *mB = b;
}

// Pooled features in the BF16 head's A-operand layout (FT_* in common.cuh):
// tiles of 128 pairs, each 32 K-chunks of 16 features; a chunk holds the
// bf16 value (hi) as a K-major no-swizzle [128 x 16] tile and the bf16
// rounding of the remainder (lo, f - hi) as a second tile FT_SUB bytes
// further.  The head multiplies both with its weights, so the features enter
// it to about 2^-16 relative.

// Pooled feature k of pair p (rel = p - first pair of the launch): float32
// [P][512] when feat is given, and always the hi / lo pair in the head's
// operand tiles, so that the head loads A chunks with bulk copies.
__device__ __forceinline__ void put_feat(float* feat, __nv_bfloat16* ftile, int p, int rel, int k,
                                         float v) {
  if (feat) feat[(size_t)p * 512 + k] = v;
  unsigned char* t = reinterpret_cast<unsigned char*>(ftile) + (size_t)(rel >> 7) * FT_TILE +
                     (size_t)(k / FT_K) * FT_CHUNK + kmajor_off(rel & 127, k % FT_K, FT_K);
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(t) = hi;
  *reinterpret_cast<__nv_bfloat16*>(t + FT_SUB) = __float2bfloat16_rn(v - __bfloat162float(hi));
}

}  // namespace
}  // namespace locc

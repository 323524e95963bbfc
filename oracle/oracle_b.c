/*
 * ORACLE (b): plain CPU forward and backward of the local-crop network.
 *
 * Test infrastructure only.  Nothing in the product library links, loads or
 * calls this file; only tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code with the CUDA path.
 *
 * What it computes, per object pair (A, B):
 *   1. Pose composition (Sec. III, "create the OBB ... by using their poses";
 *      appendix, "apply a transformation ... with the given pose"):
 *      R(q) of each unit quaternion, R_rel = R_A^T R_B, t_rel = R_A^T (t_B - t_A).
 *   2. Crop centre: the centre of the intersection region of A's box and B's
 *      box, both expressed in A's body frame (appendix, "intersection region of
 *      two AABB").  B's box in A's frame is the axis-aligned box of B's oriented
 *      box.  The margin epsilon of the appendix moves both bounds of the
 *      region equally and so leaves the centre unchanged.
 *   3. Crop selection (Sec. III, "select the features in colliding cells",
 *      read as: the surface points of each object that lie inside a ball of
 *      radius r about the crop centre): each object keeps at most kmax points,
 *      nearest first, ties to the lower point index; the rest is zero padding.
 *   4. Canonical crop frame: A's body axes with origin at the crop centre.
 *   5. Per-point encoder 3->64->128->256 with ReLU after every layer
 *      (appendix: point-wise MLP, ReLU on all layers), max-pool over the valid
 *      points of each object (an empty crop pools to 0), head on the
 *      concatenated [f_A, f_B] 512->256->256 (ReLU) -> 8 (linear).
 *   6. Epilogue: logit, contact point and normal mapped back to the world frame,
 *      penetration depth.
 *   7. Loss and gradients: binary cross-entropy on the logit (Sec. III-A loss),
 *      regression terms on point / normal / depth, alpha * mean(f^2) on the
 *      pooled embedding (the paper's alpha |f^SE|^2, alpha = 0.5).
 *
 * Steps 1-4 run in float32, one IEEE operation at a time in the fixed order
 * written below (this file must be compiled with -ffp-contract=off and without
 * -ffast-math), so that crop index sets are reproducible bit for bit.  Steps
 * 5-7 run in float64 with the float32 parameters widened.
 *
 * Operand mode "bf16" of the loss and gradient (orb_loss_grad, bf16 != 0):
 * the same float64 arithmetic, except that both operands of every product
 * that a bf16 tensor-core trainer runs as a matrix multiply are first rounded
 * to bfloat16 (orb_bf16: to float32, then to 8 significant bits, ties to
 * even).  Those products: layers 2 and 3 of the encoder and layers 1 and 2 of
 * the head in the forward pass, and in the backward pass the weight
 * gradients and the input gradients of those head layers and of encoder layer
 * 2.  Everything else stays unrounded: encoder layer 1, the head's output
 * layer, the loss, layer 3's backward (sparse: only argmax rows), biases.
 * The max-pool's argmax is then decided on the same rounded operands as in
 * such a trainer, which leaves only the float32-versus-float64 accumulation
 * between the two.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORB_FEAT 256
#define ORB_OUT 8

/* ---------------------------------------------------------------- float32 */

/* Rotation matrix of the unit quaternion (w, x, y, z); body -> world. */
static void orb_rotation(const float q[4], float R[3][3]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  R[0][0] = 1.0f - 2.0f * (yy + zz);
  R[0][1] = 2.0f * (xy - wz);
  R[0][2] = 2.0f * (xz + wy);
  R[1][0] = 2.0f * (xy + wz);
  R[1][1] = 1.0f - 2.0f * (xx + zz);
  R[1][2] = 2.0f * (yz - wx);
  R[2][0] = 2.0f * (xz - wy);
  R[2][1] = 2.0f * (yz + wx);
  R[2][2] = 1.0f - 2.0f * (xx + yy);
}

/* (a0 b0 + a1 b1) + a2 b2, each product and sum rounded to float32. */
static float orb_dot3(float a0, float a1, float a2, float b0, float b1,
                      float b2) {
  float s = a0 * b0;
  s = s + a1 * b1;
  return s + a2 * b2;
}

typedef struct {
  float Rrel[3][3];
  float trel[3];
  float RA[3][3];
  float centre[3]; /* crop centre, A frame */
  float cB[3];     /* crop centre, B frame */
} orb_frame;

void orb_pair_frame(const float poseA[7], const float poseB[7],
                    const float aabbA[6], const float aabbB[6],
                    orb_frame *fr) {
  float RA[3][3], RB[3][3];
  orb_rotation(poseA, RA);
  orb_rotation(poseB, RB);
  memcpy(fr->RA, RA, sizeof(RA));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      fr->Rrel[i][j] = orb_dot3(RA[0][i], RA[1][i], RA[2][i], RB[0][j],
                                RB[1][j], RB[2][j]);
  float dt[3];
  for (int i = 0; i < 3; ++i) dt[i] = poseB[4 + i] - poseA[4 + i];
  for (int i = 0; i < 3; ++i)
    fr->trel[i] = orb_dot3(RA[0][i], RA[1][i], RA[2][i], dt[0], dt[1], dt[2]);
  /* B's oriented box expressed as an axis-aligned box of A's frame */
  float cb[3], hb[3];
  for (int j = 0; j < 3; ++j) {
    cb[j] = (aabbB[j] + aabbB[3 + j]) * 0.5f;
    hb[j] = (aabbB[3 + j] - aabbB[j]) * 0.5f;
  }
  for (int i = 0; i < 3; ++i) {
    float c = orb_dot3(fr->Rrel[i][0], fr->Rrel[i][1], fr->Rrel[i][2], cb[0],
                       cb[1], cb[2]) +
              fr->trel[i];
    float h = orb_dot3(fabsf(fr->Rrel[i][0]), fabsf(fr->Rrel[i][1]),
                       fabsf(fr->Rrel[i][2]), hb[0], hb[1], hb[2]);
    float lo = c - h, hi = c + h;
    float a = fmaxf(aabbA[i], lo);
    float b = fminf(aabbA[3 + i], hi);
    fr->centre[i] = (a + b) * 0.5f;
  }
  float e[3];
  for (int i = 0; i < 3; ++i) e[i] = fr->centre[i] - fr->trel[i];
  for (int j = 0; j < 3; ++j)
    fr->cB[j] = orb_dot3(fr->Rrel[0][j], fr->Rrel[1][j], fr->Rrel[2][j], e[0],
                         e[1], e[2]);
}

typedef struct {
  uint32_t key;
  int32_t idx;
} orb_cand;

static int orb_cand_cmp(const void *pa, const void *pb) {
  const orb_cand *a = (const orb_cand *)pa, *b = (const orb_cand *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Select the crop of one object.  pts: [n][3] body frame; c: crop centre in
 * the same frame; rot: NULL for object A (canonical = p - c), else R_rel for
 * object B (canonical = R_rel (p - c)).  Returns the count. */
static int orb_select(const float *pts, int n, const float c[3], float r2,
                      int kmax, const float (*rot)[3], int32_t *idx_out,
                      float *xyz_out, orb_cand *scratch) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    float d0 = pts[3 * i] - c[0];
    float d1 = pts[3 * i + 1] - c[1];
    float d2 = pts[3 * i + 2] - c[2];
    float s = d0 * d0;
    s = s + d1 * d1;
    s = s + d2 * d2;
    if (s <= r2) {
      uint32_t bits;
      memcpy(&bits, &s, 4);
      scratch[m].key = bits;
      scratch[m].idx = i;
      ++m;
    }
  }
  qsort(scratch, (size_t)m, sizeof(orb_cand), orb_cand_cmp);
  int cnt = m < kmax ? m : kmax;
  for (int k = 0; k < kmax; ++k) {
    if (k < cnt) {
      int i = scratch[k].idx;
      float d0 = pts[3 * i] - c[0];
      float d1 = pts[3 * i + 1] - c[1];
      float d2 = pts[3 * i + 2] - c[2];
      idx_out[k] = i;
      if (rot == NULL) {
        xyz_out[3 * k] = d0;
        xyz_out[3 * k + 1] = d1;
        xyz_out[3 * k + 2] = d2;
      } else {
        for (int a = 0; a < 3; ++a)
          xyz_out[3 * k + a] = orb_dot3(rot[a][0], rot[a][1], rot[a][2], d0, d1,
                                        d2);
      }
    } else {
      idx_out[k] = -1;
      xyz_out[3 * k] = xyz_out[3 * k + 1] = xyz_out[3 * k + 2] = 0.0f;
    }
  }
  return cnt;
}

/* Global crop of one object (the ablation without locality, Sec. IV-B
 * GLOBAL-OCN): its first kmax samples in index order -- an area-uniform
 * subset of the whole surface -- in the same canonical frame as orb_select.
 * Returns the count. */
static int orb_select_global(const float *pts, int n, const float c[3], int kmax,
                             const float (*rot)[3], int32_t *idx_out, float *xyz_out) {
  int cnt = n < kmax ? n : kmax;
  for (int k = 0; k < kmax; ++k) {
    if (k < cnt) {
      float d0 = pts[3 * k] - c[0];
      float d1 = pts[3 * k + 1] - c[1];
      float d2 = pts[3 * k + 2] - c[2];
      idx_out[k] = k;
      if (rot == NULL) {
        xyz_out[3 * k] = d0;
        xyz_out[3 * k + 1] = d1;
        xyz_out[3 * k + 2] = d2;
      } else {
        for (int a = 0; a < 3; ++a)
          xyz_out[3 * k + a] = orb_dot3(rot[a][0], rot[a][1], rot[a][2], d0, d1, d2);
      }
    } else {
      idx_out[k] = -1;
      xyz_out[3 * k] = xyz_out[3 * k + 1] = xyz_out[3 * k + 2] = 0.0f;
    }
  }
  return cnt;
}

/* ---------------------------------------------------------------- float64 */

/* Parameter offsets into the flat float64 buffer, in this order:
 * W1[64][3] b1[64] W2[128][64] b2[128] W3[256][128] b3[256]
 * H1[256][512] c1[256] H2[256][256] c2[256] H3[8][256] c3[8]. */
static const int ORB_DIMS[6][2] = {{3, 64},    {64, 128},  {128, 256},
                                   {512, 256}, {256, 256}, {256, 8}};

int orb_n_params(void) {
  int n = 0;
  for (int l = 0; l < 6; ++l) n += ORB_DIMS[l][0] * ORB_DIMS[l][1] + ORB_DIMS[l][1];
  return n;
}

static void orb_layer_offsets(int offW[6], int offb[6]) {
  int o = 0;
  for (int l = 0; l < 6; ++l) {
    offW[l] = o;
    o += ORB_DIMS[l][0] * ORB_DIMS[l][1];
    offb[l] = o;
    o += ORB_DIMS[l][1];
  }
}

/* y = W x + b, W row-major [out][in]. */
static void orb_affine(const double *W, const double *b, const double *x,
                       int nin, int nout, double *y) {
  for (int o = 0; o < nout; ++o) {
    double s = b[o];
    for (int i = 0; i < nin; ++i) s += W[(size_t)o * nin + i] * x[i];
    y[o] = s;
  }
}

static void orb_relu(double *v, int n) {
  for (int i = 0; i < n; ++i)
    if (v[i] < 0.0) v[i] = 0.0;
}

/* bfloat16 rounding of a value held in float32: 8 significant bits (the
 * implicit one and 7 stored), round to nearest, ties to even.  Zero, inf and
 * NaN pass through; values below the normal range are not met here. */
double orb_bf16(double v) {
  const float f = (float)v;
  if (f == 0.0f || !isfinite(f)) return (double)f;
  int e;
  const double m = frexp((double)f, &e); /* f = m 2^e, 0.5 <= |m| < 1 */
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* dst[i] = orb_bf16(src[i]) when bf16, else a copy. */
static void orb_operand(const double *src, int n, int bf16, double *dst) {
  for (int i = 0; i < n; ++i) dst[i] = bf16 ? orb_bf16(src[i]) : src[i];
}

/* Per-object encoder forward of point k: h1 (layer 1, unrounded), h2
 * (layer 2 on bf16 operands in bf16 mode; Pr holds the rounded weights) and
 * h3 (layer 3 likewise), each after its ReLU. */
static void orb_encode_point(const double *P, const double *Pr, int bf16, const double x[3],
                             double h1[64], double h2[128], double h3[256]) {
  int offW[6], offb[6];
  orb_layer_offsets(offW, offb);
  double t1[64], t2[128];
  orb_affine(P + offW[0], P + offb[0], x, 3, 64, h1);
  orb_relu(h1, 64);
  orb_operand(h1, 64, bf16, t1);
  orb_affine(Pr + offW[1], P + offb[1], t1, 64, 128, h2);
  orb_relu(h2, 128);
  orb_operand(h2, 128, bf16, t2);
  orb_affine(Pr + offW[2], P + offb[2], t2, 128, 256, h3);
  orb_relu(h3, 256);
}

/* Per-object encoder of up to kmax points; writes pooled [256] and, if
 * argmax != NULL, the index of the point that realises each channel's max
 * (ties to the lower point slot; -1 when the crop is empty). */
static void orb_encode_mode(const double *P, const double *Pr, int bf16, const float *xyz,
                            int cnt, double *pooled, int *argmax) {
  for (int c = 0; c < ORB_FEAT; ++c) {
    pooled[c] = 0.0;
    if (argmax) argmax[c] = -1;
  }
  double x[3], h1[64], h2[128], h3[256];
  for (int k = 0; k < cnt; ++k) {
    for (int a = 0; a < 3; ++a) x[a] = (double)xyz[3 * k + a];
    orb_encode_point(P, Pr, bf16, x, h1, h2, h3);
    for (int c = 0; c < ORB_FEAT; ++c) {
      if (k == 0 || h3[c] > pooled[c]) {
        pooled[c] = h3[c];
        if (argmax) argmax[c] = k;
      }
    }
  }
}

static void orb_encode(const double *P, const float *xyz, int cnt, double *pooled, int *argmax) {
  orb_encode_mode(P, P, 0, xyz, cnt, pooled, argmax);
}

/* Head on f = [f_A, f_B] (512) -> raw outputs y[8] (canonical frame). */
static void orb_head(const double *P, const double *f, double *g1, double *g2,
                     double *y) {
  int offW[6], offb[6];
  orb_layer_offsets(offW, offb);
  orb_affine(P + offW[3], P + offb[3], f, 512, 256, g1);
  orb_relu(g1, 256);
  orb_affine(P + offW[4], P + offb[4], g1, 256, 256, g2);
  orb_relu(g2, 256);
  orb_affine(P + offW[5], P + offb[5], g2, 256, 8, y);
}

/* The head in either operand mode: g1 = relu(W4 f + b4), g2 = relu(W5 g1 + b5)
 * with bf16 operands in bf16 mode, y = W6 g2 + b6 unrounded. */
static void orb_head_mode(const double *P, const double *Pr, int bf16, const double *f,
                          double *g1, double *g2, double *y) {
  int offW[6], offb[6];
  orb_layer_offsets(offW, offb);
  double fr[512], g1r[256];
  orb_operand(f, 512, bf16, fr);
  orb_affine(Pr + offW[3], P + offb[3], fr, 512, 256, g1);
  orb_relu(g1, 256);
  orb_operand(g1, 256, bf16, g1r);
  orb_affine(Pr + offW[4], P + offb[4], g1r, 256, 256, g2);
  orb_relu(g2, 256);
  orb_affine(P + offW[5], P + offb[5], g2, 256, 8, y);
}

/* Raw canonical-frame outputs -> world: logit, R_A (p + c) + t_A,
 * R_A n / max(|n|, 1e-12), depth. */
static void orb_epilogue(const double *y, const orb_frame *fr,
                         const float poseA[7], double *out) {
  out[0] = y[0];
  double p[3], n[3];
  for (int i = 0; i < 3; ++i) p[i] = y[1 + i] + (double)fr->centre[i];
  double nn = sqrt(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
  if (nn < 1e-12) nn = 1e-12;
  for (int i = 0; i < 3; ++i) n[i] = y[4 + i] / nn;
  for (int i = 0; i < 3; ++i) {
    double sp = (double)poseA[4 + i], sn = 0.0;
    for (int j = 0; j < 3; ++j) {
      sp += (double)fr->RA[i][j] * p[j];
      sn += (double)fr->RA[i][j] * n[j];
    }
    out[1 + i] = sp;
    out[4 + i] = sn;
  }
  out[7] = y[7];
}

/* ------------------------------------------------------------ batch calls */

typedef struct {
  const float *points, *aabb, *poses;
  const int32_t *obj_shape, *pairs;
  int n_shapes, n_points, n_obj, n_pairs, kmax;
  float r;
  int32_t *idx_out, *cnt_out;
  float *xyz_out, *centre_out;
  const double *params;
  double *out, *feat_out;
  int status;
  int lo, hi;
  int global; /* 1: global crops (orb_select_global) */
} orb_job;

static int orb_pair_valid(const orb_job *j, int p) {
  int a = j->pairs[2 * p], b = j->pairs[2 * p + 1];
  if (a < 0 || b < 0 || a >= j->n_obj || b >= j->n_obj) return 0;
  int sa = j->obj_shape[a], sb = j->obj_shape[b];
  return sa >= 0 && sb >= 0 && sa < j->n_shapes && sb < j->n_shapes;
}

static void orb_crop_one(const orb_job *j, int p, orb_cand *scratch,
                         orb_frame *fr, int32_t *idx, int32_t *cnt,
                         float *xyz) {
  int a = j->pairs[2 * p], b = j->pairs[2 * p + 1];
  int sa = j->obj_shape[a], sb = j->obj_shape[b];
  const float *pa = j->points + (size_t)sa * j->n_points * 3;
  const float *pb = j->points + (size_t)sb * j->n_points * 3;
  orb_pair_frame(j->poses + 7 * a, j->poses + 7 * b, j->aabb + 6 * sa,
                 j->aabb + 6 * sb, fr);
  if (j->global) {
    cnt[0] = orb_select_global(pa, j->n_points, fr->centre, j->kmax, NULL, idx, xyz);
    cnt[1] = orb_select_global(pb, j->n_points, fr->cB, j->kmax, (const float(*)[3])fr->Rrel,
                               idx + j->kmax, xyz + 3 * j->kmax);
    return;
  }
  float r2 = j->r * j->r;
  cnt[0] = orb_select(pa, j->n_points, fr->centre, r2, j->kmax, NULL, idx, xyz,
                      scratch);
  cnt[1] = orb_select(pb, j->n_points, fr->cB, r2, j->kmax,
                      (const float(*)[3])fr->Rrel, idx + j->kmax,
                      xyz + 3 * j->kmax, scratch);
}

static void *orb_worker(void *arg) {
  orb_job *j = (orb_job *)arg;
  orb_cand *scratch = (orb_cand *)malloc(sizeof(orb_cand) * (size_t)j->n_points);
  int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)j->kmax);
  float *xyz = (float *)malloc(sizeof(float) * 6 * (size_t)j->kmax);
  if (!scratch || !idx || !xyz) {
    j->status = -2;
    free(scratch), free(idx), free(xyz);
    return NULL;
  }
  double f[512], g1[256], g2[256], y[8];
  for (int p = j->lo; p < j->hi; ++p) {
    if (!orb_pair_valid(j, p)) {
      j->status = -1;
      continue;
    }
    orb_frame fr;
    int32_t cnt[2];
    orb_crop_one(j, p, scratch, &fr, idx, cnt, xyz);
    if (j->idx_out) memcpy(j->idx_out + (size_t)p * 2 * j->kmax, idx, sizeof(int32_t) * 2 * j->kmax);
    if (j->cnt_out) memcpy(j->cnt_out + 2 * (size_t)p, cnt, sizeof(cnt));
    if (j->xyz_out) memcpy(j->xyz_out + (size_t)p * 6 * j->kmax, xyz, sizeof(float) * 6 * j->kmax);
    if (j->centre_out) memcpy(j->centre_out + 3 * (size_t)p, fr.centre, sizeof(fr.centre));
    if (j->params) {
      orb_encode(j->params, xyz, cnt[0], f, NULL);
      orb_encode(j->params, xyz + 3 * j->kmax, cnt[1], f + 256, NULL);
      orb_head(j->params, f, g1, g2, y);
      int a = j->pairs[2 * p];
      if (j->out) orb_epilogue(y, &fr, j->poses + 7 * a, j->out + 8 * (size_t)p);
      if (j->feat_out) memcpy(j->feat_out + 512 * (size_t)p, f, sizeof(f));
    }
  }
  free(scratch), free(idx), free(xyz);
  return NULL;
}

/* Crop selection and (if params != NULL) network forward for n_pairs pairs on
 * n_threads host threads.  Layouts: points [S][n_points][3], aabb [S][6],
 * poses [n_obj][7] (w,x,y,z,tx,ty,tz), obj_shape [n_obj], pairs [n_pairs][2];
 * outputs (each may be NULL): idx [P][2][kmax] (-1 padded), cnt [P][2],
 * xyz [P][2][kmax][3] canonical float32, centre [P][3], out [P][8] world
 * float64, feat [P][512] pooled float64.  Returns 0, -1 (bad index), -2 (OOM). */
static int orb_run_mode(const float *points, const float *aabb, int n_shapes, int n_points,
                        const float *poses, const int32_t *obj_shape, int n_obj,
                        const int32_t *pairs, int n_pairs, float r, int kmax,
                        const double *params, int32_t *idx_out, int32_t *cnt_out,
                        float *xyz_out, float *centre_out, double *out, double *feat_out,
                        int n_threads, int global);

int orb_run(const float *points, const float *aabb, int n_shapes, int n_points,
            const float *poses, const int32_t *obj_shape, int n_obj,
            const int32_t *pairs, int n_pairs, float r, int kmax,
            const double *params, int32_t *idx_out, int32_t *cnt_out,
            float *xyz_out, float *centre_out, double *out, double *feat_out,
            int n_threads) {
  return orb_run_mode(points, aabb, n_shapes, n_points, poses, obj_shape, n_obj, pairs,
                      n_pairs, r, kmax, params, idx_out, cnt_out, xyz_out, centre_out, out,
                      feat_out, n_threads, 0);
}

/* orb_run with global crops (orb_select_global) instead of local ones. */
int orb_run_global(const float *points, const float *aabb, int n_shapes, int n_points,
                   const float *poses, const int32_t *obj_shape, int n_obj,
                   const int32_t *pairs, int n_pairs, float r, int kmax,
                   const double *params, int32_t *idx_out, int32_t *cnt_out,
                   float *xyz_out, float *centre_out, double *out, double *feat_out,
                   int n_threads) {
  return orb_run_mode(points, aabb, n_shapes, n_points, poses, obj_shape, n_obj, pairs,
                      n_pairs, r, kmax, params, idx_out, cnt_out, xyz_out, centre_out, out,
                      feat_out, n_threads, 1);
}

static int orb_run_mode(const float *points, const float *aabb, int n_shapes, int n_points,
                        const float *poses, const int32_t *obj_shape, int n_obj,
                        const int32_t *pairs, int n_pairs, float r, int kmax,
                        const double *params, int32_t *idx_out, int32_t *cnt_out,
                        float *xyz_out, float *centre_out, double *out, double *feat_out,
                        int n_threads, int global) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  orb_job jobs[256];
  int per = (n_pairs + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    orb_job *j = &jobs[t];
    j->points = points, j->aabb = aabb, j->poses = poses;
    j->obj_shape = obj_shape, j->pairs = pairs;
    j->n_shapes = n_shapes, j->n_points = n_points, j->n_obj = n_obj;
    j->n_pairs = n_pairs, j->kmax = kmax, j->r = r;
    j->idx_out = idx_out, j->cnt_out = cnt_out, j->xyz_out = xyz_out;
    j->centre_out = centre_out, j->params = params, j->out = out;
    j->feat_out = feat_out, j->status = 0, j->global = global;
    j->lo = t * per;
    j->hi = (t + 1) * per < n_pairs ? (t + 1) * per : n_pairs;
    if (j->lo > j->hi) j->lo = j->hi;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, orb_worker, &jobs[t]);
  orb_worker(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  int st = 0;
  for (int t = 0; t < n_threads; ++t)
    if (jobs[t].status < st) st = jobs[t].status;
  return st;
}

/* Network only, on given crops: xyz [P][2][kmax][3], cnt [P][2] ->
 * raw canonical outputs y [P][8] and pooled feat [P][512] (either may be NULL). */
int orb_network(const double *params, const float *xyz, const int32_t *cnt,
                int n_pairs, int kmax, double *y_out, double *feat_out) {
  double f[512], g1[256], g2[256], y[8];
  for (int p = 0; p < n_pairs; ++p) {
    const float *x = xyz + (size_t)p * 6 * kmax;
    int ca = cnt[2 * p], cb = cnt[2 * p + 1];
    if (ca < 0 || cb < 0 || ca > kmax || cb > kmax) return -1;
    orb_encode(params, x, ca, f, NULL);
    orb_encode(params, x + 3 * kmax, cb, f + 256, NULL);
    orb_head(params, f, g1, g2, y);
    if (y_out) memcpy(y_out + 8 * (size_t)p, y, sizeof(y));
    if (feat_out) memcpy(feat_out + 512 * (size_t)p, f, sizeof(f));
  }
  return 0;
}

/* ---------------------------------------------------------------- backward */

/* Loss of one pair on raw canonical outputs y and pooled f:
 *   BCE(sigmoid(y0), lab)
 *   + lab * (w_pt |y[1:4] - pt|^2 + w_n (1 - cos(y[4:7], n)))
 *   + w_len * (|y[4:7]| - 1)^2       (every pair; this library's term: keeps
 *                                     the raw normal away from zero length)
 *   + w_d * huber_beta(y7 - depth)
 *   + alpha * mean(f^2).
 * tgt = {lab, pt.xyz, n.xyz, depth} in the canonical frame;
 * hp = {w_pt, w_n, w_d, beta, alpha, w_len}.
 * Writes dL/dy [8] and dL/df [512]; returns the loss. */
static double orb_pair_loss(const double *y, const double *f, const double *tgt,
                            const double *hp, double *dy, double *df) {
  double w_pt = hp[0], w_n = hp[1], w_d = hp[2], beta = hp[3], alpha = hp[4], w_len = hp[5];
  double lab = tgt[0];
  double z = y[0];
  /* BCE with logits: max(z,0) - z*lab + log(1 + exp(-|z|)) */
  double L = (z > 0 ? z : 0.0) - z * lab + log1p(exp(-fabs(z)));
  double sig = 1.0 / (1.0 + exp(-z));
  for (int i = 0; i < 8; ++i) dy[i] = 0.0;
  dy[0] = sig - lab;
  if (lab > 0) {
    for (int i = 0; i < 3; ++i) {
      double d = y[1 + i] - tgt[1 + i];
      L += lab * w_pt * d * d;
      dy[1 + i] = lab * w_pt * 2.0 * d;
    }
    double nn = sqrt(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
    double tn = sqrt(tgt[4] * tgt[4] + tgt[5] * tgt[5] + tgt[6] * tgt[6]);
    if (nn > 1e-12 && tn > 1e-12) {
      double dot = y[4] * tgt[4] + y[5] * tgt[5] + y[6] * tgt[6];
      double cs = dot / (nn * tn);
      L += lab * w_n * (1.0 - cs);
      /* d cos / d n = t/(|n||t|) - cos * n / |n|^2 */
      for (int i = 0; i < 3; ++i)
        dy[4 + i] = -lab * w_n * (tgt[4 + i] / (nn * tn) - cs * y[4 + i] / (nn * nn));
    }
  }
  if (w_len > 0) {
    double nl = sqrt(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
    if (nl > 1e-12) {
      L += w_len * (nl - 1.0) * (nl - 1.0);
      for (int i = 0; i < 3; ++i) dy[4 + i] += w_len * 2.0 * (nl - 1.0) * y[4 + i] / nl;
    }
  }
  double e = y[7] - tgt[7];
  if (fabs(e) < beta) {
    L += w_d * 0.5 * e * e / beta;
    dy[7] = w_d * e / beta;
  } else {
    L += w_d * (fabs(e) - 0.5 * beta);
    dy[7] = w_d * (e > 0 ? 1.0 : -1.0);
  }
  double sq = 0.0;
  for (int i = 0; i < 512; ++i) sq += f[i] * f[i];
  L += alpha * sq / 512.0;
  for (int i = 0; i < 512; ++i) df[i] = alpha * 2.0 * f[i] / 512.0;
  return L;
}

/* Backward through the encoder of one object: dpool [256] -> grads.  The
 * gradient of the max-pool goes to the point that realises each channel's
 * max (ties to the lower slot); ReLU passes gradient where its output > 0. */
static void orb_encode_backward(const double *P, const double *Pr, int bf16, const float *xyz,
                                int cnt, const double *dpool, double *G) {
  int offW[6], offb[6];
  orb_layer_offsets(offW, offb);
  if (cnt <= 0) return;
  double pooled[256];
  int am[256];
  orb_encode_mode(P, Pr, bf16, xyz, cnt, pooled, am);
  double x[3], h1[64], h2[128], h3[256], d3[256], d2[128], d1[64], h1r[64], d2r[128];
  for (int k = 0; k < cnt; ++k) {
    int any = 0;
    for (int c = 0; c < 256; ++c) {
      d3[c] = 0.0;
      if (am[c] == k && pooled[c] > 0.0) {
        d3[c] = dpool[c];
        any = 1;
      }
    }
    if (!any) continue;
    for (int a = 0; a < 3; ++a) x[a] = (double)xyz[3 * k + a];
    orb_encode_point(P, Pr, bf16, x, h1, h2, h3);
    /* layer 3: d3 already masked by h3 > 0 via pooled > 0 */
    for (int o = 0; o < 256; ++o) {
      if (d3[o] == 0.0) continue;
      G[offb[2] + o] += d3[o];
      for (int i = 0; i < 128; ++i) G[offW[2] + o * 128 + i] += d3[o] * h2[i];
    }
    for (int i = 0; i < 128; ++i) {
      double s = 0.0;
      for (int o = 0; o < 256; ++o) s += P[offW[2] + o * 128 + i] * d3[o];
      d2[i] = h2[i] > 0.0 ? s : 0.0;
    }
    /* layer 2 (a matrix product in bf16 mode: d2 and h1 rounded) */
    orb_operand(d2, 128, bf16, d2r);
    orb_operand(h1, 64, bf16, h1r);
    for (int o = 0; o < 128; ++o) {
      G[offb[1] + o] += d2[o];
      for (int i = 0; i < 64; ++i) G[offW[1] + o * 64 + i] += d2r[o] * h1r[i];
    }
    for (int i = 0; i < 64; ++i) {
      double s = 0.0;
      for (int o = 0; o < 128; ++o) s += Pr[offW[1] + o * 64 + i] * d2r[o];
      d1[i] = h1[i] > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < 64; ++o) {
      G[offb[0] + o] += d1[o];
      for (int i = 0; i < 3; ++i) G[offW[0] + o * 3 + i] += d1[o] * x[i];
    }
  }
}

/* Mean loss over n_pairs given crops and canonical targets tgt [P][8]
 * ({label, point, normal, depth}); hp = {w_pt, w_n, w_d, beta, alpha, w_len}.
 * Accumulates the gradient of the mean loss into grad (zeroed here). */
double orb_loss_grad(const double *params, const float *xyz, const int32_t *cnt,
                     const double *tgt, int n_pairs, int kmax, const double *hp,
                     int bf16, double *grad) {
  int offW[6], offb[6];
  orb_layer_offsets(offW, offb);
  int np = orb_n_params();
  memset(grad, 0, sizeof(double) * (size_t)np);
  /* Pr: the weights of the matrix-product layers rounded in bf16 mode */
  double *Pr = (double *)malloc(sizeof(double) * (size_t)np);
  if (!Pr) return NAN;
  memcpy(Pr, params, sizeof(double) * (size_t)np);
  if (bf16)
    for (int l = 1; l <= 4; ++l)
      for (int i = offW[l]; i < offb[l]; ++i) Pr[i] = orb_bf16(params[i]);
  double total = 0.0;
  double f[512], g1[256], g2[256], y[8], dy[8], df[512], dg2[256], dg1[256];
  double fr[512], g1r[256], dg2r[256], dg1r[256];
  for (int p = 0; p < n_pairs; ++p) {
    const float *x = xyz + (size_t)p * 6 * kmax;
    int ca = cnt[2 * p], cb = cnt[2 * p + 1];
    orb_encode_mode(params, Pr, bf16, x, ca, f, NULL);
    orb_encode_mode(params, Pr, bf16, x + 3 * kmax, cb, f + 256, NULL);
    orb_head_mode(params, Pr, bf16, f, g1, g2, y);
    total += orb_pair_loss(y, f, tgt + 8 * (size_t)p, hp, dy, df);
    double s = 1.0 / n_pairs;
    for (int i = 0; i < 8; ++i) dy[i] *= s;
    for (int i = 0; i < 512; ++i) df[i] *= s;
    /* head layer 3 (linear) */
    for (int o = 0; o < 8; ++o) {
      grad[offb[5] + o] += dy[o];
      for (int i = 0; i < 256; ++i) grad[offW[5] + o * 256 + i] += dy[o] * g2[i];
    }
    for (int i = 0; i < 256; ++i) {
      double t = 0.0;
      for (int o = 0; o < 8; ++o) t += params[offW[5] + o * 256 + i] * dy[o];
      dg2[i] = g2[i] > 0.0 ? t : 0.0;
    }
    /* head layers 2 and 1 (matrix products in bf16 mode) */
    orb_operand(dg2, 256, bf16, dg2r);
    orb_operand(g1, 256, bf16, g1r);
    for (int o = 0; o < 256; ++o) {
      grad[offb[4] + o] += dg2[o];
      for (int i = 0; i < 256; ++i) grad[offW[4] + o * 256 + i] += dg2r[o] * g1r[i];
    }
    for (int i = 0; i < 256; ++i) {
      double t = 0.0;
      for (int o = 0; o < 256; ++o) t += Pr[offW[4] + o * 256 + i] * dg2r[o];
      dg1[i] = g1[i] > 0.0 ? t : 0.0;
    }
    orb_operand(dg1, 256, bf16, dg1r);
    orb_operand(f, 512, bf16, fr);
    for (int o = 0; o < 256; ++o) {
      grad[offb[3] + o] += dg1[o];
      for (int i = 0; i < 512; ++i) grad[offW[3] + o * 512 + i] += dg1r[o] * fr[i];
    }
    for (int i = 0; i < 512; ++i) {
      double t = 0.0;
      for (int o = 0; o < 256; ++o) t += Pr[offW[3] + o * 512 + i] * dg1r[o];
      df[i] += t;
    }
    orb_encode_backward(params, Pr, bf16, x, ca, df, grad);
    orb_encode_backward(params, Pr, bf16, x + 3 * kmax, cb, df + 256, grad);
  }
  free(Pr);
  return total / n_pairs;
}

/* ------------------------------------------------------------- broadphase */

/* Broad phase (Sec. II, footnote 1: far-apart objects are ruled out before
 * the narrow phase): the world axis-aligned box of each object's posed body
 * box (centre R c + t, half extents |R| h, float32 in the fixed order of
 * orb_dot3), and every pair (i, j), i < j, of one environment whose boxes
 * overlap on all axes (|c_i - c_j| <= h_i + h_j).  Pairs are listed by
 * environment, then i, then j.  Writes at most max_pairs pairs; returns the
 * full count (or -1 on a bad shape id). */
static void orb_world_box(const float *pose, const float *aabb, float c[3], float h[3]) {
  float R[3][3];
  orb_rotation(pose, R);
  float cl[3], hl[3];
  for (int j = 0; j < 3; ++j) {
    cl[j] = (aabb[j] + aabb[3 + j]) * 0.5f;
    hl[j] = (aabb[3 + j] - aabb[j]) * 0.5f;
  }
  for (int i = 0; i < 3; ++i) {
    c[i] = orb_dot3(R[i][0], R[i][1], R[i][2], cl[0], cl[1], cl[2]) + pose[4 + i];
    h[i] = orb_dot3(fabsf(R[i][0]), fabsf(R[i][1]), fabsf(R[i][2]), hl[0], hl[1], hl[2]);
  }
}

long long orb_broadphase(const float *aabb, int n_shapes, const float *poses,
                         const int32_t *obj_shape, const int32_t *env_offsets, int n_env,
                         int32_t *pairs_out, long long max_pairs) {
  long long n = 0;
  for (int e = 0; e < n_env; ++e) {
    int o0 = env_offsets[e], o1 = env_offsets[e + 1];
    for (int i = o0; i < o1; ++i) {
      if (obj_shape[i] < 0 || obj_shape[i] >= n_shapes) return -1;
      float ci[3], hi[3];
      orb_world_box(poses + 7 * (size_t)i, aabb + 6 * (size_t)obj_shape[i], ci, hi);
      for (int j = i + 1; j < o1; ++j) {
        if (obj_shape[j] < 0 || obj_shape[j] >= n_shapes) return -1;
        float cj[3], hj[3];
        orb_world_box(poses + 7 * (size_t)j, aabb + 6 * (size_t)obj_shape[j], cj, hj);
        int ov = 1;
        for (int a = 0; a < 3; ++a)
          if (!(fabsf(ci[a] - cj[a]) <= hi[a] + hj[a])) ov = 0;
        if (ov) {
          if (n < max_pairs) {
            pairs_out[2 * n] = i;
            pairs_out[2 * n + 1] = j;
          }
          ++n;
        }
      }
    }
  }
  return n;
}

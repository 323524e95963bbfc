/*
 * ORACLE (a): plain float64 geometric contact detector on triangle meshes.
 *
 * Test infrastructure only.  Nothing in the product library links, loads or
 * calls this file; only tests, the smoke check, the benchmark's CPU-baseline
 * leg and the committed dataset / golden-value scripts under oracle/ and
 * tests/golden/ do.  It shares no code with the CUDA path.
 *
 * The paper labels a pair of posed meshes as colliding or not (Sec. III-A,
 * dataset tuples (x1, x2, q1, q2, y)) and measures distances between objects
 * (the shortest-distance vector delta of the data generation, Fig. 4; the
 * min-|sd| metric of Table 2).  It does not define a contact point, normal or
 * penetration depth for non-convex meshes; the readings below are this
 * implementation's own.
 *
 * A shape is a union of closed, outward-oriented component meshes.
 *   inside(x, S)  <=> the generalised winding number (sum of signed solid
 *                     angles / 4 pi, van Oosterom & Strackee 1983) of some
 *                     component of S at x exceeds 1/2.
 *   label y = 1   <=> some triangle of A meets some triangle of B, or some
 *                     vertex of A is inside B, or some vertex of B inside A.
 *   y = 0: gap    =  min over triangle pairs of the triangle-triangle distance
 *                    (6 point-triangle + 9 segment-segment distances); the
 *                    realising points pA, pB (ties to the lowest (tA, tB));
 *                    depth = -gap, point = (pA + pB)/2, normal = (pB - pA)/gap.
 *   y = 1: candidates are A's surface samples and A's vertices (not strictly
 *          inside another component of A) that lie inside B, then the same for
 *          B inside A.  depth = max over candidates v of the distance from v
 *          to the other shape's surface (its triangles, minus those whose three
 *          vertices are all strictly inside another of its components); q is
 *          the realising surface point; point = (v + q)/2; normal = (v - q)/|v-q|
 *          for v in A, (q - v)/|q - v| for v in B, so the normal points from A
 *          towards B.  Ties go to the earlier candidate.  With no candidate
 *          inside (edges crossing only): depth = 0, point = midpoint of the
 *          intersection segment of the lowest intersecting triangle pair,
 *          normal = normalise(nA - nB) of that pair's face normals.
 *
 * Two variants give identical results: brute force over all triangle pairs
 * and candidates, and a culled one that skips work ruled out by bounding
 * boxes (conservatively, with a 1e-12 slack).
 *
 * Geometric primitives follow C. Ericson, Real-Time Collision Detection (2005):
 * closest point on a triangle by Voronoi regions (Sec. 5.1.5) and closest points
 * of two segments (Sec. 5.1.9); segment-triangle crossing by orientation signs.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_SLACK 1e-12

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
static double clamp01(double t) { return t < 0 ? 0 : (t > 1 ? 1 : t); }

/* --------------------------------------------------------------- meshes */

typedef struct {
  int nv, nf, ncomp, ns;
  v3 *V;          /* world vertices */
  int32_t *F;     /* [nf][3] */
  int32_t *comp;  /* [nf] */
  v3 *S;          /* world surface samples */
  v3 *blo, *bhi;  /* per-face box */
  v3 *clo, *chi;  /* per-component box */
  v3 lo, hi;      /* whole-shape box */
  unsigned char *face_internal; /* all three vertices inside another comp */
  unsigned char *vert_internal; /* vertex strictly inside another comp */
} ora_shape;

static void quat_rot64(const float q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n, x /= n, y /= n, z /= n;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

static v3 xform(const double R[3][3], const double t[3], v3 p) {
  return mk(R[0][0] * p.x + R[0][1] * p.y + R[0][2] * p.z + t[0],
            R[1][0] * p.x + R[1][1] * p.y + R[1][2] * p.z + t[1],
            R[2][0] * p.x + R[2][1] * p.y + R[2][2] * p.z + t[2]);
}

static v3 vmin(v3 a, v3 b) { return mk(fmin(a.x, b.x), fmin(a.y, b.y), fmin(a.z, b.z)); }
static v3 vmax(v3 a, v3 b) { return mk(fmax(a.x, b.x), fmax(a.y, b.y), fmax(a.z, b.z)); }

/* signed solid angle of triangle (a, b, c) seen from p (van Oosterom &
 * Strackee): tan(omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|) */
static double solid_angle(v3 p, v3 A, v3 B, v3 C) {
  v3 a = sub(A, p), b = sub(B, p), c = sub(C, p);
  double la = norm(a), lb = norm(b), lc = norm(c);
  double num = dot(a, cross(b, c));
  double den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
  return 2.0 * atan2(num, den);
}

static double winding_comp(const ora_shape *s, int k, v3 p) {
  double w = 0.0;
  for (int f = 0; f < s->nf; ++f) {
    if (s->comp[f] != k) continue;
    const int32_t *t = s->F + 3 * f;
    w += solid_angle(p, s->V[t[0]], s->V[t[1]], s->V[t[2]]);
  }
  return w / (4.0 * M_PI);
}

static int in_box(v3 p, v3 lo, v3 hi) {
  return p.x >= lo.x - ORA_SLACK && p.x <= hi.x + ORA_SLACK &&
         p.y >= lo.y - ORA_SLACK && p.y <= hi.y + ORA_SLACK &&
         p.z >= lo.z - ORA_SLACK && p.z <= hi.z + ORA_SLACK;
}

/* inside the union, optionally ignoring component `skip` */
static int inside_shape(const ora_shape *s, v3 p, int skip, int culled) {
  if (culled && !in_box(p, s->lo, s->hi)) return 0;
  for (int k = 0; k < s->ncomp; ++k) {
    if (k == skip) continue;
    if (culled && !in_box(p, s->clo[k], s->chi[k])) continue;
    if (winding_comp(s, k, p) > 0.5) return 1;
  }
  return 0;
}

static int ora_build(ora_shape *s, const double *V, int nv, const int32_t *F,
                     const int32_t *comp, int nf, const float *samples, int ns,
                     const float pose[7], int culled) {
  memset(s, 0, sizeof(*s));
  double R[3][3], t[3] = {pose[4], pose[5], pose[6]};
  quat_rot64(pose, R);
  s->nv = nv, s->nf = nf, s->ns = ns;
  s->V = (v3 *)malloc(sizeof(v3) * (size_t)nv);
  s->S = (v3 *)malloc(sizeof(v3) * (size_t)(ns > 0 ? ns : 1));
  s->F = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nf);
  s->comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf);
  s->blo = (v3 *)malloc(sizeof(v3) * (size_t)nf);
  s->bhi = (v3 *)malloc(sizeof(v3) * (size_t)nf);
  s->face_internal = (unsigned char *)calloc((size_t)nf, 1);
  s->vert_internal = (unsigned char *)calloc((size_t)nv, 1);
  if (!s->V || !s->S || !s->F || !s->comp || !s->blo || !s->bhi ||
      !s->face_internal || !s->vert_internal)
    return -2;
  memcpy(s->F, F, sizeof(int32_t) * 3 * (size_t)nf);
  memcpy(s->comp, comp, sizeof(int32_t) * (size_t)nf);
  for (int i = 0; i < nv; ++i)
    s->V[i] = xform(R, t, mk(V[3 * i], V[3 * i + 1], V[3 * i + 2]));
  for (int i = 0; i < ns; ++i)
    s->S[i] = xform(R, t, mk(samples[3 * i], samples[3 * i + 1], samples[3 * i + 2]));
  s->ncomp = 0;
  for (int f = 0; f < nf; ++f)
    if (comp[f] + 1 > s->ncomp) s->ncomp = comp[f] + 1;
  s->clo = (v3 *)malloc(sizeof(v3) * (size_t)s->ncomp);
  s->chi = (v3 *)malloc(sizeof(v3) * (size_t)s->ncomp);
  int *vcomp = (int *)malloc(sizeof(int) * (size_t)nv);
  if (!s->clo || !s->chi || !vcomp) { free(vcomp); return -2; }
  for (int k = 0; k < s->ncomp; ++k) s->clo[k] = mk(INFINITY, INFINITY, INFINITY), s->chi[k] = mk(-INFINITY, -INFINITY, -INFINITY);
  s->lo = mk(INFINITY, INFINITY, INFINITY), s->hi = mk(-INFINITY, -INFINITY, -INFINITY);
  for (int i = 0; i < nv; ++i) vcomp[i] = -1;
  for (int f = 0; f < nf; ++f) {
    v3 a = s->V[F[3 * f]], b = s->V[F[3 * f + 1]], c = s->V[F[3 * f + 2]];
    s->blo[f] = vmin(vmin(a, b), c);
    s->bhi[f] = vmax(vmax(a, b), c);
    int k = comp[f];
    s->clo[k] = vmin(s->clo[k], s->blo[f]);
    s->chi[k] = vmax(s->chi[k], s->bhi[f]);
    s->lo = vmin(s->lo, s->blo[f]);
    s->hi = vmax(s->hi, s->bhi[f]);
    for (int j = 0; j < 3; ++j) vcomp[F[3 * f + j]] = k;
  }
  /* vertices strictly inside another component are not on the union surface */
  if (s->ncomp > 1) {
    for (int i = 0; i < nv; ++i)
      s->vert_internal[i] = vcomp[i] >= 0 && inside_shape(s, s->V[i], vcomp[i], culled);
    for (int f = 0; f < nf; ++f)
      s->face_internal[f] = s->vert_internal[F[3 * f]] && s->vert_internal[F[3 * f + 1]] &&
                            s->vert_internal[F[3 * f + 2]];
  }
  free(vcomp);
  return 0;
}

static void ora_free(ora_shape *s) {
  free(s->V), free(s->S), free(s->F), free(s->comp), free(s->blo), free(s->bhi);
  free(s->clo), free(s->chi), free(s->face_internal), free(s->vert_internal);
}

/* ------------------------------------------------------------ primitives */

/* Closest point of triangle abc to p (Voronoi-region walk, Ericson 5.1.5). */
static v3 closest_on_tri(v3 p, v3 a, v3 b, v3 c) {
  v3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
  double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0 && d2 <= 0) return a;                      /* vertex a */
  v3 bp = sub(p, b);
  double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0 && d4 <= d3) return b;                     /* vertex b */
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0)                     /* edge ab */
    return add(a, scl(ab, d1 / (d1 - d3)));
  v3 cp = sub(p, c);
  double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0 && d5 <= d6) return c;                     /* vertex c */
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0)                     /* edge ac */
    return add(a, scl(ac, d2 / (d2 - d6)));
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0)       /* edge bc */
    return add(b, scl(sub(c, b), (d4 - d3) / ((d4 - d3) + (d5 - d6))));
  double den = 1.0 / (va + vb + vc);                     /* face interior */
  return add(a, add(scl(ab, vb * den), scl(ac, vc * den)));
}

/* Closest points of segments p1q1 and p2q2 (Ericson 5.1.9). */
static void closest_seg_seg(v3 p1, v3 q1, v3 p2, v3 q2, v3 *c1, v3 *c2) {
  v3 d1 = sub(q1, p1), d2 = sub(q2, p2), r = sub(p1, p2);
  double a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  double s, t;
  const double eps = 1e-300;
  if (a <= eps && e <= eps) {
    s = t = 0;
  } else if (a <= eps) {
    s = 0, t = clamp01(f / e);
  } else {
    double c = dot(d1, r);
    if (e <= eps) {
      t = 0, s = clamp01(-c / a);
    } else {
      double b = dot(d1, d2), den = a * e - b * b;
      s = den != 0 ? clamp01((b * f - c * e) / den) : 0.0;
      t = (b * s + f) / e;
      if (t < 0) t = 0, s = clamp01(-c / a);
      else if (t > 1) t = 1, s = clamp01((b - c) / a);
    }
  }
  *c1 = add(p1, scl(d1, s));
  *c2 = add(p2, scl(d2, t));
}

static double orient(v3 a, v3 b, v3 c, v3 d) {
  return dot(cross(sub(b, a), sub(c, a)), sub(d, a));
}

/* Does segment pq cross triangle abc?  If so, *x is the crossing point.
 * Coplanar configurations count as not crossing. */
static int seg_tri(v3 p, v3 q, v3 a, v3 b, v3 c, v3 *x) {
  double sp = orient(a, b, c, p), sq = orient(a, b, c, q);
  if ((sp > 0 && sq > 0) || (sp < 0 && sq < 0) || (sp == 0 && sq == 0)) return 0;
  double o1 = orient(p, q, a, b), o2 = orient(p, q, b, c), o3 = orient(p, q, c, a);
  int pos = o1 >= 0 && o2 >= 0 && o3 >= 0;
  int neg = o1 <= 0 && o2 <= 0 && o3 <= 0;
  if (!pos && !neg) return 0;
  *x = add(p, scl(sub(q, p), sp / (sp - sq)));
  return 1;
}

/* Triangles T = (a0,a1,a2), U = (b0,b1,b2): number of edge crossings (0 if
 * disjoint) and their mean in *mid. */
static int tri_tri_meet(const v3 *T, const v3 *U, v3 *mid) {
  int n = 0;
  v3 acc = mk(0, 0, 0), x;
  for (int e = 0; e < 3; ++e) {
    if (seg_tri(T[e], T[(e + 1) % 3], U[0], U[1], U[2], &x)) acc = add(acc, x), ++n;
    if (seg_tri(U[e], U[(e + 1) % 3], T[0], T[1], T[2], &x)) acc = add(acc, x), ++n;
  }
  if (n) *mid = scl(acc, 1.0 / n);
  return n;
}

/* Distance between two non-intersecting triangles with realising points. */
static double tri_tri_dist(const v3 *T, const v3 *U, v3 *pT, v3 *pU) {
  double best = INFINITY;
  for (int i = 0; i < 3; ++i) {
    v3 q = closest_on_tri(T[i], U[0], U[1], U[2]);
    double d = norm(sub(T[i], q));
    if (d < best) best = d, *pT = T[i], *pU = q;
  }
  for (int i = 0; i < 3; ++i) {
    v3 q = closest_on_tri(U[i], T[0], T[1], T[2]);
    double d = norm(sub(U[i], q));
    if (d < best) best = d, *pT = q, *pU = U[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      v3 c1, c2;
      closest_seg_seg(T[i], T[(i + 1) % 3], U[j], U[(j + 1) % 3], &c1, &c2);
      double d = norm(sub(c1, c2));
      if (d < best) best = d, *pT = c1, *pU = c2;
    }
  return best;
}

static double box_dist(v3 alo, v3 ahi, v3 blo, v3 bhi) {
  double dx = fmax(0.0, fmax(alo.x - bhi.x, blo.x - ahi.x));
  double dy = fmax(0.0, fmax(alo.y - bhi.y, blo.y - ahi.y));
  double dz = fmax(0.0, fmax(alo.z - bhi.z, blo.z - ahi.z));
  return sqrt(dx * dx + dy * dy + dz * dz);
}

static double point_box_dist(v3 p, v3 lo, v3 hi) {
  return box_dist(p, p, lo, hi);
}

static void tri_of(const ora_shape *s, int f, v3 *T) {
  for (int j = 0; j < 3; ++j) T[j] = s->V[s->F[3 * f + j]];
}

/* --------------------------------------------------------------- contact */

/* Distance from p to the outer surface of s (faces not flagged internal),
 * with the realising point (ties to the lower face index). */
static double surface_dist(const ora_shape *s, v3 p, v3 *q, int culled) {
  double best = INFINITY;
  v3 T[3];
  for (int f = 0; f < s->nf; ++f) {
    if (s->face_internal[f]) continue;
    if (culled && point_box_dist(p, s->blo[f], s->bhi[f]) > best + ORA_SLACK) continue;
    tri_of(s, f, T);
    v3 c = closest_on_tri(p, T[0], T[1], T[2]);
    double d = norm(sub(p, c));
    if (d < best) best = d, *q = c;
  }
  return best;
}

static int boxes_overlap(v3 alo, v3 ahi, v3 blo, v3 bhi) {
  return alo.x <= bhi.x + ORA_SLACK && blo.x <= ahi.x + ORA_SLACK &&
         alo.y <= bhi.y + ORA_SLACK && blo.y <= ahi.y + ORA_SLACK &&
         alo.z <= bhi.z + ORA_SLACK && blo.z <= ahi.z + ORA_SLACK;
}

/* Lowest intersecting face pair (fa, fb) in lexicographic order; returns 1 if
 * any, with the crossing midpoint. */
static int first_meeting_pair(const ora_shape *A, const ora_shape *B, int culled,
                              int *fa, int *fb, v3 *mid) {
  v3 T[3], U[3];
  for (int i = 0; i < A->nf; ++i) {
    if (culled && !boxes_overlap(A->blo[i], A->bhi[i], B->lo, B->hi)) continue;
    tri_of(A, i, T);
    for (int j = 0; j < B->nf; ++j) {
      if (culled && !boxes_overlap(A->blo[i], A->bhi[i], B->blo[j], B->bhi[j])) continue;
      tri_of(B, j, U);
      if (tri_tri_meet(T, U, mid)) {
        *fa = i, *fb = j;
        return 1;
      }
    }
  }
  return 0;
}

typedef struct { double d; int i; } ora_key;
static int key_cmp(const void *a, const void *b) {
  const ora_key *x = (const ora_key *)a, *y = (const ora_key *)b;
  if (x->d != y->d) return x->d < y->d ? -1 : 1;
  return x->i - y->i;
}

/* Minimum triangle-pair distance, realising points; ties to lowest (fa, fb). */
static double min_pair_dist(const ora_shape *A, const ora_shape *B, int culled,
                            v3 *pA, v3 *pB) {
  double best = INFINITY;
  int bi = -1, bj = -1;
  v3 T[3], U[3], x, y;
  ora_key *order = (ora_key *)malloc(sizeof(ora_key) * (size_t)A->nf);
  for (int i = 0; i < A->nf; ++i) {
    order[i].i = i;
    order[i].d = culled ? box_dist(A->blo[i], A->bhi[i], B->lo, B->hi) : 0.0;
  }
  if (culled) qsort(order, (size_t)A->nf, sizeof(ora_key), key_cmp);
  for (int oi = 0; oi < A->nf; ++oi) {
    int i = order[oi].i;
    if (culled && order[oi].d > best + ORA_SLACK) break;
    tri_of(A, i, T);
    for (int j = 0; j < B->nf; ++j) {
      if (culled && box_dist(A->blo[i], A->bhi[i], B->blo[j], B->bhi[j]) > best + ORA_SLACK)
        continue;
      tri_of(B, j, U);
      double d = tri_tri_dist(T, U, &x, &y);
      if (d < best || (d == best && (i < bi || (i == bi && j < bj)))) {
        best = d, bi = i, bj = j, *pA = x, *pB = y;
      }
    }
  }
  free(order);
  return best;
}

/* out = {label, point xyz, normal xyz, depth} in the world frame. */
static int ora_contact_built(const ora_shape *A, const ora_shape *B, int culled,
                             double *out) {
  int fa = -1, fb = -1;
  v3 mid = mk(0, 0, 0);
  int meet = first_meeting_pair(A, B, culled, &fa, &fb, &mid);
  /* candidates: samples of A, surface vertices of A inside B; then B in A */
  double best = -INFINITY;
  v3 bv = mk(0, 0, 0), bq = mk(0, 0, 0);
  int b_in_a = 0, any_inside = 0;
  for (int side = 0; side < 2; ++side) {
    const ora_shape *X = side == 0 ? A : B, *Y = side == 0 ? B : A;
    for (int pass = 0; pass < 2; ++pass) {
      int n = pass == 0 ? X->ns : X->nv;
      for (int i = 0; i < n; ++i) {
        if (pass == 1 && X->vert_internal[i]) continue;
        v3 v = pass == 0 ? X->S[i] : X->V[i];
        if (!inside_shape(Y, v, -1, culled)) continue;
        any_inside = 1;
        v3 q;
        double d = surface_dist(Y, v, &q, culled);
        if (d > best) best = d, bv = v, bq = q, b_in_a = side;
      }
    }
  }
  if (!meet && !any_inside) {
    v3 pA, pB;
    double g = min_pair_dist(A, B, culled, &pA, &pB);
    v3 pt = scl(add(pA, pB), 0.5);
    v3 n = g > 0 ? scl(sub(pB, pA), 1.0 / g) : mk(0, 0, 0);
    out[0] = 0.0;
    out[1] = pt.x, out[2] = pt.y, out[3] = pt.z;
    out[4] = n.x, out[5] = n.y, out[6] = n.z;
    out[7] = -g;
    return 0;
  }
  out[0] = 1.0;
  if (any_inside) {
    v3 pt = scl(add(bv, bq), 0.5);
    v3 n = b_in_a ? sub(bq, bv) : sub(bv, bq);
    double l = norm(n);
    n = l > 0 ? scl(n, 1.0 / l) : mk(0, 0, 0);
    out[1] = pt.x, out[2] = pt.y, out[3] = pt.z;
    out[4] = n.x, out[5] = n.y, out[6] = n.z;
    out[7] = best;
  } else {
    v3 T[3], U[3];
    tri_of(A, fa, T);
    tri_of(B, fb, U);
    v3 na = cross(sub(T[1], T[0]), sub(T[2], T[0]));
    v3 nb = cross(sub(U[1], U[0]), sub(U[2], U[0]));
    na = scl(na, 1.0 / norm(na));
    nb = scl(nb, 1.0 / norm(nb));
    v3 n = sub(na, nb);
    double l = norm(n);
    n = l > 0 ? scl(n, 1.0 / l) : mk(0, 0, 0);
    out[1] = mid.x, out[2] = mid.y, out[3] = mid.z;
    out[4] = n.x, out[5] = n.y, out[6] = n.z;
    out[7] = 0.0;
  }
  return 0;
}

typedef struct {
  const double *V; int nv; const int32_t *F; const int32_t *comp; int nf;
  const float *samples; int ns;
} ora_mesh_in;

/* One pair.  Meshes in body frames (float64 vertices), samples float32 in body
 * frames, poses float32 (w,x,y,z,tx,ty,tz). */
int ora_contact(const double *VA, int nvA, const int32_t *FA, const int32_t *compA, int nfA,
                const float *SA, int nsA, const float poseA[7],
                const double *VB, int nvB, const int32_t *FB, const int32_t *compB, int nfB,
                const float *SB, int nsB, const float poseB[7], int culled, double *out) {
  ora_shape A, B;
  int st = ora_build(&A, VA, nvA, FA, compA, nfA, SA, nsA, poseA, culled);
  if (st == 0) st = ora_build(&B, VB, nvB, FB, compB, nfB, SB, nsB, poseB, culled);
  else memset(&B, 0, sizeof(B));
  if (st == 0) st = ora_contact_built(&A, &B, culled, out);
  ora_free(&A);
  ora_free(&B);
  return st;
}

/* ------------------------------------------------------ batch over pairs */

typedef struct {
  /* library: concatenated meshes with per-shape offsets */
  const double *V; const int64_t *voff;
  const int32_t *F; const int32_t *comp; const int64_t *foff;
  const float *samples; int n_samples;
  const float *poses; const int32_t *obj_shape; const int32_t *pairs;
  int culled; double *out; int lo, hi; int status;
} ora_job;

static void *ora_worker(void *arg) {
  ora_job *j = (ora_job *)arg;
  for (int p = j->lo; p < j->hi; ++p) {
    int a = j->pairs[2 * p], b = j->pairs[2 * p + 1];
    int sa = j->obj_shape[a], sb = j->obj_shape[b];
    int st = ora_contact(
        j->V + 3 * j->voff[sa], (int)(j->voff[sa + 1] - j->voff[sa]), j->F + 3 * j->foff[sa],
        j->comp + j->foff[sa], (int)(j->foff[sa + 1] - j->foff[sa]),
        j->samples + (size_t)sa * j->n_samples * 3, j->n_samples, j->poses + 7 * a,
        j->V + 3 * j->voff[sb], (int)(j->voff[sb + 1] - j->voff[sb]), j->F + 3 * j->foff[sb],
        j->comp + j->foff[sb], (int)(j->foff[sb + 1] - j->foff[sb]),
        j->samples + (size_t)sb * j->n_samples * 3, j->n_samples, j->poses + 7 * b,
        j->culled, j->out + 8 * (size_t)p);
    if (st) j->status = st;
  }
  return NULL;
}

/* Contacts of n_pairs pairs over a library of meshes: V [sum nv][3] with
 * voff [S+1] (vertex offsets), F [sum nf][3] (per-shape local indices) and
 * comp [sum nf] with foff [S+1]; samples [S][n_samples][3]. */
int ora_contact_batch(const double *V, const int64_t *voff, const int32_t *F,
                      const int32_t *comp, const int64_t *foff,
                      const float *samples, int n_samples, const float *poses,
                      const int32_t *obj_shape, const int32_t *pairs, int n_pairs,
                      int culled, double *out, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  ora_job jobs[256];
  int per = (n_pairs + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    ora_job *j = &jobs[t];
    j->V = V, j->voff = voff, j->F = F, j->comp = comp, j->foff = foff;
    j->samples = samples, j->n_samples = n_samples, j->poses = poses;
    j->obj_shape = obj_shape, j->pairs = pairs, j->culled = culled, j->out = out;
    j->status = 0;
    j->lo = t * per;
    j->hi = (t + 1) * per < n_pairs ? (t + 1) * per : n_pairs;
    if (j->lo > j->hi) j->lo = j->hi;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, ora_worker, &jobs[t]);
  ora_worker(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  int st = 0;
  for (int t = 0; t < n_threads; ++t)
    if (jobs[t].status) st = jobs[t].status;
  return st;
}

/* Winding-number inside test of points against one posed mesh (for tests). */
int ora_inside(const double *V, int nv, const int32_t *F, const int32_t *comp, int nf,
               const float pose[7], const double *pts, int n, int32_t *res) {
  ora_shape s;
  int st = ora_build(&s, V, nv, F, comp, nf, NULL, 0, pose, 1);
  if (st == 0)
    for (int i = 0; i < n; ++i)
      res[i] = inside_shape(&s, mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]), -1, 0);
  ora_free(&s);
  return st;
}

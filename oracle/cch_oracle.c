/*
 * cch_oracle.c -- CPU FP64 oracle for the two-way continuous collision
 * handling step (arXiv 2211.04045).
 *
 * TEST INFRASTRUCTURE ONLY: the slow, plain reference for parity tests, the
 * smoke check and the CPU baseline of the benchmark.  The product path never
 * loads it.  It shares no code with the CUDA path.
 *
 * Every function follows one passage of the paper (cited beside it) in the
 * paper's order and notation.  Where the paper is silent the readings used
 * are stated at the function; they are the same readings the CUDA path
 * implements independently.  Compile with -ffp-contract=off: every floating
 * point expression below is evaluated exactly as written, left to right.
 */
#include "cch_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* 3-vectors                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;

static v3 ld3(const double* p, int64_t i) { v3 r = {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; return r; }
static void st3(double* p, int64_t i, v3 v) { p[3 * i] = v.x; p[3 * i + 1] = v.y; p[3 * i + 2] = v.z; }
static v3 sub3(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 add3(v3 a, v3 b) { v3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static v3 scl3(double s, v3 a) { v3 r = {s * a.x, s * a.y, s * a.z}; return r; }
/* x + a (y - x), the forward step of Eq. forward2: y itself at a = 1 and x
 * itself at a = 0 (a vertex that does not move keeps its position exactly,
 * even when y is not finite, R2c). */
static v3 step_to(v3 x, v3 y, double a) {
  if (a == 1.0) return y;
  if (a == 0.0) return x;
  return add3(x, scl3(a, sub3(y, x)));
}
static v3 div3(v3 a, double s) { v3 r = {a.x / s, a.y / s, a.z / s}; return r; }
static double dot3(v3 a, v3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static v3 cross3(v3 a, v3 b) {
  v3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
  return r;
}
static double norm3(v3 a) { return sqrt(dot3(a, a)); }
static double det3(v3 a, v3 b, v3 c) { return dot3(a, cross3(b, c)); }
static int eq3(v3 a, v3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

/* SplitMix64 (Steele, Lea, Flood 2014): the counter-based mixer that gives
 * the random sweep order of Sec. 4.3 its priorities. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

void orc_params_default(orc_params* p) {
  /* Table 2. */
  p->d_min = 2e-3; p->d_max = 4e-3; p->delta = 1e-3; p->sigma = 1.1; p->gamma = 0.9;
  p->eps = 1e-4; p->jacobi_omega = 0.5;
  p->max_iters = 2048; p->gs_sweeps = 1; p->solver = 0; p->ccd_check = 0; p->search_mode = 2;
  p->constraint_form = 0; p->step_rule = 0; p->ccd_rounds = 8; p->colouring = 1; p->seed = 0x2211040450ULL;
}

/* ------------------------------------------------------------------------ */
/* Distances between simplices (the dist() of Eq. relationship_P and Sec. 5) */
/* ------------------------------------------------------------------------ */

/* Closest distance from p to the segment [a,b]; t = clamped parameter. */
static double ps_dist(v3 p, v3 a, v3 b, double* t_out) {
  v3 e = sub3(b, a), w = sub3(p, a), q = a;
  double ee = dot3(e, e), t = 0.0;
  if (ee > 0.0) {
    t = dot3(w, e) / ee;
    if (t <= 0.0) { t = 0.0; q = a; }
    else if (t >= 1.0) { t = 1.0; q = b; }
    else q = add3(a, scl3(t, e));
  }
  if (t_out) *t_out = t;
  return norm3(sub3(p, q));
}

/* Closest distance from p to triangle (a,b,c).  The closest point is either
 * the projection onto the plane (when it falls inside, barycentric weights
 * of Sec. 4.1 all >= 0) or lies on one of the three edges. */
/* The same distance with the closest point's barycentric weights on (a, b, c)
 * and whether it lies inside the triangle (the plane projection). */
static double pt_closest(v3 p, v3 a, v3 b, v3 c, double wt[3], int* inside) {
  v3 e1 = sub3(b, a), e2 = sub3(c, a), w = sub3(p, a);
  v3 n = cross3(e1, e2);
  double nn = dot3(n, n);
  if (nn > 0.0) {
    double u = dot3(cross3(w, e2), n) / nn, v = dot3(cross3(e1, w), n) / nn;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
      wt[0] = (1.0 - u) - v; wt[1] = u; wt[2] = v;
      *inside = 1;
      return fabs(dot3(w, n)) / sqrt(nn);
    }
  }
  *inside = 0;
  double t1, t2, t3;
  double d = ps_dist(p, a, b, &t1), d2 = ps_dist(p, b, c, &t2), d3 = ps_dist(p, c, a, &t3);
  wt[0] = 1.0 - t1; wt[1] = t1; wt[2] = 0.0;
  if (d2 < d) { d = d2; wt[0] = 0.0; wt[1] = 1.0 - t2; wt[2] = t2; }
  if (d3 < d) { d = d3; wt[0] = t3; wt[1] = 0.0; wt[2] = 1.0 - t3; }
  return d;
}
static double pt_dist(v3 p, v3 a, v3 b, v3 c) {
  v3 e1 = sub3(b, a), e2 = sub3(c, a), w = sub3(p, a);
  v3 n = cross3(e1, e2);
  double nn = dot3(n, n);
  if (nn > 0.0) {
    double u = dot3(cross3(w, e2), n) / nn; /* weight of b */
    double v = dot3(cross3(e1, w), n) / nn; /* weight of c */
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) return fabs(dot3(w, n)) / sqrt(nn);
  }
  double d = ps_dist(p, a, b, 0), d2 = ps_dist(p, b, c, 0), d3 = ps_dist(p, c, a, 0);
  if (d2 < d) d = d2;
  if (d3 < d) d = d3;
  return d;
}

/* Closest distance between segments [a,b] and [c,d]: the interior critical
 * point of |a + s(b-a) - c - t(d-c)|^2 when it lies in [0,1]^2, and the four
 * endpoint-to-segment distances; the minimum of these. */
static double ss_dist(v3 a, v3 b, v3 c, v3 d, double* s_out, double* t_out) {
  v3 d1 = sub3(b, a), d2 = sub3(d, c), r = sub3(a, c);
  double A = dot3(d1, d1), E = dot3(d2, d2), B = dot3(d1, d2), C = dot3(d1, r), F = dot3(d2, r);
  double best = INFINITY, bs = 0.0, bt = 0.0, tt, dd;
  double den = A * E - B * B;
  if (den > 0.0) {
    double s = (B * F - C * E) / den, t = (A * F - B * C) / den;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      v3 p = add3(a, scl3(s, d1)), q = add3(c, scl3(t, d2));
      best = norm3(sub3(p, q)); bs = s; bt = t;
    }
  }
  dd = ps_dist(a, c, d, &tt); if (dd < best) { best = dd; bs = 0.0; bt = tt; }
  dd = ps_dist(b, c, d, &tt); if (dd < best) { best = dd; bs = 1.0; bt = tt; }
  dd = ps_dist(c, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 0.0; }
  dd = ps_dist(d, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 1.0; }
  if (s_out) *s_out = bs;
  if (t_out) *t_out = bt;
  return best;
}

double orc_point_segment_dist(const double p[3], const double a[3], const double b[3], double* t) {
  return ps_dist(ld3(p, 0), ld3(a, 0), ld3(b, 0), t);
}
double orc_point_triangle_dist(const double p[3], const double a[3], const double b[3], const double c[3]) {
  return pt_dist(ld3(p, 0), ld3(a, 0), ld3(b, 0), ld3(c, 0));
}
double orc_segment_segment_dist(const double a[3], const double b[3], const double c[3], const double d[3],
                                double* s, double* t) {
  return ss_dist(ld3(a, 0), ld3(b, 0), ld3(c, 0), ld3(d, 0), s, t);
}
/* det[b-a, c-a, d-a]: six times the signed volume of tetrahedron abcd
 * (the volume of Eq. volume_by_det). */
double orc_signed_volume(const double a[3], const double b[3], const double c[3], const double d[3]) {
  v3 A = ld3(a, 0);
  return det3(sub3(ld3(b, 0), A), sub3(ld3(c, 0), A), sub3(ld3(d, 0), A));
}

/* ------------------------------------------------------------------------ */
/* Exact predicates: floating-point expansions (Shewchuk 1997).  An         */
/* expansion is a list of doubles, nonoverlapping and of increasing         */
/* magnitude, whose exact sum is the value; its sign is the sign of its     */
/* last nonzero component.                                                  */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b, bv = x - a, av = x - bv, br = b - bv, ar = a - av;
  *s = x; *e = ar + br;
}
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *p = x; *e = fma(a, b, -x); /* fma is correctly rounded: the error term is exact */
}
/* h = e + b (Shewchuk's GROW-EXPANSION with zero elimination). */
static int grow(int elen, const double* e, double b, double* h) {
  double q = b, s, err;
  int hl = 0;
  for (int i = 0; i < elen; i++) {
    two_sum(q, e[i], &s, &err);
    if (err != 0.0) h[hl++] = err;
    q = s;
  }
  if (q != 0.0 || hl == 0) h[hl++] = q;
  return hl;
}
typedef struct { int n; double c[512]; } expn;
static void ex_add(expn* e, double b) {
  double tmp[512];
  int n = grow(e->n, e->c, b, tmp);
  memcpy(e->c, tmp, sizeof(double) * (size_t)n);
  e->n = n;
}
/* e += sign * a * b * c, exactly. */
static void ex_add_triple(expn* e, double sign, double a, double b, double c) {
  double p, pe, p1, e1, p2, e2;
  two_prod(a, b, &p, &pe);
  two_prod(p, c, &p1, &e1);
  two_prod(pe, c, &p2, &e2);
  ex_add(e, sign * e2); ex_add(e, sign * p2); ex_add(e, sign * e1); ex_add(e, sign * p1);
}
static void ex_add_pair(expn* e, double sign, double a, double b) {
  double p, pe;
  two_prod(a, b, &p, &pe);
  ex_add(e, sign * pe); ex_add(e, sign * p);
}
static int ex_sign(const expn* e) {
  for (int i = e->n - 1; i >= 0; i--)
    if (e->c[i] != 0.0) return e->c[i] > 0.0 ? 1 : -1;
  return 0;
}
/* det3 of raw coordinates as six signed triple products. */
static void ex_det3(expn* e, double sg, v3 p, v3 q, v3 r) {
  ex_add_triple(e, sg, p.x, q.y, r.z); ex_add_triple(e, -sg, p.x, q.z, r.y);
  ex_add_triple(e, -sg, p.y, q.x, r.z); ex_add_triple(e, sg, p.y, q.z, r.x);
  ex_add_triple(e, sg, p.z, q.x, r.y); ex_add_triple(e, -sg, p.z, q.y, r.x);
}
/* Exact sign of det[b-a, c-a, d-a] = det(b,c,d) - det(a,c,d) + det(a,b,d) - det(a,b,c). */
static int o3_exact(v3 a, v3 b, v3 c, v3 d) {
  expn e; e.n = 0;
  ex_det3(&e, 1.0, b, c, d); ex_det3(&e, -1.0, a, c, d);
  ex_det3(&e, 1.0, a, b, d); ex_det3(&e, -1.0, a, b, c);
  return ex_sign(&e);
}
/* Filtered orient3d: the FP64 value decides when it exceeds a generous
 * bound on its rounding error (45 ulps of the permanent); else exact. */
static int o3(v3 a, v3 b, v3 c, v3 d) {
  v3 u = sub3(b, a), v = sub3(c, a), w = sub3(d, a);
  double det = det3(u, v, w);
  double perm = fabs(u.x) * (fabs(v.y * w.z) + fabs(v.z * w.y)) + fabs(u.y) * (fabs(v.x * w.z) + fabs(v.z * w.x)) +
                fabs(u.z) * (fabs(v.x * w.y) + fabs(v.y * w.x));
  double bound = 5e-15 * perm;
  if (det > bound) return 1;
  if (det < -bound) return -1;
  return o3_exact(a, b, c, d);
}
int orc_orient3d_exact(const double a[3], const double b[3], const double c[3], const double d[3]) {
  return o3_exact(ld3(a, 0), ld3(b, 0), ld3(c, 0), ld3(d, 0));
}
/* Exact sign of the 2-D orientation of (a,b,c) using coordinates (i,j). */
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static int o2_exact(v3 a, v3 b, v3 c, int i, int j) {
  /* (bi-ai)(cj-aj) - (bj-aj)(ci-ai) expanded into raw products */
  expn e; e.n = 0;
  double ai = comp(a, i), aj = comp(a, j), bi = comp(b, i), bj = comp(b, j), ci = comp(c, i), cj = comp(c, j);
  ex_add_pair(&e, 1.0, bi, cj); ex_add_pair(&e, -1.0, bi, aj); ex_add_pair(&e, -1.0, ai, cj);
  ex_add_pair(&e, -1.0, bj, ci); ex_add_pair(&e, 1.0, bj, ai); ex_add_pair(&e, 1.0, aj, ci);
  return ex_sign(&e);
}
/* q lies on the closed segment [a,b], all three collinear (exact compares). */
static int on_seg_collinear(v3 q, v3 a, v3 b) {
  return (q.x >= fmin(a.x, b.x) && q.x <= fmax(a.x, b.x) && q.y >= fmin(a.y, b.y) && q.y <= fmax(a.y, b.y) &&
          q.z >= fmin(a.z, b.z) && q.z <= fmax(a.z, b.z));
}
/* Closed 2-D segments [p,q], [r,s] intersect (coordinates i,j). */
static int seg2_exact(v3 p, v3 q, v3 r, v3 s, int i, int j) {
  int o1 = o2_exact(p, q, r, i, j), o2 = o2_exact(p, q, s, i, j);
  int o3v = o2_exact(r, s, p, i, j), o4 = o2_exact(r, s, q, i, j);
  if (o1 * o2 < 0 && o3v * o4 < 0) return 1;
  if (o1 == 0 && on_seg_collinear(r, p, q)) return 1;
  if (o2 == 0 && on_seg_collinear(s, p, q)) return 1;
  if (o3v == 0 && on_seg_collinear(p, r, s)) return 1;
  if (o4 == 0 && on_seg_collinear(q, r, s)) return 1;
  return 0;
}
/* A projection plane (i,j) in which three coplanar points are not collinear;
 * returns 0 when they are collinear in every projection. */
static int pick_plane(v3 a, v3 b, v3 c, int* i, int* j) {
  static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int k = 0; k < 3; k++)
    if (o2_exact(a, b, c, P[k][0], P[k][1]) != 0) { *i = P[k][0]; *j = P[k][1]; return 1; }
  return 0;
}
/* Point in closed 2-D triangle. */
static int pt_in_tri2(v3 p, v3 a, v3 b, v3 c, int i, int j) {
  int s1 = o2_exact(a, b, p, i, j), s2 = o2_exact(b, c, p, i, j), s3 = o2_exact(c, a, p, i, j);
  int pos = (s1 > 0) + (s2 > 0) + (s3 > 0), neg = (s1 < 0) + (s2 < 0) + (s3 < 0);
  return !(pos && neg);
}
/* Closed 3-D segments [p,q], [r,s] intersect. */
static int seg_seg_exact(v3 p, v3 q, v3 r, v3 s) {
  if (o3(p, q, r, s) != 0) return 0;
  /* coplanar: find a projection where the four points are not all collinear */
  int i, j;
  if (pick_plane(p, q, r, &i, &j) || pick_plane(p, q, s, &i, &j) || pick_plane(r, s, p, &i, &j) ||
      pick_plane(r, s, q, &i, &j))
    return seg2_exact(p, q, r, s, i, j);
  /* all four collinear: they overlap iff an endpoint of one lies on the other */
  return on_seg_collinear(p, r, s) || on_seg_collinear(q, r, s) || on_seg_collinear(r, p, q) ||
         on_seg_collinear(s, p, q);
}
/* Closed segment [p,q] and closed triangle (a,b,c) intersect. */
static int seg_tri_exact(v3 p, v3 q, v3 a, v3 b, v3 c) {
  int s1 = o3(a, b, c, p), s2 = o3(a, b, c, q);
  if (s1 != 0 && s1 == s2) return 0;
  int i, j;
  if (s1 == 0 && s2 == 0) {
    if (!pick_plane(a, b, c, &i, &j))
      return seg_seg_exact(p, q, a, b) || seg_seg_exact(p, q, b, c) || seg_seg_exact(p, q, c, a);
    if (pt_in_tri2(p, a, b, c, i, j) || pt_in_tri2(q, a, b, c, i, j)) return 1;
    return seg2_exact(p, q, a, b, i, j) || seg2_exact(p, q, b, c, i, j) || seg2_exact(p, q, c, a, i, j);
  }
  int t1 = o3(p, q, a, b), t2 = o3(p, q, b, c), t3 = o3(p, q, c, a);
  int pos = (t1 > 0) + (t2 > 0) + (t3 > 0), neg = (t1 < 0) + (t2 < 0) + (t3 < 0);
  if (pos && neg) return 0;
  if (pos == 0 && neg == 0) /* degenerate: segment on the triangle's line set */
    return seg_seg_exact(p, q, a, b) || seg_seg_exact(p, q, b, c) || seg_seg_exact(p, q, c, a);
  return 1;
}
/* Point p on closed triangle (a,b,c). */
static int pt_on_tri_exact(v3 p, v3 a, v3 b, v3 c) {
  if (o3(a, b, c, p) != 0) return 0;
  int i, j;
  if (!pick_plane(a, b, c, &i, &j))
    return seg_seg_exact(p, p, a, b) || seg_seg_exact(p, p, b, c) || seg_seg_exact(p, p, c, a);
  return pt_in_tri2(p, a, b, c, i, j);
}

/* ------------------------------------------------------------------------ */
/* Scene-derived data                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_topology* t;
  int64_t n;
  uint8_t* is_point;   /* vertex is a VV participant                           */
  uint8_t* is_coll;    /* vertex belongs to a triangle, collision edge or point */
  uint8_t* is_static;  /* inv_mass == 0 and x~ == x^t: never moves in the step  */
  int32_t* vc;         /* collision vertices, ascending                         */
  int64_t n_vc;
} scene;

static double rho_of(const orc_topology* t, int64_t v) { return t->radius ? t->radius[v] : 0.0; }

static void scene_init(scene* s, const orc_topology* t, const double* x_t, const double* x_tilde) {
  int64_t n = t->n_verts;
  s->t = t; s->n = n;
  s->is_point = (uint8_t*)calloc((size_t)n + 1, 1);
  s->is_coll = (uint8_t*)calloc((size_t)n + 1, 1);
  s->is_static = (uint8_t*)calloc((size_t)n + 1, 1);
  for (int64_t i = 0; i < t->n_points; i++) { s->is_point[t->points[i]] = 1; s->is_coll[t->points[i]] = 1; }
  for (int64_t i = 0; i < 3 * t->n_tris; i++) s->is_coll[t->tris[i]] = 1;
  for (int64_t i = 0; i < 2 * t->n_edges; i++) s->is_coll[t->edges[i]] = 1;
  s->vc = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  s->n_vc = 0;
  for (int64_t v = 0; v < n; v++) {
    if (s->is_coll[v]) s->vc[s->n_vc++] = (int32_t)v;
    /* R4: a vertex with zero inverse mass whose target equals its start
     * never moves in this step. */
    s->is_static[v] = (t->inv_mass[v] == 0.0 && eq3(ld3(x_t, v), ld3(x_tilde, v)));
  }
}
static void scene_free(scene* s) { free(s->is_point); free(s->is_coll); free(s->is_static); free(s->vc); }

/* ------------------------------------------------------------------------ */
/* Pairs and their canonical keys                                            */
/* ------------------------------------------------------------------------ */
/* key = kind<<62 | id1<<31 | id2, ids < 2^31.  VT: (vertex, triangle);
 * EE: (edge, edge) with id1 < id2; VV: (point, vertex). */
static uint64_t mkkey(int kind, int64_t a, int64_t b) {
  return ((uint64_t)kind << 62) | ((uint64_t)a << 31) | (uint64_t)b;
}
static int key_kind(uint64_t k) { return (int)(k >> 62); }
static int64_t key_a(uint64_t k) { return (int64_t)((k >> 31) & 0x7fffffffULL); }
static int64_t key_b(uint64_t k) { return (int64_t)(k & 0x7fffffffULL); }

/* Vertex ids of a pair: VT (a,i,j,k), EE (a,b,c,d), VV (a,b). */
static int pair_verts(const orc_topology* t, uint64_t key, int32_t v[4]) {
  int kind = key_kind(key);
  int64_t a = key_a(key), b = key_b(key);
  if (kind == ORC_VT) {
    v[0] = (int32_t)a; v[1] = t->tris[3 * b]; v[2] = t->tris[3 * b + 1]; v[3] = t->tris[3 * b + 2];
    return 4;
  }
  if (kind == ORC_EE) {
    v[0] = t->edges[2 * a]; v[1] = t->edges[2 * a + 1]; v[2] = t->edges[2 * b]; v[3] = t->edges[2 * b + 1];
    return 4;
  }
  v[0] = (int32_t)a; v[1] = (int32_t)b; v[2] = -1; v[3] = -1;
  return 2;
}

/* Distance of a pair at state x (R5): VT point-triangle minus the point's
 * radius; EE segment-segment; VV centre distance minus both radii. */
static double pair_dist(const orc_topology* t, uint64_t key, const double* x, double* s, double* tt) {
  int32_t v[4];
  int kind = key_kind(key);
  pair_verts(t, key, v);
  if (kind == ORC_VT) return pt_dist(ld3(x, v[0]), ld3(x, v[1]), ld3(x, v[2]), ld3(x, v[3])) - rho_of(t, v[0]);
  if (kind == ORC_EE) return ss_dist(ld3(x, v[0]), ld3(x, v[1]), ld3(x, v[2]), ld3(x, v[3]), s, tt);
  return (norm3(sub3(ld3(x, v[0]), ld3(x, v[1]))) - rho_of(t, v[0])) - rho_of(t, v[1]);
}

/* ------------------------------------------------------------------------ */
/* Proximity search, Sec. 3.1                                                */
/* ------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; } box;

static box box_vertex(const double* x, int64_t v, double rho) {
  box b;
  v3 p = ld3(x, v);
  b.lo[0] = p.x - rho; b.lo[1] = p.y - rho; b.lo[2] = p.z - rho;
  b.hi[0] = p.x + rho; b.hi[1] = p.y + rho; b.hi[2] = p.z + rho;
  return b;
}
static box box_of(const double* x, const int32_t* v, int nv) {
  box b;
  for (int k = 0; k < 3; k++) { b.lo[k] = x[3 * v[0] + k]; b.hi[k] = x[3 * v[0] + k]; }
  for (int i = 1; i < nv; i++)
    for (int k = 0; k < 3; k++) {
      double c = x[3 * v[i] + k];
      if (c < b.lo[k]) b.lo[k] = c;
      if (c > b.hi[k]) b.hi[k] = c;
    }
  return b;
}
/* R3: two boxes are candidates when, on every axis, the computed gap
 * fl(lo_2 - hi_1) and fl(lo_1 - hi_2) is at most D. */
static int box_near(const box* a, const box* b, double D) {
  for (int k = 0; k < 3; k++) {
    if (b->lo[k] - a->hi[k] > D) return 0;
    if (a->lo[k] - b->hi[k] > D) return 0;
  }
  return 1;
}

typedef struct { uint64_t* k; int64_t n, cap; } keyvec;
static void kv_push(keyvec* v, uint64_t k) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 1024;
    v->k = (uint64_t*)realloc(v->k, sizeof(uint64_t) * (size_t)v->cap);
  }
  v->k[v->n++] = k;
}
static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y);
}

/* Pair exclusions (R4): shared vertex, or every vertex static. */
static int all_static(const scene* s, const int32_t* v, int nv) {
  for (int i = 0; i < nv; i++)
    if (!s->is_static[v[i]]) return 0;
  return 1;
}

typedef struct { box b; double key; int32_t id; } sbox; /* for the sorted-axis window */
static int cmp_sbox(const void* a, const void* b) {
  double x = ((const sbox*)a)->key, y = ((const sbox*)b)->key;
  if (x < y) return -1;
  if (x > y) return 1;
  return ((const sbox*)a)->id - ((const sbox*)b)->id;
}

/* Candidate pairs of state x at bound D (unsorted, appended to out).
 * mode 0 tests all pairs; mode 1 visits, per query, only targets whose
 * lower bound on the widest axis lies in a window that contains every
 * target passing the box test, then applies the same box test, so both
 * modes produce the same set. */
static void candidates(const scene* s, const double* x, double D, int mode, keyvec* out) {
  const orc_topology* t = s->t;
  int64_t T = t->n_tris, E = t->n_edges, nvc = s->n_vc;
  box* tb = (box*)malloc(sizeof(box) * ((size_t)T + 1));
  box* eb = (box*)malloc(sizeof(box) * ((size_t)E + 1));
  box* vb = (box*)malloc(sizeof(box) * ((size_t)nvc + 1));
  for (int64_t i = 0; i < T; i++) tb[i] = box_of(x, t->tris + 3 * i, 3);
  for (int64_t i = 0; i < E; i++) eb[i] = box_of(x, t->edges + 2 * i, 2);
  for (int64_t i = 0; i < nvc; i++) vb[i] = box_vertex(x, s->vc[i], rho_of(t, s->vc[i]));
  if (mode == 2) mode = (nvc * T + E * E / 2 > 4000000) ? 1 : 0;

  /* widest axis of the collision vertices, and a window slack far above any
   * rounding of a coordinate difference */
  int ax = 0;
  double slack = 0.0;
  if (mode == 1) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, M = 0.0;
    for (int64_t i = 0; i < nvc; i++)
      for (int k = 0; k < 3; k++) {
        if (vb[i].lo[k] < lo[k]) lo[k] = vb[i].lo[k];
        if (vb[i].hi[k] > hi[k]) hi[k] = vb[i].hi[k];
        if (fabs(vb[i].lo[k]) > M) M = fabs(vb[i].lo[k]);
        if (fabs(vb[i].hi[k]) > M) M = fabs(vb[i].hi[k]);
      }
    for (int k = 1; k < 3; k++)
      if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
    slack = 1e-9 * (1.0 + M) + 1e-9 * D;
  }

  /* VT: collision vertex vs triangle */
  if (mode == 0) {
    for (int64_t qi = 0; qi < nvc; qi++) {
      int32_t a = s->vc[qi];
      for (int64_t tr = 0; tr < T; tr++) {
        const int32_t* tv = t->tris + 3 * tr;
        if (a == tv[0] || a == tv[1] || a == tv[2]) continue;
        int32_t v4[4] = {a, tv[0], tv[1], tv[2]};
        if (all_static(s, v4, 4)) continue;
        if (box_near(&vb[qi], &tb[tr], D)) kv_push(out, mkkey(ORC_VT, a, tr));
      }
    }
  } else {
    sbox* st = (sbox*)malloc(sizeof(sbox) * ((size_t)T + 1));
    double W = 0.0;
    for (int64_t i = 0; i < T; i++) {
      st[i].b = tb[i]; st[i].key = tb[i].lo[ax]; st[i].id = (int32_t)i;
      if (tb[i].hi[ax] - tb[i].lo[ax] > W) W = tb[i].hi[ax] - tb[i].lo[ax];
    }
    qsort(st, (size_t)T, sizeof(sbox), cmp_sbox);
    for (int64_t qi = 0; qi < nvc; qi++) {
      int32_t a = s->vc[qi];
      double from = vb[qi].lo[ax] - D - W - slack, to = vb[qi].hi[ax] + D + slack;
      int64_t lo = 0, hi = T;
      while (lo < hi) { int64_t m = (lo + hi) / 2; if (st[m].key < from) lo = m + 1; else hi = m; }
      for (int64_t k = lo; k < T && st[k].key <= to; k++) {
        int64_t tr = st[k].id;
        const int32_t* tv = t->tris + 3 * tr;
        if (a == tv[0] || a == tv[1] || a == tv[2]) continue;
        int32_t v4[4] = {a, tv[0], tv[1], tv[2]};
        if (all_static(s, v4, 4)) continue;
        if (box_near(&vb[qi], &tb[tr], D)) kv_push(out, mkkey(ORC_VT, a, tr));
      }
    }
    free(st);
  }

  /* EE: unordered pairs of collision edges */
  if (mode == 0) {
    for (int64_t e1 = 0; e1 < E; e1++)
      for (int64_t e2 = e1 + 1; e2 < E; e2++) {
        const int32_t *p = t->edges + 2 * e1, *q = t->edges + 2 * e2;
        if (p[0] == q[0] || p[0] == q[1] || p[1] == q[0] || p[1] == q[1]) continue;
        int32_t v4[4] = {p[0], p[1], q[0], q[1]};
        if (all_static(s, v4, 4)) continue;
        if (box_near(&eb[e1], &eb[e2], D)) kv_push(out, mkkey(ORC_EE, e1, e2));
      }
  } else {
    sbox* st = (sbox*)malloc(sizeof(sbox) * ((size_t)E + 1));
    double W = 0.0;
    for (int64_t i = 0; i < E; i++) {
      st[i].b = eb[i]; st[i].key = eb[i].lo[ax]; st[i].id = (int32_t)i;
      if (eb[i].hi[ax] - eb[i].lo[ax] > W) W = eb[i].hi[ax] - eb[i].lo[ax];
    }
    qsort(st, (size_t)E, sizeof(sbox), cmp_sbox);
    for (int64_t e1 = 0; e1 < E; e1++) {
      double from = eb[e1].lo[ax] - D - W - slack, to = eb[e1].hi[ax] + D + slack;
      int64_t lo = 0, hi = E;
      while (lo < hi) { int64_t m = (lo + hi) / 2; if (st[m].key < from) lo = m + 1; else hi = m; }
      for (int64_t k = lo; k < E && st[k].key <= to; k++) {
        int64_t e2 = st[k].id;
        if (e2 <= e1) continue;
        const int32_t *p = t->edges + 2 * e1, *q = t->edges + 2 * e2;
        if (p[0] == q[0] || p[0] == q[1] || p[1] == q[0] || p[1] == q[1]) continue;
        int32_t v4[4] = {p[0], p[1], q[0], q[1]};
        if (all_static(s, v4, 4)) continue;
        if (box_near(&eb[e1], &eb[e2], D)) kv_push(out, mkkey(ORC_EE, e1, e2));
      }
    }
    free(st);
  }

  /* VV: a point against every other collision vertex (a point pair once) */
  for (int64_t pi = 0; pi < t->n_points; pi++) {
    int32_t a = t->points[pi];
    box ba = box_vertex(x, a, rho_of(t, a));
    for (int64_t qi = 0; qi < nvc; qi++) {
      int32_t b = s->vc[qi];
      if (b == a) continue;
      if (s->is_point[b] && b < a) continue;
      int32_t v2[2] = {a, b};
      if (all_static(s, v2, 2)) continue;
      if (box_near(&ba, &vb[qi], D)) kv_push(out, mkkey(ORC_VV, a, b));
    }
  }
  free(tb); free(eb); free(vb);
}

int64_t orc_candidates(const orc_topology* t, const double* x, const double* x_tilde, double D, int32_t mode,
                       uint64_t* keys, int64_t cap) {
  scene s; scene_init(&s, t, x, x_tilde ? x_tilde : x);
  keyvec kv = {0, 0, 0};
  candidates(&s, x, D, mode, &kv);
  qsort(kv.k, (size_t)kv.n, sizeof(uint64_t), cmp_u64);
  for (int64_t i = 0; i < kv.n && i < cap; i++) keys[i] = kv.k[i];
  int64_t n = kv.n;
  free(kv.k); scene_free(&s);
  return n;
}

/* P = {candidate pairs with dist < D} (Eq. relationship_P with D = D^max). */
typedef struct { uint64_t* k; double* d; int64_t n, cap; } pairset;
static void ps_push(pairset* p, uint64_t k, double d) {
  if (p->n == p->cap) {
    p->cap = p->cap ? 2 * p->cap : 1024;
    p->k = (uint64_t*)realloc(p->k, sizeof(uint64_t) * (size_t)p->cap);
    p->d = (double*)realloc(p->d, sizeof(double) * (size_t)p->cap);
  }
  p->k[p->n] = k; p->d[p->n] = d; p->n++;
}
static int64_t proximity_search(const scene* s, const double* x, double D, int mode, pairset* P) {
  keyvec kv = {0, 0, 0};
  candidates(s, x, D, mode, &kv);
  qsort(kv.k, (size_t)kv.n, sizeof(uint64_t), cmp_u64);
  P->n = 0;
  for (int64_t i = 0; i < kv.n; i++) {
    double d = pair_dist(s->t, kv.k[i], x, 0, 0);
    if (d < D) ps_push(P, kv.k[i], d);
  }
  int64_t nc = kv.n;
  free(kv.k);
  return nc;
}

int64_t orc_proximity(const orc_topology* t, const double* x, const double* x_tilde, double D, int32_t mode,
                      uint64_t* keys, double* dist, int64_t cap) {
  scene s; scene_init(&s, t, x, x_tilde ? x_tilde : x);
  pairset P = {0, 0, 0, 0};
  proximity_search(&s, x, D, mode, &P);
  for (int64_t i = 0; i < P.n && i < cap; i++) { keys[i] = P.k[i]; if (dist) dist[i] = P.d[i]; }
  int64_t n = P.n;
  free(P.k); free(P.d); scene_free(&s);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Contact constraints, Sec. 4.1                                              */
/* ------------------------------------------------------------------------ */
/* Volume constraint of Eq. volume_by_det for four vertices p0..p3 whose
 * reference shape r moves p0 (and p1 when mv1 = +1) by +h n and the others
 * by -h n, h = (delta - d)/2:  c = det[Dx]/det[Dr] - 1, with the reference
 * held constant; gradient of det[p1-p0, p2-p0, p3-p0] over det[Dr]. */
static int volume_constraint(const v3 p[4], const double sgn[4], v3 n, double h, double* c0, v3 g[4]) {
  v3 r[4];
  for (int i = 0; i < 4; i++) r[i] = add3(p[i], scl3(sgn[i] * h, n));
  v3 c1 = sub3(p[1], p[0]), c2 = sub3(p[2], p[0]), c3 = sub3(p[3], p[0]);
  double dx = det3(c1, c2, c3);
  double dr = det3(sub3(r[1], r[0]), sub3(r[2], r[0]), sub3(r[3], r[0]));
  if (!(fabs(dr) >= 1e-30)) return 0;
  *c0 = dx / dr - 1.0;
  g[1] = div3(cross3(c2, c3), dr);
  g[2] = div3(cross3(c3, c1), dr);
  g[3] = div3(cross3(c1, c2), dr);
  v3 s = add3(add3(g[1], g[2]), g[3]);
  g[0] = scl3(-1.0, s);
  return 1;
}

/* Gap constraint (reading G1; the comparison constraints of Sec. 4.1's gap
 * figure): c = d/delta - 1, d the pair distance, with gradient w_v n / delta
 * at each vertex, w_v its signed closest-point weight (+ on the first
 * primitive, - on the second) and n the unit direction from the second
 * primitive's closest point to the first's. */
static void gap_constraint(double d, double delta, v3 n, const double w[4], double* c0, v3 g[4]) {
  *c0 = d / delta - 1.0;
  for (int k = 0; k < 4; k++) g[k] = scl3(w[k] / delta, n);
}

/* VT (R6): n is the unit triangle normal flipped to the vertex's side; the
 * vertex moves along +n and the triangle along -n.  d is the pair distance
 * (point radius already subtracted). */
static int vt_constraint(const v3 p[4], double d, double delta, int form, double* c0, v3 g[4]) {
  v3 nrm = cross3(sub3(p[2], p[1]), sub3(p[3], p[1]));
  double nn = dot3(nrm, nrm);
  if (!(nn > 0.0)) return 0;
  v3 nh = div3(nrm, sqrt(nn));
  double side = dot3(nh, sub3(p[0], p[1])) < 0.0 ? -1.0 : 1.0;
  v3 n = scl3(side, nh);
  if (form == 1) {
    /* gap (G1): the closest point q of the triangle; n = (p - q)/|p - q|,
     * the flipped normal when the projection is inside or p lies on it */
    double wt[3];
    int inside;
    pt_closest(p[0], p[1], p[2], p[3], wt, &inside);
    if (!inside) {
      v3 q = add3(add3(scl3(wt[0], p[1]), scl3(wt[1], p[2])), scl3(wt[2], p[3]));
      v3 dv = sub3(p[0], q);
      double L = norm3(dv);
      if (L > 0.0) n = div3(dv, L);
    }
    double w[4] = {1.0, -wt[0], -wt[1], -wt[2]};
    gap_constraint(d, delta, n, w, c0, g);
    return 1;
  }
  static const double sg[4] = {1.0, -1.0, -1.0, -1.0};
  return volume_constraint(p, sg, n, 0.5 * (delta - d), c0, g);
}

/* EE (R7): n points from the closest point of cd to that of ab; ab moves
 * along +n and cd along -n.  Near-parallel edges (sin < 1e-6) use the gap
 * form c = d/delta - 1 with the closest-point weights. */
static int ee_constraint(const v3 p[4], double d, double s, double t, double delta, int form, double* c0,
                         v3 g[4]) {
  v3 e1 = sub3(p[1], p[0]), e2 = sub3(p[3], p[2]);
  v3 nx = cross3(e1, e2);
  double nn = dot3(nx, nx);
  v3 pa = add3(p[0], scl3(s, e1)), pc = add3(p[2], scl3(t, e2));
  v3 dv = sub3(pa, pc);
  double L = norm3(dv);
  v3 n;
  if (L > 0.0) n = div3(dv, L);
  else if (nn > 0.0) n = div3(nx, sqrt(nn));
  else return 0;
  if (form == 1 || nn < 1e-12 * (dot3(e1, e1) * dot3(e2, e2))) {
    double w[4] = {1.0 - s, s, -(1.0 - t), -t};
    gap_constraint(d, delta, n, w, c0, g);
    return 1;
  }
  static const double sg[4] = {1.0, 1.0, -1.0, -1.0};
  return volume_constraint(p, sg, n, 0.5 * (delta - d), c0, g);
}

/* VV (R8): c = |x_a - x_b| / (rho_a + rho_b + delta) - 1; reduces to the
 * point constraint of Sec. 4.1 when both radii are zero. */
static int vv_constraint(const v3 p[2], double ra, double rb, double delta, double* c0, v3 g[4]) {
  v3 dv = sub3(p[0], p[1]);
  double L = norm3(dv);
  if (!(L > 0.0)) return 0;
  double R = (ra + rb) + delta;
  *c0 = L / R - 1.0;
  v3 u = div3(dv, L);
  g[0] = div3(u, R);
  g[1] = scl3(-1.0, g[0]);
  return 1;
}

int orc_contact_constraint(int kind, const double* p, const double* rho, double delta, int form, double* c0,
                           double* g) {
  v3 P[4], G[4];
  int ok;
  if (kind == ORC_VT) {
    for (int i = 0; i < 4; i++) P[i] = ld3(p, i);
    double d = pt_dist(P[0], P[1], P[2], P[3]) - rho[0];
    ok = vt_constraint(P, d, delta, form, c0, G);
  } else if (kind == ORC_EE) {
    for (int i = 0; i < 4; i++) P[i] = ld3(p, i);
    double s, t, d = ss_dist(P[0], P[1], P[2], P[3], &s, &t);
    ok = ee_constraint(P, d, s, t, delta, form, c0, G);
  } else {
    P[0] = ld3(p, 0); P[1] = ld3(p, 1);
    ok = vv_constraint(P, rho[0], rho[1], delta, c0, G);
  }
  if (ok) for (int i = 0; i < (kind == ORC_VV ? 2 : 4); i++) st3(g, i, G[i]);
  return ok;
}

/* ------------------------------------------------------------------------ */
/* Constraint records and the linearised LCP of Eq. LCP                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t v[4];
  int nv;
  double c0;      /* c(x^(l)) ; edges: unused                                  */
  v3 g[4];        /* dc/dx_v ; edges: g[0] = u/L0                              */
  double den;     /* sum_v m_v^-1 |g_v|^2                                       */
  uint64_t key;   /* canonical identity                                          */
  uint64_t prio;  /* colouring priority (R11)                                    */
  int32_t colour; /* colour class of the Gauss-Seidel sweep (Sec. 4.3)          */
  double lambda;
} cons;

/* Order of the projected Gauss-Seidel sweep (Sec. 4.3, reading R11).  The
 * paper's sweep is multi-colour Gauss-Seidel: the constraints are split into
 * colour classes in which no two share a vertex, by a randomized colouring,
 * and the classes are applied one after the other, the constraints of one
 * class in parallel.  Here the randomness is a priority per constraint,
 * splitmix64(seed ^ key) (a bijection of the unique keys, so no ties), and
 * the colouring is one of two randomized colourings, both taken over the
 * constraints in descending priority with conflicts through movable vertices
 * only (static vertices never change y): the greedy one, each constraint the
 * smallest colour not used by a higher-priority constraint sharing a movable
 * vertex with it (the Jones-Plassmann colouring), or the level one, one more
 * than the largest colour among those (the round in which the constraint's
 * priority first exceeds that of all its uncoloured conflicting constraints,
 * as in Luby's rounds).  Contacts are coloured among themselves every
 * iteration, edge-length constraints among themselves.  The sequential sweep
 * applies the contact classes in ascending colour, then the edge classes;
 * inside a class the order does not change the result (no shared movable
 * vertex), and it is taken by descending priority. */
static int cmp_cons_prio_desc(const void* a, const void* b) {
  uint64_t pa = ((const cons*)a)->prio, pb = ((const cons*)b)->prio;
  return pa > pb ? -1 : pa < pb;
}
static int cmp_cons_colour(const void* a, const void* b) {
  const cons *ca = (const cons*)a, *cb = (const cons*)b;
  if (ca->colour != cb->colour) return ca->colour < cb->colour ? -1 : 1;
  return cmp_cons_prio_desc(a, b);
}

/* colours used so far at one vertex */
typedef struct { int32_t* c; int32_t n, cap; } ilist;
static void il_push(ilist* l, int32_t v) {
  if (l->n == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 8;
    l->c = (int32_t*)realloc(l->c, sizeof(int32_t) * (size_t)l->cap);
  }
  l->c[l->n++] = v;
}

/* Level colouring of cs[0..n), sorted by descending priority: one more than
 * the largest colour of an earlier constraint sharing a movable vertex with
 * it (0 if none), kept per vertex as the largest colour there so far. */
static int32_t colour_levels(cons* cs, int64_t n, const uint8_t* movable, int64_t nverts) {
  int32_t* top = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nverts + 1));
  for (int64_t v = 0; v < nverts; v++) top[v] = -1;
  int32_t ncol = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t col = 0;
    for (int k = 0; k < cs[i].nv; k++)
      if (movable[cs[i].v[k]] && top[cs[i].v[k]] + 1 > col) col = top[cs[i].v[k]] + 1;
    cs[i].colour = col;
    if (col + 1 > ncol) ncol = col + 1;
    for (int k = 0; k < cs[i].nv; k++)
      if (movable[cs[i].v[k]]) top[cs[i].v[k]] = col;
  }
  free(top);
  return ncol;
}

/* Greedy colouring of cs[0..n), which the caller has sorted by descending
 * priority: each constraint takes the smallest colour that no earlier one
 * sharing a movable vertex with it has.  Returns the number of colours;
 * *verts receives the number of distinct movable vertices of the set. */
static int32_t colour_greedy(cons* cs, int64_t n, const uint8_t* movable, int64_t nverts, int64_t* verts) {
  ilist* used = (ilist*)calloc((size_t)nverts + 1, sizeof(ilist));
  int32_t ncol = 0;
  int64_t nv_used = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t mv[4], nm = 0, tot = 0;
    for (int k = 0; k < cs[i].nv; k++)
      if (movable[cs[i].v[k]]) mv[nm++] = cs[i].v[k];
    for (int k = 0; k < nm; k++) tot += used[mv[k]].n;
    /* colours of the earlier constraints at these vertices (at most tot of
     * them, so the smallest free colour is at most tot) */
    uint8_t* taken = (uint8_t*)calloc((size_t)tot + 1, 1);
    for (int k = 0; k < nm; k++)
      for (int32_t j = 0; j < used[mv[k]].n; j++)
        if (used[mv[k]].c[j] <= tot) taken[used[mv[k]].c[j]] = 1;
    int32_t col = 0;
    while (taken[col]) col++;
    free(taken);
    cs[i].colour = col;
    if (col + 1 > ncol) ncol = col + 1;
    for (int k = 0; k < nm; k++) {
      if (used[mv[k]].n == 0) nv_used++;
      il_push(&used[mv[k]], col);
    }
  }
  for (int64_t v = 0; v < nverts; v++) free(used[v].c);
  free(used);
  if (verts) *verts = nv_used;
  return ncol;
}

/* Largest number of constraints at one movable vertex (statistics). */
static int32_t max_vertex_degree(const cons* cs, int64_t n, const uint8_t* movable, int64_t nverts) {
  int32_t* deg = (int32_t*)calloc((size_t)nverts + 1, sizeof(int32_t));
  int32_t m = 0;
  for (int64_t i = 0; i < n; i++)
    for (int k = 0; k < cs[i].nv; k++) {
      int32_t v = cs[i].v[k];
      if (movable[v] && ++deg[v] > m) m = deg[v];
    }
  free(deg);
  return m;
}

/* One projected Gauss-Seidel update of a contact constraint linearised at
 * x^(l) (Eq. LCP): w = c(x) + sum_v g_v.(y_v - x_v); the multiplier of this
 * backward step is projected onto lambda >= 0 and the change is applied
 * through M^-1 J^T (first KKT condition). */
static void pgs_contact(cons* c, const double* x, double* y, const double* im) {
  if (!(c->den > 0.0)) return;
  double w = c->c0;
  for (int k = 0; k < c->nv; k++) w = w + dot3(c->g[k], sub3(ld3(y, c->v[k]), ld3(x, c->v[k])));
  double tl = c->lambda - w / c->den;
  double ln = tl > 0.0 ? tl : 0.0;
  double dl = ln - c->lambda;
  c->lambda = ln;
  if (dl == 0.0) return;
  for (int k = 0; k < c->nv; k++) {
    double sc = im[c->v[k]] * dl;
    st3(y, c->v[k], add3(ld3(y, c->v[k]), scl3(sc, c->g[k])));
  }
}
/* Edge-length constraint of Sec. 4.2 linearised at y^[k+1] (R9):
 * c = sigma - g.(y_i - y_j), g = u / L0. */
static void pgs_edge(cons* c, double sigma, double* y, const double* im) {
  if (!(c->den > 0.0)) return;
  double w = sigma - dot3(c->g[0], sub3(ld3(y, c->v[0]), ld3(y, c->v[1])));
  double tl = c->lambda - w / c->den;
  double ln = tl > 0.0 ? tl : 0.0;
  double dl = ln - c->lambda;
  c->lambda = ln;
  if (dl == 0.0) return;
  double si = im[c->v[0]] * dl, sj = im[c->v[1]] * dl;
  st3(y, c->v[0], sub3(ld3(y, c->v[0]), scl3(si, c->g[0])));
  st3(y, c->v[1], add3(ld3(y, c->v[1]), scl3(sj, c->g[0])));
}

static int cmp_cons_key(const void* a, const void* b) {
  uint64_t ka = ((const cons*)a)->key, kb = ((const cons*)b)->key;
  return ka < kb ? -1 : ka > kb;
}

/* Projected Jacobi (Sec. 4.3.2, R12).  The paper notes that this variant
 * needs under-relaxation to converge; summing the corrections of every
 * constraint at a vertex overshoots by up to the number of constraints
 * there.  The relaxation is therefore per constraint: omega_c = omega /
 * n_max(c), where n_max(c) is the largest number of constraints (with a
 * positive denominator) at any movable vertex of c, so that every vertex
 * moves by at most omega times a convex combination of single-constraint
 * corrections.  Every multiplier change comes from the same y with the
 * update of Eq. LCP, dl = max(0, lambda - w / den) - lambda; the applied
 * change is s_c = omega_c * dl and lambda advances by s_c, so that y stays
 * its start plus the sum of m^-1 g lambda.  Each vertex sums m^-1 s_c g over
 * its constraints in canonical order (contacts by ascending pair key, then
 * edge-length constraints by ascending edge index) and adds the sum to y.
 * The caller passes cc and ce sorted by key and the per-vertex counts. */
static double jacobi_relax(const cons* c, double omega, const int32_t* nvc, const double* im) {
  int32_t m = 0;
  for (int k = 0; k < c->nv; k++)
    if (im[c->v[k]] > 0.0 && nvc[c->v[k]] > m) m = nvc[c->v[k]];
  return omega / (double)(m > 0 ? m : 1);
}

static void jacobi_sweep(cons* cc, int64_t nc, cons* ce, int64_t ne, double sigma, double omega,
                         const int32_t* nvc, const double* x, double* y, const double* im, int64_t n) {
  double* acc = (double*)calloc(3 * (size_t)n + 3, sizeof(double));
  double* sc = (double*)malloc(sizeof(double) * ((size_t)(nc + ne) + 1));
  for (int64_t i = 0; i < nc; i++) {
    cons* c = &cc[i];
    sc[i] = 0.0;
    if (!(c->den > 0.0)) continue;
    double w = c->c0;
    for (int k = 0; k < c->nv; k++) w = w + dot3(c->g[k], sub3(ld3(y, c->v[k]), ld3(x, c->v[k])));
    double tl = c->lambda - w / c->den;
    double dl = (tl > 0.0 ? tl : 0.0) - c->lambda;
    sc[i] = jacobi_relax(c, omega, nvc, im) * dl;
  }
  for (int64_t i = 0; i < ne; i++) {
    cons* c = &ce[i];
    sc[nc + i] = 0.0;
    if (!(c->den > 0.0)) continue;
    double w = sigma - dot3(c->g[0], sub3(ld3(y, c->v[0]), ld3(y, c->v[1])));
    double tl = c->lambda - w / c->den;
    double dl = (tl > 0.0 ? tl : 0.0) - c->lambda;
    sc[nc + i] = jacobi_relax(c, omega, nvc, im) * dl;
  }
  for (int64_t i = 0; i < nc; i++) {
    if (sc[i] == 0.0) continue;
    cc[i].lambda = cc[i].lambda + sc[i];
    for (int k = 0; k < cc[i].nv; k++) {
      int32_t v = cc[i].v[k];
      st3(acc, v, add3(ld3(acc, v), scl3(im[v] * sc[i], cc[i].g[k])));
    }
  }
  for (int64_t i = 0; i < ne; i++) {
    if (sc[nc + i] == 0.0) continue;
    ce[i].lambda = ce[i].lambda + sc[nc + i];
    int32_t a = ce[i].v[0], b = ce[i].v[1];
    st3(acc, a, sub3(ld3(acc, a), scl3(im[a] * sc[nc + i], ce[i].g[0])));
    st3(acc, b, add3(ld3(acc, b), scl3(im[b] * sc[nc + i], ce[i].g[0])));
  }
  for (int64_t v = 0; v < n; v++) st3(y, v, add3(ld3(y, v), ld3(acc, v)));
  free(acc); free(sc);
}

/* Edge-length constraints for the step (R9): every listed edge, u and L0
 * from the target y^[k+1]; an edge with L0 = 0 gets a zero denominator and
 * is skipped by the sweep.  Sweep order: ascending colour of the greedy
 * colouring of the edges (R11). */
static int64_t build_edges(const orc_topology* t, const orc_params* prm, const double* ytgt, const uint8_t* movable,
                           cons** out, int32_t* ncol, int32_t* ncolours) {
  cons* ce = (cons*)calloc((size_t)t->n_len + 1, sizeof(cons));
  int64_t ne = t->n_len;
  for (int64_t e = 0; e < ne; e++) {
    int32_t i = t->len_edges[2 * e], j = t->len_edges[2 * e + 1];
    cons* c = &ce[e];
    c->v[0] = i; c->v[1] = j; c->v[2] = c->v[3] = -1; c->nv = 2;
    v3 d0 = sub3(ld3(ytgt, i), ld3(ytgt, j));
    double L0 = norm3(d0);
    if (L0 > 0.0) {
      c->g[0] = div3(div3(d0, L0), L0);
      c->den = (t->inv_mass[i] + t->inv_mass[j]) * dot3(c->g[0], c->g[0]);
    } else {
      v3 z = {0.0, 0.0, 0.0};
      c->g[0] = z;
      c->den = 0.0;
    }
    c->key = (3ULL << 62) | (uint64_t)e;
    c->prio = orc_splitmix64(prm->seed ^ c->key);
  }
  *ncol = max_vertex_degree(ce, ne, movable, t->n_verts);
  qsort(ce, (size_t)ne, sizeof(cons), cmp_cons_prio_desc);
  *ncolours = prm->colouring == 1 ? colour_levels(ce, ne, movable, t->n_verts)
                                  : colour_greedy(ce, ne, movable, t->n_verts, 0);
  qsort(ce, (size_t)ne, sizeof(cons), cmp_cons_colour);
  *out = ce;
  return ne;
}

/* Contact constraints from the active pairs of P (dist < delta) at x^(l). */
static int64_t build_contacts(const orc_topology* t, const orc_params* prm, const pairset* P, const double* x,
                              const uint8_t* movable, cons** out, int32_t* ncol, int64_t* degenerate,
                              int32_t* ncolours, int64_t* nverts_used) {
  cons* cc = (cons*)calloc((size_t)P->n + 1, sizeof(cons));
  int64_t nc = 0;
  for (int64_t i = 0; i < P->n; i++) {
    if (!(P->d[i] < prm->delta)) continue;
    uint64_t key = P->k[i];
    int kind = key_kind(key);
    cons* c = &cc[nc];
    memset(c, 0, sizeof(cons));
    c->nv = pair_verts(t, key, c->v);
    v3 p[4];
    for (int k = 0; k < c->nv; k++) p[k] = ld3(x, c->v[k]);
    int ok;
    if (kind == ORC_VT) ok = vt_constraint(p, P->d[i], prm->delta, prm->constraint_form, &c->c0, c->g);
    else if (kind == ORC_EE) {
      double s, tt, d = ss_dist(p[0], p[1], p[2], p[3], &s, &tt);
      (void)d;
      ok = ee_constraint(p, P->d[i], s, tt, prm->delta, prm->constraint_form, &c->c0, c->g);
    } else ok = vv_constraint(p, rho_of(t, c->v[0]), rho_of(t, c->v[1]), prm->delta, &c->c0, c->g);
    if (!ok) { (*degenerate)++; continue; }
    c->den = 0.0;
    for (int k = 0; k < c->nv; k++) c->den = c->den + t->inv_mass[c->v[k]] * dot3(c->g[k], c->g[k]);
    c->key = key;
    c->prio = orc_splitmix64(prm->seed ^ key);
    nc++;
  }
  *ncol = max_vertex_degree(cc, nc, movable, t->n_verts);
  qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_prio_desc);
  *ncolours = colour_greedy(cc, nc, movable, t->n_verts, nverts_used);
  if (prm->colouring == 1) *ncolours = colour_levels(cc, nc, movable, t->n_verts);
  qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_colour);
  *out = cc;
  return nc;
}

/* Backward step (Sec. 4): y^(l+1) from y^(l) by gs_sweeps projected
 * Gauss-Seidel sweeps, contacts then edges (R10), each in ascending colour
 * (R11; cc and ce arrive in that order), each backward step starting its
 * multipliers at zero. */
static void backward(const orc_topology* t, const orc_params* prm, cons* cc, int64_t nc, cons* ce, int64_t ne,
                     const double* x, double* y) {
  for (int64_t i = 0; i < nc; i++) cc[i].lambda = 0.0;
  for (int64_t i = 0; i < ne; i++) ce[i].lambda = 0.0;
  if (prm->solver == 1) {
    qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_key);
    qsort(ce, (size_t)ne, sizeof(cons), cmp_cons_key);
    /* constraints with a positive denominator at each movable vertex */
    int32_t* nvc = (int32_t*)calloc((size_t)t->n_verts + 1, sizeof(int32_t));
    for (int64_t i = 0; i < nc; i++)
      if (cc[i].den > 0.0)
        for (int k = 0; k < cc[i].nv; k++)
          if (t->inv_mass[cc[i].v[k]] > 0.0) nvc[cc[i].v[k]]++;
    for (int64_t i = 0; i < ne; i++)
      if (ce[i].den > 0.0)
        for (int k = 0; k < 2; k++)
          if (t->inv_mass[ce[i].v[k]] > 0.0) nvc[ce[i].v[k]]++;
    for (int s = 0; s < prm->gs_sweeps; s++)
      jacobi_sweep(cc, nc, ce, ne, prm->sigma, prm->jacobi_omega, nvc, x, y, t->inv_mass, t->n_verts);
    free(nvc);
    return;
  }
  for (int s = 0; s < prm->gs_sweeps; s++) {
    for (int64_t i = 0; i < nc; i++) pgs_contact(&cc[i], x, y, t->inv_mass);
    for (int64_t i = 0; i < ne; i++) pgs_edge(&ce[i], prm->sigma, y, t->inv_mass);
  }
}

int32_t orc_colouring(int32_t kind, int64_t n, const int32_t* verts, const uint64_t* prio, const double* inv_mass,
                      int64_t n_verts, int32_t* colour) {
  cons* cs = (cons*)calloc((size_t)n + 1, sizeof(cons));
  uint8_t* movable = (uint8_t*)malloc((size_t)n_verts + 1);
  for (int64_t v = 0; v < n_verts; v++) movable[v] = inv_mass[v] > 0.0;
  for (int64_t i = 0; i < n; i++) {
    int nv = 0;
    for (int k = 0; k < 4; k++)
      if (verts[4 * i + k] >= 0) cs[i].v[nv++] = verts[4 * i + k];
    cs[i].nv = nv;
    cs[i].prio = prio[i];
    cs[i].key = (uint64_t)i; /* remembers the input position */
  }
  qsort(cs, (size_t)n, sizeof(cons), cmp_cons_prio_desc);
  int32_t ncol = kind == 1 ? colour_levels(cs, n, movable, n_verts) : colour_greedy(cs, n, movable, n_verts, 0);
  for (int64_t i = 0; i < n; i++) colour[cs[i].key] = cs[i].colour;
  free(cs); free(movable);
  return ncol;
}

int64_t orc_contact_colours(const orc_topology* t, const orc_params* prm, const double* x, const double* x_tilde,
                            uint64_t* keys, int32_t* colour, int64_t cap) {
  scene s; scene_init(&s, t, x, x_tilde);
  uint8_t* movable = (uint8_t*)malloc((size_t)t->n_verts + 1);
  for (int64_t v = 0; v < t->n_verts; v++) movable[v] = t->inv_mass[v] > 0.0;
  pairset P = {0, 0, 0, 0};
  proximity_search(&s, x, prm->d_max, prm->search_mode, &P);
  cons* cc;
  int32_t ncc, colc;
  int64_t degen = 0, nvu = 0;
  int64_t nc = build_contacts(t, prm, &P, x, movable, &cc, &ncc, &degen, &colc, &nvu);
  qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_key);
  for (int64_t i = 0; i < nc && i < cap; i++) {
    keys[i] = cc[i].key;
    colour[i] = cc[i].colour;
  }
  free(cc); free(P.k); free(P.d); free(movable); scene_free(&s);
  return nc;
}

int32_t orc_edge_colours(const orc_topology* t, const orc_params* prm, int32_t* colour) {
  uint8_t* movable = (uint8_t*)malloc((size_t)t->n_verts + 1);
  for (int64_t v = 0; v < t->n_verts; v++) movable[v] = t->inv_mass[v] > 0.0;
  double* z = (double*)calloc(3 * (size_t)t->n_verts + 3, sizeof(double));
  cons* ce;
  int32_t nce, cole;
  int64_t ne = build_edges(t, prm, z, movable, &ce, &nce, &cole);
  for (int64_t i = 0; i < ne; i++) colour[ce[i].key & 0x3fffffffffffffffULL] = ce[i].colour;
  free(ce); free(z); free(movable);
  return cole;
}

int orc_backward_once(const orc_topology* t, const orc_params* prm, const double* x, const double* y_in,
                      const double* y_target, double* y_out) {
  scene s; scene_init(&s, t, x, y_target);
  uint8_t* movable = (uint8_t*)malloc((size_t)t->n_verts + 1);
  for (int64_t v = 0; v < t->n_verts; v++) movable[v] = t->inv_mass[v] > 0.0;
  pairset P = {0, 0, 0, 0};
  proximity_search(&s, x, prm->d_max, prm->search_mode, &P);
  cons *cc, *ce;
  int32_t ncc, nce, colc, cole;
  int64_t degen = 0, nvu = 0;
  int64_t nc = build_contacts(t, prm, &P, x, movable, &cc, &ncc, &degen, &colc, &nvu);
  int64_t ne = build_edges(t, prm, y_target, movable, &ce, &nce, &cole);
  memcpy(y_out, y_in, sizeof(double) * 3 * (size_t)t->n_verts);
  backward(t, prm, cc, nc, ce, ne, x, y_out);
  free(cc); free(ce); free(P.k); free(P.d); free(movable); scene_free(&s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* CCD of a linearly moving pair (Sec. 5.1's comparison scheme: the step    */
/* rule of its CCD-based variant, or a safety check of each segment).       */
/* ------------------------------------------------------------------------ */
static double cubic_at(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }

/* Roots of the coplanarity cubic in [0,1], ascending.  The interval is cut
 * at the roots of the derivative; a sign change on a monotone piece is
 * bisected 80 times. */
static int cubic_roots01(const double c[4], double* roots) {
  double cuts[4];
  int nc = 0;
  cuts[nc++] = 0.0;
  double A = 3.0 * c[3], B = 2.0 * c[2], C = c[1];
  double crit[2];
  int ncr = 0;
  if (A != 0.0) {
    double disc = B * B - 4.0 * A * C;
    if (disc >= 0.0) {
      double sq = sqrt(disc);
      double r1 = (-B - sq) / (2.0 * A), r2 = (-B + sq) / (2.0 * A);
      if (r1 > r2) { double tmp = r1; r1 = r2; r2 = tmp; }
      crit[ncr++] = r1; crit[ncr++] = r2;
    }
  } else if (B != 0.0) crit[ncr++] = -C / B;
  for (int i = 0; i < ncr; i++)
    if (crit[i] > 0.0 && crit[i] < 1.0 && crit[i] > cuts[nc - 1]) cuts[nc++] = crit[i];
  cuts[nc++] = 1.0;
  int nr = 0;
  for (int i = 0; i + 1 < nc; i++) {
    double a = cuts[i], b = cuts[i + 1], fa = cubic_at(c, a), fb = cubic_at(c, b);
    if (fa == 0.0) { if (nr == 0 || roots[nr - 1] != a) roots[nr++] = a; continue; }
    if (fb == 0.0) { roots[nr++] = b; continue; }
    if ((fa < 0.0) == (fb < 0.0)) continue;
    for (int it = 0; it < 80; it++) {
      double m = 0.5 * (a + b), fm = cubic_at(c, m);
      if (fm == 0.0) { a = b = m; break; }
      if ((fm < 0.0) == (fa < 0.0)) { a = m; fa = fm; } else b = m;
    }
    roots[nr++] = 0.5 * (a + b);
  }
  return nr;
}

#define CCD_TOUCH 1e-9
/* Smallest pair distance the forward step trusts (metres). */
#define ORC_D_FLOOR 1e-10
/* Vertices 0..3 move linearly from x0 to x1.  VT (a; i,j,k) and EE (a,b;
 * c,d): the first time in [0,1] at which the four points are coplanar and the
 * primitives touch (distance <= CCD_TOUCH); a vertex with a radius (rho[0]
 * > 0) against a triangle is not handled (returns 0).  VV (a, b) with radii:
 * the first time the centre distance reaches rho_a + rho_b. */
int orc_ccd(int kind, const double* x0, const double* x1, const double* rho, double* toi) {
  int nv = kind == ORC_VV ? 2 : 4;
  v3 p0[4], d[4];
  for (int i = 0; i < nv; i++) { p0[i] = ld3(x0, i); d[i] = sub3(ld3(x1, i), p0[i]); }
  double R = 0.0;
  if (kind == ORC_VV) R = (rho ? rho[0] : 0.0) + (rho ? rho[1] : 0.0);
  if (kind == ORC_VT && rho && rho[0] > 0.0) return 0;
  /* swept boxes of the two primitives: they can only touch if these overlap */
  {
    int na = kind == ORC_EE ? 2 : 1;
    box A, B;
    for (int k = 0; k < 3; k++) { A.lo[k] = INFINITY; A.hi[k] = -INFINITY; B.lo[k] = INFINITY; B.hi[k] = -INFINITY; }
    for (int i = 0; i < nv; i++) {
      double q[6] = {x0[3 * i], x0[3 * i + 1], x0[3 * i + 2], x1[3 * i], x1[3 * i + 1], x1[3 * i + 2]};
      box* bx = i < na ? &A : &B;
      for (int h = 0; h < 2; h++)
        for (int k = 0; k < 3; k++) {
          if (q[3 * h + k] < bx->lo[k]) bx->lo[k] = q[3 * h + k];
          if (q[3 * h + k] > bx->hi[k]) bx->hi[k] = q[3 * h + k];
        }
    }
    if (!box_near(&A, &B, CCD_TOUCH + R)) return 0;
  }
  if (kind == ORC_VV) {
    /* |r + t v|^2 = R^2: the smaller root in [0,1], if the spheres reach contact */
    v3 r = sub3(p0[0], p0[1]), v = sub3(d[0], d[1]);
    double rr = dot3(r, r), RR = (R + CCD_TOUCH) * (R + CCD_TOUCH);
    if (rr <= RR) { *toi = 0.0; return 1; }
    double vv = dot3(v, v), rv = dot3(r, v);
    if (!(vv > 0.0) || rv >= 0.0) return 0;
    double disc = rv * rv - vv * (rr - RR);
    if (disc < 0.0) return 0;
    double t = (-rv - sqrt(disc)) / vv;
    if (t >= 0.0 && t <= 1.0) { *toi = t; return 1; }
    return 0;
  }
  /* coplanarity cubic f(t) = det[a1+t b1, a2+t b2, a3+t b3] */
  v3 a[3], b[3];
  for (int k = 0; k < 3; k++) { a[k] = sub3(p0[k + 1], p0[0]); b[k] = sub3(d[k + 1], d[0]); }
  double c[4];
  c[0] = det3(a[0], a[1], a[2]);
  c[1] = (det3(b[0], a[1], a[2]) + det3(a[0], b[1], a[2])) + det3(a[0], a[1], b[2]);
  c[2] = (det3(a[0], b[1], b[2]) + det3(b[0], a[1], b[2])) + det3(b[0], b[1], a[2]);
  c[3] = det3(b[0], b[1], b[2]);
  double roots[16];
  int nr;
  if (c[0] == 0.0 && c[1] == 0.0 && c[2] == 0.0 && c[3] == 0.0) {
    /* coplanar for all t: probe nine instants */
    nr = 0;
    for (int i = 0; i <= 8; i++) roots[nr++] = i / 8.0;
  } else nr = cubic_roots01(c, roots);
  for (int r = 0; r < nr; r++) {
    double t = roots[r];
    v3 q[4];
    for (int i = 0; i < 4; i++) q[i] = add3(p0[i], scl3(t, d[i]));
    double dist = kind == ORC_VT ? pt_dist(q[0], q[1], q[2], q[3]) : ss_dist(q[0], q[1], q[2], q[3], 0, 0);
    if (dist <= CCD_TOUCH) { *toi = t; return 1; }
  }
  return 0;
}

/* Conservative CCD, an independent check of orc_ccd: 0 when the two
 * primitives certainly stay more than tol apart during the whole linear
 * motion, 1 otherwise (they may come within tol).  Over a time interval of
 * half-width h around tm, every point of one primitive moves relative to
 * every point of the other by at most V h, where V is the largest relative
 * displacement of a vertex of one against a vertex of the other (points of a
 * primitive are convex combinations of its vertices), so the distance there
 * is at least d(tm) - V h.  The interval is certified when that bound, less
 * the rounding error of d(tm) (64 units in the last place of the largest
 * coordinate), exceeds tol; otherwise it is split in two, down to 2^-44 of
 * the step and at most 2^20 evaluations in all (past either bound the
 * answer is 1). */
static double pair_dist_at(int kind, const v3* p0, const v3* d, const double* rho, double t) {
  v3 q[4];
  int nv = kind == ORC_VV ? 2 : 4;
  for (int i = 0; i < nv; i++) q[i] = add3(p0[i], scl3(t, d[i]));
  if (kind == ORC_VT) return pt_dist(q[0], q[1], q[2], q[3]) - (rho ? rho[0] : 0.0);
  if (kind == ORC_EE) return ss_dist(q[0], q[1], q[2], q[3], 0, 0);
  return (norm3(sub3(q[0], q[1])) - (rho ? rho[0] : 0.0)) - (rho ? rho[1] : 0.0);
}
static int certify(int kind, const v3* p0, const v3* d, const double* rho, double V, double err, double tol,
                   double t0, double t1, int depth, long* budget) {
  if (--*budget < 0) return 0;
  double tm = 0.5 * (t0 + t1), h = 0.5 * (t1 - t0);
  double lower = pair_dist_at(kind, p0, d, rho, tm) - V * h - err;
  if (lower > tol) return 1;
  if (depth >= 44) return 0;
  return certify(kind, p0, d, rho, V, err, tol, t0, tm, depth + 1, budget) &&
         certify(kind, p0, d, rho, V, err, tol, tm, t1, depth + 1, budget);
}
int orc_ccd_conservative(int kind, const double* x0, const double* x1, const double* rho, double tol) {
  int nv = kind == ORC_VV ? 2 : 4, na = kind == ORC_EE ? 2 : 1;
  v3 p0[4], d[4];
  double M = 0.0;
  for (int i = 0; i < nv; i++) {
    p0[i] = ld3(x0, i);
    d[i] = sub3(ld3(x1, i), p0[i]);
    for (int k = 0; k < 3; k++) {
      if (fabs(x0[3 * i + k]) > M) M = fabs(x0[3 * i + k]);
      if (fabs(x1[3 * i + k]) > M) M = fabs(x1[3 * i + k]);
    }
  }
  double V = 0.0;
  for (int i = 0; i < na; i++)
    for (int j = na; j < nv; j++) {
      double r = norm3(sub3(d[i], d[j]));
      if (r > V) V = r;
    }
  V = V * (1.0 + 1e-12);
  double err = 64.0 * 2.220446049250313e-16 * (M + (rho ? rho[0] + (nv == 2 ? rho[1] : 0.0) : 0.0)) + 1e-300;
  long budget = 1L << 20; /* interval evaluations; past it the answer is "may touch" */
  return certify(kind, p0, d, rho, V, err, tol, 0.0, 1.0, 0, &budget) ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Exact acceptance                                                          */
/* ------------------------------------------------------------------------ */
int64_t orc_count_intersections(const orc_topology* t, const double* x) {
  int64_t hits = 0;
  int64_t T = t->n_tris, E = t->n_edges;
  box* tb = (box*)malloc(sizeof(box) * ((size_t)T + 1));
  box* eb = (box*)malloc(sizeof(box) * ((size_t)E + 1));
  for (int64_t i = 0; i < T; i++) tb[i] = box_of(x, t->tris + 3 * i, 3);
  for (int64_t i = 0; i < E; i++) eb[i] = box_of(x, t->edges + 2 * i, 2);
  /* edge vs non-adjacent triangle: covers triangle-triangle intersection */
  for (int64_t e = 0; e < E; e++) {
    const int32_t* ev = t->edges + 2 * e;
    for (int64_t tr = 0; tr < T; tr++) {
      const int32_t* tv = t->tris + 3 * tr;
      if (ev[0] == tv[0] || ev[0] == tv[1] || ev[0] == tv[2] || ev[1] == tv[0] || ev[1] == tv[1] || ev[1] == tv[2])
        continue;
      if (!box_near(&eb[e], &tb[tr], 0.0)) continue;
      hits += seg_tri_exact(ld3(x, ev[0]), ld3(x, ev[1]), ld3(x, tv[0]), ld3(x, tv[1]), ld3(x, tv[2]));
    }
  }
  /* edge vs non-adjacent edge (strands) */
  for (int64_t e1 = 0; e1 < E; e1++)
    for (int64_t e2 = e1 + 1; e2 < E; e2++) {
      const int32_t *p = t->edges + 2 * e1, *q = t->edges + 2 * e2;
      if (p[0] == q[0] || p[0] == q[1] || p[1] == q[0] || p[1] == q[1]) continue;
      if (!box_near(&eb[e1], &eb[e2], 0.0)) continue;
      hits += seg_seg_exact(ld3(x, p[0]), ld3(x, p[1]), ld3(x, q[0]), ld3(x, q[1]));
    }
  /* points: a zero-radius point on a triangle is decided exactly; with a
   * radius, the FP64 gap must exceed 1e-12 */
  for (int64_t pi = 0; pi < t->n_points; pi++) {
    int32_t a = t->points[pi];
    double ra = rho_of(t, a);
    for (int64_t tr = 0; tr < T; tr++) {
      const int32_t* tv = t->tris + 3 * tr;
      if (a == tv[0] || a == tv[1] || a == tv[2]) continue;
      if (ra == 0.0) hits += pt_on_tri_exact(ld3(x, a), ld3(x, tv[0]), ld3(x, tv[1]), ld3(x, tv[2]));
      else hits += (pt_dist(ld3(x, a), ld3(x, tv[0]), ld3(x, tv[1]), ld3(x, tv[2])) - ra) <= 1e-12;
    }
    for (int64_t pj = pi + 1; pj < t->n_points; pj++) {
      int32_t b = t->points[pj];
      double g = (norm3(sub3(ld3(x, a), ld3(x, b))) - ra) - rho_of(t, b);
      hits += g <= 1e-12;
    }
  }
  free(tb); free(eb);
  return hits;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */
int orc_handle_step(const orc_topology* t, const orc_params* prm, const double* x_t, const double* x_tilde,
                    double* x_next, orc_stats* st, orc_trace* tr) {
  int64_t n = t->n_verts;
  scene s; scene_init(&s, t, x_t, x_tilde);
  orc_stats S;
  memset(&S, 0, sizeof(S));
  S.min_pair_dist = INFINITY;
  uint8_t* movable = (uint8_t*)malloc((size_t)n + 1);
  for (int64_t v = 0; v < n; v++) movable[v] = t->inv_mass[v] > 0.0;

  double* x = (double*)malloc(sizeof(double) * 3 * ((size_t)n + 1));
  double* y = (double*)malloc(sizeof(double) * 3 * ((size_t)n + 1));
  double* xn = (double*)malloc(sizeof(double) * 3 * ((size_t)n + 1));
  double* r = (double*)malloc(sizeof(double) * ((size_t)n + 1));
  double* Di = (double*)malloc(sizeof(double) * ((size_t)n + 1));
  double* alpha = (double*)malloc(sizeof(double) * ((size_t)n + 1));
  double* clampf = (double*)malloc(sizeof(double) * ((size_t)n + 1));
  /* x^(0) = x^[k], y^(0) = y^[k+1], D^(0) = 0, r^(0) = 1, P = {} */
  memcpy(x, x_t, sizeof(double) * 3 * (size_t)n);
  memcpy(y, x_tilde, sizeof(double) * 3 * (size_t)n);
  for (int64_t v = 0; v < n; v++) r[v] = 1.0;
  double D = 0.0;
  pairset P = {0, 0, 0, 0};
  cons* ce;
  int32_t nce;
  int64_t ne = build_edges(t, prm, x_tilde, movable, &ce, &nce, &S.edge_colours);
  S.max_vertex_edges = nce;
  const double hg = 0.5 * prm->gamma;
  if (tr && tr->x) memcpy(tr->x, x, sizeof(double) * 3 * (size_t)n);

  int32_t l;
  for (l = 0; l <= prm->max_iters; l++) {
    int searched = 0;
    if (D < prm->d_min) {
      S.candidates += proximity_search(&s, x, prm->d_max, prm->search_mode, &P);
      D = prm->d_max;
      S.searches++;
      searched = 1;
    } else {
      /* reuse P: refresh distances, drop pairs no longer below D^(l) */
      int64_t m = 0;
      for (int64_t i = 0; i < P.n; i++) {
        double d = pair_dist(t, P.k[i], x, 0, 0);
        if (d < D) { P.k[m] = P.k[i]; P.d[m] = d; m++; }
      }
      P.n = m;
    }
    S.pairs_evaluated += P.n;
    if (P.n > S.max_pairs) S.max_pairs = P.n;
    /* D_i (Sec. 5): shortest distance of the pairs involving i, at most
     * D^(l) (R1), and never below zero */
    for (int64_t v = 0; v < n; v++) Di[v] = D;
    for (int64_t i = 0; i < P.n; i++) {
      int32_t v4[4];
      int nv = pair_verts(t, P.k[i], v4);
      for (int k = 0; k < nv; k++)
        if (P.d[i] < Di[v4[k]]) Di[v4[k]] = P.d[i];
      if (P.d[i] < S.min_pair_dist) S.min_pair_dist = P.d[i];
    }
    /* every pair of P is closer than D^(l), so its vertices have D_i < D^(l) */
    for (int64_t v = 0; v < n; v++) S.pair_vertices += Di[v] < D;
    /* R2b: below ORC_D_FLOOR the bound D_i/2 is no larger than the rounding
     * of an FP64 position update, so such a vertex does not move */
    for (int64_t v = 0; v < n; v++)
      if (!(Di[v] >= ORC_D_FLOOR)) Di[v] = 0.0;

    /* backward step */
    cons* cc;
    int32_t ncc, colc;
    int64_t nvu = 0;
    int64_t nc = build_contacts(t, prm, &P, x, movable, &cc, &ncc, &S.degenerate, &colc, &nvu);
    S.active_contacts += nc;
    S.contact_vertices += nvu;
    if (ncc > S.max_vertex_contacts) S.max_vertex_contacts = ncc;
    if (colc > S.contact_colours) S.contact_colours = colc;
    backward(t, prm, cc, nc, ce, ne, x, y);
    free(cc);

    /* forward step, Eq. forward2 (R2).  The CCD-based rule (Sec. 5.1's
     * comparison scheme) caps every vertex by the global bound D^(l) instead
     * of its own D_i and lets the CCD below decide the step: a pair outside P
     * is at least D^(l) apart and its two sides close at most 0.9 D^(l).  A
     * vertex whose own D_i is below the floor (R2b) stays under either rule:
     * at that distance the CCD's roots are rounding noise */
    const int ccd_rule = prm->step_rule == 1;
    double Dcap = D;
    if (!(Dcap >= ORC_D_FLOOR)) Dcap = 0.0;
    S.frozen_vertices = 0;
    for (int64_t v = 0; v < n; v++) {
      v3 xv = ld3(x, v), yv = ld3(y, v);
      v3 dx = sub3(yv, xv);
      double nd = norm3(dx), a = 1.0;
      double bound = ccd_rule ? (Di[v] == 0.0 ? 0.0 : Dcap) : Di[v];
      if (nd > 0.0) {
        double q = (hg * bound) / nd;
        a = q < 1.0 ? q : 1.0;
        if (bound == 0.0) S.frozen_vertices++;
      } else if (nd != 0.0) {
        a = 0.0; /* R2c: y not finite, the vertex does not move */
      }
      alpha[v] = a;
      st3(xn, v, step_to(xv, yv, a));
    }
    /* CCD of each pair's segment x^(l) -> x^(l+1) (the safety check, or the
     * step rule): a hit at time t_hit scales the step of the pair's vertices by
     * t_hit / 2 (the smallest factor over their pairs) and the segments are tested
     * again, for at most ccd_rounds rounds; a hit after the last round keeps
     * every vertex of the scene where it is for this iteration */
    if (prm->ccd_check || ccd_rule) {
      for (int32_t round = 0;; round++) {
        for (int64_t v = 0; v < n; v++) clampf[v] = 1.0;
        int hit_any = 0;
        for (int64_t i = 0; i < P.n; i++) {
          int32_t v4[4];
          int nv = pair_verts(t, P.k[i], v4);
          double a0[12], a1[12], rr[2] = {rho_of(t, v4[0]), nv == 2 ? rho_of(t, v4[1]) : 0.0}, toi;
          for (int k = 0; k < nv; k++) { st3(a0, k, ld3(x, v4[k])); st3(a1, k, ld3(xn, v4[k])); }
          if (orc_ccd(key_kind(P.k[i]), a0, a1, rr, &toi)) {
            hit_any = 1;
            S.ccd_clamps++;
            for (int k = 0; k < nv; k++)
              if (0.5 * toi < clampf[v4[k]]) clampf[v4[k]] = 0.5 * toi;
          }
        }
        if (!hit_any) break;
        if (round >= prm->ccd_rounds) {
          for (int64_t v = 0; v < n; v++) { alpha[v] = 0.0; st3(xn, v, ld3(x, v)); }
          break;
        }
        for (int64_t v = 0; v < n; v++)
          if (clampf[v] < 1.0) {
            alpha[v] = clampf[v] * alpha[v];
            st3(xn, v, step_to(ld3(x, v), ld3(y, v), alpha[v]));
          }
      }
    }
    double mmax = 0.0, rmax = 0.0;
    for (int64_t v = 0; v < n; v++) {
      r[v] = r[v] * (1.0 - alpha[v]);
      double mv = norm3(sub3(ld3(xn, v), ld3(x, v)));
      if (mv > mmax) mmax = mv;
      if (r[v] > rmax) rmax = r[v];
    }
    if (tr && l < tr->cap_iters) {
      if (tr->y) memcpy(tr->y + 3 * (size_t)n * (size_t)l, y, sizeof(double) * 3 * (size_t)n);
      if (tr->Dl) tr->Dl[l] = D;
      if (tr->Di) memcpy(tr->Di + (size_t)n * (size_t)l, Di, sizeof(double) * (size_t)n);
      if (tr->searched) tr->searched[l] = searched;
      if (tr->n_pairs) tr->n_pairs[l] = P.n;
      if (tr->pair_keys)
        for (int64_t i = 0; i < P.n && i < tr->cap_pairs; i++) tr->pair_keys[(size_t)tr->cap_pairs * (size_t)l + (size_t)i] = P.k[i];
      if (tr->n_contacts) tr->n_contacts[l] = nc;
      if (tr->x) memcpy(tr->x + 3 * (size_t)n * (size_t)(l + 1), xn, sizeof(double) * 3 * (size_t)n);
    }
    { double* tmp = x; x = xn; xn = tmp; }
    /* D^(l+1) = D^(l) - 2 max_i |dx_i|, one ulp down (R15) */
    D = nextafter(D - 2.0 * mmax, -INFINITY);
    S.final_r_inf = rmax;
    if (rmax < prm->eps) { S.converged = 1; l++; break; }
  }
  S.iterations = l; /* iterations executed: l+1 of them when the loop runs out */
  memcpy(x_next, x, sizeof(double) * 3 * (size_t)n);
  if (st) *st = S;
  free(x); free(y); free(xn); free(r); free(Di); free(alpha); free(clampf); free(movable);
  free(P.k); free(P.d); free(ce);
  scene_free(&s);
  return 0;
}

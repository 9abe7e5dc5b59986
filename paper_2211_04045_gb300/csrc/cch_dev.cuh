// cch_dev.cuh -- device data layout and per-element arithmetic of the
// two-way collision-handling path (arXiv 2211.04045) for sm_103a.
//
// Every formula here is evaluated as written: the library is compiled with
// --fmad=false, so no multiply-add is contracted and each FP64 expression
// rounds exactly like its plain IEEE evaluation, left to right.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cch {

// ---------------------------------------------------------------------------
// layout
// ---------------------------------------------------------------------------
// Positions live as 32-byte aligned (x, y, z, w) records: one vertex gather
// touches one 32-byte sector.
struct __align__(32) P4 { double x, y, z, w; };

struct dv3 { double x, y, z; };

// vertex flag bits
enum : uint8_t { VF_STATIC = 1, VF_POINT = 2, VF_COLL = 4, VF_MOVABLE = 8 };
enum { K_VT = 0, K_EE = 1, K_VV = 2 };

// Per-scene constants (device copy).
struct SceneDesc {
  int v0, nv;      // vertex range in the pool
  int t0, nt;      // triangle range
  int e0, ne;      // collision-edge range
  int l0, nl;      // edge-length constraint range
  int q0, nq;      // point range
  int c0, nc;      // collision-vertex range (index into the vc list)
  double d_min, d_max, delta, sigma, hgamma, eps, omega;
  int form;                       // contact constraint: 0 volume, 1 gap
  double rho_max;  // largest point radius of the scene
  int max_iters, gs_sweeps, solver, ccd;
  int step_rule;                  // 0 distance bound (Eq. forward2), 1 CCD-based
  int n_ecol;                     // colours of the edge-length constraints
  uint64_t seed;
};

// Per-scene loop state, mutated on the device.
struct SceneState {
  double D;                       // D^(l)
  int iter;                       // l
  int active;                     // takes part in the current step
  int start;                      // server: (re)start this scene's step at the next launch
  int done;                       // loop of this step has ended
  int do_search;                  // iteration l runs a proximity search
  int converged;
  int searches;
  unsigned long long move_bits;   // max_i |x_i^(l+1) - x_i^(l)| (double bits)
  unsigned long long rmax_bits;   // ||r^(l+1)||_inf (double bits)
  unsigned long long mind_bits;   // min pair distance of the step
  long long pairs_eval, max_pairs, contacts, candidates, degenerate;
  int n_pairs;                    // |P| of this iteration
  int max_vcontacts;              // most contacts at one movable vertex in an iteration
  int ccd_clamps;
  double final_r;
  long long isect, uncertain;
  int bad_input;                  // x_t or x~ held a non-finite coordinate
  int ccd_live;                   // the CCD rounds of this iteration go on
  int ccd_hits[2];                // hits of the current CCD round (by parity)
  int frozen_cur;                 // vertices held by the D_i floor in this iteration
  int frozen;                     // the same count at the last finished iteration
  long long cverts;               // sum over iterations of distinct movable contact vertices
  long long pverts;               // sum over iterations of distinct vertices of P
  int ccol;                       // most contact colours of one iteration
  int pad_;
};

// Device-wide counters and flags.
struct Counters {
  int n_pairs[2];       // pairs in buffer 0 / 1
  int n_active[3];      // active contact candidates (dist < delta) per kind
  int n_cons;           // assembled contact constraints
  int vcontacts;        // most contacts at one movable vertex (this iteration)
  int overflow;         // OV_* bits
  int err;              // first error code
  int any_search;       // some active scene searches in this iteration
  int all_done;         // every active scene has finished
  unsigned long long n_cand;   // candidate pairs counted
  int n_query;          // pairs written by a query call
  int n_fcand[3];       // FP32-filter survivors per pair kind (VT, EE, VV)
  int any_refresh;      // some active scene reuses P in this iteration
  int ccd_hit;
  int n_ccol;           // colours of this iteration's contact colouring
  int n_exact[2];       // pairs whose exact FP64 distance is due: of the
                        // search's survivors [0], of the refreshed P [1]
};
enum { OV_PAIRS = 1, OV_CONTACTS = 2, OV_QUERY = 16 };
// error bits of Counters::err (ERR_COLOURS: a contact needed more colours
// than the colouring's masks hold)
enum { ERR_STACK = 2, ERR_BUDGET = 4, ERR_TREE = 8, ERR_POLL = 16, ERR_COLOURS = 32 };

// Proximity pair (SoA arrays in the pool).
struct PairBuf {
  unsigned long long* key;  // kind<<62 | local id1<<31 | local id2
  int4* v;                  // global vertex ids (VV: v.z = v.w = -1)
  double* d;                // distance at x^(l)
};

// One assembled contact constraint of Eq. LCP, linearised at x^(l).
struct __align__(16) Contact {
  int4 v;                 // vertices (VV: two, the rest -1)
  double g[12];           // dc/dx_v
  double c0;              // c(x^(l))
  double den;             // sum_v m_v^-1 |g_v|^2
  unsigned long long prio;// Gauss-Seidel priority (R11)
  unsigned long long key; // canonical identity
};

// The same constraint in FP32 (mixed precision).
struct __align__(16) ContactF {
  int4 v;
  float g[12];
  float c0, den;
  unsigned long long prio, key;
};

// BVH over one primitive class of the pool (triangles, edges or collision
// vertices).  Internal node i has children left[i], right[i]; a child index
// with the top bit set is a leaf (sorted position).  Child boxes are stored in
// the parent, rounded outward to float.
struct BVH {
  int n;                       // primitives
  unsigned long long* keys;    // sorted Morton keys (scene<<30 | morton)
  unsigned long long* keys_alt;
  int* ids;                    // sorted primitive ids
  int* ids_alt;
  int* left;                   // n-1
  int* right;
  int* parent;                 // internal parents (n-1) ; leaf parents at parent[n-1 + leaf]
  int* range_hi;               // last sorted leaf under the node (n-1)
  float4* box;                 // n-1 nodes x 3 float4: (Llo.xyz, Lhi.x) (Lhi.yz, Rlo.xy) (Rlo.z, Rhi.xyz)
  int* flag;                   // refit arrival counters (n-1)
  float4* leafbox;             // n x 2: lo, hi per sorted leaf
  int* sroot;                  // per scene: root node (leaf: top bit set), -1 if none
  unsigned int* hist;          // radix histograms
  unsigned int* hist2;
};

constexpr int LEAF = 0x40000000;

// Everything a kernel needs, passed by value.
struct Pool {
  int nv, nt, ne, nl, nq, nvc, nscene;
  int pair_cap, act_cap, cons_cap;
  P4 *x, *y, *yt, *xp;
  int mixed;               // 1: FP32 distances, contacts and projection (CCH_PREC_MIXED)
  float4* yf;              // mixed: y in float
  float4* lgf;             // mixed: edge-length constraint g (xyz), den (w) in float
  double* alpha;           // CCD mode: step size of the forward step
  unsigned long long* clampb;  // CCD mode: per-vertex clamp factor (double bits)
  float4* xf;              // x rounded to float (the FP32 distance pre-filter)
  double *im, *rho, *r;
  unsigned long long* Dv;
  int* vscene;
  uint8_t* vflag;
  int4* tv;                // i, j, k, scene
  int4* ev;                // a, b, scene, -
  int4* lv;                // i, j, scene, -
  P4* lg;                  // per edge-length constraint: g = u/L0 (xyz), den (w)
  int* edeg;               // per vertex: edge-length constraints at it
  int2* erank;             // per edge-length constraint: its rank at vertex i and
                           // at vertex j among that vertex's edges, by descending priority
  int* vlevel;             // per vertex: colour of its last applied contact
                           // (level colouring; -1 before the first)
  int* tinc_start;         // per vertex: start into tinc (nv + 1)
  int* tinc;               // incident triangle corners, ascending: triangle * 3 + corner
  int* vc;                 // collision vertices (pool ids), scene-contiguous
  int* pts;                // point vertices
  SceneDesc* sd;
  SceneState* ss;
  Counters* cnt;
  PairBuf pb[2];
  int* act;                // active contact lists, one region of act_cap per kind
                           // (VT, EE, VV): indices into the next pair buffer
  unsigned long long* fkey;  // FP32-filter survivors: 3 regions of pair_cap (VT, EE, VV)
  int4* fv;
  float* fd;               // mixed precision: the survivor's FP32 distance lower bound
  float2* fbs;             // FP64 mode: survivors' FP32 bounds (3 regions of pair_cap); +inf = dropped
  float2* fbr;             // FP64 mode: refreshed pairs' FP32 bounds (pair_cap)
  int* exq;                // FP64 mode: survivors due an exact distance (3 pair_cap)
  int* exr;                // FP64 mode: refreshed pairs due an exact distance (pair_cap)
  unsigned int* vmin;      // per vertex: smallest upper bound of a certain pair (fl_ord image)
  Contact* cons;
  unsigned char* fdone;    // contact colouring: coloured flags (cons_cap)
  int* ccol;               // per contact: colour class of the iteration (cons_cap)
  unsigned long long* cmask;  // per vertex: colours used there so far (CW words)
  int* chw;                // per vertex: mask words in use
  int* ccount;             // contacts per colour of the iteration (MAX_COLOURS)
  int* coff;               // start of each colour's contacts in corder (MAX_COLOURS + 1)
  int* cfill;              // contacts placed per colour so far (MAX_COLOURS)
  int* corder;             // contacts grouped by colour (cons_cap)
  int* ecol;               // per edge-length constraint: colour class (fixed)
  int n_ecol;              // edge colours (most over the scenes)
  int* eorder;             // edge-length constraints grouped by colour (nl)
  int* eoff;               // start of each edge colour in eorder (n_ecol + 1)
  unsigned int* bar;       // grid barrier of the sweep: arrivals since the launch
  double* lam;             // multipliers for gs_sweeps > 1 (contacts then edges)
  double* jdl;             // projected Jacobi: dl per contact, then per edge (cons_cap + nl)
  int* vlstart;            // projected Jacobi: per vertex, start into vllist (nv + 1)
  int* vllist;             // its edge-length constraints, ascending: edge * 2 + end (0 = i, 1 = j)
  BVH bt, be, bv;          // triangles, edges, collision vertices
  float4* sbox;            // per scene: Morton normalisation box (lo, hi) x2
  unsigned long long* qkeys;   // inspection output
  double* qdist;
  int qcap;
};

// ---------------------------------------------------------------------------
// FP64 vector helpers (no contraction: compiled with --fmad=false)
// ---------------------------------------------------------------------------
__device__ __forceinline__ dv3 mk(const P4& p) { return {p.x, p.y, p.z}; }
__device__ __forceinline__ dv3 vsub(dv3 a, dv3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ dv3 vadd(dv3 a, dv3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ dv3 vscl(double s, dv3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ dv3 vdiv(dv3 a, double s) { return {a.x / s, a.y / s, a.z / s}; }
__device__ __forceinline__ double vdot(dv3 a, dv3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
__device__ __forceinline__ dv3 vcross(dv3 a, dv3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double vnorm(dv3 a) { return sqrt(vdot(a, a)); }
__device__ __forceinline__ double vdet(dv3 a, dv3 b, dv3 c) { return vdot(a, vcross(b, c)); }

__device__ __forceinline__ unsigned long long dbits(double d) { return (unsigned long long)__double_as_longlong(d); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// ---------------------------------------------------------------------------
// distances between simplices
// ---------------------------------------------------------------------------
// point to segment [a,b]; t receives the clamped parameter
__device__ __forceinline__ double d_ps(dv3 p, dv3 a, dv3 b, double* tout) {
  dv3 e = vsub(b, a), w = vsub(p, a), q = a;
  double ee = vdot(e, e), t = 0.0;
  if (ee > 0.0) {
    t = vdot(w, e) / ee;
    if (t <= 0.0) { t = 0.0; q = a; }
    else if (t >= 1.0) { t = 1.0; q = b; }
    else q = vadd(a, vscl(t, e));
  }
  *tout = t;
  return vnorm(vsub(p, q));
}

// point to triangle (a,b,c): plane projection when inside, else the nearest edge
__device__ __forceinline__ double d_pt(dv3 p, dv3 a, dv3 b, dv3 c) {
  dv3 e1 = vsub(b, a), e2 = vsub(c, a), w = vsub(p, a);
  dv3 n = vcross(e1, e2);
  double nn = vdot(n, n);
  if (nn > 0.0) {
    double u = vdot(vcross(w, e2), n) / nn;
    double v = vdot(vcross(e1, w), n) / nn;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) return fabs(vdot(w, n)) / sqrt(nn);
  }
  double t;
  double d = d_ps(p, a, b, &t), d2 = d_ps(p, b, c, &t), d3 = d_ps(p, c, a, &t);
  if (d2 < d) d = d2;
  if (d3 < d) d = d3;
  return d;
}

// segment [a,b] to segment [c,d]: interior critical point if inside, and the
// four endpoint-to-segment distances; the smallest wins (first on ties)
__device__ __forceinline__ double d_ss(dv3 a, dv3 b, dv3 c, dv3 d, double* sout, double* tout) {
  dv3 d1 = vsub(b, a), d2 = vsub(d, c), r = vsub(a, c);
  double A = vdot(d1, d1), E = vdot(d2, d2), B = vdot(d1, d2), C = vdot(d1, r), F = vdot(d2, r);
  double best = __longlong_as_double(0x7ff0000000000000LL), bs = 0.0, bt = 0.0, tt, dd;
  double den = A * E - B * B;
  if (den > 0.0) {
    double s = (B * F - C * E) / den, t = (A * F - B * C) / den;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      dv3 p = vadd(a, vscl(s, d1)), q = vadd(c, vscl(t, d2));
      best = vnorm(vsub(p, q)); bs = s; bt = t;
    }
  }
  dd = d_ps(a, c, d, &tt); if (dd < best) { best = dd; bs = 0.0; bt = tt; }
  dd = d_ps(b, c, d, &tt); if (dd < best) { best = dd; bs = 1.0; bt = tt; }
  dd = d_ps(c, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 0.0; }
  dd = d_ps(d, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 1.0; }
  *sout = bs; *tout = bt;
  return best;
}

// ---------------------------------------------------------------------------
// keys and priorities
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mkkey(int kind, long long a, long long b) {
  return ((unsigned long long)kind << 62) | ((unsigned long long)a << 31) | (unsigned long long)b;
}
// SplitMix64 (Steele, Lea and Flood 2014), the mixer of the sweep priorities
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// contact constraints, Sec. 4.1
// ---------------------------------------------------------------------------
// Volume constraint: reference r_v = p_v + sgn_v h n (h = (delta - d)/2),
// c = det[p1-p0, p2-p0, p3-p0] / det[r1-r0, r2-r0, r3-r0] - 1, gradient of
// the numerator over the (constant) denominator.
__device__ __forceinline__ bool volume_cons(const dv3 p[4], const double sg[4], dv3 n, double h, double* c0,
                                            dv3 g[4]) {
  dv3 r[4];
#pragma unroll
  for (int i = 0; i < 4; i++) r[i] = vadd(p[i], vscl(sg[i] * h, n));
  dv3 c1 = vsub(p[1], p[0]), c2 = vsub(p[2], p[0]), c3 = vsub(p[3], p[0]);
  double dx = vdet(c1, c2, c3);
  double dr = vdet(vsub(r[1], r[0]), vsub(r[2], r[0]), vsub(r[3], r[0]));
  if (!(fabs(dr) >= 1e-30)) return false;
  *c0 = dx / dr - 1.0;
  g[1] = vdiv(vcross(c2, c3), dr);
  g[2] = vdiv(vcross(c3, c1), dr);
  g[3] = vdiv(vcross(c1, c2), dr);
  dv3 s = vadd(vadd(g[1], g[2]), g[3]);
  g[0] = vscl(-1.0, s);
  return true;
}

// vertex p0 against triangle (p1,p2,p3): unit normal flipped to the vertex
// closest point of triangle (a, b, c) to p: barycentric weights, and whether
// it is the plane projection (the same branches as d_pt)
__device__ __forceinline__ bool pt_weights(dv3 p, dv3 a, dv3 b, dv3 c, double wt[3]) {
  dv3 e1 = vsub(b, a), e2 = vsub(c, a), w = vsub(p, a);
  dv3 n = vcross(e1, e2);
  double nn = vdot(n, n);
  if (nn > 0.0) {
    double u = vdot(vcross(w, e2), n) / nn, v = vdot(vcross(e1, w), n) / nn;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
      wt[0] = (1.0 - u) - v; wt[1] = u; wt[2] = v;
      return true;
    }
  }
  double t1, t2, t3;
  double d = d_ps(p, a, b, &t1), d2 = d_ps(p, b, c, &t2), d3 = d_ps(p, c, a, &t3);
  wt[0] = 1.0 - t1; wt[1] = t1; wt[2] = 0.0;
  if (d2 < d) { d = d2; wt[0] = 0.0; wt[1] = 1.0 - t2; wt[2] = t2; }
  if (d3 < d) { wt[0] = t3; wt[1] = 0.0; wt[2] = 1.0 - t3; }
  return false;
}
// gap constraint (reading G1): c = d/delta - 1, gradient w_v n / delta
__device__ __forceinline__ void gap_cons(double d, double delta, dv3 n, const double w[4], double* c0, dv3 g[4]) {
  *c0 = d / delta - 1.0;
  for (int k = 0; k < 4; k++) g[k] = vscl(w[k] / delta, n);
}

// form: 0 volume (Sec. 4.1), 1 gap
__device__ __forceinline__ bool vt_cons(const dv3 p[4], double d, double delta, int form, double* c0, dv3 g[4]) {
  dv3 nrm = vcross(vsub(p[2], p[1]), vsub(p[3], p[1]));
  double nn = vdot(nrm, nrm);
  if (!(nn > 0.0)) return false;
  dv3 nh = vdiv(nrm, sqrt(nn));
  double side = vdot(nh, vsub(p[0], p[1])) < 0.0 ? -1.0 : 1.0;
  dv3 n = vscl(side, nh);
  if (form == 1) {
    double wt[3];
    if (!pt_weights(p[0], p[1], p[2], p[3], wt)) {
      dv3 q = vadd(vadd(vscl(wt[0], p[1]), vscl(wt[1], p[2])), vscl(wt[2], p[3]));
      dv3 dv = vsub(p[0], q);
      double L = vnorm(dv);
      if (L > 0.0) n = vdiv(dv, L);
    }
    const double w[4] = {1.0, -wt[0], -wt[1], -wt[2]};
    gap_cons(d, delta, n, w, c0, g);
    return true;
  }
  const double sg[4] = {1.0, -1.0, -1.0, -1.0};
  return volume_cons(p, sg, n, 0.5 * (delta - d), c0, g);
}

// edge (p0,p1) against edge (p2,p3); near-parallel edges use the gap form
__device__ __forceinline__ bool ee_cons(const dv3 p[4], double d, double s, double t, double delta, int form,
                                        double* c0, dv3 g[4]) {
  dv3 e1 = vsub(p[1], p[0]), e2 = vsub(p[3], p[2]);
  dv3 nx = vcross(e1, e2);
  double nn = vdot(nx, nx);
  dv3 pa = vadd(p[0], vscl(s, e1)), pc = vadd(p[2], vscl(t, e2));
  dv3 dv = vsub(pa, pc);
  double L = vnorm(dv);
  dv3 n;
  if (L > 0.0) n = vdiv(dv, L);
  else if (nn > 0.0) n = vdiv(nx, sqrt(nn));
  else return false;
  if (form == 1 || nn < 1e-12 * (vdot(e1, e1) * vdot(e2, e2))) {
    const double w[4] = {1.0 - s, s, -(1.0 - t), -t};
    gap_cons(d, delta, n, w, c0, g);
    return true;
  }
  const double sg[4] = {1.0, 1.0, -1.0, -1.0};
  return volume_cons(p, sg, n, 0.5 * (delta - d), c0, g);
}

// point p0 against vertex p1 with radii
__device__ __forceinline__ bool vv_cons(const dv3 p[2], double ra, double rb, double delta, double* c0, dv3 g[4]) {
  dv3 dv = vsub(p[0], p[1]);
  double L = vnorm(dv);
  if (!(L > 0.0)) return false;
  double R = (ra + rb) + delta;
  *c0 = L / R - 1.0;
  dv3 u = vdiv(dv, L);
  g[0] = vdiv(u, R);
  g[1] = vscl(-1.0, g[0]);
  return true;
}

// ---------------------------------------------------------------------------
// FP32 distance pre-filter.  The distances below are evaluated on float
// copies of the positions; their error is below FILTER_TOL * (|x|max + extent)
// (coordinate rounding 2^-24 |x| plus a few dozen float operations on vectors
// of the primitives' extent).  A pair is sent to the exact FP64 distance
// unless d32 - tol >= D, so the set of pairs closer than D is unchanged.
// ---------------------------------------------------------------------------
constexpr float FILTER_TOL = 4e-6f;
struct fv3 { float x, y, z; };
__device__ __forceinline__ fv3 fk(float4 p) { return {p.x, p.y, p.z}; }
__device__ __forceinline__ fv3 fsub(fv3 a, fv3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float fdot(fv3 a, fv3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ fv3 fcross(fv3 a, fv3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float fmaxabs(fv3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }
__device__ __forceinline__ float f_ps(fv3 p, fv3 a, fv3 b) {
  fv3 e = fsub(b, a), w = fsub(p, a);
  float ee = fdot(e, e), t = 0.f;
  if (ee > 0.f) t = fminf(fmaxf(fdot(w, e) / ee, 0.f), 1.f);
  fv3 q = {w.x - t * e.x, w.y - t * e.y, w.z - t * e.z};
  return sqrtf(fdot(q, q));
}
__device__ __forceinline__ float f_pt(fv3 p, fv3 a, fv3 b, fv3 c) {
  fv3 e1 = fsub(b, a), e2 = fsub(c, a), w = fsub(p, a);
  fv3 n = fcross(e1, e2);
  float nn = fdot(n, n);
  if (nn > 0.f) {
    float u = fdot(fcross(w, e2), n) / nn, v = fdot(fcross(e1, w), n) / nn;
    if (u >= 0.f && v >= 0.f && u + v <= 1.f) return fabsf(fdot(w, n)) * rsqrtf(nn);
  }
  return fminf(f_ps(p, a, b), fminf(f_ps(p, b, c), f_ps(p, c, a)));
}
__device__ __forceinline__ float f_ss(fv3 a, fv3 b, fv3 c, fv3 d) {
  fv3 d1 = fsub(b, a), d2 = fsub(d, c), r = fsub(a, c);
  float A = fdot(d1, d1), E = fdot(d2, d2), B = fdot(d1, d2), C = fdot(d1, r), F = fdot(d2, r);
  float best = fminf(fminf(f_ps(a, c, d), f_ps(b, c, d)), fminf(f_ps(c, a, b), f_ps(d, a, b)));
  float den = A * E - B * B;
  if (den > 0.f) {
    float s = (B * F - C * E) / den, t = (A * F - B * C) / den;
    if (s >= 0.f && s <= 1.f && t >= 0.f && t <= 1.f) {
      fv3 q = {r.x + s * d1.x - t * d2.x, r.y + s * d1.y - t * d2.y, r.z + s * d1.z - t * d2.z};
      best = fminf(best, sqrtf(fdot(q, q)));
    }
  }
  return best;
}
// A lower bound of the segment-segment distance that does not rely on the
// closest-point solution: for nearly parallel segments that solution is
// ill-conditioned in float (its denominator |d1|^2 |d2|^2 sin^2 of the angle
// loses its digits), and f_ss can then exceed the true distance by more than
// the rounding margin.  The interval gap of the projections of both segments
// onto any direction k is a lower bound of their distance; it is exact for
// the true separation direction.  The bound is the largest gap over three
// directions: the difference of f_ss's closest points, d1 x d2 and the part of
// c - a orthogonal to d1.  Projections are taken relative to a, so their
// rounding is small against FILTER_TOL (|x|max + extent).
__device__ __forceinline__ float f_gap(fv3 k, fv3 a, fv3 b, fv3 c, fv3 d) {
  float kk = fdot(k, k);
  if (!(kk > 0.f)) return 0.f;
  float pb = fdot(k, fsub(b, a)), pc = fdot(k, fsub(c, a)), pd = fdot(k, fsub(d, a));
  float g = fmaxf(fminf(pc, pd) - fmaxf(0.f, pb), fminf(0.f, pb) - fmaxf(pc, pd));
  return g > 0.f ? g / sqrtf(kk) : 0.f;
}
__device__ __forceinline__ fv3 f_seg_pt(fv3 p, fv3 a, fv3 b) {
  fv3 e = fsub(b, a), w = fsub(p, a);
  float ee = fdot(e, e), t = 0.f;
  if (ee > 0.f) t = fminf(fmaxf(fdot(w, e) / ee, 0.f), 1.f);
  return {a.x + t * e.x, a.y + t * e.y, a.z + t * e.z};
}
// Distance of f_ss (returned; an upper estimate of the true distance up to
// rounding, as the distance of two points of the segments) and, in *lower, a
// lower bound: the gap along the difference of the closest points found, and
// unless that gap already reaches `enough`, the larger of it and the gaps
// along d1 x d2 and the part of c - a orthogonal to d1.  Each gap alone is a
// valid bound, so a caller that only needs to reject pairs beyond a distance
// passes it as `enough` and skips the other two for most of them.
__device__ __forceinline__ float f_ss_bounds(fv3 a, fv3 b, fv3 c, fv3 d, float enough, float* lower) {
  fv3 d1 = fsub(b, a), d2 = fsub(d, c), r = fsub(a, c);
  float A = fdot(d1, d1), E = fdot(d2, d2), B = fdot(d1, d2), C = fdot(d1, r), F = fdot(d2, r);
  // closest points as f_ss finds them: the four endpoint projections and the
  // interior solution, whichever is nearest
  fv3 z = fsub(a, f_seg_pt(a, c, d));
  float bz = fdot(z, z);
  {
    fv3 z2 = fsub(b, f_seg_pt(b, c, d));
    float b2 = fdot(z2, z2);
    if (b2 < bz) { bz = b2; z = z2; }
    fv3 z3 = fsub(f_seg_pt(c, a, b), c);
    float b3 = fdot(z3, z3);
    if (b3 < bz) { bz = b3; z = z3; }
    fv3 z4 = fsub(f_seg_pt(d, a, b), d);
    float b4 = fdot(z4, z4);
    if (b4 < bz) { bz = b4; z = z4; }
  }
  float den = A * E - B * B;
  if (den > 0.f) {
    float s = (B * F - C * E) / den, t = (A * F - B * C) / den;
    if (s >= 0.f && s <= 1.f && t >= 0.f && t <= 1.f) {
      fv3 zi = {r.x + s * d1.x - t * d2.x, r.y + s * d1.y - t * d2.y, r.z + s * d1.z - t * d2.z};
      float bi = fdot(zi, zi);
      if (bi < bz) { bz = bi; z = zi; }
    }
  }
  float g = f_gap(z, a, b, c, d);
  if (!(g >= enough)) {
    g = fmaxf(g, f_gap(fcross(d1, d2), a, b, c, d));
    if (A > 0.f) {
      float sc = C / A;
      fv3 k = {r.x - sc * d1.x, r.y - sc * d1.y, r.z - sc * d1.z};
      g = fmaxf(g, f_gap(k, a, b, c, d));
    }
  }
  *lower = g;
  return sqrtf(bz);
}
// error margin of a float distance over these points
__device__ __forceinline__ float ftol(fv3 a, fv3 b, fv3 c, fv3 d) {
  float X = fmaxf(fmaxf(fmaxabs(a), fmaxabs(b)), fmaxf(fmaxabs(c), fmaxabs(d)));
  float M = fmaxf(fmaxf(fmaxabs(fsub(b, a)), fmaxabs(fsub(c, a))), fmaxabs(fsub(d, a)));
  return FILTER_TOL * (X + M) + 1e-30f;
}

// monotone unsigned image of a float (a < b <=> fl_ord(a) < fl_ord(b))
__device__ __forceinline__ unsigned int fl_ord(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_fl(unsigned int u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
// The exact candidate test (R3): on every axis fl(lo_b - hi_a) <= D and
// fl(lo_a - hi_b) <= D.
__device__ __forceinline__ bool box_near(dv3 alo, dv3 ahi, dv3 blo, dv3 bhi, double D) {
  if (blo.x - ahi.x > D) return false;
  if (alo.x - bhi.x > D) return false;
  if (blo.y - ahi.y > D) return false;
  if (alo.y - bhi.y > D) return false;
  if (blo.z - ahi.z > D) return false;
  if (alo.z - bhi.z > D) return false;
  return true;
}
// ---------------------------------------------------------------------------
// CCD of a linearly moving pair (the comparison scheme of Sec. 5.1, here the
// per-iteration safety check).  Same arithmetic as the oracle's CCD.
// ---------------------------------------------------------------------------
constexpr double CCD_TOUCH = 1e-9;

__device__ __forceinline__ double cubic_at(const double c[4], double t) {
  return ((c[3] * t + c[2]) * t + c[1]) * t + c[0];
}
// roots of the coplanarity cubic in [0,1], ascending: the interval is cut at
// the derivative's roots and sign changes on monotone pieces are bisected
__device__ __forceinline__ int cubic_roots01(const double c[4], double* roots) {
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
      crit[ncr++] = r1;
      crit[ncr++] = r2;
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

// kind VT (a; i,j,k) / EE (a,b; c,d) / VV (a,b) moving from p0 to p1
__device__ __forceinline__ bool ccd_pair(int kind, const dv3* p0, const dv3* p1, double ra, double rb, double* toi) {
  int nv = kind == K_VV ? 2 : 4;
  dv3 d[4];
  for (int i = 0; i < nv; i++) d[i] = vsub(p1[i], p0[i]);
  double R = kind == K_VV ? ra + rb : 0.0;
  if (kind == K_VT && ra > 0.0) return false;
  {
    int na = kind == K_EE ? 2 : 1;
    dv3 alo = p0[0], ahi = p0[0], blo = p0[na], bhi = p0[na];
    for (int i = 0; i < nv; i++) {
      dv3 q[2] = {p0[i], p1[i]};
      for (int h = 0; h < 2; h++) {
        dv3& lo = i < na ? alo : blo;
        dv3& hi = i < na ? ahi : bhi;
        if (q[h].x < lo.x) lo.x = q[h].x; if (q[h].x > hi.x) hi.x = q[h].x;
        if (q[h].y < lo.y) lo.y = q[h].y; if (q[h].y > hi.y) hi.y = q[h].y;
        if (q[h].z < lo.z) lo.z = q[h].z; if (q[h].z > hi.z) hi.z = q[h].z;
      }
    }
    if (!box_near(alo, ahi, blo, bhi, CCD_TOUCH + R)) return false;
  }
  if (kind == K_VV) {
    dv3 r = vsub(p0[0], p0[1]), v = vsub(d[0], d[1]);
    double rr = vdot(r, r), RR = (R + CCD_TOUCH) * (R + CCD_TOUCH);
    if (rr <= RR) { *toi = 0.0; return true; }
    double vv = vdot(v, v), rv = vdot(r, v);
    if (!(vv > 0.0) || rv >= 0.0) return false;
    double disc = rv * rv - vv * (rr - RR);
    if (disc < 0.0) return false;
    double t = (-rv - sqrt(disc)) / vv;
    if (t >= 0.0 && t <= 1.0) { *toi = t; return true; }
    return false;
  }
  dv3 a[3], b[3];
  for (int k = 0; k < 3; k++) { a[k] = vsub(p0[k + 1], p0[0]); b[k] = vsub(d[k + 1], d[0]); }
  double c[4];
  c[0] = vdet(a[0], a[1], a[2]);
  c[1] = (vdet(b[0], a[1], a[2]) + vdet(a[0], b[1], a[2])) + vdet(a[0], a[1], b[2]);
  c[2] = (vdet(a[0], b[1], b[2]) + vdet(b[0], a[1], b[2])) + vdet(b[0], b[1], a[2]);
  c[3] = vdet(b[0], b[1], b[2]);
  double roots[16];
  int nr;
  if (c[0] == 0.0 && c[1] == 0.0 && c[2] == 0.0 && c[3] == 0.0) {
    nr = 0;
    for (int i = 0; i <= 8; i++) roots[nr++] = i / 8.0;
  } else nr = cubic_roots01(c, roots);
  for (int r = 0; r < nr; r++) {
    double t = roots[r];
    dv3 q[4];
    for (int i = 0; i < 4; i++) q[i] = vadd(p0[i], vscl(t, d[i]));
    double s, u;
    double dist = kind == K_VT ? d_pt(q[0], q[1], q[2], q[3]) : d_ss(q[0], q[1], q[2], q[3], &s, &u);
    if (dist <= CCD_TOUCH) { *toi = t; return true; }
  }
  return false;
}

// ---------------------------------------------------------------------------
// acceptance: FP64 orientation with an error bound (45 ulps of the
// permanent); 2 = the sign is not certain
// ---------------------------------------------------------------------------
__device__ __forceinline__ int o3f(dv3 a, dv3 b, dv3 c, dv3 d) {
  dv3 u = vsub(b, a), v = vsub(c, a), w = vsub(d, a);
  double det = vdet(u, v, w);
  double perm = fabs(u.x) * (fabs(v.y * w.z) + fabs(v.z * w.y)) + fabs(u.y) * (fabs(v.x * w.z) + fabs(v.z * w.x)) +
                fabs(u.z) * (fabs(v.x * w.y) + fabs(v.y * w.x));
  double bound = 5e-15 * perm;
  if (det > bound) return 1;
  if (det < -bound) return -1;
  return 2;
}
// 1: segment [p,q] meets triangle (a,b,c); 0: disjoint; 2: not decided.
// When an orientation is uncertain the pair is (nearly) coplanar or passes
// near the triangle's boundary, and then it is disjoint if the segment stays
// more than tol from the triangle's edges and the endpoints from the triangle.
__device__ __forceinline__ int seg_tri_test(dv3 p, dv3 q, dv3 a, dv3 b, dv3 c, double tol) {
  int s1 = o3f(a, b, c, p), s2 = o3f(a, b, c, q);
  bool unsure = s1 == 2 || s2 == 2;
  if (!unsure) {
    if (s1 == s2) return 0;
    int t1 = o3f(p, q, a, b), t2 = o3f(p, q, b, c), t3 = o3f(p, q, c, a);
    if (t1 != 2 && t2 != 2 && t3 != 2) {
      int pos = (t1 > 0) + (t2 > 0) + (t3 > 0), neg = (t1 < 0) + (t2 < 0) + (t3 < 0);
      return (pos && neg) ? 0 : 1;
    }
  }
  double s, t;
  double m = d_pt(p, a, b, c);
  m = fmin(m, d_pt(q, a, b, c));
  m = fmin(m, d_ss(p, q, a, b, &s, &t));
  m = fmin(m, d_ss(p, q, b, c, &s, &t));
  m = fmin(m, d_ss(p, q, c, a, &s, &t));
  return m > tol ? 0 : 2;
}

// ---------------------------------------------------------------------------
// FP32 versions of the contact constraints (mixed precision): the same
// formulas as vt_cons / ee_cons / vv_cons evaluated in float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ fv3 fadd3(fv3 a, fv3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ fv3 fscl3(float s, fv3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ fv3 fdiv3(fv3 a, float s) { return {a.x / s, a.y / s, a.z / s}; }
__device__ __forceinline__ float fdet3(fv3 a, fv3 b, fv3 c) { return fdot(a, fcross(b, c)); }
__device__ __forceinline__ float f_ps_t(fv3 p, fv3 a, fv3 b, float* tout) {
  fv3 e = fsub(b, a), w = fsub(p, a), q = a;
  float ee = fdot(e, e), t = 0.f;
  if (ee > 0.f) {
    t = fdot(w, e) / ee;
    if (t <= 0.f) { t = 0.f; q = a; }
    else if (t >= 1.f) { t = 1.f; q = b; }
    else q = fadd3(a, fscl3(t, e));
  }
  *tout = t;
  fv3 r = fsub(p, q);
  return sqrtf(fdot(r, r));
}
__device__ __forceinline__ void f_ss_st(fv3 a, fv3 b, fv3 c, fv3 d, float* sout, float* tout) {
  fv3 d1 = fsub(b, a), d2 = fsub(d, c), r = fsub(a, c);
  float A = fdot(d1, d1), E = fdot(d2, d2), B = fdot(d1, d2), C = fdot(d1, r), F = fdot(d2, r);
  float best = 3.4e38f, bs = 0.f, bt = 0.f, tt, dd;
  float den = A * E - B * B;
  if (den > 0.f) {
    float s = (B * F - C * E) / den, t = (A * F - B * C) / den;
    if (s >= 0.f && s <= 1.f && t >= 0.f && t <= 1.f) {
      fv3 q = fsub(fadd3(a, fscl3(s, d1)), fadd3(c, fscl3(t, d2)));
      best = sqrtf(fdot(q, q)); bs = s; bt = t;
    }
  }
  dd = f_ps_t(a, c, d, &tt); if (dd < best) { best = dd; bs = 0.f; bt = tt; }
  dd = f_ps_t(b, c, d, &tt); if (dd < best) { best = dd; bs = 1.f; bt = tt; }
  dd = f_ps_t(c, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 0.f; }
  dd = f_ps_t(d, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 1.f; }
  *sout = bs; *tout = bt;
}
__device__ __forceinline__ bool volume_cons_f(const fv3 p[4], const float sg[4], fv3 n, float h, float* c0, fv3 g[4]) {
  fv3 r[4];
  for (int i = 0; i < 4; i++) r[i] = fadd3(p[i], fscl3(sg[i] * h, n));
  fv3 c1 = fsub(p[1], p[0]), c2 = fsub(p[2], p[0]), c3 = fsub(p[3], p[0]);
  float dx = fdet3(c1, c2, c3);
  float dr = fdet3(fsub(r[1], r[0]), fsub(r[2], r[0]), fsub(r[3], r[0]));
  if (!(fabsf(dr) >= 1e-30f)) return false;
  *c0 = dx / dr - 1.f;
  g[1] = fdiv3(fcross(c2, c3), dr);
  g[2] = fdiv3(fcross(c3, c1), dr);
  g[3] = fdiv3(fcross(c1, c2), dr);
  g[0] = fscl3(-1.f, fadd3(fadd3(g[1], g[2]), g[3]));
  return true;
}
__device__ __forceinline__ void gap_cons_f(float d, float delta, fv3 n, const float w[4], float* c0, fv3 g[4]) {
  *c0 = d / delta - 1.f;
  for (int k = 0; k < 4; k++) g[k] = fscl3(w[k] / delta, n);
}
__device__ __forceinline__ bool vt_cons_f(const fv3 p[4], float d, float delta, int form, float* c0, fv3 g[4]) {
  fv3 nrm = fcross(fsub(p[2], p[1]), fsub(p[3], p[1]));
  float nn = fdot(nrm, nrm);
  if (!(nn > 0.f)) return false;
  fv3 nh = fdiv3(nrm, sqrtf(nn));
  float side = fdot(nh, fsub(p[0], p[1])) < 0.f ? -1.f : 1.f;
  fv3 n = fscl3(side, nh);
  if (form == 1) {
    // closest point of the triangle, as in the FP64 form
    fv3 e1 = fsub(p[2], p[1]), e2 = fsub(p[3], p[1]), w = fsub(p[0], p[1]);
    float u = fdot(fcross(w, e2), nrm) / nn, v = fdot(fcross(e1, w), nrm) / nn;
    float wt[3];
    if (u >= 0.f && v >= 0.f && u + v <= 1.f) {
      wt[0] = (1.f - u) - v; wt[1] = u; wt[2] = v;
    } else {
      float t1, t2, t3;
      float da = f_ps_t(p[0], p[1], p[2], &t1), db = f_ps_t(p[0], p[2], p[3], &t2), dc = f_ps_t(p[0], p[3], p[1], &t3);
      wt[0] = 1.f - t1; wt[1] = t1; wt[2] = 0.f;
      if (db < da) { da = db; wt[0] = 0.f; wt[1] = 1.f - t2; wt[2] = t2; }
      if (dc < da) { wt[0] = t3; wt[1] = 0.f; wt[2] = 1.f - t3; }
      fv3 q = fadd3(fadd3(fscl3(wt[0], p[1]), fscl3(wt[1], p[2])), fscl3(wt[2], p[3]));
      fv3 dv = fsub(p[0], q);
      float L = sqrtf(fdot(dv, dv));
      if (L > 0.f) n = fdiv3(dv, L);
    }
    const float gw[4] = {1.f, -wt[0], -wt[1], -wt[2]};
    gap_cons_f(d, delta, n, gw, c0, g);
    return true;
  }
  const float sg[4] = {1.f, -1.f, -1.f, -1.f};
  return volume_cons_f(p, sg, n, 0.5f * (delta - d), c0, g);
}
__device__ __forceinline__ bool ee_cons_f(const fv3 p[4], float d, float s, float t, float delta, int form, float* c0,
                                          fv3 g[4]) {
  fv3 e1 = fsub(p[1], p[0]), e2 = fsub(p[3], p[2]);
  fv3 nx = fcross(e1, e2);
  float nn = fdot(nx, nx);
  fv3 dv = fsub(fadd3(p[0], fscl3(s, e1)), fadd3(p[2], fscl3(t, e2)));
  float L = sqrtf(fdot(dv, dv));
  fv3 n;
  if (L > 0.f) n = fdiv3(dv, L);
  else if (nn > 0.f) n = fdiv3(nx, sqrtf(nn));
  else return false;
  if (form == 1 || nn < 1e-12f * (fdot(e1, e1) * fdot(e2, e2))) {
    const float w[4] = {1.f - s, s, -(1.f - t), -t};
    gap_cons_f(d, delta, n, w, c0, g);
    return true;
  }
  const float sg[4] = {1.f, 1.f, -1.f, -1.f};
  return volume_cons_f(p, sg, n, 0.5f * (delta - d), c0, g);
}
__device__ __forceinline__ bool vv_cons_f(const fv3 p[2], float ra, float rb, float delta, float* c0, fv3 g[4]) {
  fv3 dv = fsub(p[0], p[1]);
  float L = sqrtf(fdot(dv, dv));
  if (!(L > 0.f)) return false;
  float R = (ra + rb) + delta;
  *c0 = L / R - 1.f;
  g[0] = fdiv3(fdiv3(dv, L), R);
  g[1] = fscl3(-1.f, g[0]);
  return true;
}

// Smallest pair distance the forward step trusts: below it D_i/2 is no larger
// than the rounding of an FP64 position update, so the vertex stays put.
constexpr double D_FLOOR = 1e-10;

}  // namespace cch

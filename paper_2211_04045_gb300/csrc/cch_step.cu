// cch_step.cu -- one iteration of Algorithm 1 on sm_103a: distance refresh
// of the reused proximity set (Sec. 3.1), contact assembly (Sec. 4.1),
// the projected Gauss-Seidel or Jacobi backward step (Sec. 4.3),
// the forward step (Sec. 5) and the loop control (Algorithm 1).
#include "cch_host.h"
#include "cch_step.h"

namespace cch {

static int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

// ---------------------------------------------------------------------------
// step set-up
// ---------------------------------------------------------------------------
// per scene: D^(0) = 0 < D^min, so the first iteration searches (D <- D^max)
// mode 0: every scene becomes active and starts; mode 2: only scenes whose
// start flag is set (a server admitting requests while others run)
__global__ void k_scene_init(Pool P, int mode) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.nscene; s += gridDim.x * blockDim.x) {
    SceneState& S = P.ss[s];
    if (mode == 2 && !S.start) continue;
    S.active = 1;
    S.D = P.sd[s].d_max;
    S.iter = 0;
    S.done = 0;
    S.do_search = 1;
    S.converged = 0;
    S.searches = 0;
    S.move_bits = 0;
    S.rmax_bits = 0;
    S.mind_bits = 0x7ff0000000000000ULL;
    S.pairs_eval = S.max_pairs = S.contacts = S.candidates = S.degenerate = 0;
    S.n_pairs = 0;
    S.max_vcontacts = 0;
    S.ccd_clamps = 0;
    S.final_r = 1.0;
    S.isect = S.uncertain = 0;
    S.bad_input = 0;
    S.frozen_cur = S.frozen = 0;
    S.cverts = 0;
    S.pverts = 0;
    S.ccol = 0;
  }
}

// x^(0) = x_t, y^(0) = y^[k+1] = x_tilde, r^(0) = 1; static flags (R4)
__global__ void k_vert_init(Pool P, double* const* ptrs, int mode) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    if (!P.ss[s].active || (mode == 2 && !P.ss[s].start)) continue;
    int i = v - P.sd[s].v0;
    const double* xt = ptrs[3 * s];
    const double* xl = ptrs[3 * s + 1];
    P4 a = {xt[3 * i], xt[3 * i + 1], xt[3 * i + 2], 0.0};
    P4 b = {xl[3 * i], xl[3 * i + 1], xl[3 * i + 2], 0.0};
    if (!(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(b.x) && isfinite(b.y) && isfinite(b.z))) {
      // the scene's step is not run; the call reports CCH_E_INVALID_ARG
      P.ss[s].bad_input = 1;
      P.ss[s].done = 1;
    }
    P.x[v] = a;
    P.xf[v] = make_float4((float)a.x, (float)a.y, (float)a.z, 0.f);
    P.y[v] = b;
    P.yt[v] = b;
    if (P.yf) P.yf[v] = make_float4((float)b.x, (float)b.y, (float)b.z, 0.f);
    P.r[v] = 1.0;
    P.Dv[v] = 0x7ff0000000000000ULL;
    if (P.clampb) P.clampb[v] = 0x3ff0000000000000ULL;
    uint8_t f = P.vflag[v] & (uint8_t)~VF_STATIC;
    if (P.im[v] == 0.0 && a.x == b.x && a.y == b.y && a.z == b.z) f |= VF_STATIC;
    P.vflag[v] = f;
  }
}

// edge-length constraints of the step (R9): g = u / L0 from y^[k+1]
__global__ void k_edge_prep(Pool P, int mode) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nl; e += gridDim.x * blockDim.x) {
    int4 l = P.lv[e];
    if (!P.ss[l.z].active || (mode == 2 && !P.ss[l.z].start)) continue;
    dv3 d0 = vsub(mk(P.yt[l.x]), mk(P.yt[l.y]));
    double L0 = vnorm(d0);
    P4 o = {0.0, 0.0, 0.0, 0.0};
    if (L0 > 0.0) {
      dv3 g = vdiv(vdiv(d0, L0), L0);
      o = {g.x, g.y, g.z, (P.im[l.x] + P.im[l.y]) * vdot(g, g)};
    }
    P.lg[e] = o;
    if (P.lgf) P.lgf[e] = make_float4((float)o.x, (float)o.y, (float)o.z, (float)o.w);
  }
}

// ---------------------------------------------------------------------------
// distance refresh of a reused P (Sec. 3.1): keep pairs still below D^(l)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pair_dist(const Pool& P, unsigned long long key, int4 v) {
  int kind = (int)(key >> 62);
  if (kind == K_VT) return d_pt(mk(P.x[v.x]), mk(P.x[v.y]), mk(P.x[v.z]), mk(P.x[v.w])) - P.rho[v.x];
  if (kind == K_EE) {
    double s, t;
    return d_ss(mk(P.x[v.x]), mk(P.x[v.y]), mk(P.x[v.z]), mk(P.x[v.w]), &s, &t);
  }
  return (vnorm(vsub(mk(P.x[v.x]), mk(P.x[v.y]))) - P.rho[v.x]) - P.rho[v.y];
}

// Distance refresh, FP64 mode: pass A records every reused pair's FP32 bounds
// and the smallest upper bound of the certain pairs per vertex; pass B keeps
// the pairs below D^(l), with exact distances only where they decide
// something (see needs_exact).  Mixed precision: one pass, the FP32 lower
// bound is the distance.
__global__ void k_refresh_bounds(Pool P, int cur) {
  if (!P.cnt->any_refresh) return;
  int n = min(P.cnt->n_pairs[cur], P.pair_cap);
  const PairBuf B = P.pb[cur];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 v = B.v[i];
    const SceneState& S = P.ss[P.vscene[v.x]];
    if (!S.active || S.done || S.do_search) continue;
    float2 b = pair_bounds32(P, B.key[i], v);
    P.fbr[i] = b;
    if (b.x < __double2float_ru(S.D) && (double)b.y < S.D) note_upper(P, v, b.y);
  }
}

__global__ void k_refresh(Pool P, int cur, int nxt) {
  if (!P.cnt->any_refresh) return;
  int n = P.cnt->n_pairs[cur];
  if (n > P.pair_cap) n = P.pair_cap;
  const PairBuf B = P.pb[cur];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 v = B.v[i];
    int s = P.vscene[v.x];
    const SceneState& S = P.ss[s];
    if (!S.active || S.done || S.do_search) continue;
    unsigned long long key = B.key[i];
    if (P.mixed) {
      // mixed precision: the FP32 lower bound is the pair's distance
      float lower = pair_bounds32(P, key, v).x;
      if (lower >= __double2float_ru(S.D)) continue;
      if ((double)lower < S.D) emit_pair(P, nxt, s, key, v, (double)lower);
      continue;
    }
    float2 b = P.fbr[i];
    if (b.x >= __double2float_ru(S.D)) continue;
    if (needs_exact(P, v, b, S.D, P.sd[s].delta)) {
      // the FP64 distance runs in k_exact_refresh, over a dense list
      int e = claim(&P.cnt->n_exact[1], P.pair_cap);
      if (e >= 0) P.exr[e] = i;
    } else {
      emit_pair(P, nxt, s, key, v, (double)b.x);  // certainly in P; its distance decides nothing
    }
  }
}

// exact FP64 distances of the refreshed pairs k_refresh left due, one per
// thread over the dense list
__global__ void k_exact_refresh(Pool P, int cur, int nxt) {
  if (!P.cnt->any_refresh) return;
  int n = min(P.cnt->n_exact[1], P.pair_cap);
  const PairBuf B = P.pb[cur];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int i = P.exr[j];
    int4 v = B.v[i];
    unsigned long long key = B.key[i];
    int s = P.vscene[v.x];
    double d = pair_dist(P, key, v);
    if (d < P.ss[s].D) emit_pair(P, nxt, s, key, v, d);
  }
}

// ---------------------------------------------------------------------------
// contact assembly at x^(l) (Sec. 4.1, linearisation of Sec. 4)
// ---------------------------------------------------------------------------
// mixed precision: the constraint in FP32 from the float positions
__device__ __forceinline__ void assemble_f(Pool& P, int s, const SceneDesc& S, int kind, unsigned long long key,
                                           int4 v, float d) {
  fv3 q[4], g[4];
  float c0 = 0.f;
  bool ok;
  q[0] = fk(P.xf[v.x]);
  q[1] = fk(P.xf[v.y]);
  int nv = 2;
  float delta = (float)S.delta;
  if (kind == K_VV) {
    ok = vv_cons_f(q, (float)P.rho[v.x], (float)P.rho[v.y], delta, &c0, g);
    g[2] = g[3] = {0.f, 0.f, 0.f};
  } else {
    q[2] = fk(P.xf[v.z]);
    q[3] = fk(P.xf[v.w]);
    nv = 4;
    if (kind == K_VT) ok = vt_cons_f(q, d, delta, S.form, &c0, g);
    else {
      float ps, pt;
      f_ss_st(q[0], q[1], q[2], q[3], &ps, &pt);
      ok = ee_cons_f(q, d, ps, pt, delta, S.form, &c0, g);
    }
  }
  if (!ok) {
    atomicAdd((unsigned long long*)&P.ss[s].degenerate, 1ull);
    return;
  }
  int vid[4] = {v.x, v.y, v.z, v.w};
  float den = 0.f;
  for (int k = 0; k < nv; k++) den = den + (float)P.im[vid[k]] * fdot(g[k], g[k]);
  int idx = claim(&P.cnt->n_cons, P.cons_cap);
  if (idx < 0) {
    atomicOr(&P.cnt->overflow, OV_CONTACTS);
    return;
  }
  ContactF c;
  c.v = v;
  for (int k = 0; k < 4; k++) {
    c.g[3 * k] = g[k].x;
    c.g[3 * k + 1] = g[k].y;
    c.g[3 * k + 2] = g[k].z;
  }
  c.c0 = c0;
  c.den = den;
  c.key = key;
  c.prio = splitmix64(S.seed ^ key);
  ((ContactF*)P.cons)[idx] = c;
  scene_count(P, s, [&](int n) { atomicAdd((unsigned long long*)&P.ss[s].contacts, (unsigned long long)n); });
}

__global__ void k_assemble(Pool P, int nxt) {
  int n0 = min(P.cnt->n_active[0], P.act_cap), n1 = min(P.cnt->n_active[1], P.act_cap);
  int n = n0 + n1 + min(P.cnt->n_active[2], P.act_cap);
  const PairBuf B = P.pb[nxt];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = i < n0 ? P.act[i] : (i < n0 + n1 ? P.act[P.act_cap + (i - n0)] : P.act[2 * (size_t)P.act_cap + (i - n0 - n1)]);
    unsigned long long key = B.key[p];
    int4 v = B.v[p];
    double d = B.d[p];
    int s = P.vscene[v.x];
    const SceneDesc& S = P.sd[s];
    int kind = (int)(key >> 62);
    if (P.mixed) {
      assemble_f(P, s, S, kind, key, v, (float)d);
      continue;
    }
    dv3 q[4];
    dv3 g[4];
    double c0 = 0.0;
    bool ok;
    q[0] = mk(P.x[v.x]);
    q[1] = mk(P.x[v.y]);
    int nv = 2;
    if (kind == K_VV) {
      ok = vv_cons(q, P.rho[v.x], P.rho[v.y], S.delta, &c0, g);
      g[2] = g[3] = {0.0, 0.0, 0.0};
    } else {
      q[2] = mk(P.x[v.z]);
      q[3] = mk(P.x[v.w]);
      nv = 4;
      if (kind == K_VT) ok = vt_cons(q, d, S.delta, S.form, &c0, g);
      else {
        double ps, pt;
        d_ss(q[0], q[1], q[2], q[3], &ps, &pt);
        ok = ee_cons(q, d, ps, pt, S.delta, S.form, &c0, g);
      }
    }
    if (!ok) {
      atomicAdd((unsigned long long*)&P.ss[s].degenerate, 1ull);
      continue;
    }
    int vid[4] = {v.x, v.y, v.z, v.w};
    double den = 0.0;
    for (int k = 0; k < nv; k++) den = den + P.im[vid[k]] * vdot(g[k], g[k]);
    int idx = claim(&P.cnt->n_cons, P.cons_cap);
    if (idx < 0) {
      atomicOr(&P.cnt->overflow, OV_CONTACTS);
      continue;
    }
    Contact c;
    c.v = v;
    for (int k = 0; k < 4; k++) {
      c.g[3 * k] = g[k].x;
      c.g[3 * k + 1] = g[k].y;
      c.g[3 * k + 2] = g[k].z;
    }
    c.c0 = c0;
    c.den = den;
    c.key = key;
    c.prio = splitmix64(S.seed ^ key);
    P.cons[idx] = c;
    scene_count(P, s, [&](int n) { atomicAdd((unsigned long long*)&P.ss[s].contacts, (unsigned long long)n); });
  }
}

// ---------------------------------------------------------------------------
// Order of the backward step's sweep (Sec. 4.3, readings R10 and R11):
// contacts, then edge-length constraints, each by descending priority
// splitmix64(seed ^ key).  Every constraint's rank among the constraints at
// each of its movable vertices is all the sweep needs: per-vertex incidence
// lists of the contacts are built each iteration (count, scan, scatter,
// rank); the ranks of the edge-length constraints depend on the topology
// only and are computed once per scene.
// ---------------------------------------------------------------------------
struct ContactAcc {
  const Contact* c;
  __device__ int4 verts(int i) const { return c[i].v; }
  __device__ unsigned long long prio(int i) const { return c[i].prio; }
};
struct ContactFAcc {
  const ContactF* c;
  __device__ int4 verts(int i) const { return c[i].v; }
  __device__ unsigned long long prio(int i) const { return c[i].prio; }
};

__device__ __forceinline__ bool movable(const Pool& P, int v) { return v >= 0 && (P.vflag[v] & VF_MOVABLE); }

// one more distinct movable vertex with a contact in this iteration (statistics)
__device__ __forceinline__ void count_contact_vertex(Pool& P, int s) {
  scene_count(P, s, [&](int n) { atomicAdd((unsigned long long*)&P.ss[s].cverts, (unsigned long long)n); });
}

template <class Acc>
__global__ void k_inc_count(Pool P, Acc acc, OrderBufs B) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int4 v = acc.verts(c);
    int vv[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < 4; k++)
      if (movable(P, vv[k])) atomicAdd(&B.vstart[vv[k]], 1);
  }
}

template <class Acc>
__global__ void k_inc_scatter(Pool P, Acc acc, OrderBufs B) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int4 v = acc.verts(c);
    unsigned long long p = acc.prio(c);
    int vv[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < 4; k++)
      if (movable(P, vv[k])) {
        int slot = B.vstart[vv[k]] + atomicAdd(&B.vfill[vv[k]], 1);
        B.iprio[slot] = p;
        B.iid[slot] = 4 * c + k;
      }
  }
}

// rank of each incidence at its vertex by descending priority (priorities
// are a bijection of the unique pair keys: no ties); the vertex with the most
// contacts is recorded for the statistics
template <class Acc>
__global__ void k_inc_rank(Pool P, Acc acc, OrderBufs B) {
  int total = B.vstart[P.nv];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
    int id = B.iid[s];
    int4 v = acc.verts(id >> 2);
    int vv[4] = {v.x, v.y, v.z, v.w};
    int vert = vv[id & 3];
    int a = B.vstart[vert], b = B.vstart[vert + 1];
    unsigned long long p = B.iprio[s];
    int r = 0;
    for (int t = a; t < b; t++) r += B.iprio[t] > p;
    B.rank[id] = r;
    if (r == 0) {
      atomicMax(&P.cnt->vcontacts, b - a);
      count_contact_vertex(P, P.vscene[vert]);
    }
  }
}

// Exclusive scan of m ints in place, in three launches: every block of 1024
// threads scans a tile of SCAN_TILE ints (8 per thread) and writes the tile's
// total, one block scans the totals, and every element adds its tile's
// offset.
constexpr int SCAN_TILE = 8192;
__global__ void __launch_bounds__(1024) k_scan_tiles(int* a, int m, int* tsum) {
  __shared__ int wtot[32];
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * 8;
  int v[8];
  if (base + 8 <= m) {
    int4 p = *(const int4*)(a + base), q = *(const int4*)(a + base + 4);
    v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
  } else {
    for (int k = 0; k < 8; k++) v[k] = base + k < m ? a[base + k] : 0;
  }
  int sum = 0;
  for (int k = 0; k < 8; k++) sum += v[k];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wtot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int t = wtot[lane], ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    wtot[lane] = ti - t;
  }
  __syncthreads();
  int run = wtot[w] + inc - sum;
  for (int k = 0; k < 8; k++) {
    if (base + k < m) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == blockDim.x - 1) tsum[blockIdx.x] = run;
}
__global__ void k_scan_add(int* a, int m, const int* tsum) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (i >= SCAN_TILE) a[i] += tsum[i / SCAN_TILE];
}

// exclusive scan of m ints, in place, one block of 1024 threads
__global__ void k_scan_ints(int* a, int m) {
  __shared__ int part[1024];
  int per = (m + 1023) / 1024;
  int lo = threadIdx.x * per, hi = min(lo + per, m);
  int sum = 0;
  for (int i = lo; i < hi; i++) sum += a[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = lo; i < hi; i++) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
}

static void scan_ints(Runtime& R, int* a, int m, cudaStream_t st) {
  int tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<tiles, 1024, 0, st>>>(a, m, R.obuf.tsum);
  k_scan_ints<<<1, 1024, 0, st>>>(R.obuf.tsum, tiles);
  k_scan_add<<<grid_for(m, 256), 256, 0, st>>>(a, m, R.obuf.tsum);
  R.launches += 2;  // the third is counted with the caller's kernels
}

// ---------------------------------------------------------------------------
// Backward step: projected Gauss-Seidel (Eq. LCP), one constraint at a time.
// y is read and written through L2 (ld.cg / st.cg): a constraint applied on
// one SM is seen by the next constraint at the same vertex on another.
// ---------------------------------------------------------------------------
__device__ __forceinline__ dv3 ldy(const Pool& P, int v) {
  const double* p = (const double*)(P.y + v);
  return {__ldcg(p), __ldcg(p + 1), __ldcg(p + 2)};
}
__device__ __forceinline__ void sty(Pool& P, int v, dv3 a) {
  double* p = (double*)(P.y + v);
  __stcg(p, a.x);
  __stcg(p + 1, a.y);
  __stcg(p + 2, a.z);
}

// One projected Gauss-Seidel update of a contact (FP64) or edge-length
// constraint.  The vertex ids come from the caller, so that every load the
// update needs (y, x, the constraint record) is issued at once; the
// arithmetic is the same sequence as the oracle's.  lam: multipliers when
// gs_sweeps > 1 (zero at the first sweep).
__device__ __forceinline__ void pgs_contact(Pool& P, int ci, const int* vid, double* lam, bool first) {
  const Contact& c = P.cons[ci];
  int nv = vid[2] < 0 ? 2 : 4;
  dv3 yv[4], xv[4];
  for (int k = 0; k < nv; k++) {
    yv[k] = ldy(P, vid[k]);
    xv[k] = mk(P.x[vid[k]]);
  }
  double den = c.den, w = c.c0;
  if (!(den > 0.0)) return;
  for (int k = 0; k < nv; k++) {
    dv3 g = {c.g[3 * k], c.g[3 * k + 1], c.g[3 * k + 2]};
    w = w + vdot(g, vsub(yv[k], xv[k]));
  }
  double l0 = lam && !first ? lam[ci] : 0.0;
  double tl = l0 - w / den;
  double ln = tl > 0.0 ? tl : 0.0;
  double dl = ln - l0;
  if (lam) lam[ci] = ln;
  if (dl == 0.0) return;
  for (int k = 0; k < nv; k++) {
    double sc = P.im[vid[k]] * dl;
    dv3 g = {c.g[3 * k], c.g[3 * k + 1], c.g[3 * k + 2]};
    sty(P, vid[k], vadd(yv[k], vscl(sc, g)));
  }
}

// mixed precision: the same updates in FP32 on the float copy of y
__device__ __forceinline__ float4 ldyf(const Pool& P, int v) { return __ldcg(P.yf + v); }
__device__ __forceinline__ void pgs_contact_f(Pool& P, int ci, const int* vid, double* lam, bool first) {
  const ContactF& c = ((const ContactF*)P.cons)[ci];
  int nv = vid[2] < 0 ? 2 : 4;
  float4 yv[4], xv[4];
  for (int k = 0; k < nv; k++) {
    yv[k] = ldyf(P, vid[k]);
    xv[k] = P.xf[vid[k]];
  }
  float den = c.den, w = c.c0;
  if (!(den > 0.f)) return;
  for (int k = 0; k < nv; k++)
    w = w + (c.g[3 * k] * (yv[k].x - xv[k].x) + c.g[3 * k + 1] * (yv[k].y - xv[k].y) +
             c.g[3 * k + 2] * (yv[k].z - xv[k].z));
  float l0 = lam && !first ? (float)lam[ci] : 0.f;
  float tl = l0 - w / den;
  float ln = tl > 0.f ? tl : 0.f;
  float dl = ln - l0;
  if (lam) lam[ci] = ln;
  if (dl == 0.f) return;
  for (int k = 0; k < nv; k++) {
    float sc = (float)P.im[vid[k]] * dl;
    float4 o = make_float4(yv[k].x + sc * c.g[3 * k], yv[k].y + sc * c.g[3 * k + 1], yv[k].z + sc * c.g[3 * k + 2], 0.f);
    __stcg(P.yf + vid[k], o);
  }
}
__device__ __forceinline__ void pgs_edge_f(Pool& P, int e, int i, int j, double* lam, bool first) {
  float4 gd = P.lgf[e];
  float4 yi = ldyf(P, i), yj = ldyf(P, j);
  float sigma = (float)P.sd[P.vscene[i]].sigma;
  if (!(gd.w > 0.f)) return;
  float w = sigma - (gd.x * (yi.x - yj.x) + gd.y * (yi.y - yj.y) + gd.z * (yi.z - yj.z));
  float l0 = lam && !first ? (float)lam[e] : 0.f;
  float tl = l0 - w / gd.w;
  float ln = tl > 0.f ? tl : 0.f;
  float dl = ln - l0;
  if (lam) lam[e] = ln;
  if (dl == 0.f) return;
  float si = (float)P.im[i] * dl, sj = (float)P.im[j] * dl;
  __stcg(P.yf + i, make_float4(yi.x - si * gd.x, yi.y - si * gd.y, yi.z - si * gd.z, 0.f));
  __stcg(P.yf + j, make_float4(yj.x + sj * gd.x, yj.y + sj * gd.y, yj.z + sj * gd.z, 0.f));
}

__device__ __forceinline__ void pgs_edge(Pool& P, int e, int i, int j, double* lam, bool first) {
  P4 gd = P.lg[e];
  dv3 yi = ldy(P, i), yj = ldy(P, j);
  double sigma = P.sd[P.vscene[i]].sigma;
  if (!(gd.w > 0.0)) return;
  dv3 g = {gd.x, gd.y, gd.z};
  double w = sigma - vdot(g, vsub(yi, yj));
  double l0 = lam && !first ? lam[e] : 0.0;
  double tl = l0 - w / gd.w;
  double ln = tl > 0.0 ? tl : 0.0;
  double dl = ln - l0;
  if (lam) lam[e] = ln;
  if (dl == 0.0) return;
  double si = P.im[i] * dl, sj = P.im[j] * dl;
  sty(P, i, vsub(yi, vscl(si, g)));
  sty(P, j, vadd(yj, vscl(sj, g)));
}

// ---------------------------------------------------------------------------
// Multi-colour Gauss-Seidel (Sec. 4.3, readings R10 and R11).  The
// constraints are split into colour classes of the greedy colouring in
// descending priority: each constraint takes the smallest colour not used by
// a higher-priority constraint sharing a movable vertex with it.  Contacts
// are coloured among themselves every iteration (k_colour, below), the
// edge-length constraints once per scene (on the host, from the topology).
// The sweep then applies the contact classes in ascending colour, then the
// edge classes, one class per phase of a persistent kernel, with a grid
// barrier between phases; the constraints of one class share no movable
// vertex, so the result equals the sequential sweep in that order bit for
// bit.
//
// The colouring itself is a dataflow over per-vertex counters: a contact is
// coloured once the counter of every one of its movable vertices (contacts
// coloured there so far) equals its rank at that vertex by priority.  It then
// reads the colours already used at those vertices from per-vertex bit masks,
// takes the smallest free one, records it in the masks and increments the
// counters.  Contacts that share no movable vertex do not wait for each
// other, so the colours equal the sequential greedy colouring.
// ---------------------------------------------------------------------------
constexpr int CW = 32;                  // 64-bit mask words per vertex
constexpr int MAX_COLOURS = 64 * CW;    // colours one iteration may use

// the vertices an item waits on and the counter values it waits for
struct ItemWait {
  int v[4];
  int t[4];  // -1: no wait (vertex absent or not movable); else the rank
};
__device__ __forceinline__ void contact_wait(const Pool& P, const OrderBufs& B, int i, ItemWait& w) {
  int4 v = P.mixed ? ((const ContactF*)P.cons)[i].v : P.cons[i].v;
  w.v[0] = v.x; w.v[1] = v.y; w.v[2] = v.z; w.v[3] = v.w;
  for (int k = 0; k < 4; k++) w.t[k] = movable(P, w.v[k]) ? __ldg(&B.rank[4 * i + k]) : -1;
}
// Synchronisation at GPU scope: counters are polled with acquire loads, so
// the loads that find an item ready also make its predecessors' writes
// visible; after the item's own writes, one release fence precedes relaxed
// increments of its counters.  (A release on each increment costs one fence
// per vertex.)
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_relaxed_add(int* p, int v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// contacts still to be coloured at the item's vertices before it (0: ready)
__device__ __forceinline__ int item_gap(const OrderBufs& B, const ItemWait& w) {
  int gap = 0;
  for (int k = 0; k < 4; k++)
    if (w.t[k] >= 0) gap = max(gap, w.t[k] - ld_acquire(&B.vdone[w.v[k]]));
  return gap;
}

// Colours contact i (its turn has come at every movable vertex): the
// smallest colour absent from the masks of its movable vertices.  A vertex at
// which i is the first contact (rank 0) has an empty set; its mask words are
// rewritten rather than read (they hold an earlier iteration's colours).
__device__ __forceinline__ void colour_apply(Pool& P, const OrderBufs& B, int i, const ItemWait& w, int& maxcol) {
  // (the acquire loads that found the item ready order the reads below)
  // the words in use and the first four mask words (256 colours) of every
  // movable vertex, all loaded at once; later words only when those are full
  int hw[4];
  ulonglong2 w01[4], w23[4];
  for (int k = 0; k < 4; k++) {
    hw[k] = 0;
    w01[k] = w23[k] = make_ulonglong2(0ULL, 0ULL);
    if (w.t[k] > 0) {
      const unsigned long long* mk = P.cmask + (size_t)w.v[k] * CW;
      hw[k] = __ldcg(&P.chw[w.v[k]]);
      w01[k] = __ldcg((const ulonglong2*)mk);
      w23[k] = __ldcg((const ulonglong2*)(mk + 2));
    }
  }
  unsigned long long m4[4] = {0ULL, 0ULL, 0ULL, 0ULL};
  for (int k = 0; k < 4; k++) {
    if (hw[k] > 0) m4[0] |= w01[k].x;
    if (hw[k] > 1) m4[1] |= w01[k].y;
    if (hw[k] > 2) m4[2] |= w23[k].x;
    if (hw[k] > 3) m4[3] |= w23[k].y;
  }
  int col = -1;
  for (int wd = 0; wd < 4 && col < 0; wd++)
    if (m4[wd] != ~0ULL) col = wd * 64 + __ffsll((long long)~m4[wd]) - 1;
  for (int wd = 4; wd < CW && col < 0; wd++) {
    unsigned long long m = 0ULL;
    for (int k = 0; k < 4; k++)
      if (wd < hw[k]) m |= __ldcg(&P.cmask[(size_t)w.v[k] * CW + wd]);
    if (m != ~0ULL) col = wd * 64 + __ffsll((long long)~m) - 1;
  }
  if (col < 0) {  // more than MAX_COLOURS colours at these vertices
    atomicOr(&P.cnt->err, ERR_COLOURS);
    col = MAX_COLOURS - 1;
  }
  int wd = col >> 6;
  unsigned long long bit = 1ULL << (col & 63);
  for (int k = 0; k < 4; k++) {
    if (w.t[k] < 0) continue;
    unsigned long long* mk = P.cmask + (size_t)w.v[k] * CW;
    if (wd < hw[k]) {
      __stcg(mk + wd, __ldcg(mk + wd) | bit);
    } else {
      for (int z = hw[k]; z < wd; z++) __stcg(mk + z, 0ULL);
      __stcg(mk + wd, bit);
      __stcg(&P.chw[w.v[k]], wd + 1);
    }
  }
  P.ccol[i] = col;
  maxcol = max(maxcol, col + 1);
  fence_acq_rel();
  for (int k = 0; k < 4; k++)
    if (w.t[k] >= 0) red_relaxed_add(&B.vdone[w.v[k]], 1);
}

__device__ __forceinline__ unsigned long long contact_prio(const Pool& P, int i) {
  return P.mixed ? ((const ContactF*)P.cons)[i].prio : P.cons[i].prio;
}

// All blocks are resident (cooperative launch).  Each thread takes up to 32
// contacts (i = tid + k * nth), sorts them by descending priority and colours
// them one after the other, waiting before each only for its own vertex
// counters.  The highest-priority uncoloured contact of the whole pool is at
// the head of its thread's list and ready, so the colouring always
// progresses.  With more contacts than 32 per thread, every thread polls all
// of its pending contacts each round instead.  Waits are bounded and set
// ERR_POLL past the bound.
__global__ void __launch_bounds__(256, 2) k_colour(Pool P, OrderBufs B, int max_polls) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  int maxcol = 0;
  long long polls = 0;
  if (n <= 32 * nth) {
    int items[32];
    unsigned long long keys[32];
    int m = 0;
    for (int i = tid; i < n; i += nth) {
      unsigned long long key = ~contact_prio(P, i);
      int j = m++;
      while (j > 0 && keys[j - 1] > key) {
        items[j] = items[j - 1];
        keys[j] = keys[j - 1];
        j--;
      }
      items[j] = i;
      keys[j] = key;
    }
    // The lanes of a warp advance together: each round every lane checks
    // its head item; the lanes whose head is ready colour it, and the warp
    // sleeps only when none is (a lane spinning alone would take issue
    // slots from a lane of its warp that could proceed).  The sleep grows
    // by about a microsecond per contact still ahead of the nearest head
    // item (each of them is at least one dependent hop away), so that
    // far-from-ready warps do not crowd L2 with counter loads.
    int j = 0;
    ItemWait w;
    bool has = m > 0;
    if (has) contact_wait(P, B, items[0], w);
    while (__any_sync(0xffffffffu, has)) {
      int gap = has ? item_gap(B, w) : 1 << 30;
      bool ready = has && gap == 0;
      if (__any_sync(0xffffffffu, ready)) {
        if (ready) {
          colour_apply(P, B, items[j], w, maxcol);
          has = ++j < m;
          if (has) contact_wait(P, B, items[j], w);
        }
        continue;
      }
      if (++polls > max_polls) {  // the same count in every lane
        if ((threadIdx.x & 31) == 0) atomicOr(&P.cnt->err, ERR_POLL);
        break;
      }
      int g = __reduce_min_sync(0xffffffffu, gap);
      __nanosleep(min(32 + 1024 * (g - 1), 8192));
    }
  } else {
    // more contacts than that: poll every pending one each round
    for (;;) {
      bool pending = false, progressed = false;
      for (int i = tid; i < n; i += nth) {
        if (P.fdone[i]) continue;
        ItemWait w;
        contact_wait(P, B, i, w);
        if (item_gap(B, w) == 0) {
          colour_apply(P, B, i, w, maxcol);
          P.fdone[i] = 1;
          progressed = true;
        } else {
          pending = true;
        }
      }
      if (!pending) break;
      if (!progressed) {
        if (++polls > max_polls) {
          atomicOr(&P.cnt->err, ERR_POLL);
          break;
        }
        __nanosleep(32);
      }
    }
  }
  unsigned mx = __reduce_max_sync(0xffffffffu, (unsigned)maxcol);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&P.cnt->n_ccol, (int)mx);
}

// per-scene colour counts of the iteration (statistics), aggregated per warp
// and the number of contacts of each colour (a block histogram in shared
// memory, added to ccount; the sweep sizes its single-block tail from it)
__global__ void __launch_bounds__(256) k_colour_stats(Pool P) {
  __shared__ int hist[MAX_COLOURS];
  for (int c = threadIdx.x; c < MAX_COLOURS; c += blockDim.x) hist[c] = 0;
  __syncthreads();
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 v = P.mixed ? ((const ContactF*)P.cons)[i].v : P.cons[i].v;
    int s = P.vscene[v.x];
    int c = P.ccol[i];
    scene_reduce(P, s, c + 1, cg::greater<int>(), [&](int m, int) { atomicMax(&P.ss[s].ccol, m); });
    if ((unsigned)c < (unsigned)MAX_COLOURS) atomicAdd(&hist[c], 1);
  }
  __syncthreads();
  int ncc = min(P.cnt->n_ccol, MAX_COLOURS);
  for (int c = threadIdx.x; c < ncc; c += blockDim.x)
    if (hist[c]) atomicAdd(&P.ccount[c], hist[c]);
}

// Grid barrier of a cooperative launch (every block resident): one arrival
// counter, zeroed before the launch.  Each block adds one per barrier, so the
// k-th barrier is passed once the counter reaches k * gridDim.x; a block
// polls it at most max_polls times, after which the wait sets ERR_POLL, and
// leaves a wait once another block has given up.  Returns false when the
// barrier failed; the caller then returns.  The release fence before the
// arrival publishes the block's writes (ordered before thread 0 by the block
// barrier); a waiting block acquires them through the load that sees the
// count, which the later arrivals' additions carry forward.
__device__ __forceinline__ bool grid_barrier(Pool& P, unsigned& target, int max_polls) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    target += gridDim.x;
    fence_acq_rel();
    red_relaxed_add((int*)P.bar, 1);
    long long polls = 0;
    while ((int)(ld_acquire_u32(P.bar) - target) < 0) {
      if (++polls > max_polls || ((polls & 255) == 0 && (ld_relaxed(&P.cnt->err) & ERR_POLL))) {
        atomicOr(&P.cnt->err, ERR_POLL);
        ok = 0;
        break;
      }
      __nanosleep(16);
    }
  }
  __syncthreads();
  return ok != 0;
}

// the edge-length constraints of scenes that are not running take no part
__device__ __forceinline__ bool edge_live(const Pool& P, int e) {
  const SceneState& S = P.ss[P.lv[e].z];
  return S.active && !S.done;
}

// ---------------------------------------------------------------------------
// Multi-colour Gauss-Seidel with the level colouring (R11, colouring = 1):
// a constraint's colour is one more than the largest colour among the
// higher-priority constraints sharing a movable vertex with it, the round in
// which its priority first exceeds that of all its uncoloured conflicting
// constraints.  Conflicting constraints are then applied in priority order,
// so sweeping the classes in ascending colour is the sequential sweep in
// descending priority, and no colouring pass is needed: this kernel applies
// each constraint once the counter of every one of its movable vertices
// (constraints applied there so far) equals its rank there by priority, and
// then increments those counters.  Constraints that share no movable vertex
// commute, so the result is exactly the sequential sweep.  Sweep s of
// gs_sweeps starts at counter s * (constraints at the vertex), so counters
// need no reset between sweeps.  In the first sweep each contact records its
// colour (its chain length at its vertices) for the statistics.
//
// All blocks are resident (cooperative launch).  Each thread takes up to 32
// constraints (i = tid + k * nth), sorts them into the sweep order and
// applies them one after the other, waiting before each only for its own
// vertex counters.  The earliest pending constraint of the whole sweep is at
// the head of its thread's list and is ready, so the sweep always progresses.
// With more constraints than 32 per thread, every thread polls all of its
// pending constraints each round instead.  Waits are bounded and set
// ERR_POLL past the bound.
// ---------------------------------------------------------------------------
struct LevelCtx {
  int nc;          // contacts (items [0, nc)); edge-length constraints follow
  int sweep;
  double* lam;     // contact multipliers (gs_sweeps > 1), else null
  double* elam;    // edge multipliers
  bool dataflow;   // level sweep: record levels (first sweep) and advance the vertex counters
};

__device__ __forceinline__ int contacts_at(const OrderBufs& B, int v) {
  return __ldg(&B.vstart[v + 1]) - __ldg(&B.vstart[v]);
}
// counter value at which a constraint of rank r among the contacts (edge:
// among the edges) of v may be applied in sweep s
__device__ __forceinline__ int target_at(const Pool& P, const OrderBufs& B, int v, int s, int r, bool edge) {
  int nct = contacts_at(B, v);
  return s * (nct + __ldg(&P.edeg[v])) + (edge ? nct : 0) + r;
}
__device__ __forceinline__ void level_wait(const Pool& P, const OrderBufs& B, const LevelCtx& X, int i, ItemWait& w) {
  if (i < X.nc) {
    int4 v = P.mixed ? ((const ContactF*)P.cons)[i].v : P.cons[i].v;
    w.v[0] = v.x; w.v[1] = v.y; w.v[2] = v.z; w.v[3] = v.w;
    for (int k = 0; k < 4; k++)
      w.t[k] = movable(P, w.v[k]) ? target_at(P, B, w.v[k], X.sweep, __ldg(&B.rank[4 * i + k]), false) : -1;
  } else {
    int e = i - X.nc;
    int4 l = P.lv[e];
    int2 r = __ldg(&P.erank[e]);
    w.v[0] = l.x; w.v[1] = l.y; w.v[2] = w.v[3] = -1;
    w.t[0] = movable(P, l.x) ? target_at(P, B, l.x, X.sweep, r.x, true) : -1;
    w.t[1] = movable(P, l.y) ? target_at(P, B, l.y, X.sweep, r.y, true) : -1;
    w.t[2] = w.t[3] = -1;
  }
}
// (the acquire loads of item_gap that found the item ready order its reads)
__device__ __forceinline__ void level_apply(Pool& P, const OrderBufs& B, const LevelCtx& X, int i,
                                            const ItemWait& w) {
  bool first = X.sweep == 0;
  int lvl = 0;
  if (first && i < X.nc) {
    for (int k = 0; k < 4; k++)
      if (w.t[k] >= 0) lvl = max(lvl, __ldcg(&P.vlevel[w.v[k]]) + 1);
    P.ccol[i] = lvl;
  }
  if (i < X.nc) {
    if (P.mixed) pgs_contact_f(P, i, w.v, X.lam, first);
    else pgs_contact(P, i, w.v, X.lam, first);
  } else {
    if (P.mixed) pgs_edge_f(P, i - X.nc, w.v[0], w.v[1], X.elam, first);
    else pgs_edge(P, i - X.nc, w.v[0], w.v[1], X.elam, first);
  }
  if (first && i < X.nc)
    for (int k = 0; k < 4; k++)
      if (w.t[k] >= 0) __stcg(&P.vlevel[w.v[k]], lvl);
  fence_acq_rel();
  for (int k = 0; k < 4; k++)
    if (w.t[k] >= 0) red_relaxed_add(&B.vdone[w.v[k]], 1);
}

// edge-length constraints of scenes that are not running take no part
__device__ __forceinline__ bool level_live(const Pool& P, const LevelCtx& X, int i) {
  if (i < X.nc) return true;
  return edge_live(P, i - X.nc);
}
// sweep-order key: contacts (class 0) before edges (class 1), then
// descending priority; compared as (class, ~prio) ascending
__device__ __forceinline__ unsigned long long level_prio(const Pool& P, const LevelCtx& X, int i) {
  if (i < X.nc) return contact_prio(P, i);
  int e = i - X.nc;
  const SceneDesc& d = P.sd[P.lv[e].z];
  return splitmix64(d.seed ^ ((3ULL << 62) | (unsigned long long)(e - d.l0)));
}

// Quad form of the FP64 sweep.  FP64 runs at 2 lanes per cycle per SM on
// this part and a warp instruction holds the pipe for all 32 lanes, active or
// not, so a thread applying a 4-vertex contact alone (about 75 FP64
// instructions, most lanes of its warp idle) makes the dependent chain long.
// Here four lanes share one list and apply its head together: lane k owns
// vertex k of the head constraint, polls that vertex's counter, loads its y,
// x and gradient block, and computes its term g_k.(y_k - x_k); the quad
// gathers the four terms and every lane forms w = (((c0 + t0) + t1) + t2) + t3,
// the same sum in the same order as pgs_contact, then updates its own vertex.
// Each lane's arithmetic is that of pgs_contact for its vertex, so the result
// is bit for bit the same, at about 30 FP64 instructions per constraint.  An
// edge-length constraint is applied by lanes 0 and 1 (vertices i and j).
//
// A quad's list is split over its lanes: lane k takes items
// q + nq * (k + 4 m) and sorts them; the quad's head is the first of the
// four lanes' heads in the sweep order (contacts, then edges, by descending
// priority, ties by index), found with two shuffles.  The quad applies its
// head once the head's counters are ready, as the thread form below does.
constexpr int NO_ITEM = 0x7fffffff;  // an exhausted list's head
__device__ __forceinline__ bool sweep_before(int ia, unsigned long long ka, int ib, unsigned long long kb, int nc) {
  bool ea = ia >= nc, eb = ib >= nc;
  if (ea != eb) return eb;
  if (ka != kb) return ka < kb;
  return ia < ib;
}
__device__ __forceinline__ int quad_head(unsigned mask, int item, unsigned long long key, int nc) {
  for (int o = 1; o <= 2; o <<= 1) {
    int io = __shfl_xor_sync(mask, item, o);
    unsigned long long ko = __shfl_xor_sync(mask, key, o);
    if (sweep_before(io, ko, item, key, nc)) {
      item = io;
      key = ko;
    }
  }
  return item;
}
// lane lk's vertex of item i and the counter value it waits for (-1: none)
__device__ __forceinline__ void quad_vertex(const Pool& P, const OrderBufs& B, const LevelCtx& X, int i, int lk,
                                            int& vk, int& tk) {
  vk = -1;
  tk = -1;
  if (i < X.nc) {
    int4 v = P.cons[i].v;
    vk = lk == 0 ? v.x : lk == 1 ? v.y : lk == 2 ? v.z : v.w;
    if (movable(P, vk)) tk = target_at(P, B, vk, X.sweep, __ldg(&B.rank[4 * i + lk]), false);
  } else if (lk < 2) {
    int e = i - X.nc;
    int4 l = P.lv[e];
    int2 r = __ldg(&P.erank[e]);
    vk = lk == 0 ? l.x : l.y;
    if (movable(P, vk)) tk = target_at(P, B, vk, X.sweep, lk == 0 ? r.x : r.y, true);
  }
}
// contact ci, applied by the quads of `mask` (all four lanes of each)
__device__ __forceinline__ void quad_contact(Pool& P, OrderBufs& B, const LevelCtx& X, unsigned mask, int ci, int lk,
                                             int vk, int tk) {
  const Contact& c = P.cons[ci];
  bool first = X.sweep == 0, rec = first && X.dataflow;
  dv3 yk = {0.0, 0.0, 0.0}, gk = yk;
  double tkm = 0.0;
  if (vk >= 0) {
    yk = ldy(P, vk);
    dv3 xk = mk(P.x[vk]);
    gk = {c.g[3 * lk], c.g[3 * lk + 1], c.g[3 * lk + 2]};
    tkm = vdot(gk, vsub(yk, xk));
  }
  int lv = rec && tk >= 0 ? __ldcg(&P.vlevel[vk]) + 1 : 0;
  int base = (threadIdx.x & 31) & ~3;
  double t[4];
  for (int k = 0; k < 4; k++) t[k] = __shfl_sync(mask, tkm, base + k);
  lv = max(lv, __shfl_xor_sync(mask, lv, 1));
  lv = max(lv, __shfl_xor_sync(mask, lv, 2));
  double den = c.den, w = c.c0;
  if (den > 0.0) {
    int nv = c.v.z < 0 ? 2 : 4;
    for (int k = 0; k < nv; k++) w = w + t[k];
    double l0 = X.lam && !first ? X.lam[ci] : 0.0;
    double tl = l0 - w / den;
    double ln = tl > 0.0 ? tl : 0.0;
    double dl = ln - l0;
    if (X.lam && lk == 0) X.lam[ci] = ln;
    if (dl != 0.0 && vk >= 0) {
      double sc = P.im[vk] * dl;
      sty(P, vk, vadd(yk, vscl(sc, gk)));
    }
  }
  if (!X.dataflow) return;
  if (rec) {
    if (lk == 0) P.ccol[ci] = lv;
    if (tk >= 0) __stcg(&P.vlevel[vk], lv);
  }
  fence_acq_rel();
  if (tk >= 0) red_relaxed_add(&B.vdone[vk], 1);
}
// edge-length constraint e, applied by lanes 0 (vertex i) and 1 (vertex j)
__device__ __forceinline__ void quad_edge(Pool& P, OrderBufs& B, const LevelCtx& X, int e, int lk, int vk, int tk) {
  if (lk < 2) {
    P4 gd = P.lg[e];
    int4 l = P.lv[e];
    dv3 yi = ldy(P, l.x), yj = ldy(P, l.y);
    double sigma = P.sd[P.vscene[l.x]].sigma;
    if (gd.w > 0.0) {
      dv3 g = {gd.x, gd.y, gd.z};
      double w = sigma - vdot(g, vsub(yi, yj));
      double l0 = X.elam && X.sweep != 0 ? X.elam[e] : 0.0;
      double tl = l0 - w / gd.w;
      double ln = tl > 0.0 ? tl : 0.0;
      double dl = ln - l0;
      if (X.elam && lk == 0) X.elam[e] = ln;
      if (dl != 0.0) {
        if (lk == 0) sty(P, l.x, vsub(yi, vscl(P.im[l.x] * dl, g)));
        else sty(P, l.y, vadd(yj, vscl(P.im[l.y] * dl, g)));
      }
    }
  }
  fence_acq_rel();
  if (tk >= 0) red_relaxed_add(&B.vdone[vk], 1);
}

__global__ void __launch_bounds__(256, 2) k_level_sweep(Pool P, OrderBufs B, int sweep, int sweeps, int max_polls) {
  LevelCtx X;
  X.nc = min(P.cnt->n_cons, P.cons_cap);
  X.sweep = sweep;
  X.dataflow = true;
  X.lam = sweeps > 1 ? P.lam : nullptr;
  X.elam = X.lam ? P.lam + P.cons_cap : nullptr;
  int n = X.nc + P.nl;
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  long long polls = 0;
  if (!P.mixed && n <= 32 * nth) {
    const unsigned FULL = 0xffffffffu;
    int lk = threadIdx.x & 3, nq = nth >> 2, q = tid >> 2;
    // this lane's share of its quad's items in sweep order (at most 32)
    int items[32];
    unsigned long long keys[32];
    int m = 0;
    for (int i = q + nq * lk; i < n; i += 4 * nq) {
      if (!level_live(P, X, i)) continue;
      unsigned long long key = ~level_prio(P, X, i);
      int j = m++;
      while (j > 0 && sweep_before(i, key, items[j - 1], keys[j - 1], X.nc)) {
        items[j] = items[j - 1];
        keys[j] = keys[j - 1];
        j--;
      }
      items[j] = i;
      keys[j] = key;
    }
    int j = 0;
    int cur = quad_head(FULL, m > 0 ? items[0] : NO_ITEM, m > 0 ? keys[0] : ~0ULL, X.nc);
    int vk = -1, tk = -1;
    if (cur != NO_ITEM) quad_vertex(P, B, X, cur, lk, vk, tk);
    // as below: the quads of a warp advance together and the warp sleeps
    // only when no quad's head is ready.  (Polling several items per quad
    // instead of the head only was measured slower: more counter loads per
    // round, and the head is the item the sweep waits for.)
    while (__any_sync(FULL, cur != NO_ITEM)) {
      bool has = cur != NO_ITEM;
      int gap = has && tk >= 0 ? tk - ld_acquire(&B.vdone[vk]) : 0;
      gap = max(gap, __shfl_xor_sync(FULL, gap, 1));
      gap = max(gap, __shfl_xor_sync(FULL, gap, 2));
      if (!has) gap = 1 << 30;
      bool ready = has && gap == 0;
      unsigned cm = __ballot_sync(FULL, ready && cur < X.nc);
      unsigned em = __ballot_sync(FULL, ready && cur >= X.nc);
      if (cm | em) {
        if (ready) {
          if (cur < X.nc) quad_contact(P, B, X, cm, cur, lk, vk, tk);
          else quad_edge(P, B, X, cur - X.nc, lk, vk, tk);
          if (j < m && items[j] == cur) j++;  // the lane that held the head
          cur = quad_head(cm | em, j < m ? items[j] : NO_ITEM, j < m ? keys[j] : ~0ULL, X.nc);
          vk = tk = -1;
          if (cur != NO_ITEM) quad_vertex(P, B, X, cur, lk, vk, tk);
        }
        continue;
      }
      if (++polls > max_polls) {  // the same count in every lane
        if ((threadIdx.x & 31) == 0) atomicOr(&P.cnt->err, ERR_POLL);
        break;
      }
      int g = __reduce_min_sync(FULL, gap);
      __nanosleep(min(32 + 1024 * (g - 1), 8192));
    }
  } else if (n <= 32 * nth) {
    // this thread's items in sweep order (insertion sort, at most 32)
    int items[32];
    unsigned long long keys[32];
    int m = 0;
    for (int i = tid; i < n; i += nth) {
      if (!level_live(P, X, i)) continue;
      unsigned long long key = ~level_prio(P, X, i);
      bool edge = i >= X.nc;
      int j = m++;
      while (j > 0 && ((items[j - 1] >= X.nc) > edge || ((items[j - 1] >= X.nc) == edge && keys[j - 1] > key))) {
        items[j] = items[j - 1];
        keys[j] = keys[j - 1];
        j--;
      }
      items[j] = i;
      keys[j] = key;
    }
    // The lanes of a warp advance together: each round every lane checks
    // its head item; the lanes whose head is ready apply it, and the warp
    // sleeps only when none is.  The sleep grows by about a microsecond per
    // constraint still ahead of the nearest head item (each is at least one
    // dependent hop away), so that far-from-ready warps do not crowd L2 with
    // counter loads.
    int j = 0;
    ItemWait w;
    bool has = m > 0;
    if (has) level_wait(P, B, X, items[0], w);
    while (__any_sync(0xffffffffu, has)) {
      int gap = has ? item_gap(B, w) : 1 << 30;
      bool ready = has && gap == 0;
      if (__any_sync(0xffffffffu, ready)) {
        if (ready) {
          level_apply(P, B, X, items[j], w);
          has = ++j < m;
          if (has) level_wait(P, B, X, items[j], w);
        }
        continue;
      }
      if (++polls > max_polls) {  // the same count in every lane
        if ((threadIdx.x & 31) == 0) atomicOr(&P.cnt->err, ERR_POLL);
        break;
      }
      int g = __reduce_min_sync(0xffffffffu, gap);
      __nanosleep(min(32 + 1024 * (g - 1), 8192));
    }
  } else {
    // more items than that: poll every pending item each round
    for (;;) {
      bool pending = false, progressed = false;
      for (int i = tid; i < n; i += nth) {
        if (P.fdone[i] || !level_live(P, X, i)) continue;
        ItemWait w;
        level_wait(P, B, X, i, w);
        if (item_gap(B, w) == 0) {
          level_apply(P, B, X, i, w);
          P.fdone[i] = 1;
          progressed = true;
        } else {
          pending = true;
        }
      }
      if (!pending) break;
      if (!progressed) {
        if (++polls > max_polls) {
          atomicOr(&P.cnt->err, ERR_POLL);
          break;
        }
        __nanosleep(32);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Colour-class sweep of the greedy colouring (colouring = 0).  k_colour_order
// groups the contacts by colour (a counting sort on the histogram of
// k_colour_stats; the order within a colour is immaterial, its contacts share
// no movable vertex); the edge-length constraints were grouped once on the
// host.  k_colour_sweep then applies, gs_sweeps times, the contact classes
// in ascending colour and then the edge classes, one class per phase of a
// persistent kernel with a grid barrier after each.  A class's contacts are
// contiguous, so its work spreads over the fewest warps: in FP64 a quad of
// lanes applies each contact (quad_contact, bit for bit pgs_contact), in
// mixed precision one thread each; edges take one thread each.  The last
// contact classes are small: from the first class after which at most
// TAIL_MAX contacts remain, block 0 alone applies the rest, separated by block
// barriers only, while the other blocks wait at the next grid barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apply_contact(Pool& P, const LevelCtx& X, int i) {
  int4 v = ((const ContactF*)P.cons)[i].v;
  int vid[4] = {v.x, v.y, v.z, v.w};
  pgs_contact_f(P, i, vid, X.lam, X.sweep == 0);
}
__device__ __forceinline__ void apply_edge(Pool& P, const LevelCtx& X, int e) {
  int4 l = P.lv[e];
  if (P.mixed) pgs_edge_f(P, e, l.x, l.y, X.elam, X.sweep == 0);
  else pgs_edge(P, e, l.x, l.y, X.elam, X.sweep == 0);
}
// exclusive prefix of ccount[0, ncc) into off[0, ncc] (one block)
__device__ __forceinline__ void colour_offsets(const Pool& P, int ncc, int* off) {
  __shared__ int part[256];
  int per = (ncc + blockDim.x - 1) / blockDim.x, a = threadIdx.x * per, sum = 0;
  for (int c = a; c < min(a + per, ncc); c++) sum += P.ccount[c];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < (int)blockDim.x; t++) {
      int v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int c = a; c < min(a + per, ncc); c++) {
    off[c] = run;
    run += P.ccount[c];
  }
  if (threadIdx.x == blockDim.x - 1) off[ncc] = run;
  __syncthreads();
}
__global__ void __launch_bounds__(256) k_colour_order(Pool P) {
  __shared__ int off[MAX_COLOURS + 1];
  int ncc = min(P.cnt->n_ccol, MAX_COLOURS);
  colour_offsets(P, ncc, off);
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c <= ncc; c += blockDim.x) P.coff[c] = off[c];
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = P.ccol[i];
    if ((unsigned)c < (unsigned)ncc) P.corder[off[c] + atomicAdd(&P.cfill[c], 1)] = i;
  }
}

constexpr int TAIL_MAX = 2048;
// contacts [a, b) of corder, applied by `quads` quads (quad q of them is this lane's)
__device__ __forceinline__ void colour_class(Pool& P, OrderBufs& B, const LevelCtx& X, int a, int b, int q, int quads,
                                             int th, int threads) {
  if (P.mixed) {
    for (int k = a + th; k < b; k += threads) apply_contact(P, X, __ldg(&P.corder[k]));
    return;
  }
  int lk = threadIdx.x & 3;
  for (int base = a; base < b; base += quads) {  // the same trip count in every lane
    int k = base + q;
    int ci = k < b ? __ldcg(&P.corder[k]) : -1;
    unsigned cm = __ballot_sync(0xffffffffu, ci >= 0);
    if (ci >= 0) {
      int4 v = P.cons[ci].v;
      int vk = lk == 0 ? v.x : lk == 1 ? v.y : lk == 2 ? v.z : v.w;
      quad_contact(P, B, X, cm, ci, lk, vk, -1);
    }
  }
}
__global__ void __launch_bounds__(256, 1) k_colour_sweep(Pool P, OrderBufs B, int sweeps, int max_polls) {
  LevelCtx X;
  X.nc = min(P.cnt->n_cons, P.cons_cap);
  X.lam = sweeps > 1 ? P.lam : nullptr;
  X.elam = X.lam ? P.lam + P.cons_cap : nullptr;
  X.dataflow = false;
  int ncc = min(P.cnt->n_ccol, MAX_COLOURS), nec = P.n_ecol;
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  unsigned target = 0;
  // first colour of the single-block tail (every block finds the same one)
  int ctail = ncc;
  if (gridDim.x > 1) {
    int rest = 0;
    while (ctail > 0 && rest + P.ccount[ctail - 1] <= TAIL_MAX) rest += P.ccount[--ctail];
  }
  for (int sw = 0; sw < sweeps; sw++) {
    X.sweep = sw;
    for (int c = 0; c < ctail; c++) {
      colour_class(P, B, X, __ldg(&P.coff[c]), __ldg(&P.coff[c + 1]), tid >> 2, nth >> 2, tid, nth);
      if (!grid_barrier(P, target, max_polls)) return;
    }
    if (ctail < ncc) {
      if (blockIdx.x == 0)
        for (int c = ctail; c < ncc; c++) {
          colour_class(P, B, X, __ldg(&P.coff[c]), __ldg(&P.coff[c + 1]), threadIdx.x >> 2, blockDim.x >> 2,
                       threadIdx.x, blockDim.x);
          __syncthreads();
        }
      if (!grid_barrier(P, target, max_polls)) return;
    }
    for (int c = 0; c < nec; c++) {
      int a = __ldg(&P.eoff[c]), b = __ldg(&P.eoff[c + 1]);
      for (int k = a + tid; k < b; k += nth) {
        int e = __ldg(&P.eorder[k]);
        if (edge_live(P, e)) apply_edge(P, X, e);
      }
      if (!grid_barrier(P, target, max_polls)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// Backward step, projected Jacobi variant (Sec. 4.3.2, R12).  Every
// multiplier change dl = max(0, lambda - w/den) - lambda is computed from the
// same y.  Constraint c is under-relaxed by omega_c = omega / n_max(c), the
// largest number of constraints at one of its movable vertices, so that a
// vertex moves by at most omega times a convex combination of the
// single-constraint corrections (an unrelaxed sum overshoots by up to the
// vertex's constraint count and diverges).  The applied change
// s_c = omega_c * dl also advances the multiplier.  Each vertex sums
// m^-1 s_c g over its constraints in canonical order (contacts by ascending
// pair key, then edge-length constraints by ascending index) and adds the sum
// to y.  The per-vertex sums are segmented reductions over a vertex-major
// incidence list sorted by key, so the result does not depend on the order in
// which contacts were appended.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool scene_running(const Pool& P, int s) {
  const SceneState& S = P.ss[s];
  return S.active && !S.done;
}

// incidences (contact, movable vertex) of every contact that can move y
__global__ void k_jac_count(Pool P, OrderBufs B) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int4 v;
    bool live;
    if (P.mixed) {
      const ContactF& cf = ((const ContactF*)P.cons)[c];
      v = cf.v;
      live = cf.den > 0.f;
    } else {
      v = P.cons[c].v;
      live = P.cons[c].den > 0.0;
    }
    if (!live) continue;
    int vv[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < 4; k++)
      if (movable(P, vv[k])) atomicAdd(&B.vstart[vv[k]], 1);
  }
}
__global__ void k_jac_scatter(Pool P, OrderBufs B) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int4 v;
    unsigned long long key;
    bool live;
    if (P.mixed) {
      const ContactF& cf = ((const ContactF*)P.cons)[c];
      v = cf.v;
      key = cf.key;
      live = cf.den > 0.f;
    } else {
      v = P.cons[c].v;
      key = P.cons[c].key;
      live = P.cons[c].den > 0.0;
    }
    if (!live) continue;
    int vv[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < 4; k++)
      if (movable(P, vv[k])) {
        int slot = B.vstart[vv[k]] + atomicAdd(&B.vfill[vv[k]], 1);
        B.iprio[slot] = key;
        B.iid[slot] = 4 * c + k;
      }
  }
}
// place each incidence at its key rank inside its vertex's segment
// (B.rank becomes the key-sorted incidence list; pair keys are unique)
__global__ void k_jac_rank(Pool P, OrderBufs B) {
  int total = B.vstart[P.nv];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
    int id = B.iid[s];
    int4 v = P.mixed ? ((const ContactF*)P.cons)[id >> 2].v : P.cons[id >> 2].v;
    int vv[4] = {v.x, v.y, v.z, v.w};
    int vert = vv[id & 3];
    int a = B.vstart[vert], b = B.vstart[vert + 1];
    unsigned long long key = B.iprio[s];
    int r = 0;
    for (int t = a; t < b; t++) r += B.iprio[t] < key;
    B.rank[a + r] = id;
  }
}

// constraints at each movable vertex: its contacts (the scattered count in
// vfill) plus its edge-length constraints with a positive denominator
__global__ void k_jac_nv(Pool P, OrderBufs B) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int m = 0;
    if (P.vflag[v] & VF_MOVABLE) {
      m = B.vfill[v];
      if (m > 0) count_contact_vertex(P, P.vscene[v]);
      for (int j = P.vlstart[v]; j < P.vlstart[v + 1]; j++) {
        int e = P.vllist[j] >> 1;
        m += P.mixed ? (P.lgf[e].w > 0.f) : (P.lg[e].w > 0.0);
      }
    }
    B.vdone[v] = m;
  }
}
__device__ __forceinline__ int nmax_at(const Pool& P, const OrderBufs& B, int v, int m) {
  return (v >= 0 && (P.vflag[v] & VF_MOVABLE) && B.vdone[v] > m) ? B.vdone[v] : m;
}
__device__ __forceinline__ double relax(double omega, int m) { return omega / (double)(m > 0 ? m : 1); }

// s = omega_c dl of every contact and edge-length constraint from the same y
__global__ void k_jac_dl(Pool P, OrderBufs B, int sweep) {
  int n = min(P.cnt->n_cons, P.cons_cap);
  double* lam = P.sd[0].gs_sweeps > 1 ? P.lam : nullptr;
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int ci = tid; ci < n; ci += nth) {
    if (P.mixed) {
      const ContactF& c = ((const ContactF*)P.cons)[ci];
      float dl = 0.f;
      if (c.den > 0.f) {
        int vid[4] = {c.v.x, c.v.y, c.v.z, c.v.w};
        int nv = vid[2] < 0 ? 2 : 4;
        float w = c.c0;
        for (int k = 0; k < nv; k++) {
          float4 yv = P.yf[vid[k]], xv = P.xf[vid[k]];
          w = w + (c.g[3 * k] * (yv.x - xv.x) + c.g[3 * k + 1] * (yv.y - xv.y) + c.g[3 * k + 2] * (yv.z - xv.z));
        }
        float l0 = lam && sweep > 0 ? (float)lam[ci] : 0.f;
        float tl = l0 - w / c.den;
        int m = 0;
        for (int k = 0; k < nv; k++) m = nmax_at(P, B, vid[k], m);
        dl = (float)P.sd[P.vscene[vid[0]]].omega / (float)(m > 0 ? m : 1) * ((tl > 0.f ? tl : 0.f) - l0);
        if (lam) lam[ci] = (double)(l0 + dl);
      }
      P.jdl[ci] = (double)dl;
      continue;
    }
    const Contact& c = P.cons[ci];
    double dl = 0.0;
    if (c.den > 0.0) {
      int vid[4] = {c.v.x, c.v.y, c.v.z, c.v.w};
      int nv = vid[2] < 0 ? 2 : 4;
      double w = c.c0;
      for (int k = 0; k < nv; k++) {
        dv3 g = {c.g[3 * k], c.g[3 * k + 1], c.g[3 * k + 2]};
        w = w + vdot(g, vsub(mk(P.y[vid[k]]), mk(P.x[vid[k]])));
      }
      double l0 = lam && sweep > 0 ? lam[ci] : 0.0;
      double tl = l0 - w / c.den;
      int m = 0;
      for (int k = 0; k < nv; k++) m = nmax_at(P, B, vid[k], m);
      dl = relax(P.sd[P.vscene[vid[0]]].omega, m) * ((tl > 0.0 ? tl : 0.0) - l0);
      if (lam) lam[ci] = l0 + dl;
    }
    P.jdl[ci] = dl;
  }
  double* elam = lam ? lam + P.cons_cap : nullptr;
  double* edl = P.jdl + P.cons_cap;
  for (int e = tid; e < P.nl; e += nth) {
    int4 l = P.lv[e];
    double dl = 0.0;
    if (!scene_running(P, l.z)) {
      edl[e] = 0.0;
      continue;
    }
    if (P.mixed) {
      float4 gd = P.lgf[e];
      float dlf = 0.f;
      if (gd.w > 0.f) {
        float4 yi = P.yf[l.x], yj = P.yf[l.y];
        float w = (float)P.sd[l.z].sigma - (gd.x * (yi.x - yj.x) + gd.y * (yi.y - yj.y) + gd.z * (yi.z - yj.z));
        float l0 = elam && sweep > 0 ? (float)elam[e] : 0.f;
        float tl = l0 - w / gd.w;
        int m = nmax_at(P, B, l.y, nmax_at(P, B, l.x, 0));
        dlf = (float)P.sd[l.z].omega / (float)(m > 0 ? m : 1) * ((tl > 0.f ? tl : 0.f) - l0);
        if (elam) elam[e] = (double)(l0 + dlf);
      }
      edl[e] = (double)dlf;
      continue;
    }
    P4 gd = P.lg[e];
    if (gd.w > 0.0) {
      dv3 g = {gd.x, gd.y, gd.z};
      double w = P.sd[l.z].sigma - vdot(g, vsub(mk(P.y[l.x]), mk(P.y[l.y])));
      double l0 = elam && sweep > 0 ? elam[e] : 0.0;
      double tl = l0 - w / gd.w;
      int m = nmax_at(P, B, l.y, nmax_at(P, B, l.x, 0));
      dl = relax(P.sd[l.z].omega, m) * ((tl > 0.0 ? tl : 0.0) - l0);
      if (elam) elam[e] = l0 + dl;
    }
    edl[e] = dl;
  }
}

// per-vertex segmented sum in canonical order, then y += omega * sum
__global__ void k_jac_apply(Pool P, OrderBufs B) {
  const double* edl = P.jdl + P.cons_cap;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    if (!scene_running(P, s)) continue;
    double im = P.im[v];
    int a = B.vstart[v], b = B.vstart[v + 1];
    int ea = P.vlstart[v], eb = P.vlstart[v + 1];
    if (!(P.vflag[v] & VF_MOVABLE)) a = b = ea = eb = 0;
    if (P.mixed) {
      float imf = (float)im;
      float ax = 0.f, ay = 0.f, az = 0.f;
      for (int j = a; j < b; j++) {
        int id = B.rank[j];
        float dl = (float)P.jdl[id >> 2];
        if (dl == 0.f) continue;
        const float* g = ((const ContactF*)P.cons)[id >> 2].g + 3 * (id & 3);
        float sc = imf * dl;
        ax = ax + sc * g[0];
        ay = ay + sc * g[1];
        az = az + sc * g[2];
      }
      for (int j = ea; j < eb; j++) {
        int ent = P.vllist[j];
        float dl = (float)edl[ent >> 1];
        if (dl == 0.f) continue;
        float4 g = P.lgf[ent >> 1];
        float sc = (ent & 1) ? imf * dl : -(imf * dl);
        ax = ax + sc * g.x;
        ay = ay + sc * g.y;
        az = az + sc * g.z;
      }
      float4 y = P.yf[v];
      P.yf[v] = make_float4(y.x + ax, y.y + ay, y.z + az, 0.f);
      continue;
    }
    dv3 acc = {0.0, 0.0, 0.0};
    for (int j = a; j < b; j++) {
      int id = B.rank[j];
      double dl = P.jdl[id >> 2];
      if (dl == 0.0) continue;
      const double* g = P.cons[id >> 2].g + 3 * (id & 3);
      acc = vadd(acc, vscl(im * dl, dv3{g[0], g[1], g[2]}));
    }
    for (int j = ea; j < eb; j++) {
      int ent = P.vllist[j];
      double dl = edl[ent >> 1];
      if (dl == 0.0) continue;
      P4 g = P.lg[ent >> 1];
      dv3 t = vscl(im * dl, dv3{g.x, g.y, g.z});
      acc = (ent & 1) ? vadd(acc, t) : vsub(acc, t);
    }
    P4 y = P.y[v];
    dv3 yn = vadd(mk(y), acc);
    P.y[v] = {yn.x, yn.y, yn.z, 0.0};
  }
}

// ---------------------------------------------------------------------------
// Forward step, Eq. forward2 (R2): alpha_i = min(0.5 gamma D_i / |y_i - x_i|, 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scene_max(const Pool& P, unsigned long long* dst, int s, unsigned long long v) {
  scene_reduce(P, s, v, cg::greater<unsigned long long>(), [&](unsigned long long m, int) { atomicMax(dst, m); });
}

// x + a (y - x): y itself at a = 1, x itself at a = 0 (a vertex that does
// not move keeps its position exactly, even when y is not finite)
__device__ __forceinline__ dv3 step_to(dv3 x, dv3 y, double a) {
  if (a == 1.0) return y;
  if (a == 0.0) return x;
  return vadd(x, vscl(a, vsub(y, x)));
}

__global__ void k_forward(Pool P) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    const SceneState& S = P.ss[s];
    if (!S.active || S.done) continue;
    // CCD-based rule: the global bound D^(l) caps every vertex that is not
    // floored, the CCD rounds decide the rest
    unsigned long long dvb = P.Dv[v];
    if (dvb != 0x7ff0000000000000ULL) {
      // a vertex of a pair of P (statistics)
      scene_count(P, s, [&](int n) { atomicAdd((unsigned long long*)&P.ss[s].pverts, (unsigned long long)n); });
    }
    // the vertex's own D_i; below the floor (R2b) the vertex does not move,
    // under either rule
    double own = bitsd(dvb);
    if (S.D < own) own = S.D;
    double Di = P.sd[s].step_rule ? S.D : own;
    bool floored = !(Di >= D_FLOOR) || !(own >= D_FLOOR);
    if (floored) Di = 0.0;
    P.Dv[v] = 0x7ff0000000000000ULL;
    P4 xv4 = P.x[v];
    dv3 yv;
    if (P.yf) {
      float4 f = P.yf[v];
      yv = {(double)f.x, (double)f.y, (double)f.z};
    } else yv = mk(P.y[v]);
    dv3 xv = mk(xv4);
    double nd = vnorm(vsub(yv, xv)), a = 1.0;
    if (nd > 0.0) {
      double q = (P.sd[s].hgamma * Di) / nd;
      a = q < 1.0 ? q : 1.0;
    } else if (nd != 0.0) {
      a = 0.0;  // R2c: y not finite, the vertex does not move
    }
    if (floored && nd > 0.0) {
      // held by the D_i floor although its target is elsewhere (statistics)
      scene_count(P, s, [&](int n) { atomicAdd(&P.ss[s].frozen_cur, n); });
    }
    dv3 xn = step_to(xv, yv, a);
    P.x[v] = {xn.x, xn.y, xn.z, 0.0};
    P.xf[v] = make_float4((float)xn.x, (float)xn.y, (float)xn.z, 0.f);
    if (P.alpha) {
      // CCD mode: tentative x; k_ccd_fix applies the clamps, r and the reductions
      P.xp[v] = xv4;
      P.alpha[v] = a;
      continue;
    }
    double r = P.r[v] * (1.0 - a);
    P.r[v] = r;
    double mv = vnorm(vsub(xn, xv));
    scene_max(P, &P.ss[s].move_bits, s, dbits(mv));
    scene_max(P, &P.ss[s].rmax_bits, s, dbits(r));
  }
}

// ---------------------------------------------------------------------------
// CCD of every pair's segment x^(l) -> x^(l+1) (the safety check, or the
// CCD-based step rule of Sec. 5.1): a hit at time t scales the step of the
// pair's vertices by t/2 (the smallest factor over their pairs), and the
// segments are tested again.  Round k runs k_ccd_pairs then k_ccd_apply; a
// scene whose round finds no hit leaves the rounds; a hit in the test after
// the last round keeps every vertex of the scene in place (k_ccd_fix).
// ---------------------------------------------------------------------------
__global__ void k_ccd_begin(Pool P) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < P.nscene) {
    P.ss[s].ccd_live = 1;
    P.ss[s].ccd_hits[0] = 0;
    P.ss[s].ccd_hits[1] = 0;
  }
}

__global__ void k_ccd_pairs(Pool P, int nxt, int round) {
  int n = min(P.cnt->n_pairs[nxt], P.pair_cap);
  const PairBuf B = P.pb[nxt];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 v = B.v[i];
    int s = P.vscene[v.x];
    const SceneState& S = P.ss[s];
    if (!S.active || S.done || !S.ccd_live) continue;
    int kind = (int)(B.key[i] >> 62);
    int vid[4] = {v.x, v.y, v.z, v.w};
    int nv = kind == K_VV ? 2 : 4;
    dv3 p0[4], p1[4];
    for (int k = 0; k < nv; k++) {
      p0[k] = mk(P.xp[vid[k]]);
      p1[k] = mk(P.x[vid[k]]);
    }
    double toi;
    if (ccd_pair(kind, p0, p1, P.rho[v.x], kind == K_VV ? P.rho[v.y] : 0.0, &toi)) {
      unsigned long long cb = dbits(0.5 * toi);
      for (int k = 0; k < nv; k++) atomicMin(&P.clampb[vid[k]], cb);
      atomicAdd(&P.ss[s].ccd_clamps, 1);
      atomicAdd(&P.ss[s].ccd_hits[round & 1], 1);
    }
  }
}

__device__ __forceinline__ dv3 y_of(const Pool& P, int v) {
  if (P.yf) {
    float4 f = P.yf[v];
    return {(double)f.x, (double)f.y, (double)f.z};
  }
  return mk(P.y[v]);
}

// Round `round` (< ccd_rounds) found hits: scale the clamped steps.  The
// counter of the next round is cleared here (nothing reads it in this launch).
__global__ void k_ccd_apply(Pool P, int round) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    SceneState& S = P.ss[s];
    if (!S.active || S.done) continue;
    if (v == P.sd[s].v0) S.ccd_hits[(round + 1) & 1] = 0;
    if (S.ccd_hits[round & 1] == 0) {
      if (v == P.sd[s].v0) S.ccd_live = 0;
      continue;
    }
    double c = bitsd(P.clampb[v]);
    if (c < 1.0) {
      double a = c * P.alpha[v];
      P.alpha[v] = a;
      dv3 xn = step_to(mk(P.xp[v]), y_of(P, v), a);
      P.x[v] = {xn.x, xn.y, xn.z, 0.0};
      P.xf[v] = make_float4((float)xn.x, (float)xn.y, (float)xn.z, 0.f);
      P.clampb[v] = dbits(1.0);
    }
  }
}

// After the last round: a remaining hit keeps the scene in place; then r and
// the reductions of the forward step.
__global__ void k_ccd_fix(Pool P, int round) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    const SceneState& S = P.ss[s];
    if (!S.active || S.done) continue;
    double a = P.alpha[v];
    dv3 xv = mk(P.xp[v]);
    dv3 xn = mk(P.x[v]);
    if (S.ccd_live && S.ccd_hits[round & 1] > 0) {
      a = 0.0;
      xn = xv;
      P.x[v] = {xn.x, xn.y, xn.z, 0.0};
      P.xf[v] = make_float4((float)xn.x, (float)xn.y, (float)xn.z, 0.f);
    }
    P.clampb[v] = dbits(1.0);
    double r = P.r[v] * (1.0 - a);
    P.r[v] = r;
    double mv = vnorm(vsub(xn, xv));
    scene_max(P, &P.ss[s].move_bits, s, dbits(mv));
    scene_max(P, &P.ss[s].rmax_bits, s, dbits(r));
  }
}

// ---------------------------------------------------------------------------
// Loop control (Algorithm 1): D^(l+1) = D^(l) - 2 max|dx| one ulp down (R15);
// stop at ||r||_inf < eps or after iteration L; search when D < D^min.
// ---------------------------------------------------------------------------
__global__ void k_control(Pool P, int cur) {
  Counters* C = P.cnt;
  __shared__ int any_search, running, any_refresh;
  if (threadIdx.x == 0) { any_search = 0; running = 0; any_refresh = 0; }
  __syncthreads();
  for (int s = threadIdx.x; s < P.nscene; s += blockDim.x) {
    SceneState& S = P.ss[s];
    if (!S.active || S.done) continue;
    const SceneDesc& d = P.sd[s];
    double m = bitsd(S.move_bits), rmax = bitsd(S.rmax_bits);
    S.pairs_eval += S.n_pairs;
    if (S.n_pairs > S.max_pairs) S.max_pairs = S.n_pairs;
    if (S.do_search) S.searches++;
    S.n_pairs = 0;
    S.D = nextafter(S.D - 2.0 * m, -__longlong_as_double(0x7ff0000000000000LL));
    S.iter++;
    S.final_r = rmax;
    S.move_bits = 0;
    S.rmax_bits = 0;
    S.frozen = S.frozen_cur;
    S.frozen_cur = 0;
    if (C->vcontacts > S.max_vcontacts) S.max_vcontacts = C->vcontacts;
    if (rmax < d.eps) {
      S.done = 1;
      S.converged = 1;
    } else if (S.iter > d.max_iters) {
      S.done = 1;
    } else {
      S.do_search = S.D < d.d_min;
      if (S.do_search) {
        S.D = d.d_max;
        atomicOr(&any_search, 1);
      } else {
        atomicOr(&any_refresh, 1);
      }
      atomicOr(&running, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    C->any_search = any_search;
    C->any_refresh = any_refresh;
    C->n_fcand[0] = C->n_fcand[1] = C->n_fcand[2] = 0;
    C->all_done = running ? 0 : 1;
    C->n_pairs[cur] = 0;
    C->n_active[0] = C->n_active[1] = C->n_active[2] = 0;
    C->n_cons = 0;
    C->vcontacts = 0;
    C->n_ccol = 0;
    C->n_exact[0] = C->n_exact[1] = 0;
  }
}

__global__ void k_output(Pool P, double* const* ptrs, int only) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    if (!P.ss[s].active || (only >= 0 && s != only)) continue;
    int i = v - P.sd[s].v0;
    double* xo = ptrs[3 * s + 2];
    P4 p = P.x[v];
    xo[3 * i] = p.x;
    xo[3 * i + 1] = p.y;
    xo[3 * i + 2] = p.z;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <class K, class... A>
static cudaError_t coop_launch(K kern, int blocks, int threads, cudaStream_t st, A... args) {
  void* argv[] = {(void*)&args...};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(threads), argv, 0, st);
}

// Resident blocks of the cooperative kernels: the colouring and the
// level-colouring sweep (which = 0), and the colour-class sweep (which = 1).
int coop_grid(int threads, int which) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (which == 0) {
    int per2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_colour, threads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_level_sweep, threads, 0);
    if (per2 < per) per = per2;
  } else {
    // one block per SM: a class spans a few hundred warps at most, and every
    // block more is one more arrival at each grid barrier
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_colour_sweep, threads, 0);
    if (per > 1) per = 1;
  }
  if (per < 1) per = 1;
  return sms * per;
}

__global__ void k_clear_start(Pool P) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < P.nscene) P.ss[s].start = 0;
}

// mode 0: all scenes start (counters reset); mode 2: only the flagged scenes
// start, the others keep their loop state and the shared counters
void step_init(Runtime& R, cudaStream_t st, int mode) {
  Pool& P = R.pool;
  if (mode == 0) cudaMemsetAsync(P.cnt, 0, sizeof(Counters), st);
  k_scene_init<<<(P.nscene + 127) / 128, 128, 0, st>>>(P, mode);
  k_vert_init<<<grid_for(P.nv, 256), 256, 0, st>>>(P, R.d_ptrs, mode);
  R.launches += 2;
  if (P.nl) {
    k_edge_prep<<<grid_for(P.nl, 256), 256, 0, st>>>(P, mode);
    R.launches++;
  }
  if (mode == 2) {
    k_clear_start<<<(P.nscene + 127) / 128, 128, 0, st>>>(P);
    R.launches++;
  }
}

void set_any_search(Runtime& R, cudaStream_t st) {
  int one = 1;
  cudaMemcpyAsync(&R.pool.cnt->any_search, &one, sizeof(int), cudaMemcpyHostToDevice, st);
}

cudaError_t iteration(Runtime& R, int cur, cudaStream_t st) {
  Pool& P = R.pool;
  int nxt = 1 - cur;
  prof_mark(R, PG_REFIT, 0, st);
  if (!R.refit_only) bvh_build_all(R, st, 1);
  bvh_refit_all(R, st, 0);
  prof_mark(R, PG_REFIT, 1, st);
  for (int c = 0; c < 3; c++) {
    prof_mark(R, PG_VT + c, 0, st);
    query_class(R, c, nxt, 0, 0.0, st);
    prof_mark(R, PG_VT + c, 1, st);
  }
  prof_mark(R, PG_FINAL, 0, st);
  if (!P.mixed) cudaMemsetAsync(P.vmin, 0xff, sizeof(unsigned int) * (size_t)P.nv, st);
  finalize_search(R, nxt, 0, 0.0, st);
  prof_mark(R, PG_FINAL, 1, st);
  prof_mark(R, PG_REFRESH, 0, st);
  if (!P.mixed) {
    k_refresh_bounds<<<grid_for(P.pair_cap, 256), 256, 0, st>>>(P, cur);
    R.launches++;
  }
  k_refresh<<<grid_for(P.pair_cap, 256), 256, 0, st>>>(P, cur, nxt);
  if (!P.mixed) {
    k_exact_refresh<<<grid_for(P.pair_cap, 256), 256, 0, st>>>(P, cur, nxt);
    R.launches++;
  }
  prof_mark(R, PG_REFRESH, 1, st);
  prof_mark(R, PG_ASSEMBLE, 0, st);
  k_assemble<<<grid_for(P.act_cap, 128), 128, 0, st>>>(P, nxt);
  prof_mark(R, PG_ASSEMBLE, 1, st);
  prof_mark(R, PG_ORDER, 0, st);
  cudaError_t e = cudaSuccess;
  const OrderBufs& B = R.obuf;
  cudaMemsetAsync(B.vstart, 0, sizeof(int) * ((size_t)P.nv + 1), st);
  cudaMemsetAsync(B.vfill, 0, sizeof(int) * (size_t)P.nv, st);
  if (R.solver == 1) {  // projected Jacobi
    k_jac_count<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, B);
    scan_ints(R, B.vstart, P.nv + 1, st);
    k_jac_scatter<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, B);
    k_jac_rank<<<grid_for(4LL * P.cons_cap, 256), 256, 0, st>>>(P, B);
    k_jac_nv<<<grid_for(P.nv, 256), 256, 0, st>>>(P, B);
    prof_mark(R, PG_ORDER, 1, st);
    prof_mark(R, PG_SWEEP, 0, st);
    for (int sw = 0; sw < R.sweeps; sw++) {
      k_jac_dl<<<grid_for((long long)P.cons_cap + P.nl, 256), 256, 0, st>>>(P, B, sw);
      k_jac_apply<<<grid_for(P.nv, 256), 256, 0, st>>>(P, B);
    }
    prof_mark(R, PG_SWEEP, 1, st);
    R.launches += 5 + 2 * R.sweeps;
  } else {  // projected Gauss-Seidel in colour classes
    cudaMemsetAsync(B.vdone, 0, sizeof(int) * (size_t)P.nv, st);
    if (R.colouring == 1) cudaMemsetAsync(P.vlevel, 0xff, sizeof(int) * (size_t)P.nv, st);
    if (P.mixed) {
      ContactFAcc acc{(const ContactF*)P.cons};
      k_inc_count<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
      scan_ints(R, B.vstart, P.nv + 1, st);
      k_inc_scatter<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
      k_inc_rank<<<grid_for(4LL * P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
    } else {
      ContactAcc acc{P.cons};
      k_inc_count<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
      scan_ints(R, B.vstart, P.nv + 1, st);
      k_inc_scatter<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
      k_inc_rank<<<grid_for(4LL * P.cons_cap, 256), 256, 0, st>>>(P, acc, B);
    }
    prof_mark(R, PG_ORDER, 1, st);
    if (R.colouring == 1) {
      // level colouring: the dataflow sweep applies the classes in order
      prof_mark(R, PG_SWEEP, 0, st);
      for (int sw = 0; sw < R.sweeps && e == cudaSuccess; sw++) {
        cudaMemsetAsync(P.fdone, 0, (size_t)P.cons_cap + P.nl, st);
        e = coop_launch(k_level_sweep, R.coop_blocks, 256, st, P, B, sw, R.sweeps, R.max_polls);
      }
      prof_mark(R, PG_SWEEP, 1, st);
      prof_mark(R, PG_COLOUR, 0, st);
      cudaMemsetAsync(P.ccount, 0, sizeof(int) * MAX_COLOURS, st);
      if (e == cudaSuccess) k_colour_stats<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P);
      prof_mark(R, PG_COLOUR, 1, st);
      R.launches += 5 + R.sweeps;
    } else {
      prof_mark(R, PG_COLOUR, 0, st);
      cudaMemsetAsync(P.fdone, 0, (size_t)P.cons_cap, st);
      cudaMemsetAsync(P.ccount, 0, sizeof(int) * MAX_COLOURS, st);
      e = coop_launch(k_colour, R.coop_blocks, 256, st, P, B, R.max_polls);
      if (e == cudaSuccess) k_colour_stats<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P);
      cudaMemsetAsync(P.cfill, 0, sizeof(int) * MAX_COLOURS, st);
      if (e == cudaSuccess) k_colour_order<<<grid_for(P.cons_cap, 256), 256, 0, st>>>(P);
      prof_mark(R, PG_COLOUR, 1, st);
      prof_mark(R, PG_SWEEP, 0, st);
      cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned int), st);
      if (e == cudaSuccess) e = coop_launch(k_colour_sweep, R.sweep_blocks, 256, st, P, B, R.sweeps, R.max_polls);
      prof_mark(R, PG_SWEEP, 1, st);
      R.launches += 8;
    }
  }
  if (e != cudaSuccess) return e;
  prof_mark(R, PG_FORWARD, 0, st);
  k_forward<<<grid_for(P.nv, 256), 256, 0, st>>>(P);
  if (P.alpha) {
    k_ccd_begin<<<(P.nscene + 127) / 128, 128, 0, st>>>(P);
    for (int k = 0; k < R.ccd_rounds; k++) {
      k_ccd_pairs<<<grid_for(P.pair_cap, 128), 128, 0, st>>>(P, nxt, k);
      k_ccd_apply<<<grid_for(P.nv, 256), 256, 0, st>>>(P, k);
    }
    k_ccd_pairs<<<grid_for(P.pair_cap, 128), 128, 0, st>>>(P, nxt, R.ccd_rounds);
    k_ccd_fix<<<grid_for(P.nv, 256), 256, 0, st>>>(P, R.ccd_rounds);
    R.launches += 3 + 2 * R.ccd_rounds;
  }
  prof_mark(R, PG_FORWARD, 1, st);
  prof_mark(R, PG_CONTROL, 0, st);
  k_control<<<1, 256, 0, st>>>(P, cur);
  prof_mark(R, PG_CONTROL, 1, st);
  R.launches += 4;
  return cudaGetLastError();
}


__global__ void k_reset_accept(Pool P) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < P.nscene) P.ss[s].isect = P.ss[s].uncertain = 0;
}
void reset_accept(Runtime& R, cudaStream_t st) {
  k_reset_accept<<<(R.pool.nscene + 127) / 128, 128, 0, st>>>(R.pool);
  R.launches++;
}

void output(Runtime& R, cudaStream_t st) {
  Pool& P = R.pool;
  k_output<<<grid_for(P.nv, 256), 256, 0, st>>>(P, R.d_ptrs, -1);
  R.launches++;
}

void output_scene(Runtime& R, int s, cudaStream_t st) {
  Pool& P = R.pool;
  const SceneDesc& d = R.sd[s];
  (void)d;
  k_output<<<grid_for(R.sd[s].nv, 256), 256, 0, st>>>(P, R.d_ptrs, s);
  R.launches++;
}

}  // namespace cch

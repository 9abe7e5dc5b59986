// cch_capi.cu -- host runtime and the C ABI declared in include/cch.h.
//
// A cch_scene owns a pool: the concatenated arrays of one or more scenes
// (per-scene offset tables in SceneDesc), their BVHs, the proximity-pair and
// contact buffers, and the per-scene loop state.  A step runs Algorithm 1 on
// every scene of the pool at once; each scene keeps its own D^(l), search
// flag and termination, so batched results equal single-scene results.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <algorithm>
#include <vector>

#include "../../include/cch.h"
#include "cch_host.h"
#include "cch_step.h"

using namespace cch;

struct cch_scene {
  Runtime R;
  int n_scenes = 0;
  std::vector<int64_t> nverts;  // per scene
};

namespace {

#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

cch_status cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return CCH_E_OOM;
  return CCH_E_CUDA;
}

template <class T>
cudaError_t dalloc_in(std::vector<void*>& list, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
  if (e != cudaSuccess) return e;
  list.push_back(q);
  *p = (T*)q;
  return cudaSuccess;
}
template <class T>
cudaError_t dalloc(Runtime& R, T** p, size_t count) {
  return dalloc_in(R.allocs, p, count);
}

void free_all(Runtime& R) {
  for (void* p : R.allocs) cudaFree(p);
  R.allocs.clear();
  for (void* p : R.pair_allocs) cudaFree(p);
  R.pair_allocs.clear();
  if (R.graph) cudaGraphExecDestroy(R.graph);
  R.graph = nullptr;
  if (R.h_ptrs) cudaFreeHost(R.h_ptrs);
  if (R.h_cnt) cudaFreeHost(R.h_cnt);
  if (R.h_ss) cudaFreeHost(R.h_ss);
  R.h_ptrs = nullptr;
  R.h_cnt = nullptr;
  R.h_ss = nullptr;
  for (int g = 0; g < PG_N; g++)
    for (int k = 0; k < 2; k++)
      if (R.pev[g][k]) {
        cudaEventDestroy(R.pev[g][k]);
        R.pev[g][k] = nullptr;
      }
  if (R.ev0) cudaEventDestroy(R.ev0);
  if (R.ev1) cudaEventDestroy(R.ev1);
  R.ev0 = R.ev1 = nullptr;
}

bool finite_nonneg(const double* a, int64_t n) {
  for (int64_t i = 0; i < n; i++)
    if (!std::isfinite(a[i]) || a[i] < 0.0) return false;
  return true;
}

cch_status validate_topology(const cch_topology* t) {
  if (!t || t->n_verts <= 0 || t->n_verts >= (1LL << 30) || !t->inv_mass) return CCH_E_INVALID_ARG;
  if (t->n_tris < 0 || t->n_edges < 0 || t->n_len < 0 || t->n_points < 0) return CCH_E_INVALID_ARG;
  if ((t->n_tris && !t->tris) || (t->n_edges && !t->edges) || (t->n_len && !t->len_edges) ||
      (t->n_points && !t->points))
    return CCH_E_INVALID_ARG;
  if (t->n_tris >= (1LL << 31) || t->n_edges >= (1LL << 31) || t->n_len >= (1LL << 31)) return CCH_E_INVALID_ARG;
  if (!finite_nonneg(t->inv_mass, t->n_verts)) return CCH_E_INVALID_ARG;
  if (t->point_radius && !finite_nonneg(t->point_radius, t->n_verts)) return CCH_E_INVALID_ARG;
  int64_t n = t->n_verts;
  for (int64_t i = 0; i < t->n_tris; i++) {
    const int32_t* v = t->tris + 3 * i;
    for (int k = 0; k < 3; k++)
      if (v[k] < 0 || v[k] >= n) return CCH_E_INVALID_ARG;
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return CCH_E_INVALID_ARG;
  }
  for (int64_t i = 0; i < t->n_edges; i++) {
    const int32_t* v = t->edges + 2 * i;
    if (v[0] < 0 || v[0] >= n || v[1] < 0 || v[1] >= n || v[0] == v[1]) return CCH_E_INVALID_ARG;
  }
  for (int64_t i = 0; i < t->n_len; i++) {
    const int32_t* v = t->len_edges + 2 * i;
    if (v[0] < 0 || v[0] >= n || v[1] < 0 || v[1] >= n || v[0] == v[1]) return CCH_E_INVALID_ARG;
  }
  for (int64_t i = 0; i < t->n_points; i++)
    if (t->points[i] < 0 || t->points[i] >= n) return CCH_E_INVALID_ARG;
  return CCH_OK;
}

cch_status validate_params(const cch_params* p) {
  if (!p) return CCH_E_INVALID_ARG;
  if (!(p->d_min > 0.0) || !(p->d_max > p->d_min) || !(p->delta > 0.0) || !(p->delta <= p->d_min))
    return CCH_E_INVALID_ARG;
  if (!(p->sigma > 0.0) || !(p->gamma > 0.0 && p->gamma < 1.0) || !(p->eps >= 0.0)) return CCH_E_INVALID_ARG;
  if (p->max_iters < 0 || p->gs_sweeps < 1 || p->gs_sweeps > 64) return CCH_E_INVALID_ARG;
  if (p->precision != CCH_PREC_FP64 && p->precision != CCH_PREC_MIXED) return CCH_E_INVALID_ARG;
  if (p->solver != CCH_SOLVER_GAUSS_SEIDEL && p->solver != CCH_SOLVER_JACOBI) return CCH_E_INVALID_ARG;
  if (p->constraint_form != CCH_FORM_VOLUME && p->constraint_form != CCH_FORM_GAP) return CCH_E_INVALID_ARG;
  if (p->step_rule != CCH_STEP_DISTANCE && p->step_rule != CCH_STEP_CCD) return CCH_E_INVALID_ARG;
  if (p->ccd_rounds < 0 || p->ccd_rounds > 64) return CCH_E_INVALID_ARG;
  if (p->iters_per_launch < 0 || p->iters_per_launch > 4096) return CCH_E_INVALID_ARG;
  if (p->max_polls < 0 || p->pair_capacity < 0 || p->sweep_blocks < 0) return CCH_E_INVALID_ARG;
  if (p->colouring != CCH_COLOUR_GREEDY && p->colouring != CCH_COLOUR_LEVEL) return CCH_E_INVALID_ARG;
  return CCH_OK;
}

// Status of a device error word: a bounded wait that ran out (the sweep's
// counters) is a timeout; a tree bound (stack, visit budget, climb) is a
// capacity error.
cch_status device_status(int err) { return (err & ERR_POLL) ? CCH_E_TIMEOUT : CCH_E_CAPACITY; }

// Pair-buffer capacities; grown on overflow.
void set_caps(Runtime& R, int pair_cap) {
  R.pool.pair_cap = pair_cap;
  R.pool.act_cap = pair_cap;
  R.pool.cons_cap = pair_cap;
}

cudaError_t alloc_pairs(Runtime& R) {
  Pool& P = R.pool;
  std::vector<void*>& L = R.pair_allocs;
  cudaError_t e;
  for (int b = 0; b < 2; b++) {
    if ((e = dalloc_in(L, &P.pb[b].key, P.pair_cap)) != cudaSuccess) return e;
    if ((e = dalloc_in(L, &P.pb[b].v, P.pair_cap)) != cudaSuccess) return e;
    if ((e = dalloc_in(L, &P.pb[b].d, P.pair_cap)) != cudaSuccess) return e;
  }
  if ((e = dalloc_in(L, &P.act, 3 * (size_t)P.act_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.fkey, 3 * (size_t)P.pair_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.fv, 3 * (size_t)P.pair_cap)) != cudaSuccess) return e;
  P.fd = nullptr;
  P.fbs = nullptr;
  P.fbr = nullptr;
  if (P.mixed && (e = dalloc_in(L, &P.fd, 3 * (size_t)P.pair_cap)) != cudaSuccess) return e;
  P.exq = nullptr;
  P.exr = nullptr;
  if (!P.mixed) {
    if ((e = dalloc_in(L, &P.fbs, 3 * (size_t)P.pair_cap)) != cudaSuccess) return e;
    if ((e = dalloc_in(L, &P.fbr, (size_t)P.pair_cap)) != cudaSuccess) return e;
    if ((e = dalloc_in(L, &P.exq, 3 * (size_t)P.pair_cap)) != cudaSuccess) return e;
    if ((e = dalloc_in(L, &P.exr, (size_t)P.pair_cap)) != cudaSuccess) return e;
  }
  if ((e = dalloc_in(L, &P.cons, P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.fdone, (size_t)P.cons_cap + P.nl)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.ccol, (size_t)P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.corder, (size_t)P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &R.obuf.iprio, 4 * (size_t)P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &R.obuf.iid, 4 * (size_t)P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &R.obuf.rank, 4 * (size_t)P.cons_cap)) != cudaSuccess) return e;
  if ((e = dalloc_in(L, &P.lam, (size_t)P.cons_cap + P.nl)) != cudaSuccess) return e;
  P.jdl = nullptr;
  if (R.solver == CCH_SOLVER_JACOBI && (e = dalloc_in(L, &P.jdl, (size_t)P.cons_cap + P.nl)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

// Frees the pair-sized buffers (re-allocated when they grow).
void free_pairs(Runtime& R) {
  for (void* p : R.pair_allocs) cudaFree(p);
  R.pair_allocs.clear();
}

cudaError_t alloc_bvh(Runtime& R, BVH& B, int n, int nscene) {
  cudaError_t e;
  B.n = n;
  int ni = n > 1 ? n - 1 : 1;
  int ntiles = (n + 2047) / 2048 + 1;
  if ((e = dalloc(R, &B.keys, n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.keys_alt, n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.ids, n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.ids_alt, n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.left, ni)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.right, ni)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.parent, ni + n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.range_hi, ni)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.box, 3 * ni)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.flag, ni)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.leafbox, 2 * (size_t)n)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.sroot, nscene)) != cudaSuccess) return e;
  if ((e = dalloc(R, &B.hist, 256 * (size_t)ntiles)) != cudaSuccess) return e;
  B.hist2 = nullptr;
  return cudaSuccess;
}

template <class T>
cudaError_t upload(Runtime& R, T** dst, const std::vector<T>& src) {
  cudaError_t e = dalloc(R, dst, src.size());
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  return e;
}

cch_status build_pool(cch_scene* S, const cch_topology* topos, int n_scenes, const cch_params* prm,
                      const cch_params* scene_prm, void* stream) {
  Runtime& R = S->R;
  Pool& P = R.pool;
  R.stream = (cudaStream_t)stream;
  S->n_scenes = n_scenes;
  // host tables
  std::vector<P4> zero4;
  std::vector<double> im, rho;
  std::vector<int> vscene, vc, pts;
  std::vector<uint8_t> vflag;
  std::vector<int4> tv, ev, lv;
  int nv = 0, nt = 0, ne = 0, nl = 0, nq = 0;
  for (int s = 0; s < n_scenes; s++) {
    const cch_topology& t = topos[s];
    SceneDesc d{};
    d.v0 = nv; d.nv = (int)t.n_verts;
    d.t0 = nt; d.nt = (int)t.n_tris;
    d.e0 = ne; d.ne = (int)t.n_edges;
    d.l0 = nl; d.nl = (int)t.n_len;
    d.q0 = nq; d.nq = (int)t.n_points;
    d.c0 = (int)vc.size();
    // the scene's physical parameters (its own when given), the pool's method
    const cch_params* q = scene_prm ? &scene_prm[s] : prm;
    d.d_min = q->d_min; d.d_max = q->d_max; d.delta = q->delta; d.sigma = q->sigma;
    d.hgamma = 0.5 * q->gamma; d.eps = q->eps; d.omega = prm->jacobi_omega;
    d.form = prm->constraint_form;
    d.max_iters = q->max_iters; d.gs_sweeps = prm->gs_sweeps; d.solver = prm->solver; d.ccd = prm->ccd_check;
    d.step_rule = prm->step_rule;
    d.seed = q->seed;
    d.rho_max = 0.0;
    if (t.point_radius)
      for (int64_t v = 0; v < t.n_verts; v++)
        if (t.point_radius[v] > d.rho_max) d.rho_max = t.point_radius[v];
    std::vector<uint8_t> f(t.n_verts, 0);
    for (int64_t i = 0; i < t.n_points; i++) f[t.points[i]] |= VF_POINT | VF_COLL;
    for (int64_t i = 0; i < 3 * t.n_tris; i++) f[t.tris[i]] |= VF_COLL;
    for (int64_t i = 0; i < 2 * t.n_edges; i++) f[t.edges[i]] |= VF_COLL;
    for (int64_t v = 0; v < t.n_verts; v++) {
      if (t.inv_mass[v] > 0.0) f[v] |= VF_MOVABLE;
      im.push_back(t.inv_mass[v]);
      rho.push_back(t.point_radius ? t.point_radius[v] : 0.0);
      vscene.push_back(s);
      vflag.push_back(f[v]);
      if (f[v] & VF_COLL) vc.push_back(nv + (int)v);
    }
    d.nc = (int)vc.size() - d.c0;
    for (int64_t i = 0; i < t.n_tris; i++)
      tv.push_back(make_int4(nv + t.tris[3 * i], nv + t.tris[3 * i + 1], nv + t.tris[3 * i + 2], s));
    for (int64_t i = 0; i < t.n_edges; i++)
      ev.push_back(make_int4(nv + t.edges[2 * i], nv + t.edges[2 * i + 1], s, 0));
    for (int64_t i = 0; i < t.n_len; i++)
      lv.push_back(make_int4(nv + t.len_edges[2 * i], nv + t.len_edges[2 * i + 1], s, 0));
    for (int64_t i = 0; i < t.n_points; i++) pts.push_back(nv + t.points[i]);
    nv += (int)t.n_verts; nt += (int)t.n_tris; ne += (int)t.n_edges; nl += (int)t.n_len; nq += (int)t.n_points;
    R.sd.push_back(d);
    S->nverts.push_back(t.n_verts);
    if (q->max_iters > R.max_iters) R.max_iters = q->max_iters;
  }
  P.nv = nv; P.nt = nt; P.ne = ne; P.nl = nl; P.nq = nq; P.nvc = (int)vc.size(); P.nscene = n_scenes;
  R.scene_bits = 0;
  while ((1 << R.scene_bits) < n_scenes) R.scene_bits++;
  R.sweeps = prm->gs_sweeps;
  R.solver = prm->solver;
  R.colouring = prm->colouring;
  R.ccd = prm->ccd_check || prm->step_rule == CCH_STEP_CCD;
  R.ccd_rounds = prm->ccd_rounds;
  // the CCD-based step relies on the root-finding CCD, which can miss a
  // tangential touch at a double root of the coplanarity cubic: the exact
  // acceptance of x^{t+1} always runs with it
  R.accept = prm->accept_check || prm->step_rule == CCH_STEP_CCD;
  R.validate = prm->validate_input;
  R.iters_per_check = prm->iters_per_launch > 0 ? prm->iters_per_launch : 16;
  R.refit_only = prm->bvh_refit_only ? 1 : 0;
  R.coop_blocks = coop_grid(256, 0);
  R.sweep_blocks = coop_grid(256, 1);
  if (prm->sweep_blocks > 0 && prm->sweep_blocks < R.coop_blocks) R.coop_blocks = prm->sweep_blocks;
  if (prm->sweep_blocks > 0 && prm->sweep_blocks < R.sweep_blocks) R.sweep_blocks = prm->sweep_blocks;
  R.max_polls = prm->max_polls > 0 ? prm->max_polls : 1 << 22;

  CK(dalloc(R, &P.x, nv));
  CK(dalloc(R, &P.y, nv));
  CK(dalloc(R, &P.yt, nv));
  CK(cudaMemset(P.x, 0, sizeof(P4) * nv));
  CK(dalloc(R, &P.xf, nv));
  CK(cudaMemset(P.xf, 0, sizeof(float4) * nv));
  P.mixed = prm->precision == CCH_PREC_MIXED;
  P.yf = nullptr;
  P.lgf = nullptr;
  if (P.mixed) {
    CK(dalloc(R, &P.yf, nv));
    CK(dalloc(R, &P.lgf, nl));
  }
  P.xp = nullptr;
  P.alpha = nullptr;
  P.clampb = nullptr;
  if (R.ccd) {
    CK(dalloc(R, &P.xp, nv));
    CK(dalloc(R, &P.alpha, nv));
    CK(dalloc(R, &P.clampb, nv));
  }
  CK(upload(R, &P.im, im));
  CK(upload(R, &P.rho, rho));
  CK(dalloc(R, &P.r, nv));
  CK(dalloc(R, &P.Dv, nv));
  CK(upload(R, &P.vscene, vscene));
  CK(upload(R, &P.vflag, vflag));
  CK(upload(R, &P.tv, tv));
  CK(upload(R, &P.ev, ev));
  CK(upload(R, &P.lv, lv));
  CK(dalloc(R, &P.lg, nl));
  CK(upload(R, &P.vc, vc));
  CK(upload(R, &P.pts, pts));
  CK(upload(R, &P.sd, R.sd));
  CK(dalloc(R, &P.ss, n_scenes));
  CK(cudaMemset(P.ss, 0, sizeof(SceneState) * n_scenes));
  CK(dalloc(R, &P.cnt, 1));
  CK(cudaMemset(P.cnt, 0, sizeof(Counters)));
  CK(dalloc(R, &P.cmask, (size_t)nv * 32));
  CK(dalloc(R, &P.chw, nv));
  CK(dalloc(R, &P.vlevel, nv));
  CK(dalloc(R, &P.ccount, 2048));
  CK(cudaMemset(P.ccount, 0, 2048 * sizeof(int)));
  CK(dalloc(R, &P.coff, 2048 + 1));
  CK(dalloc(R, &P.cfill, 2048));
  CK(dalloc(R, &P.bar, 2));
  CK(cudaMemset(P.bar, 0, 2 * sizeof(unsigned int)));
  CK(dalloc(R, &P.vmin, nv));
  P.vlstart = nullptr;
  P.vllist = nullptr;
  if (R.solver == CCH_SOLVER_JACOBI) {
    // per-vertex lists of edge-length constraints in ascending edge order
    // (the canonical summation order of the Jacobi update)
    std::vector<int> vls((size_t)nv + 1, 0), vll(2 * (size_t)nl);
    for (int e = 0; e < nl; e++) {
      vls[lv[e].x + 1]++;
      vls[lv[e].y + 1]++;
    }
    for (int v = 0; v < nv; v++) vls[v + 1] += vls[v];
    std::vector<int> fill(vls.begin(), vls.end() - 1);
    for (int e = 0; e < nl; e++) {
      vll[fill[lv[e].x]++] = 2 * e;
      vll[fill[lv[e].y]++] = 2 * e + 1;
    }
    CK(upload(R, &P.vlstart, vls));
    CK(upload(R, &P.vllist, vll));
  }
  {
    // per-vertex lists of incident triangle corners (the pre-passes' gathers)
    std::vector<int> ts((size_t)nv + 1, 0), tl(3 * (size_t)nt);
    for (int t = 0; t < nt; t++) {
      ts[tv[t].x + 1]++;
      ts[tv[t].y + 1]++;
      ts[tv[t].z + 1]++;
    }
    for (int v = 0; v < nv; v++) ts[v + 1] += ts[v];
    std::vector<int> fill(ts.begin(), ts.end() - 1);
    for (int t = 0; t < nt; t++) {
      tl[fill[tv[t].x]++] = 3 * t;
      tl[fill[tv[t].y]++] = 3 * t + 1;
      tl[fill[tv[t].z]++] = 3 * t + 2;
    }
    CK(upload(R, &P.tinc_start, ts));
    CK(upload(R, &P.tinc, tl));
  }
  CK(dalloc(R, &P.sbox, 2 * (size_t)n_scenes));
  CK(alloc_bvh(R, P.bt, nt, n_scenes));
  CK(alloc_bvh(R, P.be, ne, n_scenes));
  CK(alloc_bvh(R, P.bv, P.nvc, n_scenes));
  P.qcap = 1 << 16;
  CK(dalloc(R, &P.qkeys, P.qcap));
  CK(dalloc(R, &P.qdist, P.qcap));
  CK(cudaMallocHost(&R.h_ptrs, sizeof(double*) * 3 * n_scenes));
  CK(cudaMallocHost(&R.h_cnt, sizeof(Counters)));
  CK(cudaMallocHost(&R.h_ss, sizeof(SceneState) * n_scenes));
  CK(dalloc(R, &R.d_ptrs, 3 * (size_t)n_scenes));
  CK(cudaEventCreate(&R.ev0));
  CK(cudaEventCreate(&R.ev1));
  CK(dalloc(R, &R.obuf.vstart, (size_t)nv + 1));
  CK(dalloc(R, &R.obuf.tsum, ((size_t)nv + 1) / 8192 + 2));
  CK(dalloc(R, &R.obuf.vfill, nv));
  CK(dalloc(R, &R.obuf.vdone, nv));
  {
    // Colour classes of the edge-length constraints (topology only; Sec.
    // 4.3, reading R11): taken by descending priority splitmix64(seed ^ key),
    // key = 3 << 62 | local edge index, each edge gets the smallest colour
    // not used by an earlier edge at one of its movable vertices.
    std::vector<unsigned long long> eprio(nl);
    std::vector<int> order(nl), edeg(nv, 0);
    for (int e = 0; e < nl; e++) {
      const SceneDesc& d = R.sd[lv[e].z];
      eprio[e] = splitmix64(d.seed ^ ((3ULL << 62) | (unsigned long long)(e - d.l0)));
      order[e] = e;
      edeg[lv[e].x]++;
      edeg[lv[e].y]++;
    }
    R.max_vedges = 0;
    for (int v = 0; v < nv; v++)
      if ((vflag[v] & VF_MOVABLE) && edeg[v] > R.max_vedges) R.max_vedges = edeg[v];
    std::sort(order.begin(), order.end(), [&](int p, int q) { return eprio[p] > eprio[q]; });
    // greedy: the smallest colour not used at its movable ends so far; level:
    // one more than the largest colour there so far
    std::vector<std::vector<int>> used(nv);
    std::vector<int> top(nv, -1);
    std::vector<int> ecol(nl, 0);
    std::vector<char> taken;
    P.n_ecol = 0;
    for (int e : order) {
      int ends[2] = {lv[e].x, lv[e].y};
      int c = 0;
      if (R.colouring == CCH_COLOUR_LEVEL) {
        for (int v : ends)
          if ((vflag[v] & VF_MOVABLE) && top[v] + 1 > c) c = top[v] + 1;
        for (int v : ends)
          if (vflag[v] & VF_MOVABLE) top[v] = c;
      } else {
        size_t tot = 0;
        for (int v : ends)
          if (vflag[v] & VF_MOVABLE) tot += used[v].size();
        taken.assign(tot + 1, 0);
        for (int v : ends)
          if (vflag[v] & VF_MOVABLE)
            for (int u : used[v])
              if ((size_t)u <= tot) taken[u] = 1;
        while (taken[c]) c++;
        for (int v : ends)
          if (vflag[v] & VF_MOVABLE) used[v].push_back(c);
      }
      ecol[e] = c;
      SceneDesc& d = R.sd[lv[e].z];
      if (c + 1 > d.n_ecol) d.n_ecol = c + 1;
      if (c + 1 > P.n_ecol) P.n_ecol = c + 1;
    }
    CK(upload(R, &P.ecol, ecol));
    // the edges grouped by colour, ascending index within a colour (the
    // colour-class sweep applies one group per phase)
    std::vector<int> eoff((size_t)P.n_ecol + 1, 0), eorder(nl);
    for (int e = 0; e < nl; e++) eoff[ecol[e] + 1]++;
    for (int c = 0; c < P.n_ecol; c++) eoff[c + 1] += eoff[c];
    {
      std::vector<int> fill(eoff.begin(), eoff.end() - 1);
      for (int e = 0; e < nl; e++) eorder[fill[ecol[e]]++] = e;
    }
    CK(upload(R, &P.eorder, eorder));
    CK(upload(R, &P.eoff, eoff));
    CK(cudaMemcpy(P.sd, R.sd.data(), sizeof(SceneDesc) * R.sd.size(), cudaMemcpyHostToDevice));
    // the level colouring's dataflow sweep waits on each edge's rank among
    // the edges of each of its vertices, by descending priority
    std::vector<int> estart((size_t)nv + 1, 0), elist(2 * (size_t)nl);
    for (int v = 0; v < nv; v++) estart[v + 1] = estart[v] + edeg[v];
    std::vector<int> fill(estart.begin(), estart.end() - 1);
    for (int e = 0; e < nl; e++) {
      elist[fill[lv[e].x]++] = 2 * e;
      elist[fill[lv[e].y]++] = 2 * e + 1;
    }
    std::vector<int2> erank(nl);
    for (int v = 0; v < nv; v++) {
      int a = estart[v], b = estart[v + 1];
      std::sort(elist.begin() + a, elist.begin() + b,
                [&](int p, int q) { return eprio[p >> 1] > eprio[q >> 1]; });
      for (int r = 0; r < b - a; r++) {
        int ent = elist[a + r];
        if (ent & 1) erank[ent >> 1].y = r;
        else erank[ent >> 1].x = r;
      }
    }
    CK(upload(R, &P.edeg, edeg));
    CK(upload(R, &P.erank, erank));
  }
  // pair-sized buffers last (they are re-allocated on growth)
  long long guess = prm->pair_capacity > 0 ? (long long)prm->pair_capacity : 4LL * (nt + ne + nq) + 4096;
  if (guess > (1LL << 30)) guess = 1LL << 30;
  set_caps(R, (int)guess);
  CK(alloc_pairs(R));
  return CCH_OK;
}

cch_status grow_pairs(Runtime& R) {
  long long cap = 2LL * R.pool.pair_cap;
  if (cap > (1LL << 30)) return CCH_E_CAPACITY;
  CK(cudaStreamSynchronize(R.stream));
  free_pairs(R);
  set_caps(R, (int)cap);
  CK(alloc_pairs(R));
  if (R.graph) cudaGraphExecDestroy(R.graph);
  R.graph = nullptr;
  return CCH_OK;
}

// Two iterations (pair buffers 0 -> 1 -> 0) captured as one graph.
cudaError_t capture_graph(Runtime& R) {
  if (R.graph) {
    cudaGraphExecDestroy(R.graph);
    R.graph = nullptr;
  }
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g;
  long long before = R.launches;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = iteration(R, 0, cs);
    cudaError_t e2 = iteration(R, 1, cs);
    R.graph_launches = R.launches - before;
    R.launches = before;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && (e1 != cudaSuccess || e2 != cudaSuccess)) e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&R.graph, g, 0);
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  cudaGetLastError();
  return e;
}

void fill_stats(const Runtime& R, int s, const SceneState& S, cch_step_stats* st, float ms) {
  st->iterations = S.iter;
  st->searches = S.searches;
  st->converged = S.converged;
  st->ccd_clamps = S.ccd_clamps;
  st->pairs_evaluated = S.pairs_eval;
  st->max_pairs = S.max_pairs;
  st->active_contacts = S.contacts;
  st->candidates = S.candidates;
  st->degenerate = S.degenerate;
  st->max_vertex_contacts = S.max_vcontacts;
  st->max_vertex_edges = R.max_vedges;
  // the sweep's critical path: one phase per colour class
  st->gs_depth = R.solver == CCH_SOLVER_GAUSS_SEIDEL ? S.ccol + R.sd[s].n_ecol : 0;
  st->final_r_inf = S.final_r;
  union { unsigned long long u; double d; } b;
  b.u = S.mind_bits;
  st->min_pair_dist = b.d;
  st->intersections = S.isect;
  st->uncertain = S.uncertain;
  st->device_ms = ms;
  st->frozen_vertices = S.frozen;
  st->contact_vertices = S.cverts;
  st->pair_vertices = S.pverts;
  st->contact_colours = S.ccol;
  st->edge_colours = R.sd[s].n_ecol;
}

// Accumulates the event times of the kernel groups recorded since the last call.
void prof_collect(Runtime& R) {
  if (!R.profiling || !R.prof_used) return;
  for (int g = 0; g < PG_N; g++)
    if (R.prof_used & (1u << g)) {
      cudaEventSynchronize(R.pev[g][1]);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, R.pev[g][0], R.pev[g][1]) == cudaSuccess) {
        R.prof_ms[g] += ms;
        R.prof_n[g]++;
      }
    }
  R.prof_used = 0;
}

// Runs Algorithm 1 on every scene of the pool; pointer table already set.
cch_status run_step(cch_scene* S, cch_step_stats* stats) {
  Runtime& R = S->R;
  Pool& P = R.pool;
  cudaStream_t st = R.stream;
  for (int attempt = 0; attempt < 24; attempt++) {
    CK(cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3 * S->n_scenes, cudaMemcpyHostToDevice, st));
    long long launches0 = R.launches;
    CK(cudaEventRecord(R.ev0, st));
    prof_mark(R, PG_SETUP, 0, st);
    step_init(R, st, 0);
    set_any_search(R, st);
    bvh_build_all(R, st);
    prof_mark(R, PG_SETUP, 1, st);
    prof_collect(R);
    CK(cudaGetLastError());
    if (R.validate) {
      // the method assumes x^t is intersection-free (Sec. 3)
      bvh_refit_all(R, st, 1);
      accept_queries(R, st);
      CK(cudaMemcpyAsync(R.h_ss, P.ss, sizeof(SceneState) * S->n_scenes, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int s = 0; s < S->n_scenes; s++)
        if (R.h_ss[s].isect > 0) return CCH_E_INPUT_NOT_FEASIBLE;
      reset_accept(R, st);
    }
    if (R.use_graphs && !R.profiling && !R.graph) {
      if (capture_graph(R) != cudaSuccess) R.use_graphs = 0;
    }
    int cur = 0, iters = 0;
    int limit = R.max_iters + 2;
    bool overflow = false;
    while (iters < limit) {
      int chunk = R.iters_per_check;
      if (R.use_graphs && !R.profiling && R.graph) {
        for (int k = 0; k < chunk; k += 2) {
          CK(cudaGraphLaunch(R.graph, st));
          R.launches += R.graph_launches;
        }
        iters += (chunk + 1) / 2 * 2;
      } else {
        for (int k = 0; k < chunk; k++) {
          CK(iteration(R, cur, st));
          prof_collect(R);
          cur = 1 - cur;
        }
        iters += chunk;
      }
      CK(cudaMemcpyAsync(R.h_cnt, P.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (R.h_cnt->err && getenv("CCH_DEBUG"))
        fprintf(stderr, "cch: iteration %d err=%d overflow=%d n_cons=%d pairs=%d/%d\n", iters,
                R.h_cnt->err, R.h_cnt->overflow, R.h_cnt->n_cons,
                R.h_cnt->n_pairs[0], R.h_cnt->n_pairs[1]);
      if (R.h_cnt->err) return device_status(R.h_cnt->err);
      if (R.h_cnt->overflow & (OV_PAIRS | OV_CONTACTS)) {
        overflow = true;
        break;
      }
      if (R.h_cnt->all_done) break;
    }
    if (overflow) {
      cch_status g = grow_pairs(R);
      if (g != CCH_OK) return g;
      continue;
    }
    if (R.accept) {
      // exact-filtered intersection test of x^{t+1}
      bvh_refit_all(R, st, 1);
      accept_queries(R, st);
    }
    prof_mark(R, PG_OUTPUT, 0, st);
    output(R, st);
    prof_mark(R, PG_OUTPUT, 1, st);
    CK(cudaEventRecord(R.ev1, st));
    CK(cudaMemcpyAsync(R.h_ss, P.ss, sizeof(SceneState) * S->n_scenes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    prof_collect(R);
    for (int s = 0; s < S->n_scenes; s++)
      if (R.h_ss[s].bad_input) return CCH_E_INVALID_ARG;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, R.ev0, R.ev1);
    if (stats)
      for (int s = 0; s < S->n_scenes; s++) {
        fill_stats(R, s, R.h_ss[s], &stats[s], ms);
        stats[s].kernel_launches = R.launches - launches0;
      }
    return CCH_OK;
  }
  return CCH_E_CAPACITY;
}

}  // namespace

extern "C" {

cch_status cch_params_default(cch_params* p) {
  if (!p) return CCH_E_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->d_min = 2e-3;
  p->d_max = 4e-3;
  p->delta = 1e-3;
  p->sigma = 1.1;
  p->gamma = 0.9;
  p->eps = 1e-4;
  p->jacobi_omega = 0.5;
  p->max_iters = 2048;
  p->gs_sweeps = 1;
  p->precision = CCH_PREC_FP64;
  p->solver = CCH_SOLVER_GAUSS_SEIDEL;
  p->ccd_check = 0;
  p->accept_check = 0;
  p->validate_input = 0;
  p->iters_per_launch = 16;
  p->bvh_refit_only = 1;
  p->constraint_form = CCH_FORM_VOLUME;
  p->step_rule = CCH_STEP_DISTANCE;
  p->ccd_rounds = 8;
  p->colouring = CCH_COLOUR_LEVEL;
  p->seed = 0x2211040450ULL;
  return CCH_OK;
}

const char* cch_status_string(cch_status s) {
  switch (s) {
    case CCH_OK: return "ok";
    case CCH_E_INVALID_ARG: return "invalid argument";
    case CCH_E_OOM: return "out of device memory";
    case CCH_E_BUDGET: return "HBM budget exceeded";
    case CCH_E_CUDA: return "CUDA error";
    case CCH_E_CAPACITY: return "internal capacity exceeded";
    case CCH_E_TIMEOUT: return "bounded device loop timed out";
    case CCH_E_INPUT_NOT_FEASIBLE: return "input state intersects";
    case CCH_E_CANCELLED: return "cancelled";
    case CCH_E_STATE: return "invalid state";
  }
  return "unknown status";
}

cch_status cch_create_batch_params(const cch_topology* topos, int32_t n_scenes, const cch_params* prm,
                                   const cch_params* scene_prm, void* stream,
                            cch_scene** out) {
  if (!out || !topos || n_scenes <= 0 || n_scenes > (1 << 20)) return CCH_E_INVALID_ARG;
  *out = nullptr;
  cch_status v = validate_params(prm);
  if (v != CCH_OK) return v;
  long long tot = 0;
  for (int s = 0; s < n_scenes; s++) {
    v = validate_topology(&topos[s]);
    if (v != CCH_OK) return v;
    tot += topos[s].n_verts;
    if (scene_prm && (v = validate_params(&scene_prm[s])) != CCH_OK) return v;
  }
  if (tot >= (1LL << 30)) return CCH_E_INVALID_ARG;
  cch_scene* S = new cch_scene();
  cch_status r = build_pool(S, topos, n_scenes, prm, scene_prm, stream);
  if (r != CCH_OK) {
    free_all(S->R);
    delete S;
    return r;
  }
  *out = S;
  return CCH_OK;
}

cch_status cch_create_batch(const cch_topology* topos, int32_t n_scenes, const cch_params* prm, void* stream,
                            cch_scene** out) {
  return cch_create_batch_params(topos, n_scenes, prm, nullptr, stream, out);
}

cch_status cch_create_scene(const cch_topology* topo, const cch_params* prm, void* stream, cch_scene** out) {
  return cch_create_batch(topo, 1, prm, stream, out);
}

cch_status cch_batch_handle_step(cch_scene* S, const double* const* x_t, const double* const* x_tilde,
                                 double* const* x_next, cch_step_stats* stats) {
  if (!S || !x_t || !x_tilde || !x_next) return CCH_E_INVALID_ARG;
  for (int s = 0; s < S->n_scenes; s++) {
    if (!x_t[s] || !x_tilde[s] || !x_next[s]) return CCH_E_INVALID_ARG;
    S->R.h_ptrs[3 * s] = (double*)x_t[s];
    S->R.h_ptrs[3 * s + 1] = (double*)x_tilde[s];
    S->R.h_ptrs[3 * s + 2] = x_next[s];
  }
  return run_step(S, stats);
}

cch_status cch_handle_step(cch_scene* S, const double* x_t, const double* x_tilde, double* x_next,
                           cch_step_stats* stats) {
  if (!S || S->n_scenes != 1) return CCH_E_INVALID_ARG;
  return cch_batch_handle_step(S, &x_t, &x_tilde, &x_next, stats);
}

cch_status cch_handle_step_host(cch_scene* S, const double* x_t, const double* x_tilde, double* x_next,
                                cch_step_stats* stats) {
  if (!S || S->n_scenes != 1 || !x_t || !x_tilde || !x_next) return CCH_E_INVALID_ARG;
  size_t bytes = sizeof(double) * 3 * (size_t)S->nverts[0];
  double *dt = nullptr, *dl = nullptr;
  cudaStream_t st = S->R.stream;
  // staging buffers of the scene, allocated on first use
  static_assert(sizeof(double) == 8, "");
  CK(cudaMallocAsync(&dt, bytes, st));
  CK(cudaMallocAsync(&dl, bytes, st));
  cudaError_t e = cudaMemcpyAsync(dt, x_t, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dl, x_tilde, bytes, cudaMemcpyHostToDevice, st);
  cch_status r = e == cudaSuccess ? cch_handle_step(S, dt, dl, dt, stats) : cuda_fail(e);
  if (r == CCH_OK) {
    e = cudaMemcpyAsync(x_next, dt, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e);
  }
  cudaFreeAsync(dt, st);
  cudaFreeAsync(dl, st);
  cudaStreamSynchronize(st);
  return r;
}

// Autotuner of the launch configuration.  Candidate
// values are timed on a probe (one step from the caller's inputs, capped at
// probe_iters iterations) by coordinate descent: iterations per graph launch
// group, the block size of the BVH queries, BVH refit against rebuild, and
// warp-packet against thread-per-query traversal.  The configuration does not change results; every probe's output
// is compared bitwise with the first and the outcome reported.
namespace {
struct TuneCfg {
  int g, block, refit, packet;
};
cch_status time_probe(cch_scene* S, const TuneCfg& c, double* ms, std::vector<double>& out, double* dout,
                      size_t n3) {
  Runtime& R = S->R;
  if (R.iters_per_check != c.g || R.query_block != c.block || R.refit_only != c.refit || R.packet != c.packet) {
    if (R.graph) cudaGraphExecDestroy(R.graph);
    R.graph = nullptr;
  }
  R.iters_per_check = c.g;
  R.query_block = c.block;
  R.refit_only = c.refit;
  R.packet = c.packet;
  double best = 1e300;
  for (int rep = 0; rep < 2; rep++) {
    cch_step_stats st;
    cch_status r = run_step(S, &st);
    if (r != CCH_OK) return r;
    if (st.device_ms < best) best = st.device_ms;
  }
  *ms = best;
  out.resize(n3);
  CK(cudaMemcpy(out.data(), dout, sizeof(double) * n3, cudaMemcpyDeviceToHost));
  return CCH_OK;
}
}  // namespace

cch_status cch_autotune(cch_scene* S, const double* x_t, const double* x_tilde, int32_t probe_iters,
                        cch_tune_result* out) {
  if (!S || S->n_scenes != 1 || !x_t || !x_tilde || !out || probe_iters < 1 || probe_iters > 4096)
    return CCH_E_INVALID_ARG;
  Runtime& R = S->R;
  size_t n3 = 3 * (size_t)S->nverts[0];
  double* dout = nullptr;
  CK(cudaMalloc(&dout, sizeof(double) * (n3 > 0 ? n3 : 1)));
  R.h_ptrs[0] = (double*)x_t;
  R.h_ptrs[1] = (double*)x_tilde;
  R.h_ptrs[2] = dout;
  // cap the probe's loop at probe_iters
  std::vector<SceneDesc> capped = R.sd;
  for (auto& d : capped) d.max_iters = probe_iters;
  int saved_max = R.max_iters;
  cudaError_t e = cudaMemcpy(R.pool.sd, capped.data(), sizeof(SceneDesc) * capped.size(), cudaMemcpyHostToDevice);
  R.max_iters = probe_iters;
  TuneCfg best{R.iters_per_check, R.query_block, R.refit_only, R.packet};
  double best_ms = 0.0, default_ms = 0.0;
  int trials = 0, consistent = 1;
  std::vector<double> ref, got;
  cch_status r = e == cudaSuccess ? time_probe(S, best, &best_ms, ref, dout, n3) : cuda_fail(e);
  default_ms = best_ms;
  trials++;
  static const int gs[] = {4, 8, 16, 32, 64}, blocks[] = {64, 128, 256}, binary[] = {1, 0};
  for (int stage = 0; stage < 4 && r == CCH_OK; stage++) {
    int nc = stage == 0 ? 5 : (stage == 1 ? 3 : 2);
    for (int k = 0; k < nc && r == CCH_OK; k++) {
      TuneCfg c = best;
      if (stage == 0) c.g = gs[k];
      if (stage == 1) c.block = blocks[k];
      if (stage == 2) c.refit = binary[k];
      if (stage == 3) c.packet = binary[k];
      if (c.g == best.g && c.block == best.block && c.refit == best.refit && c.packet == best.packet) continue;
      double ms = 0.0;
      r = time_probe(S, c, &ms, got, dout, n3);
      trials++;
      if (r != CCH_OK) break;
      if (got != ref) consistent = 0;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  // restore the loop bound, keep the fastest configuration
  cudaMemcpy(R.pool.sd, R.sd.data(), sizeof(SceneDesc) * R.sd.size(), cudaMemcpyHostToDevice);
  R.max_iters = saved_max;
  if (R.graph) cudaGraphExecDestroy(R.graph);
  R.graph = nullptr;
  R.iters_per_check = best.g;
  R.query_block = best.block;
  R.refit_only = best.refit;
  R.packet = best.packet;
  cudaFree(dout);
  if (r != CCH_OK) return r;
  out->iters_per_launch = best.g;
  out->query_block = best.block;
  out->bvh_refit_only = best.refit;
  out->trials = trials;
  out->consistent = consistent;
  out->packet_traversal = best.packet;
  out->best_ms = best_ms;
  out->default_ms = default_ms;
  return CCH_OK;
}

cch_status cch_destroy(cch_scene* S) {
  if (!S) return CCH_E_INVALID_ARG;
  cudaStreamSynchronize(S->R.stream);
  free_all(S->R);
  delete S;
  return CCH_OK;
}

cch_status cch_set_max_polls(cch_scene* S, int32_t max_polls) {
  if (!S || max_polls < 0) return CCH_E_INVALID_ARG;
  S->R.max_polls = max_polls > 0 ? max_polls : 1 << 22;
  if (S->R.graph) cudaGraphExecDestroy(S->R.graph);  // the bound is a kernel argument
  S->R.graph = nullptr;
  return CCH_OK;
}

namespace {
// P as the first search of a step forms it (want_candidates = 2): the
// step's own search kernels at D^max write the pair buffer, which is copied
// out.
cch_status query_step_search(cch_scene* S, const double* x, const double* x_ref, uint64_t* keys, double* dist,
                             int64_t cap, int64_t* count) {
  Runtime& R = S->R;
  Pool& P = R.pool;
  cudaStream_t st = R.stream;
  for (int attempt = 0; attempt < 32; attempt++) {
    R.h_ptrs[0] = (double*)x;
    R.h_ptrs[1] = (double*)x_ref;
    R.h_ptrs[2] = nullptr;
    CK(cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3, cudaMemcpyHostToDevice, st));
    step_init(R, st, 0);
    set_any_search(R, st);
    bvh_build_all(R, st);
    bvh_refit_all(R, st, 1);
    for (int c = 0; c < 3; c++) query_class(R, c, 1, 0, 0.0, st);
    if (!P.mixed) CK(cudaMemsetAsync(P.vmin, 0xff, sizeof(unsigned int) * (size_t)P.nv, st));
    finalize_search(R, 1, 0, 0.0, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(R.h_cnt, P.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (R.h_cnt->err) return device_status(R.h_cnt->err);
    if (R.h_cnt->overflow & (OV_PAIRS | OV_CONTACTS)) {
      cch_status g = grow_pairs(R);
      if (g != CCH_OK) return g;
      continue;
    }
    int n = R.h_cnt->n_pairs[1];
    *count = n;
    int64_t m = n < cap ? n : cap;
    if (m > 0) {
      CK(cudaMemcpy(keys, P.pb[1].key, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost));
      if (dist) CK(cudaMemcpy(dist, P.pb[1].d, sizeof(double) * m, cudaMemcpyDeviceToHost));
    }
    return CCH_OK;
  }
  return CCH_E_CAPACITY;
}
}  // namespace

cch_status cch_query_pairs(cch_scene* S, const double* x, const double* x_ref, double D, int32_t want_candidates,
                           uint64_t* keys, double* dist, int64_t cap, int64_t* count) {
  if (!S || !x || !x_ref || !count || !(D >= 0.0) || cap < 0 || (cap > 0 && !keys)) return CCH_E_INVALID_ARG;
  if (S->n_scenes != 1 || want_candidates < 0 || want_candidates > 2) return CCH_E_INVALID_ARG;
  if (want_candidates == 2) return query_step_search(S, x, x_ref, keys, dist, cap, count);
  Runtime& R = S->R;
  Pool& P = R.pool;
  cudaStream_t st = R.stream;
  for (int attempt = 0; attempt < 32; attempt++) {
    R.h_ptrs[0] = (double*)x;
    R.h_ptrs[1] = (double*)x_ref;
    R.h_ptrs[2] = nullptr;
    CK(cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3, cudaMemcpyHostToDevice, st));
    step_init(R, st, 0);
    bvh_build_all(R, st);
    bvh_refit_all(R, st, 1);
    search_queries(R, 0, want_candidates ? 1 : 2, D, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(R.h_cnt, P.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (R.h_cnt->err) return device_status(R.h_cnt->err);
    if (R.h_cnt->overflow & OV_PAIRS) {
      // the FP32-filter survivors outgrew the pair-sized buffers
      cch_status g = grow_pairs(R);
      if (g != CCH_OK) return g;
      continue;
    }
    int n = R.h_cnt->n_query;
    if (n < 0) return CCH_E_CAPACITY;  // more than 2^31 results
    if (n > P.qcap) {
      // grow the inspection buffers and retry
      int cap2 = P.qcap;
      while (cap2 < n) cap2 *= 2;
      P.qcap = cap2;
      CK(dalloc(R, &P.qkeys, P.qcap));
      CK(dalloc(R, &P.qdist, P.qcap));
      continue;
    }
    *count = n;
    int64_t m = n < cap ? n : cap;
    if (m > 0) {
      CK(cudaMemcpy(keys, P.qkeys, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost));
      if (dist) CK(cudaMemcpy(dist, P.qdist, sizeof(double) * m, cudaMemcpyDeviceToHost));
    }
    return CCH_OK;
  }
  return CCH_E_CAPACITY;
}

// ---- proximity query without device allocation -----------------------------
// The pair list that the query kernels write before it is copied to the host
// lives in this fixed array instead of the scene's growable buffers, so the
// call below allocates nothing.  Keys occupy the first half, distances the
// second.  Every GPU that loads the library holds it until the process ends.
static __device__ __align__(256) unsigned char g_query_scratch[CCH_NOALLOC_MAX_PAIRS * 16];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a stand-in symbol, not the device address).
static cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_query_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

cch_status cch_query_pairs_noalloc(cch_scene* S, const double* x, const double* x_ref, double D,
                                   int32_t want_candidates, uint64_t* keys, double* dist, int64_t cap,
                                   int64_t* count) {
  if (!S || !x || !x_ref || !count || !(D >= 0.0) || cap < 0 || (cap > 0 && !keys)) return CCH_E_INVALID_ARG;
  if (S->n_scenes != 1 || want_candidates < 0 || want_candidates > 1) return CCH_E_INVALID_ARG;
  Runtime& R = S->R;
  cudaStream_t st = R.stream;
  void* scratch = nullptr;
  CK(scratch_address(&scratch));
  // run the query kernels with the fixed array as their output buffer
  Pool saved = R.pool;
  R.pool.qkeys = (unsigned long long*)scratch;
  R.pool.qdist = (double*)((unsigned char*)scratch + CCH_NOALLOC_MAX_PAIRS * 8);
  R.pool.qcap = CCH_NOALLOC_MAX_PAIRS;
  R.h_ptrs[0] = (double*)x;
  R.h_ptrs[1] = (double*)x_ref;
  R.h_ptrs[2] = nullptr;
  cudaError_t e = cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    step_init(R, st, 0);
    bvh_build_all(R, st);
    bvh_refit_all(R, st, 1);
    search_queries(R, 0, want_candidates ? 1 : 2, D, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(R.h_cnt, R.pool.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  Pool used = R.pool;
  R.pool = saved;
  if (e != cudaSuccess) return cuda_fail(e);
  if (R.h_cnt->err) return device_status(R.h_cnt->err);
  // the scene's pair buffers overflowed: the query's result is incomplete
  // and its full count unknown
  if (R.h_cnt->overflow & OV_PAIRS) {
    *count = -1;
    return CCH_E_CAPACITY;
  }
  int64_t n = R.h_cnt->n_query;
  if (n < 0) n = (int64_t)1 << 31;  // the counter passed 2^31
  *count = n;
  // more pairs than the array holds
  if (n > CCH_NOALLOC_MAX_PAIRS) return CCH_E_CAPACITY;
  int64_t m = n < cap ? n : cap;
  if (m > 0) {
    CK(cudaMemcpy(keys, used.qkeys, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost));
    if (dist) CK(cudaMemcpy(dist, used.qdist, sizeof(double) * m, cudaMemcpyDeviceToHost));
  }
  return CCH_OK;
}

cch_status cch_normal_flow_target(cch_scene* S, const double* x, double beta, double alpha, double sign,
                                  int32_t iters, double* y) {
  if (!S || S->n_scenes != 1 || !x || !y || x == y || iters < 0 || iters > 64) return CCH_E_INVALID_ARG;
  if (!std::isfinite(beta) || !std::isfinite(alpha) || !std::isfinite(sign)) return CCH_E_INVALID_ARG;
  Runtime& R = S->R;
  cudaStream_t st = R.stream;
  // the second buffer of the Jacobi steps: the pool's y array (free between steps)
  double* tmp = nullptr;
  if (iters > 0) {
    static_assert(sizeof(P4) >= 3 * sizeof(double), "");
    tmp = (double*)R.pool.y;
  }
  normal_flow(R, x, y, tmp, sign * beta, alpha, iters, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return CCH_OK;
}

cch_status cch_friction_filter(cch_scene* S, const double* x, const double* y, double* y_out, double mu,
                               double reach, double sep) {
  if (!S || S->n_scenes != 1 || !x || !y || !y_out) return CCH_E_INVALID_ARG;
  if (!(mu >= 0.0) || !(reach > 0.0) || !(sep >= 0.0) || !std::isfinite(mu) || !std::isfinite(reach) ||
      !std::isfinite(sep))
    return CCH_E_INVALID_ARG;
  Runtime& R = S->R;
  Pool& P = R.pool;
  cudaStream_t st = R.stream;
  // positions and target into the pool, BVHs at x
  R.h_ptrs[0] = (double*)x;
  R.h_ptrs[1] = (double*)y;
  R.h_ptrs[2] = nullptr;
  CK(cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3, cudaMemcpyHostToDevice, st));
  step_init(R, st, 0);
  bvh_build_all(R, st);
  bvh_refit_all(R, st, 1);
  friction(R, mu, reach, sep, y_out, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(R.h_cnt, P.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(R.h_ss, P.ss, sizeof(SceneState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (R.h_ss[0].bad_input) return CCH_E_INVALID_ARG;
  if (R.h_cnt->err) return device_status(R.h_cnt->err);
  return CCH_OK;
}

cch_status cch_set_profiling(cch_scene* S, int32_t on) {
  if (!S) return CCH_E_INVALID_ARG;
  Runtime& R = S->R;
  if (on && !R.pev[0][0])
    for (int g = 0; g < PG_N; g++)
      for (int k = 0; k < 2; k++) CK(cudaEventCreate(&R.pev[g][k]));
  R.profiling = on ? 1 : 0;
  for (int g = 0; g < PG_N; g++) {
    R.prof_ms[g] = 0.0;
    R.prof_n[g] = 0;
  }
  R.prof_used = 0;
  return CCH_OK;
}

cch_status cch_get_profile(cch_scene* S, double* ms, int64_t* count, int32_t n) {
  if (!S || !ms || !count || n < 0) return CCH_E_INVALID_ARG;
  for (int g = 0; g < n && g < PG_N; g++) {
    ms[g] = S->R.prof_ms[g];
    count[g] = S->R.prof_n[g];
  }
  return CCH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: resident scenes, a request queue and continuous batching
// ---------------------------------------------------------------------------
namespace {

struct OwnedTopo {  // host copy of a resident scene's topology
  std::vector<double> inv_mass, radius;
  std::vector<int32_t> tris, edges, len_edges, points;
  cch_topology view() const {
    cch_topology t{};
    t.n_verts = (int64_t)inv_mass.size();
    t.inv_mass = inv_mass.data();
    t.point_radius = radius.empty() ? nullptr : radius.data();
    t.n_tris = (int64_t)tris.size() / 3;
    t.tris = tris.data();
    t.n_edges = (int64_t)edges.size() / 2;
    t.edges = edges.data();
    t.n_len = (int64_t)len_edges.size() / 2;
    t.len_edges = len_edges.data();
    t.n_points = (int64_t)points.size();
    t.points = points.data();
    return t;
  }
};

using Clock = std::chrono::steady_clock;

struct Request {
  int scene = -1;
  const double* xt = nullptr;
  const double* xl = nullptr;
  double* xn = nullptr;
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  cch_status status = CCH_OK;
  cch_step_stats stats{};
};

// Device bytes a resident scene is expected to need (pool arrays, BVHs,
// pair-sized buffers at their initial capacity).
size_t scene_bytes(const cch_topology& t) {
  size_t prims = (size_t)(t.n_tris + t.n_edges + t.n_points);
  return 512 * (size_t)t.n_verts + 1600 * prims + 128 * (size_t)t.n_len + (1 << 20);
}

}  // namespace

struct cch_server {
  cch_params prm{};
  size_t budget = 0, used = 0;
  int max_active = 1;
  cudaStream_t stream = nullptr;
  std::vector<OwnedTopo> topos;
  std::vector<cch_params> sprm;   // per resident scene: its parameters
  cch_scene* pool = nullptr;      // built from every resident scene
  int pool_scenes = 0;            // scenes the pool was built with
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<int64_t> running;   // per scene: ticket in flight, or -1
  uint64_t next_ticket = 1;
  bool stop = false;
  cch_status fatal = CCH_OK;
  std::thread th;
};

namespace {

// Runs on the server's thread.  Between graph launches it retires finished
// requests and admits queued ones into free slots; admitted scenes start at
// iteration 0 while the others continue (per-scene loop state).
void server_loop(cch_server* sv) {
  std::unique_lock<std::mutex> lk(sv->mu);
  int cur = 0;
  std::vector<int> ends;
  while (!sv->stop) {
    int n_running = 0;
    for (int64_t t : sv->running) n_running += t >= 0;
    // rebuild the pool when scenes were added and nothing is in flight
    if (n_running == 0 && (!sv->pool || sv->pool_scenes != (int)sv->topos.size()) && !sv->topos.empty()) {
      if (sv->pool) cch_destroy(sv->pool);
      sv->pool = nullptr;
      std::vector<cch_topology> views;
      for (auto& t : sv->topos) views.push_back(t.view());
      int ns = (int)views.size();
      lk.unlock();
      cch_scene* p = nullptr;
      cch_status st = cch_create_batch_params(views.data(), ns, &sv->prm, sv->sprm.data(), sv->stream, &p);
      lk.lock();
      if (st != CCH_OK) {
        sv->fatal = st;
        for (auto& kv : sv->reqs)
          if (kv.second.state == 0) { kv.second.state = 2; kv.second.status = st; kv.second.t_done = Clock::now(); }
        sv->queue.clear();
        sv->cv_done.notify_all();
        sv->cv_work.wait(lk);
        continue;
      }
      sv->pool = p;
      sv->pool_scenes = ns;
      sv->running.assign(ns, -1);
      // nothing runs: the shared counters start clean
      cudaMemsetAsync(p->R.pool.cnt, 0, sizeof(Counters), sv->stream);
      cudaMemsetAsync(p->R.pool.ss, 0, sizeof(SceneState) * ns, sv->stream);
      cur = 0;
    }
    // admit queued requests into free slots
    std::vector<int> starting;
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      Request& r = sv->reqs[*it];
      if (r.scene < sv->pool_scenes && sv->running[r.scene] < 0 && n_running < sv->max_active) {
        sv->running[r.scene] = (int64_t)*it;
        r.state = 1;
        starting.push_back(r.scene);
        n_running++;
        it = sv->queue.erase(it);
      } else ++it;
    }
    if (n_running == 0) {
      sv->cv_work.wait(lk);
      continue;
    }
    cch_scene* S = sv->pool;
    Runtime& R = S->R;
    Pool& P = R.pool;
    cudaStream_t st = sv->stream;
    for (int s : starting) {
      Request& r = sv->reqs[(uint64_t)sv->running[s]];
      R.h_ptrs[3 * s] = (double*)r.xt;
      R.h_ptrs[3 * s + 1] = (double*)r.xl;
      R.h_ptrs[3 * s + 2] = r.xn;
    }
    lk.unlock();
    cudaError_t e = cudaSuccess;
    if (!starting.empty()) {
      e = cudaMemcpyAsync(R.d_ptrs, R.h_ptrs, sizeof(double*) * 3 * S->n_scenes, cudaMemcpyHostToDevice, st);
      static const int one = 1;
      for (int s : starting)
        if (e == cudaSuccess) e = cudaMemcpyAsync(&P.ss[s].start, &one, sizeof(int), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) {
        step_init(R, st, 2);
        set_any_search(R, st);
        bvh_build_all(R, st);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess && R.use_graphs && !R.graph && capture_graph(R) != cudaSuccess) R.use_graphs = 0;
    // one launch boundary: G iterations for every running scene
    for (int k = 0; k < R.iters_per_check && e == cudaSuccess; k += (R.use_graphs && R.graph) ? 2 : 1) {
      if (R.use_graphs && R.graph) {
        e = cudaGraphLaunch(R.graph, st);
        R.launches += R.graph_launches;
      } else {
        e = iteration(R, cur, st);
        cur = 1 - cur;
      }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.h_ss, P.ss, sizeof(SceneState) * S->n_scenes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.h_cnt, P.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    bool regrow = e == cudaSuccess && (R.h_cnt->overflow & (OV_PAIRS | OV_CONTACTS));
    bool broken = e != cudaSuccess || R.h_cnt->err;
    ends.clear();
    if (!broken && !regrow)
      for (int s = 0; s < S->n_scenes; s++)
        if (R.h_ss[s].active && R.h_ss[s].done) {
          output_scene(R, s, st);
          static const int zero = 0;
          cudaMemcpyAsync(&P.ss[s].active, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
          ends.push_back(s);
        }
    if (!ends.empty()) e = cudaStreamSynchronize(st);
    if (regrow && grow_pairs(R) != CCH_OK) broken = true;
    lk.lock();
    auto now = Clock::now();
    if (broken || e != cudaSuccess) {
      // fail every request in flight; the pool is rebuilt for the next ones
      for (size_t s = 0; s < sv->running.size(); s++)
        if (sv->running[s] >= 0) {
          Request& r = sv->reqs[(uint64_t)sv->running[s]];
          r.state = 2;
          r.status = e != cudaSuccess ? cuda_fail(e) : device_status(R.h_cnt->err);
          r.t_done = now;
          sv->running[s] = -1;
        }
      cch_destroy(sv->pool);
      sv->pool = nullptr;
      sv->pool_scenes = 0;
      cudaGetLastError();
      sv->cv_done.notify_all();
      continue;
    }
    if (regrow) {
      // larger buffers: every request in flight starts again from its inputs
      for (size_t s = 0; s < sv->running.size(); s++)
        if (sv->running[s] >= 0) {
          sv->queue.push_front((uint64_t)sv->running[s]);
          sv->reqs[(uint64_t)sv->running[s]].state = 0;
          sv->running[s] = -1;
        }
      static const int zero = 0;
      for (int s = 0; s < S->n_scenes; s++) cudaMemcpyAsync(&P.ss[s].active, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(P.cnt, 0, sizeof(Counters), st);
      cudaStreamSynchronize(st);
      continue;
    }
    for (int s : ends) {
      Request& r = sv->reqs[(uint64_t)sv->running[s]];
      fill_stats(R, s, R.h_ss[s], &r.stats, 0.f);
      r.state = 2;
      r.status = R.h_ss[s].bad_input ? CCH_E_INVALID_ARG : CCH_OK;
      r.t_done = now;
      r.stats.device_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
      sv->running[s] = -1;
    }
    if (!ends.empty()) sv->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

cch_status cch_server_create(size_t hbm_budget_bytes, const cch_params* prm, int32_t max_active, void* cuda_stream,
                             cch_server** out) {
  if (!out || max_active <= 0 || hbm_budget_bytes == 0) return CCH_E_INVALID_ARG;
  *out = nullptr;
  cch_status v = validate_params(prm);
  if (v != CCH_OK) return v;
  cch_server* sv = new cch_server();
  sv->prm = *prm;
  sv->budget = hbm_budget_bytes;
  sv->max_active = max_active;
  sv->stream = (cudaStream_t)cuda_stream;
  sv->th = std::thread(server_loop, sv);
  *out = sv;
  return CCH_OK;
}

cch_status cch_server_add_scene(cch_server* sv, const cch_topology* topo, int32_t* scene_id) {
  if (!sv) return CCH_E_INVALID_ARG;
  return cch_server_add_scene_params(sv, topo, &sv->prm, scene_id);
}

cch_status cch_server_add_scene_params(cch_server* sv, const cch_topology* topo, const cch_params* scene_prm,
                                       int32_t* scene_id) {
  if (!sv || !scene_id || !scene_prm) return CCH_E_INVALID_ARG;
  cch_status v = validate_topology(topo);
  if (v != CCH_OK) return v;
  if ((v = validate_params(scene_prm)) != CCH_OK) return v;
  size_t need = scene_bytes(*topo);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->used + need > sv->budget) return CCH_E_BUDGET;
  OwnedTopo t;
  t.inv_mass.assign(topo->inv_mass, topo->inv_mass + topo->n_verts);
  if (topo->point_radius) t.radius.assign(topo->point_radius, topo->point_radius + topo->n_verts);
  t.tris.assign(topo->tris, topo->tris + 3 * topo->n_tris);
  t.edges.assign(topo->edges, topo->edges + 2 * topo->n_edges);
  t.len_edges.assign(topo->len_edges, topo->len_edges + 2 * topo->n_len);
  t.points.assign(topo->points, topo->points + topo->n_points);
  sv->topos.push_back(std::move(t));
  sv->sprm.push_back(*scene_prm);
  sv->used += need;
  *scene_id = (int32_t)sv->topos.size() - 1;
  sv->cv_work.notify_all();
  return CCH_OK;
}

cch_status cch_server_submit(cch_server* sv, int32_t scene_id, const double* x_t, const double* x_tilde,
                             double* x_next, uint64_t* ticket) {
  if (!sv || !x_t || !x_tilde || !x_next || !ticket) return CCH_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (scene_id < 0 || scene_id >= (int32_t)sv->topos.size()) return CCH_E_INVALID_ARG;
  if (sv->stop) return CCH_E_STATE;
  uint64_t t = sv->next_ticket++;
  Request r;
  r.scene = scene_id;
  r.xt = x_t;
  r.xl = x_tilde;
  r.xn = x_next;
  r.t_submit = Clock::now();
  sv->reqs[t] = r;
  sv->queue.push_back(t);
  *ticket = t;
  sv->cv_work.notify_all();
  return CCH_OK;
}

cch_status cch_server_wait(cch_server* sv, uint64_t ticket, cch_step_stats* stats, double* latency_ms) {
  if (!sv) return CCH_E_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return CCH_E_INVALID_ARG;
  sv->cv_done.wait(lk, [&] { return it->second.state == 2; });
  Request r = it->second;
  sv->reqs.erase(it);
  if (stats) *stats = r.stats;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  return r.status;
}

cch_status cch_server_destroy(cch_server* sv) {
  if (!sv) return CCH_E_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (auto& kv : sv->reqs)
      if (kv.second.state != 2) { kv.second.state = 2; kv.second.status = CCH_E_CANCELLED; }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  if (sv->pool) cch_destroy(sv->pool);
  delete sv;
  return CCH_OK;
}

}  // extern "C"

// cch_host.h -- declarations shared by the CUDA translation units of the
// library: the host runtime object and the device helpers used by both the
// proximity search and the per-iteration kernels.
#pragma once
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cuda_runtime.h>

#include <vector>

#include "cch_dev.cuh"

namespace cch {
namespace cg = cooperative_groups;

// Kernel groups timed by the profiling mode (CUDA events on the stream).
enum ProfGroup {
  PG_REFIT, PG_VT, PG_EE, PG_VV, PG_REFRESH, PG_ASSEMBLE, PG_ORDER, PG_SWEEP, PG_FORWARD, PG_CONTROL, PG_SETUP,
  PG_OUTPUT, PG_FINAL, PG_COLOUR, PG_N
};

// Per-vertex incidence lists of the contacts of one iteration (see
// cch_step.cu): the order of the backward step's sweep at each vertex.
struct OrderBufs {
  int* vstart;               // N+1: incidence counts, scanned in place to bucket starts
  int* vfill;                // N: bucket fill cursors
  int* vdone;                // N: constraints applied at the vertex so far
  unsigned long long* iprio; // incidences: priority (Jacobi: key)
  int* iid;                  // incidences: constraint * 4 + slot
  int* rank;                 // constraint * 4 + slot: rank at that vertex
  int* tsum;                 // tile totals of the multi-block scan of vstart
};

// Host-side runtime of one pool of scenes (a single scene, a batch, or the
// resident scenes of a server).
struct Runtime {
  Pool pool{};                       // device pointers and sizes
  std::vector<SceneDesc> sd;         // host copy of the scene table
  std::vector<void*> allocs;         // device allocations of the pool
  std::vector<void*> pair_allocs;    // pair-sized buffers (grown on overflow)
  cudaStream_t stream = nullptr;
  int scene_bits = 0;                // bits of the scene index in Morton keys
  int coop_blocks = 0;               // grid of the cooperative colouring kernel
  int sweep_blocks = 0;              // grid of the cooperative sweep kernel
  int max_polls = 1 << 22;           // bound of one device wait (polls)
  int sweeps = 1, solver = 0, ccd = 0, accept = 0, validate = 0;
  int colouring = 1;                 // cch_colouring of the Gauss-Seidel sweep
  int ccd_rounds = 8;  // CCD clamp rounds per iteration
  int max_iters = 0;                 // max over scenes
  int iters_per_check = 16;          // G: iterations per graph launch group (autotuned)
  int query_block = 128;             // threads per block of the BVH queries (autotuned)
  int refit_only = 1;                // 0: rebuild the BVH at every search (autotuned)
  int packet = 1;                    // warp-packet BVH traversal for the searches (autotuned)
  int use_graphs = 1;
  cudaGraphExec_t graph = nullptr;   // two captured iterations
  int graph_pair_cap = -1;
  double** d_ptrs = nullptr;         // device table: x_t, x_tilde, x_next per scene
  double** h_ptrs = nullptr;         // pinned host copy of the table
  Counters* h_cnt = nullptr;         // pinned host copy of the counters
  SceneState* h_ss = nullptr;        // pinned host copy of the scene states
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int max_vedges = 0;                // most edge-length constraints at one movable vertex
  OrderBufs obuf{};                  // sweep order of the contacts
  long long launches = 0;            // kernels launched by this runtime
  long long graph_launches = 0;      // kernels in one captured graph
  int profiling = 0;                 // time kernel groups with events
  unsigned prof_used = 0;
  cudaEvent_t pev[PG_N][2] = {};
  double prof_ms[PG_N] = {};
  long long prof_n[PG_N] = {};
};

inline void prof_mark(Runtime& R, int g, int which, cudaStream_t st) {
  if (!R.profiling) return;
  cudaEventRecord(R.pev[g][which], st);
  R.prof_used |= 1u << g;
}

__device__ __forceinline__ bool searching(const Pool& P, int s) {
  const SceneState& S = P.ss[s];
  return S.active && !S.done && S.do_search;
}

// Warp aggregation of a per-scene value: the active lanes of one scene combine
// their values with op, and one lane per scene calls done(result, lanes).  In
// a pool of one scene every lane shares the scene, so the whole coalesced
// group reduces at once (no partition by scene); min, max and sums of
// integers do not depend on the order, so both forms give the same result.
template <class T, class Op, class Done>
__device__ __forceinline__ void scene_reduce(const Pool& P, int s, T v, Op op, Done done) {
  cg::coalesced_group g = cg::coalesced_threads();
  if (P.nscene == 1) {
    T r = cg::reduce(g, v, op);
    if (g.thread_rank() == 0) done(r, (int)g.size());
    return;
  }
  auto part = cg::labeled_partition(g, s);
  T r = cg::reduce(part, v, op);
  if (part.thread_rank() == 0) done(r, (int)part.size());
}
// lanes of one scene counted once per warp
template <class Done>
__device__ __forceinline__ void scene_count(const Pool& P, int s, Done done) {
  cg::coalesced_group g = cg::coalesced_threads();
  if (P.nscene == 1) {
    if (g.thread_rank() == 0) done((int)g.size());
    return;
  }
  auto part = cg::labeled_partition(g, s);
  if (part.thread_rank() == 0) done((int)part.size());
}

__device__ __forceinline__ int append_idx(int* ctr) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(ctr, (int)g.size());
  return g.shfl(base, 0) + (int)g.thread_rank();
}

// Claims a slot below cap in an append counter, or returns -1 once the
// buffer is full.  The counter is read before the atomic add, so it stops
// growing soon after it reaches cap (only warps already past the read still
// add) and can never wrap around, whatever the number of appends.
__device__ __forceinline__ int claim(int* ctr, int cap) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = cap;
  if (g.thread_rank() == 0 && *(volatile int*)ctr < cap) base = atomicAdd(ctr, (int)g.size());
  int idx = g.shfl(base, 0) + (int)g.thread_rank();
  return idx < cap ? idx : -1;
}

// FP32 bounds (lower, upper) of a pair's FP64 distance from the float copy of
// the positions: d32 -/+ FILTER_TOL * (|x|max + extent), rounded outward.
// VT: point-triangle minus the point's radius; EE: segment-segment, whose
// lower bound is the separating-axis gap of f_ss_bounds; VV: centre distance
// minus both radii.  The lower bound is the one the search's FP32 filter
// uses.
__device__ __forceinline__ float2 pair_bounds32(const Pool& P, unsigned long long key, int4 v) {
  int kind = (int)(key >> 62);
  fv3 a = fk(P.xf[v.x]), b = fk(P.xf[v.y]);
  if (kind == K_VV) {
    fv3 d = fsub(a, b);
    float dd = sqrtf(fdot(d, d)), t = ftol(a, b, b, b);
    double r = P.rho[v.x] + P.rho[v.y];
    return make_float2(__fsub_rd(__fsub_rd(dd, __double2float_ru(r)), t),
                       __fadd_ru(__fsub_ru(dd, __double2float_rd(r)), t));
  }
  fv3 c = fk(P.xf[v.z]), d = fk(P.xf[v.w]);
  float t = ftol(a, b, c, d);
  if (kind == K_VT) {
    float dd = f_pt(a, b, c, d);
    double r = P.rho[v.x];
    return make_float2(__fsub_rd(__fsub_rd(dd, __double2float_ru(r)), t),
                       __fadd_ru(__fsub_ru(dd, __double2float_rd(r)), t));
  }
  // upper: a distance between two points of the segments; lower: the
  // separating-axis bound (see f_ss_bounds)
  float lo, dd = f_ss_bounds(a, b, c, d, __int_as_float(0x7f800000), &lo);
  return make_float2(__fsub_rd(lo, t), __fadd_ru(dd, t));
}

// Exact FP64 distances are needed only where they decide something: a pair
// whose upper bound is below D is certainly in P, and its exact distance is
// needed only if it may be a contact (lower < delta) or the closest pair at
// one of its vertices (lower <= the smallest upper bound among the certain
// pairs there).  Pass A records those smallest upper bounds per vertex.
__device__ __forceinline__ void min_at(unsigned int* p, unsigned int u) {
  if (u < __ldcg(p)) atomicMin(p, u);  // most pairs at a vertex are not its closest: skip their atomics
}
__device__ __forceinline__ void note_upper(Pool& P, int4 v, float up) {
  unsigned int u = fl_ord(up);
  min_at(&P.vmin[v.x], u);
  min_at(&P.vmin[v.y], u);
  if (v.z >= 0) min_at(&P.vmin[v.z], u);
  if (v.w >= 0) min_at(&P.vmin[v.w], u);
}
__device__ __forceinline__ bool needs_exact(const Pool& P, int4 v, float2 b, double D, double delta) {
  if (!((double)b.y < D) || (double)b.x < delta) return true;
  unsigned int lo = fl_ord(b.x);
  if (lo <= P.vmin[v.x] || lo <= P.vmin[v.y]) return true;
  if (v.z >= 0 && lo <= P.vmin[v.z]) return true;
  return v.w >= 0 && lo <= P.vmin[v.w];
}

// per-vertex minimum of the bits of non-negative doubles; a pair that is not
// the closest at the vertex so far skips the atomic
__device__ __forceinline__ void dmin_at(unsigned long long* p, unsigned long long b) {
  if (b < __ldcg(p)) atomicMin(p, b);
}

// Record one pair of P found at iteration l (search or refresh).
// mode 0: normal; 1: inspection of candidates; 2: inspection of P.
__device__ __forceinline__ void emit_pair(Pool& P, int nxt, int s, unsigned long long key, int4 v, double d) {
  const SceneDesc& S = P.sd[s];
  int idx = claim(&P.cnt->n_pairs[nxt], P.pair_cap);
  if (idx < 0) {
    atomicOr(&P.cnt->overflow, OV_PAIRS);
    return;
  }
  PairBuf& B = P.pb[nxt];
  B.key[idx] = key;
  B.v[idx] = v;
  B.d[idx] = d;
  unsigned long long db = dbits(d > 0.0 ? d : 0.0);
  dmin_at(&P.Dv[v.x], db);
  dmin_at(&P.Dv[v.y], db);
  if (v.z >= 0) dmin_at(&P.Dv[v.z], db);
  if (v.w >= 0) dmin_at(&P.Dv[v.w], db);
  scene_reduce(P, s, db, cg::less<unsigned long long>(), [&](unsigned long long m, int n) {
    atomicMin(&P.ss[s].mind_bits, m);
    atomicAdd(&P.ss[s].n_pairs, n);
  });
  if (d < S.delta) {
    // one list per kind, so that the assembly's warps run one kind's arithmetic
    int kind = (int)(key >> 62), a;
    if (kind == K_VT) a = claim(&P.cnt->n_active[0], P.act_cap);
    else if (kind == K_EE) a = claim(&P.cnt->n_active[1], P.act_cap);
    else a = claim(&P.cnt->n_active[2], P.act_cap);
    if (a >= 0) P.act[(size_t)kind * P.act_cap + a] = idx;
    else atomicOr(&P.cnt->overflow, OV_CONTACTS);
  }
}

__device__ __forceinline__ void emit_query(Pool& P, unsigned long long key, double d) {
  int idx = append_idx(&P.cnt->n_query);
  if ((unsigned)idx < (unsigned)P.qcap) {
    P.qkeys[idx] = key;
    P.qdist[idx] = d;
  } else atomicOr(&P.cnt->overflow, OV_QUERY);
}

__device__ __forceinline__ bool is_static(const Pool& P, int v) { return (P.vflag[v] & VF_STATIC) != 0; }


// conservative float box test of the BVH traversal: every axis gap of the
// two boxes, rounded down, at most Df
__device__ __forceinline__ bool fbox_near(float4 lo, float4 hi, float3 qlo, float3 qhi, float Df) {
  return __fsub_rd(lo.x, qhi.x) <= Df && __fsub_rd(qlo.x, hi.x) <= Df && __fsub_rd(lo.y, qhi.y) <= Df &&
         __fsub_rd(qlo.y, hi.y) <= Df && __fsub_rd(lo.z, qhi.z) <= Df && __fsub_rd(qlo.z, hi.z) <= Df;
}

// traversal skeleton: calls leaf(pos) for every leaf whose box passes the
// conservative float test against the query box
template <class LeafFn>
__device__ __forceinline__ void traverse(const BVH& B, int root, float3 qlo, float3 qhi, float Df, int min_pos,
                                         Counters* cnt, LeafFn leaf) {
  if (root < 0) return;
  if (root & LEAF) {
    int l = root & ~LEAF;
    if (l > min_pos) {
      float4 lo = B.leafbox[2 * l], hi = B.leafbox[2 * l + 1];
      if (fbox_near(lo, hi, qlo, qhi, Df)) leaf(l);
    }
    return;
  }
  int stack[64];
  int sp = 0;
  stack[sp++] = root;
  // a valid tree visits each internal node at most once per query
  int budget = B.n + 2;
  while (sp > 0) {
    if (--budget < 0) {
      atomicOr(&cnt->err, ERR_BUDGET);
      return;
    }
    int node = stack[--sp];
    if (B.range_hi[node] <= min_pos) continue;
    float4 a = B.box[3 * node], b = B.box[3 * node + 1], d = B.box[3 * node + 2];
    float4 llo = make_float4(a.x, a.y, a.z, 0.f), lhi = make_float4(a.w, b.x, b.y, 0.f);
    float4 rlo = make_float4(b.z, b.w, d.x, 0.f), rhi = make_float4(d.y, d.z, d.w, 0.f);
    int L = B.left[node], R = B.right[node];
    bool hl = fbox_near(llo, lhi, qlo, qhi, Df), hr = fbox_near(rlo, rhi, qlo, qhi, Df);
    if (hr) {
      if (R & LEAF) { if ((R & ~LEAF) > min_pos) leaf(R & ~LEAF); }
      else if (sp < 64) stack[sp++] = R;
      else atomicOr(&cnt->err, ERR_STACK);
    }
    if (hl) {
      if (L & LEAF) { if ((L & ~LEAF) > min_pos) leaf(L & ~LEAF); }
      else if (sp < 64) stack[sp++] = L;
      else atomicOr(&cnt->err, ERR_STACK);
    }
  }
}

__device__ __forceinline__ float3 f3rd(dv3 a) {
  return make_float3(__double2float_rd(a.x), __double2float_rd(a.y), __double2float_rd(a.z));
}
__device__ __forceinline__ float3 f3ru(dv3 a) {
  return make_float3(__double2float_ru(a.x), __double2float_ru(a.y), __double2float_ru(a.z));
}


// launchers (cch_bvh.cu)
void bvh_build_all(Runtime& R, cudaStream_t st, int gated = 0);
void bvh_refit_all(Runtime& R, cudaStream_t st, int force);
void search_queries(Runtime& R, int nxt, int mode, double Dq, cudaStream_t st);
void query_class(Runtime& R, int c, int nxt, int mode, double Dq, cudaStream_t st);
void accept_queries(Runtime& R, cudaStream_t st);
void finalize_search(Runtime& R, int nxt, int mode, double Dq, cudaStream_t st);

}  // namespace cch

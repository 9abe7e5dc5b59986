// cch_bvh.cu -- proximity search of Sec. 3.1 on sm_103a.
//
// The paper's search is a grid spatial hash; this implementation uses a linear BVH
// built from a radix sort of Morton codes (Karras 2012), one tree per
// primitive class (triangles, collision edges, collision vertices) over the
// whole pool.  The scene index sits above the Morton bits of every key, so
// each scene owns a subtree and queries start at their scene's root.  The
// tree only prunes: float boxes rounded outward and a round-down gap test
// never reject a pair that the exact FP64 candidate test accepts, and every
// leaf reached goes through that exact test, so the candidate set does not
// depend on the tree.
#include <cooperative_groups.h>
#include "cch_host.h"

namespace cg = cooperative_groups;
namespace cch {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int expand10(unsigned int v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

// class accessors: FP64 box and scene of primitive id of class c
// c = 0 triangles, 1 collision edges, 2 collision vertices
__device__ __forceinline__ void prim_box(const Pool& P, int c, int id, dv3& lo, dv3& hi, int& scene) {
  if (c == 0) {
    int4 t = P.tv[id];
    dv3 a = mk(P.x[t.x]), b = mk(P.x[t.y]), d = mk(P.x[t.z]);
    lo = a; hi = a;
    if (b.x < lo.x) lo.x = b.x; if (b.x > hi.x) hi.x = b.x;
    if (b.y < lo.y) lo.y = b.y; if (b.y > hi.y) hi.y = b.y;
    if (b.z < lo.z) lo.z = b.z; if (b.z > hi.z) hi.z = b.z;
    if (d.x < lo.x) lo.x = d.x; if (d.x > hi.x) hi.x = d.x;
    if (d.y < lo.y) lo.y = d.y; if (d.y > hi.y) hi.y = d.y;
    if (d.z < lo.z) lo.z = d.z; if (d.z > hi.z) hi.z = d.z;
    scene = t.w;
  } else if (c == 1) {
    int4 e = P.ev[id];
    dv3 a = mk(P.x[e.x]), b = mk(P.x[e.y]);
    lo = a; hi = a;
    if (b.x < lo.x) lo.x = b.x; if (b.x > hi.x) hi.x = b.x;
    if (b.y < lo.y) lo.y = b.y; if (b.y > hi.y) hi.y = b.y;
    if (b.z < lo.z) lo.z = b.z; if (b.z > hi.z) hi.z = b.z;
    scene = e.z;
  } else {
    int v = P.vc[id];
    dv3 a = mk(P.x[v]);
    double r = P.rho[v];
    lo = {a.x - r, a.y - r, a.z - r};
    hi = {a.x + r, a.y + r, a.z + r};
    scene = P.vscene[v];
  }
}

// Conservative float version used for pruning: boxes rounded outward, gaps
// rounded down, D rounded up; it never rejects what box_near accepts.
__device__ __forceinline__ BVH& bvh_of(Pool& P, int c) { return c == 0 ? P.bt : (c == 1 ? P.be : P.bv); }
__device__ __forceinline__ int nprim(const Pool& P, int c) { return c == 0 ? P.nt : (c == 1 ? P.ne : P.nvc); }

// ---------------------------------------------------------------------------
// build
// ---------------------------------------------------------------------------
// gated: run only in iterations that search (BVH rebuilt at every search)
__device__ __forceinline__ bool gate_off(const Pool& P, int gated) { return gated && !P.cnt->any_search; }

__global__ void k_scene_bounds_reset(Pool P, int gated) {
  if (gate_off(P, gated)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.nscene) {
    unsigned int* b = (unsigned int*)(P.sbox + 2 * i);
    b[0] = b[1] = b[2] = 0xffffffffu;
    b[4] = b[5] = b[6] = 0u;
  }
}
// bounds of the collision vertices of every scene (ordered-int float atomics)
__global__ void k_scene_bounds(Pool P, int gated) {
  if (gate_off(P, gated)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nvc; i += gridDim.x * blockDim.x) {
    int v = P.vc[i];
    int s = P.vscene[v];
    if (!P.ss[s].active) continue;
    P4 p = P.x[v];
    unsigned int* b = (unsigned int*)(P.sbox + 2 * s);
    atomicMin(&b[0], fl_ord(__double2float_rd(p.x)));
    atomicMin(&b[1], fl_ord(__double2float_rd(p.y)));
    atomicMin(&b[2], fl_ord(__double2float_rd(p.z)));
    atomicMax(&b[4], fl_ord(__double2float_ru(p.x)));
    atomicMax(&b[5], fl_ord(__double2float_ru(p.y)));
    atomicMax(&b[6], fl_ord(__double2float_ru(p.z)));
  }
}

__global__ void k_morton(Pool P, int c, int gated) {
  if (gate_off(P, gated)) return;
  BVH& B = bvh_of(P, c);
  int n = nprim(P, c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dv3 lo, hi;
    int s;
    prim_box(P, c, i, lo, hi, s);
    const unsigned int* b = (const unsigned int*)(P.sbox + 2 * s);
    float bl[3] = {ord_fl(b[0]), ord_fl(b[1]), ord_fl(b[2])};
    float bh[3] = {ord_fl(b[4]), ord_fl(b[5]), ord_fl(b[6])};
    float cen[3] = {(float)(0.5 * (lo.x + hi.x)), (float)(0.5 * (lo.y + hi.y)), (float)(0.5 * (lo.z + hi.z))};
    unsigned int q[3];
    for (int k = 0; k < 3; k++) {
      float ext = bh[k] - bl[k];
      float u = ext > 0.f ? (cen[k] - bl[k]) / ext : 0.f;
      u = fminf(fmaxf(u, 0.f), 1.f);
      q[k] = min((unsigned int)(u * 1024.f), 1023u);
    }
    unsigned long long m = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    B.keys[i] = ((unsigned long long)s << 30) | m;
    B.ids[i] = i;
  }
}

// LSD radix sort, 8-bit digits, tiles of 2048 keys (256 threads x 8).  Pass 1
// counts digits per tile; pass 2 scans the digit-major table; pass 3 ranks
// each key stably inside its tile (per-warp match + per-warp prefix) and
// scatters it.
constexpr int RS_THREADS = 256, RS_ITEMS = 8, RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_radix_hist(const unsigned long long* keys, int n, int shift, unsigned int* hist, int ntiles,
                             const int* gate) {
  if (gate && !*gate) return;
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; k++) {
    int i = base + k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m entries in one block of 1024 threads
__global__ void k_scan_1block(unsigned int* a, int m, const int* gate) {
  if (gate && !*gate) return;
  __shared__ unsigned int part[1024];
  int per = (m + 1023) / 1024;
  int lo = threadIdx.x * per, hi = min(lo + per, m);
  unsigned int s = 0;
  for (int i = lo; i < hi; i++) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = lo; i < hi; i++) {
    unsigned int v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void k_radix_scatter(const unsigned long long* kin, const int* vin, unsigned long long* kout, int* vout,
                                int n, int shift, const unsigned int* hist, int ntiles, const int* gate) {
  if (gate && !*gate) return;
  __shared__ unsigned int wc[8][256];    // per-warp digit counts, then prefixes
  __shared__ unsigned int gb[256];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    for (int k = 0; k < 8; k++) wc[k][d] = 0;
    gb[d] = hist[d * ntiles + blockIdx.x];
  }
  __syncthreads();
  int base = blockIdx.x * RS_TILE + w * (RS_ITEMS * 32);
  unsigned long long kk[RS_ITEMS];
  int vv[RS_ITEMS];
  unsigned int rank[RS_ITEMS], dig[RS_ITEMS];
  for (int r = 0; r < RS_ITEMS; r++) {
    int i = base + r * 32 + lane;
    bool ok = i < n;
    kk[r] = ok ? kin[i] : 0ull;
    vv[r] = ok ? vin[i] : 0;
    unsigned int d = ok ? (unsigned int)((kk[r] >> shift) & 255) : 256u + lane;
    dig[r] = d;
    unsigned int peers = __match_any_sync(0xffffffffu, d);
    unsigned int before = __popc(peers & ((1u << lane) - 1u));
    unsigned int cur = ok ? wc[w][d] : 0;
    rank[r] = cur + before;
    __syncwarp();
    if (ok && before == 0) wc[w][d] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, per digit
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    unsigned int run = 0;
    for (int k = 0; k < 8; k++) {
      unsigned int c = wc[k][d];
      wc[k][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < RS_ITEMS; r++) {
    int i = base + r * 32 + lane;
    if (i < n) {
      unsigned int d = dig[r];
      unsigned int pos = gb[d] + wc[w][d] + rank[r];
      kout[pos] = kk[r];
      vout[pos] = vv[r];
    }
  }
}

__device__ __forceinline__ int delta_k(const unsigned long long* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  unsigned long long a = k[i], b = k[j];
  if (a == b) return 64 + __clz(i ^ j);
  return __clzll(a ^ b);
}

// Karras 2012: internal node i covers a contiguous range of sorted leaves
__global__ void k_karras(Pool P, int c, int gated) {
  if (gate_off(P, gated)) return;
  BVH& B = bvh_of(P, c);
  int n = B.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    const unsigned long long* K = B.keys;
    int d = (delta_k(K, n, i, i + 1) - delta_k(K, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta_k(K, n, i, i - d);
    int lmax = 2;
    while (delta_k(K, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (delta_k(K, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta_k(K, n, i, j);
    int s = 0;
    int t = l;
    do {
      t = (t + 1) >> 1;
      if (delta_k(K, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? (LEAF | gamma) : gamma;
    int right = (hi == gamma + 1) ? (LEAF | (gamma + 1)) : gamma + 1;
    B.left[i] = left;
    B.right[i] = right;
    B.range_hi[i] = hi;
    if (left & LEAF) B.parent[n - 1 + (left & ~LEAF)] = i; else B.parent[left] = i;
    if (right & LEAF) B.parent[n - 1 + (right & ~LEAF)] = i; else B.parent[right] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 1) B.parent[0] = -1;
    if (n == 1) B.parent[n - 1 + 0] = -1;
  }
}

__device__ __forceinline__ int scene_of_pos(const BVH& B, int pos) { return (int)(B.keys[pos] >> 30); }

// the root of each scene's subtree: the highest node whose leaves all belong to one scene
__global__ void k_scene_roots(Pool P, int c, int gated) {
  if (gate_off(P, gated)) return;
  BVH& B = bvh_of(P, c);
  int n = B.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n - 1; i += gridDim.x * blockDim.x) {
    int lo, hi, par;
    int node;
    if (i < n - 1) {
      node = i;
      // leftmost leaf: descend left
      int cur = i, steps = 0;
      while (!(cur & LEAF) && ++steps < 256) cur = B.left[cur];
      if (!(cur & LEAF)) { atomicOr(&P.cnt->err, ERR_TREE); continue; }
      lo = cur & ~LEAF;
      hi = B.range_hi[i];
      par = B.parent[i];
    } else {
      int leaf = i - (n - 1);
      node = LEAF | leaf;
      lo = hi = leaf;
      par = B.parent[i];
    }
    int s = scene_of_pos(B, lo);
    if (scene_of_pos(B, hi) != s) continue;
    bool top = par < 0;
    if (!top) {
      int plo;
      int cur = par, steps = 0;
      while (!(cur & LEAF) && ++steps < 256) cur = B.left[cur];
      if (!(cur & LEAF)) { atomicOr(&P.cnt->err, ERR_TREE); continue; }
      plo = cur & ~LEAF;
      int phi = B.range_hi[par];
      top = scene_of_pos(B, plo) != s || scene_of_pos(B, phi) != s;
    }
    if (top) B.sroot[s] = node;
  }
}

__device__ __forceinline__ void child_box(const BVH& B, int child, float4& lo, float4& hi) {
  if (child & LEAF) {
    int l = child & ~LEAF;
    lo = B.leafbox[2 * l];
    hi = B.leafbox[2 * l + 1];
  } else {
    float4 a = B.box[3 * child], b = B.box[3 * child + 1], d = B.box[3 * child + 2];
    // left (a.xyz, a.w b.x b.y) right (b.z b.w d.x, d.y d.z d.w)
    lo = make_float4(fminf(a.x, b.z), fminf(a.y, b.w), fminf(a.z, d.x), 0.f);
    hi = make_float4(fmaxf(a.w, d.y), fmaxf(b.x, d.z), fmaxf(b.y, d.w), 0.f);
  }
}

// ---------------------------------------------------------------------------
// queries
// ---------------------------------------------------------------------------
// FP32 lower bound of an edge-edge distance for the search's filter: the gap
// along the closest points' difference rejects most distant pairs; a pair it
// does not reject gets the full separating-axis bound
__device__ __forceinline__ float ee_lower(fv3 a, fv3 b, fv3 c, fv3 d, float Df) {
  float t = ftol(a, b, c, d), lo;
  f_ss_bounds(a, b, c, d, __fadd_ru(Df, t), &lo);
  return __fsub_rd(lo, t);
}

// A pair that the FP32 filter could not reject; the exact FP64 distance is
// evaluated later by k_finalize with one pair per thread (full warps instead
// of the few lanes still active inside a divergent traversal).
__device__ __forceinline__ void push_survivor(Pool& P, int kind, unsigned long long key, int4 v, float lower) {
  int idx = claim(&P.cnt->n_fcand[kind], P.pair_cap);
  if (idx < 0) {
    atomicOr(&P.cnt->overflow, OV_PAIRS);
    return;
  }
  size_t o = (size_t)kind * P.pair_cap + idx;
  P.fkey[o] = key;
  P.fv[o] = v;
  if (P.fd) P.fd[o] = lower;
}

__device__ __forceinline__ void add_candidates(Pool& P, int s, long long n) {
  if (n == 0) return;
  scene_reduce(P, s, n, cg::plus<long long>(), [&](long long t, int) {
    atomicAdd((unsigned long long*)&P.ss[s].candidates, (unsigned long long)t);
  });
}

// ---------------------------------------------------------------------------
// Packet traversal for the step's searches.  The 32 lanes of a warp take 32
// consecutive queries in Morton order (close in space) and descend the tree
// together as a wavefront: every stack entry is a node and the mask of the
// queries whose traversal reaches it.  Each step pops up to 32 entries, one
// per lane; a lane loads its node's two child boxes and tests them against
// each query of its mask, so a child is reached by exactly the queries whose
// own traversal would reach it (box test and, for the edge-edge search, the
// later-leaves rule applied per query).  A step thus has up to 32 node loads
// in flight instead of one, and the number of steps is about the depth of
// the traversed region rather than its node count.  Lanes of different
// scenes descend in turn, each from its scene's root.
// ---------------------------------------------------------------------------
constexpr int WAVE_STACK = 512;    // entries per warp: (node, query mask)
constexpr int WAVE_RESERVE = 128;  // kept free for depth-first steps (deeper than any tree here)

// a query of the wavefront: its box, D (lo.w) and the last sorted leaf
// position it skips (hi.w, as int bits; -1: none)
struct WaveQuery {
  float4 lo, hi;
};

// Leaf work runs from a per-warp queue: a (query, leaf) pair reached by the
// traversal first passes the cheap checks (pre), and the pairs that pass are
// queued; whenever 32 are queued, the whole warp evaluates them at once
// (work), each lane fetching its entry's query data from the query's lane.
// The distance bounds thus run with all lanes busy.
constexpr int PACKET_QUEUE = 96;  // at most 31 pending plus 32 per round

// pre(valid, q, leaf) and work(valid, q, leaf) are called by all 32 lanes
// together (they may shuffle query data from lane q); valid marks the lanes
// that hold a pair.  Returns the warp's number of pairs that passed pre.
template <class PreFn, class WorkFn>
__device__ __forceinline__ long long traverse_wave(const BVH& B, int root, bool act, float3 qlo, float3 qhi, float Df,
                                                   int min_pos, WaveQuery* qs, int2* stack, int* qlane, int* qleaf,
                                                   Counters* cnt, PreFn pre, WorkFn work) {
  const unsigned FULL = 0xffffffffu;
  int lane = threadIdx.x & 31;
  if (root < 0) return 0;
  int qn = 0;  // identical in every lane
  long long passed = 0;
  auto enqueue = [&](bool want, int q, int l) {
    unsigned m = __ballot_sync(FULL, want);
    if (!m) return;
    if (want) {
      int at = qn + __popc(m & ((1u << lane) - 1u));
      qlane[at] = q;
      qleaf[at] = l;
    }
    qn += __popc(m);
    passed += want;
    __syncwarp();
  };
  auto drain = [&](bool all) {
    int base = 0;
    for (; base + 32 <= qn || (all && base < qn); base += 32) {
      int e = base + lane;
      bool valid = e < qn;
      work(valid, valid ? qlane[e] : 0, valid ? qleaf[e] : 0);
    }
    __syncwarp();
    int rest = qn - base;  // fewer than 32 left (none when all)
    if (rest > 0) {
      int a = lane < rest ? qlane[base + lane] : 0, b = lane < rest ? qleaf[base + lane] : 0;
      __syncwarp();
      if (lane < rest) {
        qlane[lane] = a;
        qleaf[lane] = b;
      }
    }
    qn = rest > 0 ? rest : 0;
    __syncwarp();
  };
  auto reduce = [&](long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
  };
  if (root & LEAF) {  // a scene of one primitive: each lane tests the leaf itself
    int l = root & ~LEAF;
    bool hit = false;
    if (act && l > min_pos) {
      float4 lo = B.leafbox[2 * l], hi = B.leafbox[2 * l + 1];
      hit = fbox_near(lo, hi, qlo, qhi, Df);
    }
    enqueue(hit && pre(hit, lane, l), lane, l);
    drain(true);
    return reduce(passed);
  }
  qs[lane].lo = make_float4(qlo.x, qlo.y, qlo.z, Df);
  qs[lane].hi = make_float4(qhi.x, qhi.y, qhi.z, __int_as_float(min_pos));
  unsigned amask = __ballot_sync(FULL, act);
  __syncwarp();
  if (!amask) return 0;
  if (lane == 0) stack[0] = make_int2(root, (int)amask);
  int sp = 1;  // identical in every lane
  int budget = B.n + 2;
  __syncwarp();
  while (sp > 0) {
    // A popped entry pushes at most two, so popping k grows the stack by at
    // most k: up to WAVE_STACK - WAVE_RESERVE entries the warp pops up to 32
    // at once, beyond that one at a time (depth first, growing the stack by
    // at most the depth of the subtree under way before it shrinks again).
    int room = WAVE_STACK - WAVE_RESERVE - sp;
    int k = room > 0 ? min(min(sp, 32), room) : (sp < WAVE_STACK ? 1 : 0);
    if (k <= 0 || (budget -= k) < 0) {
      if (lane == 0) atomicOr(&cnt->err, k <= 0 ? ERR_STACK : ERR_BUDGET);
      break;
    }
    int2 ent = lane < k ? stack[sp - k + lane] : make_int2(0, 0);
    sp -= k;
    __syncwarp();
    unsigned ml = 0u, mr = 0u;
    int L = 0, R = 0;
    if (lane < k) {
      int node = ent.x;
      unsigned m = (unsigned)ent.y;
      float4 a = B.box[3 * node], b = B.box[3 * node + 1], d = B.box[3 * node + 2];
      float4 llo = make_float4(a.x, a.y, a.z, 0.f), lhi = make_float4(a.w, b.x, b.y, 0.f);
      float4 rlo = make_float4(b.z, b.w, d.x, 0.f), rhi = make_float4(d.y, d.z, d.w, 0.f);
      L = B.left[node];
      R = B.right[node];
      int rh = B.range_hi[node];
      while (m) {
        int q = __ffs(m) - 1;
        m &= m - 1u;
        WaveQuery Q = qs[q];
        int qmin = __float_as_int(Q.hi.w);
        if (!(rh > qmin)) continue;
        float3 lo3 = make_float3(Q.lo.x, Q.lo.y, Q.lo.z), hi3 = make_float3(Q.hi.x, Q.hi.y, Q.hi.z);
        if (fbox_near(rlo, rhi, lo3, hi3, Q.lo.w) && (!(R & LEAF) || (R & ~LEAF) > qmin)) mr |= 1u << q;
        if (fbox_near(llo, lhi, lo3, hi3, Q.lo.w) && (!(L & LEAF) || (L & ~LEAF) > qmin)) ml |= 1u << q;
      }
    }
    // inner children with queries go on the stack
    bool pr = mr && !(R & LEAF), pl = ml && !(L & LEAF);
    unsigned br = __ballot_sync(FULL, pr), bl = __ballot_sync(FULL, pl);
    unsigned lt = (1u << lane) - 1u;
    int at = sp + __popc(br & lt) + __popc(bl & lt);
    if (pr) stack[at] = make_int2(R, (int)mr);
    if (pl) stack[at + (pr ? 1 : 0)] = make_int2(L, (int)ml);
    sp += __popc(br) + __popc(bl);
    // leaf children: one (query, leaf) pair per lane and round
    unsigned lr = (R & LEAF) ? mr : 0u, ll = (L & LEAF) ? ml : 0u;
    while (__any_sync(FULL, lr | ll)) {
      int q = -1, l = 0;
      if (lr) {
        q = __ffs(lr) - 1;
        lr &= lr - 1u;
        l = R & ~LEAF;
      } else if (ll) {
        q = __ffs(ll) - 1;
        ll &= ll - 1u;
        l = L & ~LEAF;
      }
      bool v = q >= 0;
      bool want = pre(v, v ? q : 0, l) && v;
      enqueue(want, q, l);
      if (qn >= 32) drain(false);
    }
    __syncwarp();
  }
  drain(true);
  return reduce(passed);
}

// vertex-triangle pairs of the step's searches, queries in the Morton order
// of the collision vertices
__global__ void __launch_bounds__(256) k_pquery_vt(Pool P) {
  __shared__ int2 stacks[8][WAVE_STACK];
  __shared__ WaveQuery wq[8][32];
  __shared__ int qlanes[8][PACKET_QUEUE], qleaves[8][PACKET_QUEUE];
  if (!P.cnt->any_search) return;
  const unsigned FULL = 0xffffffffu;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  int nq = P.bv.n;
  for (int base = gw * 32; base < nq; base += nw * 32) {
    int i = base + lane;
    int a = -1, s = -1;
    bool pend = false;
    if (i < nq) {
      a = P.vc[P.bv.ids[i]];
      s = P.vscene[a];
      pend = searching(P, s);
    }
    double ra = a >= 0 ? P.rho[a] : 0.0;
    dv3 xa = a >= 0 ? mk(P.x[a]) : dv3{0.0, 0.0, 0.0};
    dv3 alo = {xa.x - ra, xa.y - ra, xa.z - ra}, ahi = {xa.x + ra, xa.y + ra, xa.z + ra};
    float3 qlo = f3rd(alo), qhi = f3ru(ahi);
    float Df = s >= 0 ? __double2float_ru(P.sd[s].d_max) : 0.f;
    float raf = __double2float_ru(ra);  // rounded up: the bound stays below the distance
    fv3 fa = a >= 0 ? fk(P.xf[a]) : fv3{0.f, 0.f, 0.f};
    bool sa = a >= 0 && is_static(P, a);
    while (__any_sync(FULL, pend)) {
      int leader = __ffs(__ballot_sync(FULL, pend)) - 1;
      int sc = __shfl_sync(FULL, s, leader);
      bool mine = pend && s == sc;
      const SceneDesc& S = P.sd[sc];
      long long nc = traverse_wave(P.bt, P.bt.sroot[sc], mine, qlo, qhi, Df, -1, wq[warp], stacks[warp],
                                   qlanes[warp], qleaves[warp], P.cnt,
        [&](bool valid, int q, int pos) {
          // the query's vertex; a triangle at it or a static pair is skipped
          int qa = __shfl_sync(FULL, a, q);
          bool qs = __shfl_sync(FULL, sa, q);
          if (!valid) return false;
          int4 tv = P.tv[P.bt.ids[pos]];
          if (qa == tv.x || qa == tv.y || qa == tv.z) return false;
          return !(qs && is_static(P, tv.x) && is_static(P, tv.y) && is_static(P, tv.z));
        },
        [&](bool valid, int src, int pos) {
          // the queuing lane's query: the vertex, its float position and radius bound, D
          int qa = __shfl_sync(FULL, a, src);
          float ax = __shfl_sync(FULL, fa.x, src), ay = __shfl_sync(FULL, fa.y, src), az = __shfl_sync(FULL, fa.z, src);
          float qr = __shfl_sync(FULL, raf, src), qD = __shfl_sync(FULL, Df, src);
          if (!valid) return;
          int t = P.bt.ids[pos];
          int4 tv = P.tv[t];
          fv3 qf = {ax, ay, az};
          fv3 f1 = fk(P.xf[tv.x]), f2 = fk(P.xf[tv.y]), f3 = fk(P.xf[tv.z]);
          float lower = __fsub_rd(__fsub_rd(f_pt(qf, f1, f2, f3), qr), ftol(qf, f1, f2, f3));
          if (lower >= qD) return;
          push_survivor(P, K_VT, mkkey(K_VT, qa - S.v0, t - S.t0), make_int4(qa, tv.x, tv.y, tv.z), lower);
        });
      if (lane == 0 && nc) atomicAdd((unsigned long long*)&P.ss[sc].candidates, (unsigned long long)nc);
      if (mine) pend = false;
    }
  }
}

// edge-edge pairs of the step's searches: each edge (at sorted leaf position
// i) against the later leaves of its scene
__global__ void __launch_bounds__(256) k_pquery_ee(Pool P) {
  __shared__ int2 stacks[8][WAVE_STACK];
  __shared__ WaveQuery wq[8][32];
  __shared__ int qlanes[8][PACKET_QUEUE], qleaves[8][PACKET_QUEUE];
  if (!P.cnt->any_search) return;
  const unsigned FULL = 0xffffffffu;
  const BVH& B = P.be;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int base = gw * 32; base < B.n; base += nw * 32) {
    int i = base + lane;
    int e1 = -1, s = -1;
    int4 ea = make_int4(-1, -1, -1, -1);
    bool pend = false;
    if (i < B.n) {
      e1 = B.ids[i];
      ea = P.ev[e1];
      s = ea.z;
      pend = searching(P, s);
    }
    dv3 alo = {0.0, 0.0, 0.0}, ahi = {0.0, 0.0, 0.0};
    if (e1 >= 0) {
      int sc;
      prim_box(P, 1, e1, alo, ahi, sc);
    }
    float3 qlo = f3rd(alo), qhi = f3ru(ahi);
    float Df = s >= 0 ? __double2float_ru(P.sd[s].d_max) : 0.f;
    bool sa = e1 >= 0 && is_static(P, ea.x) && is_static(P, ea.y);
    while (__any_sync(FULL, pend)) {
      int leader = __ffs(__ballot_sync(FULL, pend)) - 1;
      int sc = __shfl_sync(FULL, s, leader);
      bool mine = pend && s == sc;
      const SceneDesc& S = P.sd[sc];
      long long nc = traverse_wave(B, B.sroot[sc], mine, qlo, qhi, Df, i, wq[warp], stacks[warp], qlanes[warp],
                                   qleaves[warp], P.cnt,
        [&](bool valid, int q, int pos) {
          // the query edge; an edge sharing a vertex with it or a static pair is skipped
          int qx = __shfl_sync(FULL, ea.x, q), qy = __shfl_sync(FULL, ea.y, q);
          bool qs = __shfl_sync(FULL, sa, q);
          if (!valid) return false;
          int4 eb = P.ev[B.ids[pos]];
          if (qx == eb.x || qx == eb.y || qy == eb.x || qy == eb.y) return false;
          return !(qs && is_static(P, eb.x) && is_static(P, eb.y));
        },
        [&](bool valid, int src, int pos) {
          // the queuing lane's query edge and D
          int q1 = __shfl_sync(FULL, e1, src);
          int qx = __shfl_sync(FULL, ea.x, src), qy = __shfl_sync(FULL, ea.y, src);
          float qD = __shfl_sync(FULL, Df, src);
          if (!valid) return;
          int e2 = B.ids[pos];
          int4 eb = P.ev[e2];
          // the bound in key order (lower edge id first), whichever edge is the query
          bool qlow = q1 < e2;
          int4 A = qlow ? make_int4(qx, qy, 0, 0) : eb, Bv = qlow ? eb : make_int4(qx, qy, 0, 0);
          fv3 fa0 = fk(P.xf[A.x]), fa1 = fk(P.xf[A.y]), fb0 = fk(P.xf[Bv.x]), fb1 = fk(P.xf[Bv.y]);
          float lower = ee_lower(fa0, fa1, fb0, fb1, qD);
          if (lower >= qD) return;
          push_survivor(P, K_EE, mkkey(K_EE, min(q1, e2) - S.e0, max(q1, e2) - S.e0),
                        make_int4(A.x, A.y, Bv.x, Bv.y), lower);
        });
      if (lane == 0 && nc) atomicAdd((unsigned long long*)&P.ss[sc].candidates, (unsigned long long)nc);
      if (mine) pend = false;
    }
  }
}

// vertex-triangle pairs: every collision vertex against its scene's triangles
__global__ void __launch_bounds__(256) k_query_vt(Pool P, int nxt, int mode, double Dq) {
  if (mode == 0 && !P.cnt->any_search) return;
  for (int qi = blockIdx.x * blockDim.x + threadIdx.x; qi < P.nvc; qi += gridDim.x * blockDim.x) {
    int a = P.vc[qi];
    int s = P.vscene[a];
    if (mode == 0 && !searching(P, s)) continue;
    const SceneDesc& S = P.sd[s];
    double D = mode == 0 ? S.d_max : Dq;
    dv3 xa = mk(P.x[a]);
    double ra = P.rho[a];
    dv3 alo = {xa.x - ra, xa.y - ra, xa.z - ra}, ahi = {xa.x + ra, xa.y + ra, xa.z + ra};
    float Df = __double2float_ru(D);
    float raf = __double2float_ru(ra);  // rounded up: the bound stays below the distance
    fv3 fa = fk(P.xf[a]);
    bool sa = is_static(P, a);
    long long ncand = 0;
    traverse(P.bt, P.bt.sroot[s], f3rd(alo), f3ru(ahi), Df, -1, P.cnt, [&](int pos) {
      int t = P.bt.ids[pos];
      int4 tv = P.tv[t];
      if (a == tv.x || a == tv.y || a == tv.z) return;
      if (sa && is_static(P, tv.x) && is_static(P, tv.y) && is_static(P, tv.z)) return;
      unsigned long long key = mkkey(K_VT, a - S.v0, t - S.t0);
      if (mode == 1) {
        dv3 lo, hi;
        int sc;
        prim_box(P, 0, t, lo, hi, sc);
        if (box_near(alo, ahi, lo, hi, D)) emit_query(P, key, 0.0);
        return;
      }
      ncand++;
      fv3 f1 = fk(P.xf[tv.x]), f2 = fk(P.xf[tv.y]), f3 = fk(P.xf[tv.z]);
      float lower = __fsub_rd(__fsub_rd(f_pt(fa, f1, f2, f3), raf), ftol(fa, f1, f2, f3));
      if (lower >= Df) return;
      push_survivor(P, K_VT, key, make_int4(a, tv.x, tv.y, tv.z), lower);
    });
    if (mode == 0) add_candidates(P, s, ncand);
  }
}

// edge-edge pairs: each edge (at sorted leaf position i) against the later leaves of its scene
__global__ void __launch_bounds__(256) k_query_ee(Pool P, int nxt, int mode, double Dq) {
  if (mode == 0 && !P.cnt->any_search) return;
  const BVH& B = P.be;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n; i += gridDim.x * blockDim.x) {
    int e1 = B.ids[i];
    int4 ea = P.ev[e1];
    int s = ea.z;
    if (mode == 0 && !searching(P, s)) continue;
    const SceneDesc& S = P.sd[s];
    double D = mode == 0 ? S.d_max : Dq;
    dv3 alo, ahi;
    int sc;
    prim_box(P, 1, e1, alo, ahi, sc);
    float Df = __double2float_ru(D);
    bool sa = is_static(P, ea.x) && is_static(P, ea.y);
    fv3 fa0 = fk(P.xf[ea.x]), fa1 = fk(P.xf[ea.y]);
    long long ncand = 0;
    traverse(B, B.sroot[s], f3rd(alo), f3ru(ahi), Df, i, P.cnt, [&](int pos) {
      int e2 = B.ids[pos];
      int4 eb = P.ev[e2];
      if (ea.x == eb.x || ea.x == eb.y || ea.y == eb.x || ea.y == eb.y) return;
      if (sa && is_static(P, eb.x) && is_static(P, eb.y)) return;
      int lo_e = min(e1, e2), hi_e = max(e1, e2);
      unsigned long long key = mkkey(K_EE, lo_e - S.e0, hi_e - S.e0);
      if (mode == 1) {
        dv3 lo, hi;
        int sc2;
        prim_box(P, 1, e2, lo, hi, sc2);
        if (box_near(alo, ahi, lo, hi, D)) emit_query(P, key, 0.0);
        return;
      }
      ncand++;
      fv3 fb0 = fk(P.xf[eb.x]), fb1 = fk(P.xf[eb.y]);
      // the bound is evaluated in key order (lower edge id first), whichever
      // edge is the query, so that it does not depend on the tree: in mixed
      // precision it is the pair's distance
      bool qlo = lo_e == e1;
      float lower = qlo ? ee_lower(fa0, fa1, fb0, fb1, Df) : ee_lower(fb0, fb1, fa0, fa1, Df);
      if (lower >= Df) return;
      int4 A = qlo ? ea : eb, Bv = qlo ? eb : ea;
      push_survivor(P, K_EE, key, make_int4(A.x, A.y, Bv.x, Bv.y), lower);
    });
    if (mode == 0) add_candidates(P, s, ncand);
  }
}

// vertex-vertex pairs: each point against every collision vertex of its scene
__global__ void __launch_bounds__(256) k_query_vv(Pool P, int nxt, int mode, double Dq) {
  if (mode == 0 && !P.cnt->any_search) return;
  for (int qi = blockIdx.x * blockDim.x + threadIdx.x; qi < P.nq; qi += gridDim.x * blockDim.x) {
    int a = P.pts[qi];
    int s = P.vscene[a];
    if (mode == 0 && !searching(P, s)) continue;
    const SceneDesc& S = P.sd[s];
    double D = mode == 0 ? S.d_max : Dq;
    dv3 xa = mk(P.x[a]);
    double ra = P.rho[a];
    dv3 alo = {xa.x - ra, xa.y - ra, xa.z - ra}, ahi = {xa.x + ra, xa.y + ra, xa.z + ra};
    float Df = __double2float_ru(D);
    bool sa = is_static(P, a);
    long long ncand = 0;
    traverse(P.bv, P.bv.sroot[s], f3rd(alo), f3ru(ahi), Df, -1, P.cnt, [&](int pos) {
      int b = P.vc[P.bv.ids[pos]];
      if (b == a) return;
      if ((P.vflag[b] & VF_POINT) && b < a) return;
      if (sa && is_static(P, b)) return;
      dv3 xb = mk(P.x[b]);
      double rb = P.rho[b];
      dv3 blo = {xb.x - rb, xb.y - rb, xb.z - rb}, bhi = {xb.x + rb, xb.y + rb, xb.z + rb};
      unsigned long long key = mkkey(K_VV, a - S.v0, b - S.v0);
      if (mode == 1) {
        if (box_near(alo, ahi, blo, bhi, D)) emit_query(P, key, 0.0);
        return;
      }
      ncand++;
      fv3 fa = fk(P.xf[a]), fb = fk(P.xf[b]);
      fv3 dd = fsub(fa, fb);
      float lower = __fsub_rd(__fsub_rd(sqrtf(fdot(dd, dd)), __double2float_ru(ra + rb)), ftol(fa, fb, fb, fb));
      if (lower >= Df) return;
      push_survivor(P, K_VV, key, make_int4(a, b, -1, -1), lower);
    });
    if (mode == 0) add_candidates(P, s, ncand);
  }
}

// Exact stage of the search: FP64 distance, then the exact FP64 box test of
// R3 (implied by dist < D up to rounding; evaluated so that P equals the
// oracle's set), for every FP32-filter survivor.  The three kinds occupy
// separate regions, so a warp almost always runs one kind's arithmetic.
// exact FP64 distance of a pair (R5) and the exact candidate box test (R3)
__device__ __forceinline__ double exact_dist(const Pool& P, int kind, int4 v) {
  dv3 a = mk(P.x[v.x]), b = mk(P.x[v.y]);
  if (kind == K_VV) return (vnorm(vsub(a, b)) - P.rho[v.x]) - P.rho[v.y];
  dv3 c = mk(P.x[v.z]), e = mk(P.x[v.w]);
  if (kind == K_VT) return d_pt(a, b, c, e) - P.rho[v.x];
  double ps, pt;
  return d_ss(a, b, c, e, &ps, &pt);
}
__device__ __forceinline__ bool exact_box(const Pool& P, int kind, int4 v, double D) {
  dv3 a = mk(P.x[v.x]), b = mk(P.x[v.y]);
  dv3 alo, ahi, blo, bhi;
  if (kind == K_VV) {
    double ra = P.rho[v.x], rb = P.rho[v.y];
    alo = {a.x - ra, a.y - ra, a.z - ra}; ahi = {a.x + ra, a.y + ra, a.z + ra};
    blo = {b.x - rb, b.y - rb, b.z - rb}; bhi = {b.x + rb, b.y + rb, b.z + rb};
  } else {
    dv3 c = mk(P.x[v.z]), e = mk(P.x[v.w]);
    if (kind == K_VT) {
      double ra = P.rho[v.x];
      alo = {a.x - ra, a.y - ra, a.z - ra}; ahi = {a.x + ra, a.y + ra, a.z + ra};
      blo = {fmin(fmin(b.x, c.x), e.x), fmin(fmin(b.y, c.y), e.y), fmin(fmin(b.z, c.z), e.z)};
      bhi = {fmax(fmax(b.x, c.x), e.x), fmax(fmax(b.y, c.y), e.y), fmax(fmax(b.z, c.z), e.z)};
    } else {
      alo = {fmin(a.x, b.x), fmin(a.y, b.y), fmin(a.z, b.z)}; ahi = {fmax(a.x, b.x), fmax(a.y, b.y), fmax(a.z, b.z)};
      blo = {fmin(c.x, e.x), fmin(c.y, e.y), fmin(c.z, e.z)}; bhi = {fmax(c.x, e.x), fmax(c.y, e.y), fmax(c.z, e.z)};
    }
  }
  return box_near(alo, ahi, blo, bhi, D);
}

__device__ __forceinline__ void survivor_at(const Pool& P, int i, int& kind, size_t& o) {
  int n0 = min(P.cnt->n_fcand[0], P.pair_cap), n1 = min(P.cnt->n_fcand[1], P.pair_cap);
  kind = i < n0 ? K_VT : (i < n0 + n1 ? K_EE : K_VV);
  int j = kind == K_VT ? i : (kind == K_EE ? i - n0 : i - n0 - n1);
  o = (size_t)kind * P.pair_cap + j;
}
__device__ __forceinline__ int survivors(const Pool& P) {
  return min(P.cnt->n_fcand[0], P.pair_cap) + min(P.cnt->n_fcand[1], P.pair_cap) +
         min(P.cnt->n_fcand[2], P.pair_cap);
}

// Step searches in FP64, pass A: FP32 bounds and the exact box test of every
// survivor, smallest upper bound of the certain pairs per vertex.
__global__ void k_final_bounds(Pool P) {
  if (!P.cnt->any_search) return;
  int total = survivors(P);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int kind;
    size_t o;
    survivor_at(P, i, kind, o);
    int4 v = P.fv[o];
    double D = P.sd[P.vscene[v.x]].d_max;
    float2 b = pair_bounds32(P, P.fkey[o], v);
    // a distance below D bounds every axis gap of the boxes, so the exact box
    // test passes whenever the upper bound is below D by more than the
    // rounding of the box corners; it runs only for the other pairs
    if ((double)b.y < D * (1.0 - 1e-12)) note_upper(P, v, b.y);
    else if (!exact_box(P, kind, v, D)) b = make_float2(INFINITY, INFINITY);
    else if ((double)b.y < D) note_upper(P, v, b.y);
    P.fbs[o] = b;
  }
}

// The exact stage of a search: P = survivors with an FP64 distance below D
// that pass the exact box test.  mode 0 (the step, FP64): pass B, exact
// distances only where they decide something; mixed precision: the FP32
// lower bound is the distance; modes 1, 2 (inspection): everything exact.
__global__ void k_finalize(Pool P, int nxt, int mode, double Dq) {
  if (mode == 0 && !P.cnt->any_search) return;
  int total = survivors(P);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int kind;
    size_t o;
    survivor_at(P, i, kind, o);
    unsigned long long key = P.fkey[o];
    int4 v = P.fv[o];
    int s = P.vscene[v.x];
    double D = mode == 0 ? P.sd[s].d_max : Dq;
    if (mode == 0 && P.mixed) {
      // mixed precision: the FP32 lower bound is the pair's distance
      double d = (double)P.fd[o];
      if (d < D) emit_pair(P, nxt, s, key, v, d);
      continue;
    }
    if (mode == 0) {
      float2 b = P.fbs[o];
      if (!(b.x < INFINITY)) continue;  // failed the exact box test
      if (needs_exact(P, v, b, D, P.sd[s].delta)) {
        // the FP64 distance runs in k_exact_survivors, over a dense list
        int e = claim(&P.cnt->n_exact[0], 3 * P.pair_cap);
        if (e >= 0) P.exq[e] = i;
      } else {
        emit_pair(P, nxt, s, key, v, (double)b.x);  // certainly in P; its distance decides nothing
      }
      continue;
    }
    double d = exact_dist(P, kind, v);
    if (!(d < D) || !exact_box(P, kind, v, D)) continue;
    if (mode == 2) emit_query(P, key, d);
    else emit_pair(P, nxt, s, key, v, d);
  }
}

// The exact FP64 distances of the survivors k_finalize left due, one per
// thread over the dense list (the survivors of one kind stay together), so
// that no lane of a warp idles through the FP64 arithmetic.
__global__ void k_exact_survivors(Pool P, int nxt) {
  if (!P.cnt->any_search) return;
  int n = min(P.cnt->n_exact[0], 3 * P.pair_cap);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int i = P.exq[j], kind;
    size_t o;
    survivor_at(P, i, kind, o);
    int4 v = P.fv[o];
    int s = P.vscene[v.x];
    double d = exact_dist(P, kind, v);
    if (d < P.sd[s].d_max) emit_pair(P, nxt, s, P.fkey[o], v, d);
  }
}

// ---------------------------------------------------------------------------
// Acceptance of x^{t+1}: no non-adjacent edge crosses a triangle, no two
// non-adjacent edges meet, and no point touches a triangle or another point.
// Certain hits go to SceneState::isect, undecided pairs to ::uncertain.
// ---------------------------------------------------------------------------
constexpr double ACCEPT_TOL = 1e-11;

__device__ __forceinline__ void accept_count(Pool& P, int s, int r) {
  if (r == 1) atomicAdd((unsigned long long*)&P.ss[s].isect, 1ull);
  else if (r == 2) atomicAdd((unsigned long long*)&P.ss[s].uncertain, 1ull);
}

__global__ void __launch_bounds__(128) k_accept_edges(Pool P) {
  const BVH& B = P.be;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n; i += gridDim.x * blockDim.x) {
    int e1 = B.ids[i];
    int4 ea = P.ev[e1];
    int s = ea.z;
    if (!P.ss[s].active) continue;
    dv3 alo, ahi;
    int sc;
    prim_box(P, 1, e1, alo, ahi, sc);
    dv3 p = mk(P.x[ea.x]), q = mk(P.x[ea.y]);
    // edge against triangles
    traverse(P.bt, P.bt.sroot[s], f3rd(alo), f3ru(ahi), 0.f, -1, P.cnt, [&](int pos) {
      int t = P.bt.ids[pos];
      int4 tv = P.tv[t];
      if (ea.x == tv.x || ea.x == tv.y || ea.x == tv.z || ea.y == tv.x || ea.y == tv.y || ea.y == tv.z) return;
      dv3 lo, hi;
      int sct;
      prim_box(P, 0, t, lo, hi, sct);
      if (!box_near(alo, ahi, lo, hi, 0.0)) return;
      accept_count(P, s, seg_tri_test(p, q, mk(P.x[tv.x]), mk(P.x[tv.y]), mk(P.x[tv.z]), ACCEPT_TOL));
    });
    // edge against later edges
    traverse(B, B.sroot[s], f3rd(alo), f3ru(ahi), 0.f, i, P.cnt, [&](int pos) {
      int e2 = B.ids[pos];
      int4 eb = P.ev[e2];
      if (ea.x == eb.x || ea.x == eb.y || ea.y == eb.x || ea.y == eb.y) return;
      dv3 lo, hi;
      int sc2;
      prim_box(P, 1, e2, lo, hi, sc2);
      if (!box_near(alo, ahi, lo, hi, 0.0)) return;
      dv3 c = mk(P.x[eb.x]), d = mk(P.x[eb.y]);
      int r = 0;
      if (o3f(p, q, c, d) == 2) {
        double ps, pt;
        r = d_ss(p, q, c, d, &ps, &pt) > ACCEPT_TOL ? 0 : 2;
      }
      accept_count(P, s, r);
    });
  }
}

__global__ void __launch_bounds__(128) k_accept_points(Pool P) {
  for (int qi = blockIdx.x * blockDim.x + threadIdx.x; qi < P.nq; qi += gridDim.x * blockDim.x) {
    int a = P.pts[qi];
    int s = P.vscene[a];
    if (!P.ss[s].active) continue;
    dv3 xa = mk(P.x[a]);
    double ra = P.rho[a];
    dv3 alo = {xa.x - ra, xa.y - ra, xa.z - ra}, ahi = {xa.x + ra, xa.y + ra, xa.z + ra};
    traverse(P.bt, P.bt.sroot[s], f3rd(alo), f3ru(ahi), __double2float_ru(1e-12), -1, P.cnt, [&](int pos) {
      int t = P.bt.ids[pos];
      int4 tv = P.tv[t];
      if (a == tv.x || a == tv.y || a == tv.z) return;
      double d = d_pt(xa, mk(P.x[tv.x]), mk(P.x[tv.y]), mk(P.x[tv.z]));
      int r;
      if (ra > 0.0) r = (d - ra) <= 1e-12 ? 1 : 0;
      else r = d > ACCEPT_TOL ? 0 : 2;
      accept_count(P, s, r);
    });
    double Dq = ra + P.sd[s].rho_max + 1e-12;
    traverse(P.bv, P.bv.sroot[s], f3rd(xa), f3ru(xa), __double2float_ru(Dq), -1, P.cnt, [&](int pos) {
      int b = P.vc[P.bv.ids[pos]];
      if (b <= a || !(P.vflag[b] & VF_POINT)) return;
      double g = (vnorm(vsub(xa, mk(P.x[b]))) - ra) - P.rho[b];
      accept_count(P, s, g <= 1e-12 ? 1 : 0);
    });
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

__global__ void k_copy_sorted(unsigned long long* kd, int* id, const unsigned long long* ks, const int* is, int n,
                              const int* gate) {
  if (gate && !*gate) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    kd[i] = ks[i];
    id[i] = is[i];
  }
}
__global__ void k_sroot_reset(Pool P, int c, int gated) {
  if (gate_off(P, gated)) return;
  BVH& B = bvh_of(P, c);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.nscene; s += gridDim.x * blockDim.x) B.sroot[s] = -1;
}

// Rebuild of one BVH: Morton codes, radix sort, Karras hierarchy, scene
// roots.  gated = 1 inside the iteration graph: every kernel returns at once
// unless the iteration searches.
void bvh_build(Runtime& R, int c, cudaStream_t st, int gated) {
  Pool& P = R.pool;
  BVH& B = c == 0 ? P.bt : (c == 1 ? P.be : P.bv);
  int n = B.n;
  if (n == 0) return;
  const int* gate = gated ? &P.cnt->any_search : nullptr;
  k_morton<<<grid_for(n, 256), 256, 0, st>>>(P, c, gated);
  R.launches++;
  int bits = 30 + R.scene_bits;
  int ntiles = (n + RS_TILE - 1) / RS_TILE;
  unsigned long long *k0 = B.keys, *k1 = B.keys_alt;
  int *v0 = B.ids, *v1 = B.ids_alt;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; p++) {
    int shift = 8 * p;
    k_radix_hist<<<ntiles, 256, 0, st>>>(k0, n, shift, B.hist, ntiles, gate);
    k_scan_1block<<<1, 1024, 0, st>>>(B.hist, 256 * ntiles, gate);
    k_radix_scatter<<<ntiles, 256, 0, st>>>(k0, v0, k1, v1, n, shift, B.hist, ntiles, gate);
    R.launches += 3;
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  if (k0 != B.keys) {
    k_copy_sorted<<<grid_for(n, 256), 256, 0, st>>>(B.keys, B.ids, k0, v0, n, gate);
    R.launches++;
  }
  k_sroot_reset<<<1, 128, 0, st>>>(P, c, gated);
  if (n > 1) k_karras<<<grid_for(n - 1, 256), 256, 0, st>>>(P, c, gated);
  else k_karras<<<1, 32, 0, st>>>(P, c, gated);
  k_scene_roots<<<grid_for(2 * n - 1, 256), 256, 0, st>>>(P, c, gated);
  R.launches += 3;
}

void bvh_build_all(Runtime& R, cudaStream_t st, int gated) {
  Pool& P = R.pool;
  k_scene_bounds_reset<<<(P.nscene + 127) / 128, 128, 0, st>>>(P, gated);
  k_scene_bounds<<<grid_for(P.nvc, 256), 256, 0, st>>>(P, gated);
  R.launches += 2;
  for (int c = 0; c < 3; c++) bvh_build(R, c, st, gated);
}

// All three trees at once: the arrival flags of every internal node, then
// per leaf its box and the climb (the second child to arrive at a node writes
// the node's boxes from its children's, which the first wrote before its
// arrival), so that the three climbs overlap instead of running one after the
// other.
__device__ __forceinline__ int class_of(const Pool& P, int i, int& j, bool internal) {
  int n0 = internal ? max(P.bt.n - 1, 0) : P.bt.n, n1 = internal ? max(P.be.n - 1, 0) : P.be.n;
  if (i < n0) { j = i; return 0; }
  if (i < n0 + n1) { j = i - n0; return 1; }
  j = i - n0 - n1;
  return 2;
}
__global__ void k_refit_reset_all(Pool P, int force) {
  if (!force && !P.cnt->any_search) return;
  int n = max(P.bt.n - 1, 0) + max(P.be.n - 1, 0) + max(P.bv.n - 1, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int j, c = class_of(P, i, j, true);
    bvh_of(P, c).flag[j] = 0;
  }
}
__global__ void k_refit_all(Pool P, int force) {
  if (!force && !P.cnt->any_search) return;
  int total = P.bt.n + P.be.n + P.bv.n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int i, c = class_of(P, t, i, false);
    BVH& B = bvh_of(P, c);
    int n = B.n;
    {
      dv3 lo, hi;
      int s;
      prim_box(P, c, B.ids[i], lo, hi, s);
      B.leafbox[2 * i] = make_float4(__double2float_rd(lo.x), __double2float_rd(lo.y), __double2float_rd(lo.z), 0.f);
      B.leafbox[2 * i + 1] =
          make_float4(__double2float_ru(hi.x), __double2float_ru(hi.y), __double2float_ru(hi.z), 0.f);
    }
    if (n < 2) continue;
    int node = B.parent[n - 1 + i];
    int climb = 0;
    while (node >= 0) {
      if (++climb > 256) {  // deeper than any Karras tree over 64-bit keys
        atomicOr(&P.cnt->err, ERR_TREE);
        break;
      }
      __threadfence();
      if (atomicAdd(&B.flag[node], 1) == 0) break;
      __threadfence();
      float4 llo, lhi, rlo, rhi;
      child_box(B, B.left[node], llo, lhi);
      child_box(B, B.right[node], rlo, rhi);
      B.box[3 * node] = make_float4(llo.x, llo.y, llo.z, lhi.x);
      B.box[3 * node + 1] = make_float4(lhi.y, lhi.z, rlo.x, rlo.y);
      B.box[3 * node + 2] = make_float4(rlo.z, rhi.x, rhi.y, rhi.z);
      node = B.parent[node];
    }
  }
}

void bvh_refit_all(Runtime& R, cudaStream_t st, int force) {
  Pool& P = R.pool;
  long long ni = (long long)max(P.bt.n - 1, 0) + max(P.be.n - 1, 0) + max(P.bv.n - 1, 0);
  long long nl = (long long)P.bt.n + P.be.n + P.bv.n;
  if (nl == 0) return;
  if (ni > 0) {
    k_refit_reset_all<<<grid_for(ni, 256), 256, 0, st>>>(P, force);
    R.launches++;
  }
  k_refit_all<<<grid_for(nl, 256), 256, 0, st>>>(P, force);
  R.launches++;
}

void query_class(Runtime& R, int c, int nxt, int mode, double Dq, cudaStream_t st) {
  Pool& P = R.pool;
  int bs = R.query_block;
  if (mode == 0 && R.packet) {
    if (c == 0 && P.nvc && P.nt) {
      k_pquery_vt<<<grid_for(P.nvc, bs), bs, 0, st>>>(P);
      R.launches++;
      return;
    }
    if (c == 1 && P.ne > 1) {
      k_pquery_ee<<<grid_for(P.ne, bs), bs, 0, st>>>(P);
      R.launches++;
      return;
    }
  }
  if (c == 0 && P.nvc && P.nt) {
    k_query_vt<<<grid_for(P.nvc, bs), bs, 0, st>>>(P, nxt, mode, Dq);
    R.launches++;
  }
  if (c == 1 && P.ne > 1) {
    k_query_ee<<<grid_for(P.ne, bs), bs, 0, st>>>(P, nxt, mode, Dq);
    R.launches++;
  }
  if (c == 2 && P.nq && P.nvc) {
    k_query_vv<<<grid_for(P.nq, bs), bs, 0, st>>>(P, nxt, mode, Dq);
    R.launches++;
  }
}

void finalize_search(Runtime& R, int nxt, int mode, double Dq, cudaStream_t st) {
  Pool& P = R.pool;
  if (mode == 0 && !P.mixed) {
    k_final_bounds<<<grid_for(3LL * P.pair_cap, 256), 256, 0, st>>>(P);
    R.launches++;
  }
  k_finalize<<<grid_for(3LL * P.pair_cap, 256), 256, 0, st>>>(P, nxt, mode, Dq);
  R.launches++;
  if (mode == 0 && !P.mixed) {
    k_exact_survivors<<<grid_for(3LL * P.pair_cap, 256), 256, 0, st>>>(P, nxt);
    R.launches++;
  }
}

void search_queries(Runtime& R, int nxt, int mode, double Dq, cudaStream_t st) {
  for (int c = 0; c < 3; c++) query_class(R, c, nxt, mode, Dq, st);
  if (mode != 1) finalize_search(R, nxt, mode, Dq, st);
}

void accept_queries(Runtime& R, cudaStream_t st) {
  Pool& P = R.pool;
  if (P.ne) {
    k_accept_edges<<<grid_for(P.ne, 128), 128, 0, st>>>(P);
    R.launches++;
  }
  if (P.nq) {
    k_accept_points<<<grid_for(P.nq, 128), 128, 0, st>>>(P);
    R.launches++;
  }
}

}  // namespace cch

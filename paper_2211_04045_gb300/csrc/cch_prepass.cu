// cch_prepass.cu -- the two pre-passes that produce the target x~ of the
// extra workloads, on the scene's own topology and BVHs:
//   - the target of the globally injective normal flow (Sec. 7.4, Eq. normal
//     flow): the surface pushed along its area-weighted vertex normals, then
//     smoothed by Jacobi steps of the cotangent Laplacian;
//   - friction by velocity filtering (Sec. 6.3): every vertex-triangle pair
//     closer than `reach` whose frictionless target would leave it closer
//     than `sep` gets a normal correction and a Coulomb-bounded tangential
//     one, shared by inverse mass.
// Every per-vertex sum is a gather in a fixed order (no atomics), so both
// pre-passes are bitwise reproducible.
#include "cch_host.h"
#include "cch_step.h"

namespace cch {

static int grid_of(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

__device__ __forceinline__ dv3 ld_aos(const double* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ void st_aos(double* p, int i, dv3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}

// ---------------------------------------------------------------------------
// normal flow
// ---------------------------------------------------------------------------
// y = x + (sign beta) n(x), n the normalised sum over the incident triangles
// (a, b, c) of (b - a) x (c - a) (area-weighted vertex normal)
__global__ void k_nf_push(Pool P, const double* x, double* y, double sb) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    dv3 s = {0.0, 0.0, 0.0};
    for (int j = P.tinc_start[v]; j < P.tinc_start[v + 1]; j++) {
      int4 t = P.tv[P.tinc[j] / 3];
      dv3 a = ld_aos(x, t.x), b = ld_aos(x, t.y), c = ld_aos(x, t.z);
      s = vadd(s, vcross(vsub(b, a), vsub(c, a)));
    }
    double L = vnorm(s);
    dv3 n = vdiv(s, L > 0.0 ? L : 1.0);
    st_aos(y, v, vadd(ld_aos(x, v), vscl(sb, n)));
  }
}

// One Jacobi step y_out = y + alpha Lap(y) of the cotangent Laplacian with the
// mixed Voronoi areas of Meyer et al. (2003): in each incident triangle with
// the vertex at corner k, the edges to corners k+1 and k+2 carry half the
// cotangents of the angles opposite them, and the vertex's area share is the
// Voronoi part (|e|^2 cot over its two edges, / 8) in a non-obtuse triangle,
// half the area at an obtuse corner and a quarter at the other corners.
__global__ void k_nf_smooth(Pool P, const double* y, double* yo, double alpha) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    dv3 lap = {0.0, 0.0, 0.0};
    double A = 0.0;
    for (int j = P.tinc_start[v]; j < P.tinc_start[v + 1]; j++) {
      int ent = P.tinc[j];
      int4 t = P.tv[ent / 3];
      int k = ent % 3;
      dv3 p[3] = {ld_aos(y, t.x), ld_aos(y, t.y), ld_aos(y, t.z)};
      double area2 = vnorm(vcross(vsub(p[1], p[0]), vsub(p[2], p[0])));
      double safe2 = area2 > 0.0 ? area2 : 1.0;
      double dots[3], cot[3];
      for (int i = 0; i < 3; i++) {
        dots[i] = vdot(vsub(p[(i + 1) % 3], p[i]), vsub(p[(i + 2) % 3], p[i]));
        cot[i] = dots[i] / safe2;
      }
      bool obtuse = dots[0] < 0.0 || dots[1] < 0.0 || dots[2] < 0.0;
      int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      dv3 e1 = vsub(p[k1], p[k]), e2 = vsub(p[k2], p[k]);
      lap = vadd(lap, vscl(0.5 * cot[k2], e1));
      lap = vadd(lap, vscl(0.5 * cot[k1], e2));
      double vor = (vdot(e1, e1) * cot[k2] + vdot(e2, e2) * cot[k1]) / 8.0;
      A = A + (!obtuse ? vor : (dots[k] < 0.0 ? area2 / 4.0 : area2 / 8.0));
    }
    dv3 l = vdiv(lap, A > 0.0 ? A : 1.0);
    st_aos(yo, v, vadd(ld_aos(y, v), vscl(alpha, l)));
  }
}

// ---------------------------------------------------------------------------
// friction by velocity filtering
// ---------------------------------------------------------------------------
// closest point of triangle (a, b, c) to p as barycentric weights, by the
// Voronoi regions of the triangle: the corners, the edges, else the interior
// (Ericson, Real-Time Collision Detection, Sec. 5.1.5)
__device__ __forceinline__ void closest_weights(dv3 p, dv3 a, dv3 b, dv3 c, double w[3]) {
  dv3 ab = vsub(b, a), ac = vsub(c, a), ap = vsub(p, a), bp = vsub(p, b), cp = vsub(p, c);
  double d1 = vdot(ab, ap), d2 = vdot(ac, ap), d3 = vdot(ab, bp), d4 = vdot(ac, bp), d5 = vdot(ab, cp),
         d6 = vdot(ac, cp);
  double va = d3 * d6 - d5 * d4, vb = d5 * d2 - d1 * d6, vc = d1 * d4 - d3 * d2;
  if (d1 <= 0.0 && d2 <= 0.0) { w[0] = 1.0; w[1] = 0.0; w[2] = 0.0; return; }
  if (d3 >= 0.0 && d4 <= d3) { w[0] = 0.0; w[1] = 1.0; w[2] = 0.0; return; }
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    double t = d1 / (d1 - d3);
    w[0] = 1.0 - t; w[1] = t; w[2] = 0.0;
    return;
  }
  if (d6 >= 0.0 && d5 <= d6) { w[0] = 0.0; w[1] = 0.0; w[2] = 1.0; return; }
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    double t = d2 / (d2 - d6);
    w[0] = 1.0 - t; w[1] = 0.0; w[2] = t;
    return;
  }
  if (va <= 0.0 && d4 - d3 >= 0.0 && d5 - d6 >= 0.0) {
    double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    w[0] = 0.0; w[1] = 1.0 - t; w[2] = t;
    return;
  }
  double den = (va + vb) + vc;
  double v_ = vb / den, w_ = vc / den;
  w[0] = (1.0 - v_) - w_; w[1] = v_; w[2] = w_;
}

struct FrictionArgs {
  double mu, reach, sep;
};

// The contact of point vertex pv with triangle t (positions x in P.x, the
// frictionless target in P.y): false if it is not a contact; else du (the
// pair's relative correction), W and the closest-point weights.
__device__ __forceinline__ bool friction_pair(const Pool& P, int pv, int4 t, const FrictionArgs& F, double w[3],
                                              dv3& du, double& W) {
  if (pv == t.x || pv == t.y || pv == t.z) return false;
  double ip = P.im[pv], i0 = P.im[t.x], i1 = P.im[t.y], i2 = P.im[t.z];
  if (!(ip > 0.0 || i0 > 0.0 || i1 > 0.0 || i2 > 0.0)) return false;
  dv3 p = mk(P.x[pv]), a = mk(P.x[t.x]), b = mk(P.x[t.y]), c = mk(P.x[t.z]);
  closest_weights(p, a, b, c, w);
  dv3 q = vadd(vadd(vscl(w[0], a), vscl(w[1], b)), vscl(w[2], c));
  dv3 pq = vsub(p, q);
  double d = vnorm(pq);
  if (!(d < F.reach && d > 0.0)) return false;
  dv3 nrm = vdiv(pq, d);
  dv3 dyp = vsub(mk(P.y[pv]), p);
  dv3 dy0 = vsub(mk(P.y[t.x]), a), dy1 = vsub(mk(P.y[t.y]), b), dy2 = vsub(mk(P.y[t.z]), c);
  dv3 u = vsub(dyp, vadd(vadd(vscl(w[0], dy0), vscl(w[1], dy1)), vscl(w[2], dy2)));
  double un = vdot(u, nrm);
  double pen = F.sep - (d + un);
  W = ip + ((w[0] * w[0] * i0 + w[1] * w[1] * i1) + w[2] * w[2] * i2);
  if (!(pen > 0.0 && W > 0.0)) return false;
  dv3 ut = vsub(u, vscl(un, nrm));
  double lt = vnorm(ut);
  double f = fmin(F.mu * pen, lt);
  du = vsub(vscl(pen, nrm), vscl(f / (lt > 0.0 ? lt : 1.0), ut));
  return true;
}

// Per vertex v: the corrections of its contacts as the point (against the
// triangles within reach) and as a triangle corner (against the points within
// reach of its incident triangles), averaged over the contacts that move it.
// The points are the collision vertices; pairs come from the BVHs built at x.
__global__ void __launch_bounds__(128) k_friction(Pool P, FrictionArgs F, double* out) {
  float Rf = __double2float_ru(F.reach);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x) {
    int s = P.vscene[v];
    double iv = P.im[v];
    dv3 corr = {0.0, 0.0, 0.0};
    double cnt = 0.0;
    dv3 xv = mk(P.x[v]);
    if (P.vflag[v] & VF_COLL) {
      traverse(P.bt, P.bt.sroot[s], f3rd(xv), f3ru(xv), Rf, -1, P.cnt, [&](int pos) {
        int4 t = P.tv[P.bt.ids[pos]];
        double w[3], W;
        dv3 du;
        if (!friction_pair(P, v, t, F, w, du, W)) return;
        corr = vadd(corr, vscl(iv / W, du));
        cnt += iv > 0.0 ? 1.0 : 0.0;
      });
    }
    for (int j = P.tinc_start[v]; j < P.tinc_start[v + 1]; j++) {
      int ent = P.tinc[j];
      int4 t = P.tv[ent / 3];
      int k = ent % 3;
      dv3 lo, hi;
      {
        dv3 a = mk(P.x[t.x]), b = mk(P.x[t.y]), c = mk(P.x[t.z]);
        lo = {fmin(fmin(a.x, b.x), c.x), fmin(fmin(a.y, b.y), c.y), fmin(fmin(a.z, b.z), c.z)};
        hi = {fmax(fmax(a.x, b.x), c.x), fmax(fmax(a.y, b.y), c.y), fmax(fmax(a.z, b.z), c.z)};
      }
      traverse(P.bv, P.bv.sroot[s], f3rd(lo), f3ru(hi), Rf, -1, P.cnt, [&](int pos) {
        int pv = P.vc[P.bv.ids[pos]];
        double w[3], W;
        dv3 du;
        if (!friction_pair(P, pv, t, F, w, du, W)) return;
        corr = vsub(corr, vscl(w[k] * iv / W, du));
        cnt += (iv > 0.0 && w[k] != 0.0) ? 1.0 : 0.0;
      });
    }
    dv3 y = mk(P.y[v]);
    st_aos(out, v - P.sd[s].v0, vadd(y, vdiv(corr, cnt > 1.0 ? cnt : 1.0)));
  }
}

// ---------------------------------------------------------------------------
// host launchers (single scene; positions already in the pool for friction)
// ---------------------------------------------------------------------------
void normal_flow(Runtime& R, const double* x, double* y, double* tmp, double sb, double alpha, int iters,
                 cudaStream_t st) {
  Pool& P = R.pool;
  int g = grid_of(P.nv, 256);
  // y0 in y (iters even) or tmp (iters odd), so that the last step writes y
  double* a = (iters % 2) ? tmp : y;
  double* b = (iters % 2) ? y : tmp;
  k_nf_push<<<g, 256, 0, st>>>(P, x, a, sb);
  for (int i = 0; i < iters; i++) {
    k_nf_smooth<<<g, 256, 0, st>>>(P, a, b, alpha);
    double* c = a;
    a = b;
    b = c;
  }
  R.launches += 1 + iters;
}

void friction(Runtime& R, double mu, double reach, double sep, double* out, cudaStream_t st) {
  FrictionArgs F{mu, reach, sep};
  k_friction<<<grid_of(R.pool.nv, 128), 128, 0, st>>>(R.pool, F, out);
  R.launches++;
}

}  // namespace cch

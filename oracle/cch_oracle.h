/*
 * cch_oracle.h -- CPU FP64 oracle for the two-way continuous collision
 * handling step (Wang et al., "Fast GPU-Based Two-Way Continuous Collision
 * Handling", arXiv 2211.04045).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library never
 * links, loads or calls it.  It shares no code, header or table with the CUDA
 * path.
 *
 * All floating point is IEEE binary64, compiled without FP contraction
 * (-ffp-contract=off) so that every expression is evaluated exactly as
 * written.  Vertex arrays are AoS, n x 3 doubles; index arrays are int32.
 */
#ifndef CCH_ORACLE_H
#define CCH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pair kinds of the proximity set P (Sec. 3.1, Sec. 4.1). */
enum { ORC_VT = 0, ORC_EE = 1, ORC_VV = 2 };

/* Mesh topology and per-vertex data of one scene (host pointers). */
typedef struct {
  int64_t n_verts;
  const double* inv_mass;     /* n_verts; 0 = fixed or kinematic            */
  const double* radius;       /* n_verts or NULL (all 0); used by points     */
  int64_t n_tris;  const int32_t* tris;       /* 3 per triangle (VT targets) */
  int64_t n_edges; const int32_t* edges;      /* 2 per collision edge (EE)   */
  int64_t n_len;   const int32_t* len_edges;  /* 2 per edge-length constraint*/
  int64_t n_points; const int32_t* points;    /* VV participants (sand)      */
} orc_topology;

/* Parameters of Algorithm 1 (Table 2 defaults: see orc_params_default). */
typedef struct {
  double d_min, d_max;   /* proximity-search bounds D^min, D^max            */
  double delta;          /* contact activation threshold                    */
  double sigma;          /* edge-length violation ratio limit                */
  double gamma;          /* forward-step damping factor                      */
  double eps;            /* termination threshold on ||r||_inf               */
  double jacobi_omega;   /* under-relaxation of the projected Jacobi variant */
  int32_t max_iters;     /* L (the loop runs l = 0..L inclusive)            */
  int32_t gs_sweeps;     /* projected Gauss-Seidel sweeps per backward step  */
  int32_t solver;        /* 0 = projected Gauss-Seidel, 1 = projected Jacobi */
  int32_t ccd_check;     /* 1 = run the segment CCD safety check each iter   */
  int32_t search_mode;   /* 0 = all pairs, 1 = sorted-axis window, 2 = auto  */
  int32_t constraint_form; /* 0 = volume (Sec. 4.1), 1 = gap (the comparison */
                           /*     constraints of Sec. 4.1's gap figure)      */
  int32_t step_rule;     /* 0 = distance bound of Eq. forward2; 1 = CCD-based
                            step size (the comparison scheme of Sec. 5.1)     */
  int32_t ccd_rounds;    /* CCD clamp rounds before the scene's step is
                            frozen for the iteration (CCD check and rule)     */
  int32_t colouring;     /* randomized colouring of the Gauss-Seidel sweep
                            (R11): 0 greedy (smallest free colour), 1 level
                            (the round in which the constraint's priority
                            first exceeds its uncoloured neighbours')         */
  uint64_t seed;         /* colouring priorities (R11)                        */
} orc_params;

typedef struct {
  int32_t iterations, searches, converged, ccd_clamps;
  int64_t pairs_evaluated;   /* sum over iterations of |P|                    */
  int64_t max_pairs;         /* max over iterations of |P|                    */
  int64_t active_contacts;   /* sum over iterations of active contacts        */
  int64_t candidates;        /* sum over searches of box-test candidates      */
  int64_t degenerate;        /* contacts skipped as degenerate                */
  int32_t max_vertex_contacts; /* most contacts at one movable vertex (max over */
                               /* iterations): a lower bound on any colouring   */
  int32_t max_vertex_edges;    /* most edge-length constraints at one vertex    */
  double final_r_inf;
  double min_pair_dist;      /* min pair distance seen over the whole step    */
  int32_t frozen_vertices;   /* vertices held by the D_i floor (1e-10 m) at the
                                last iteration although y_i differs from x_i  */
  int32_t contact_colours;   /* most colours of one iteration's contact
                                colouring (Gauss-Seidel, Sec. 4.3)            */
  int64_t contact_vertices;  /* sum over iterations of the distinct movable
                                vertices of the contact constraints           */
  int32_t edge_colours;      /* colours of the edge-length constraints        */
  int32_t reserved_;
  int64_t pair_vertices;     /* sum over iterations of the distinct vertices
                                of the pairs of P                             */
} orc_stats;

/* Optional per-iteration record (tests only).  Any pointer may be NULL. */
typedef struct {
  int32_t cap_iters;
  double* x;          /* (cap_iters+1) * n * 3 : x^(l), l = 0..iterations    */
  double* y;          /* cap_iters * n * 3     : y^(l+1)                      */
  double* Dl;         /* cap_iters : D^(l) in force during iteration l        */
  double* Di;         /* cap_iters * n : D_i of iteration l                   */
  int32_t* searched;  /* cap_iters                                            */
  int64_t* n_pairs;   /* cap_iters : |P| used by iteration l                   */
  int64_t cap_pairs;
  uint64_t* pair_keys;/* cap_iters * cap_pairs : keys of P (ascending)         */
  int64_t* n_contacts;/* cap_iters                                            */
} orc_trace;

void orc_params_default(orc_params* p);

/* ---- geometry (Sec. 4.1, Sec. 5) ---- */
double orc_point_segment_dist(const double p[3], const double a[3], const double b[3], double* t);
double orc_point_triangle_dist(const double p[3], const double a[3], const double b[3], const double c[3]);
double orc_segment_segment_dist(const double a[3], const double b[3], const double c[3], const double d[3],
                                double* s, double* t);
double orc_signed_volume(const double a[3], const double b[3], const double c[3], const double d[3]);
int orc_orient3d_exact(const double a[3], const double b[3], const double c[3], const double d[3]);
uint64_t orc_splitmix64(uint64_t x);

/* ---- proximity search (Sec. 3.1) ---- */
/* Candidate set: non-adjacent, not-all-static pairs whose boxes are within
 * D per axis.  Writes up to cap keys (ascending); returns the total count. */
int64_t orc_candidates(const orc_topology* t, const double* x, const double* x_tilde, double D,
                       int32_t mode, uint64_t* keys, int64_t cap);
/* P = candidates with distance < D.  Returns |P|; keys ascending. */
int64_t orc_proximity(const orc_topology* t, const double* x, const double* x_tilde, double D,
                      int32_t mode, uint64_t* keys, double* dist, int64_t cap);

/* ---- one constraint (Sec. 4.1, 4.2) ---- */
/* kind VT/EE/VV with vertex positions p[4][3] (VV uses 2), radii rho[2]
 * (VT: rho[0] of the vertex; VV: both), form 0 (volume) or 1 (gap).
 * Returns 1 if assembled, 0 if skipped as degenerate; c0 and g[4][3] receive
 * the constraint value and gradient at x. */
int orc_contact_constraint(int kind, const double* p, const double* rho, double delta, int form,
                           double* c0, double* g);

/* ---- one backward step (Sec. 4), used by single-constraint pins ---- */
/* Runs a search at D^max on x, assembles contacts and edge constraints,
 * sweeps once, starting from y_in.  y_out receives y^(l+1). */
int orc_backward_once(const orc_topology* t, const orc_params* prm, const double* x,
                      const double* y_in, const double* y_target, double* y_out);

/* ---- colouring of the Gauss-Seidel sweep (Sec. 4.3) ---- */
/* Colouring of n constraints with vertex lists verts[4*i..4*i+3] (-1 =
 * absent) and priorities prio[i], taken by descending priority: kind 0
 * greedy, each gets the smallest colour not used by an earlier constraint
 * sharing a movable vertex with it; kind 1 level, one more than the largest
 * colour among those (0 if none).  colour[i] receives it; returns the number
 * of colours. */
int32_t orc_colouring(int32_t kind, int64_t n, const int32_t* verts, const uint64_t* prio, const double* inv_mass,
                      int64_t n_verts, int32_t* colour);
/* The contact constraints that a backward step at state x builds from a
 * search at D^max (keys ascending) and the colour of each; returns the count
 * (up to cap written). */
int64_t orc_contact_colours(const orc_topology* t, const orc_params* prm, const double* x, const double* x_tilde,
                            uint64_t* keys, int32_t* colour, int64_t cap);
/* Colours of the edge-length constraints (in the topology's edge order). */
int32_t orc_edge_colours(const orc_topology* t, const orc_params* prm, int32_t* colour);

/* ---- CCD (comparison scheme of Sec. 5.1, used as a safety check) ---- */
/* Vertices 0..3 move linearly from x0 to x1 (VT: a,i,j,k; EE: a,b,c,d; VV:
 * a,b with radii rho[0..1]; rho may be NULL).  Returns 1 and the first time
 * of impact in [0,1] if they touch. */
int orc_ccd(int kind, const double* x0, const double* x1, const double* rho, double* toi);

/* Conservative counterpart used to check orc_ccd: 0 when the primitives
 * certainly stay more than tol apart over the whole motion (bound: distance
 * at an interval's midpoint minus the largest relative vertex displacement
 * over half the interval, with bisection), 1 when that cannot be shown. */
int orc_ccd_conservative(int kind, const double* x0, const double* x1, const double* rho, double tol);

/* ---- exact acceptance ---- */
/* Number of intersecting non-adjacent primitive pairs in state x, decided by
 * exact predicates (segment-triangle, vertex-triangle, segment-segment, and
 * sphere overlap for points). */
int64_t orc_count_intersections(const orc_topology* t, const double* x);

/* ---- Algorithm 1 ---- */
int orc_handle_step(const orc_topology* t, const orc_params* prm, const double* x_t,
                    const double* x_tilde, double* x_next, orc_stats* stats, orc_trace* trace);

#ifdef __cplusplus
}
#endif
#endif

/*
 * cch.h -- C ABI of the GB300 two-way continuous collision handling library.
 *
 * The library implements one collision-handling call of Wang et al., "Fast
 * GPU-Based Two-Way Continuous Collision Handling" (arXiv 2211.04045): given
 * an intersection-free state x^t and an unconstrained target x~ it runs
 * Algorithm 1 (interleaved backward and forward steps, Sec. 3-5) on the GPU
 * and returns an intersection-free x^{t+1}.
 *
 * Conventions shared by every entry point
 *   - Every function returns cch_status; none aborts, traps or exits.
 *   - Position arrays are AoS float64, n_verts x 3, C-contiguous.  Unless a
 *     name ends in _host they are DEVICE pointers on the device that was
 *     current when the scene was created, and must stay valid until the call
 *     returns.  The call is stream-ordered on the scene's stream and returns
 *     after the result has been written (it synchronises that stream).
 *   - Topology and parameters are copied at creation; the caller keeps
 *     ownership of every pointer it passes.
 *   - Invalid arguments (NULL, negative sizes, out-of-range indices) are
 *     rejected with CCH_E_INVALID_ARG before any device work.  Non-finite
 *     coordinates in x_t or x_tilde are detected on the device when the step
 *     starts: that scene runs no iteration and the call (or the server
 *     request) returns CCH_E_INVALID_ARG, x_next then being unspecified.
 *   - Not reaching ||r||_inf < eps within L iterations is NOT an error: the
 *     result is still intersection-free (Sec. 3, end of the Algorithm 1
 *     discussion) and stats.converged = 0 reports it.
 *   - A scene object may be used by one host thread at a time.
 */
#ifndef CCH_H
#define CCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CCH_OK = 0,
  CCH_E_INVALID_ARG = 1,       /* bad pointer, size, index or value            */
  CCH_E_OOM = 2,               /* device allocation failed                     */
  CCH_E_BUDGET = 3,            /* a server's HBM budget would be exceeded      */
  CCH_E_CUDA = 4,              /* a CUDA runtime call failed                   */
  CCH_E_CAPACITY = 5,          /* an internal bound was exceeded (buffers past
                                  2^30 pairs, BVH traversal or sweep bounds)   */
  CCH_E_TIMEOUT = 6,           /* a bounded device wait ran out (the colouring's
                                  vertex counters or the sweep's grid barrier);
                                  the context stays usable                     */
  CCH_E_INPUT_NOT_FEASIBLE = 7,/* validate_input: x_t already intersects       */
  CCH_E_CANCELLED = 8,         /* a server request was cancelled               */
  CCH_E_STATE = 9              /* call not valid in the object's current state */
} cch_status;

typedef enum { CCH_PREC_FP64 = 0, CCH_PREC_MIXED = 1 } cch_precision;
/* Backward step (Sec. 4.3): gs_sweeps multi-colour projected Gauss-Seidel
 * sweeps per iteration (the contact colour classes in ascending colour, then
 * the edge-length classes; each group coloured by cch_colouring), or
 * the projected Jacobi variant (Sec. 4.3.2) with per-constraint
 * under-relaxation jacobi_omega / (most constraints at one of its vertices). */
typedef enum { CCH_SOLVER_GAUSS_SEIDEL = 0, CCH_SOLVER_JACOBI = 1 } cch_solver;
/* Randomized colouring of the multi-colour Gauss-Seidel sweep (Sec. 4.3), over
 * the constraints in descending priority splitmix64(seed ^ key), conflicts
 * through movable vertices only.  CCH_COLOUR_GREEDY: each constraint takes the
 * smallest colour not used by a higher-priority conflicting constraint (the
 * Jones-Plassmann colouring; fewest classes, computed by a colouring pass each
 * iteration, then one class per phase).  CCH_COLOUR_LEVEL (default): one more
 * than the largest such colour, the round in which its priority first exceeds
 * that of all its uncoloured conflicting constraints (Luby's rounds); the
 * classes then follow the priorities, and a dataflow sweep applies them
 * without a colouring pass. */
typedef enum { CCH_COLOUR_GREEDY = 0, CCH_COLOUR_LEVEL = 1 } cch_colouring;
/* Contact constraints: the volume-based constraints of Sec. 4.1 (default), or
 * the gap constraints c = d/delta - 1 the paper compares them with (gradient:
 * the closest-point weights times the unit separation direction, over delta).
 * Vertex-vertex pairs use the distance form in both. */
typedef enum { CCH_FORM_VOLUME = 0, CCH_FORM_GAP = 1 } cch_constraint_form;

/* Step size of the forward step.  CCH_STEP_DISTANCE: Eq. forward2,
 * alpha_i = min(0.5 gamma D_i / |y_i - x_i|, 1), safe by construction (Sec.
 * 5).  CCH_STEP_CCD: the CCD-based scheme Sec. 5.1 compares it with: every
 * vertex is capped by the global bound 0.5 gamma D^(l) (a pair outside P is at
 * least D^(l) apart, so only pairs of P can meet), and the CCD of each pair's
 * segment decides the rest: a hit at time t scales the step of the pair's
 * vertices by t/2, and the segments are tested again (ccd_rounds). */
typedef enum { CCH_STEP_DISTANCE = 0, CCH_STEP_CCD = 1 } cch_step_rule;

/* Parameters of Algorithm 1.  cch_params_default() fills Table 2's values
 * (L = 2048, eps = 1e-4, D^min = 2 mm, D^max = 4 mm, delta = 1 mm,
 * sigma = 1.1, gamma = 0.9). */
typedef struct {
  double d_min;          /* D^min: search again when D^(l) falls below it      */
  double d_max;          /* D^max: bound of each proximity search              */
  double delta;          /* contact activation threshold (Sec. 4.1)            */
  double sigma;          /* edge-length violation ratio limit (Sec. 4.2)       */
  double gamma;          /* forward-step damping factor (Eq. forward2)         */
  double eps;            /* termination threshold on ||r||_inf                 */
  double jacobi_omega;   /* under-relaxation of the projected Jacobi solver    */
  int32_t max_iters;     /* L; the loop runs l = 0..L (at most L+1 iterations) */
  int32_t gs_sweeps;     /* Gauss-Seidel sweeps per backward step (Sec 4.3.1)  */
  int32_t precision;     /* cch_precision                                      */
  int32_t solver;        /* cch_solver                                         */
  int32_t ccd_check;     /* 1: CCD of every pair's segment each iteration, with
                            the time-of-impact clamp (Sec. 5.1 scheme as a
                            safety net; always on under CCH_STEP_CCD)          */
  int32_t accept_check;  /* 1: exact-filtered intersection test of x^{t+1}
                            (always on under CCH_STEP_CCD: its root-finding
                            CCD can miss a tangential touch)                   */
  int32_t validate_input;/* 1: the same test on x^t before the loop            */
  int32_t iters_per_launch; /* iterations captured per CUDA-graph launch (G)   */
  int32_t bvh_refit_only;   /* 1: rebuild the BVH at the first search of a step
                               and only refit it at later searches             */
  int32_t constraint_form;  /* cch_constraint_form                             */
  int32_t step_rule;        /* cch_step_rule                                   */
  int32_t ccd_rounds;       /* CCD clamp rounds per iteration, 0..64 (default
                               8); a hit that remains after the last round
                               keeps every vertex of the scene in place for the
                               iteration                                       */
  uint64_t seed;         /* priorities of the randomized colouring (Sec. 4.3)  */
  int32_t max_polls;     /* bound on the polls of one bounded device wait (the
                            colouring's vertex counters, the sweep's grid
                            barrier); past it the call returns CCH_E_TIMEOUT.
                            0 = the default 2^22                               */
  int32_t pair_capacity; /* initial capacity of the pair buffers, in pairs
                            (0 = 4 (T + E + Q) + 4096); they double on
                            overflow and the step is run again                 */
  int32_t sweep_blocks;  /* blocks of the cooperative sweep kernels (0 = every
                            block that fits on the device at once)             */
  int32_t colouring;     /* cch_colouring of the Gauss-Seidel sweep            */
} cch_params;

/* Mesh of one scene (host pointers, copied at creation).
 * Collision vertices are the vertices of tris, edges and points; every
 * collision vertex is tested against every triangle (vertex-triangle pairs),
 * collision edges against each other (edge-edge), and points against every
 * collision vertex (vertex-vertex, e.g. sand grains). */
typedef struct {
  int64_t n_verts;
  const double* inv_mass;      /* n_verts; 0 = fixed or scripted (kinematic)   */
  const double* point_radius;  /* n_verts or NULL (all 0)                      */
  int64_t n_tris;   const int32_t* tris;       /* 3 per triangle               */
  int64_t n_edges;  const int32_t* edges;      /* 2 per collision edge         */
  int64_t n_len;    const int32_t* len_edges;  /* 2 per edge-length constraint */
  int64_t n_points; const int32_t* points;     /* vertex ids of point bodies   */
} cch_topology;

typedef struct {
  int32_t iterations;        /* Algorithm 1 iterations executed               */
  int32_t searches;          /* proximity searches                            */
  int32_t converged;         /* ||r||_inf < eps reached                       */
  int32_t ccd_clamps;        /* CCD hits, summed over the rounds of every
                                iteration (0 expected under CCH_STEP_DISTANCE) */
  int64_t pairs_evaluated;   /* sum over iterations of |P|                    */
  int64_t max_pairs;         /* max over iterations of |P|                    */
  int64_t active_contacts;   /* sum over iterations of contacts (dist<delta)  */
  int64_t candidates;        /* sum over searches of box-test candidates      */
  int64_t degenerate;        /* contacts skipped as degenerate                */
  int32_t max_vertex_contacts; /* most contacts at one movable vertex in an
                                iteration (a lower bound on the colours of
                                any colouring of them)                        */
  int32_t max_vertex_edges;  /* most edge-length constraints at one vertex    */
  double final_r_inf;        /* ||r^(l+1)||_inf at exit                       */
  double min_pair_dist;      /* smallest pair distance seen in the step       */
  int64_t intersections;     /* accept_check: intersecting pairs in x^{t+1}   */
  int64_t uncertain;         /* accept_check: pairs the FP64 filter could not
                                certify (expected 0)                          */
  double device_ms;          /* device time of the call (CUDA events)         */
  int64_t kernel_launches;   /* kernels this call launched (graph nodes count) */
  int32_t gs_depth;          /* phases of one Gauss-Seidel sweep, one per
                                colour class: contact_colours + edge_colours
                                (the sweep's critical path)                   */
  int32_t frozen_vertices;   /* vertices held in place at the last iteration
                                because their D_i fell below 1e-10 m (the
                                floor under which D_i/2 is no larger than the
                                rounding of a position update) although their
                                y_i differs from x_i                          */
  int64_t contact_vertices;  /* sum over iterations of the distinct movable
                                vertices of the contact constraints           */
  int32_t contact_colours;   /* most colours of one iteration's contact
                                colouring (Gauss-Seidel, cch_colouring)       */
  int32_t edge_colours;      /* colours of the edge-length constraints        */
  int64_t pair_vertices;     /* sum over iterations of the distinct vertices
                                of the pairs of P                             */
} cch_step_stats;

typedef struct cch_scene cch_scene;
typedef struct cch_server cch_server;

cch_status cch_params_default(cch_params* p);
const char* cch_status_string(cch_status s);

/* Create one resident scene on the current device.  cuda_stream may be NULL
 * (the legacy default stream) or a cudaStream_t.  Algorithm 1 input line:
 * the mesh and the bounds [D^min, D^max], L and eps. */
cch_status cch_create_scene(const cch_topology* topo, const cch_params* prm, void* cuda_stream, cch_scene** out);

/* Create a batch: n_scenes independent scenes that every step call handles
 * together in one set of launches (per-scene offset tables, per-scene loop
 * control).  Each scene's result equals what a scene of its own returns. */
cch_status cch_create_batch(const cch_topology* topos, int32_t n_scenes, const cch_params* prm, void* cuda_stream,
                            cch_scene** out);

/* As cch_create_batch, with each scene's own physical parameters (Table 2):
 * d_min, d_max, delta, sigma, gamma, eps, max_iters and seed come from
 * scene_prm[s] (n_scenes entries, each validated like prm); every other
 * field, the method and its launch configuration, from prm.  A scene of the
 * batch then returns what cch_create_scene with scene_prm[s] returns, when
 * the method fields agree.  scene_prm NULL: cch_create_batch.  The arrays are
 * read during the call only; an invalid entry returns CCH_E_INVALID_ARG
 * before any device work. */
cch_status cch_create_batch_params(const cch_topology* topos, int32_t n_scenes, const cch_params* prm,
                                   const cch_params* scene_prm, void* cuda_stream, cch_scene** out);

/* One collision-handling call, Algorithm 1: x^(0) = x_t, y^(0) = x_tilde;
 * x_next receives x^(l+1).  Device pointers, n_verts x 3 float64 each;
 * x_next may alias x_t.  stats may be NULL. */
cch_status cch_handle_step(cch_scene* s, const double* x_t, const double* x_tilde, double* x_next,
                           cch_step_stats* stats);

/* Same call with HOST buffers: the library copies x_t and x_tilde to the
 * device and x_next back (pageable or pinned memory). */
cch_status cch_handle_step_host(cch_scene* s, const double* x_t, const double* x_tilde, double* x_next,
                                cch_step_stats* stats);

/* Batched call: arrays of n_scenes device pointers (scene order of
 * cch_create_batch); stats is an array of n_scenes entries or NULL. */
cch_status cch_batch_handle_step(cch_scene* s, const double* const* x_t, const double* const* x_tilde,
                                 double* const* x_next, cch_step_stats* stats);

/* ---- autotuning of the launch configuration ------------------------------
 * Times candidate launch configurations on a probe: one step from x_t and
 * x_tilde (device pointers of the single scene), capped at probe_iters
 * iterations (1..4096), run twice per candidate.  Coordinate descent over:
 * iterations per graph launch group G in {4, 8, 16, 32, 64}; threads per block
 * of the BVH queries in {64, 128, 256}; BVH refit at later searches against a
 * rebuild at every search; packet traversal (32 queries per warp descend as
 * a wavefront, each stack entry holding the queries that reach its node)
 * against one traversal per thread.  The fastest configuration is kept for the scene's
 * later steps.  Results never depend on the configuration: each probe's output
 * is compared bitwise with the first (consistent = 1).  Allocates one scratch
 * output of n_verts x 3 doubles for the duration of the call. */
typedef struct {
  int32_t iters_per_launch;  /* chosen G                                      */
  int32_t query_block;       /* chosen threads per block of the BVH queries   */
  int32_t bvh_refit_only;    /* chosen: 1 refit, 0 rebuild at every search    */
  int32_t trials;            /* configurations timed                          */
  int32_t consistent;        /* 1: every probe gave the same x_next bitwise    */
  int32_t packet_traversal;  /* chosen: 1 packet (wavefront), 0 thread-per-query */
  double best_ms;            /* probe time with the chosen configuration      */
  double default_ms;         /* probe time with the configuration at entry    */
} cch_tune_result;

cch_status cch_autotune(cch_scene* s, const double* x_t, const double* x_tilde, int32_t probe_iters,
                        cch_tune_result* out);

cch_status cch_destroy(cch_scene* s);

/* ---- inspection (tests) ------------------------------------------------ */
/* Candidate set (Sec. 3.1 broad phase: non-adjacent, not-all-static pairs
 * whose boxes are within D on every axis) and proximity set
 * P = {candidates with dist < D} of scene 0 at state x (device pointer),
 * with the static-vertex flags taken from (x_t, x_tilde) = (x, x_ref).
 * want_candidates: 1 the candidate set; 0 P with exact FP64 distances;
 * 2 P exactly as the first search of a step forms it, at the scene's D^max
 * (D is ignored), with the distances the step records: in mixed precision
 * the FP32 lower bounds that decide membership there, in FP64 the exact
 * distance where it decides something and an FP32 lower bound otherwise.
 * keys (host, capacity cap) receive the canonical pair keys
 * kind<<62 | id1<<31 | id2 in unspecified order, dist (host, may be NULL)
 * the matching distances; *count receives the full size even when it
 * exceeds cap. */
cch_status cch_query_pairs(cch_scene* s, const double* x, const double* x_ref, double D, int32_t want_candidates,
                           uint64_t* keys, double* dist, int64_t cap, int64_t* count);

/* Bound of the scene's bounded device waits (the colouring's vertex counters
 * and the sweep's grid barrier), in polls; 0 restores the default 2^22.  A
 * wait that runs out makes the step return CCH_E_TIMEOUT and leaves the
 * scene usable for the next call. */
cch_status cch_set_max_polls(cch_scene* s, int32_t max_polls);

/* ---- proximity query without device allocation ----------------------------
 * The same query as cch_query_pairs for callers that must not allocate device
 * memory while they run: real-time loops that reserve all of their memory up
 * front and may not touch the allocator once they are running (an allocation
 * can stall on the device or fail when memory is short), and hosts whose own
 * memory manager owns the GPU's memory and forbids direct cudaMalloc.  The
 * paper has no counterpart; this is a deployment variant of the query above.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The pair
 * list the query kernels produce is written to one fixed array inside the
 * library (CCH_NOALLOC_MAX_PAIRS pairs, 16 bytes each, 2 MiB per GPU, held by
 * every GPU that loads the library until the process exits) and copied to
 * keys/dist from there.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress, once per device, with that device
 * current).  Like every call of this library it synchronises the scene's
 * stream and copies its results to the host before it returns.
 * want_candidates is 0 or 1.
 * Results: as cch_query_pairs.  When more than CCH_NOALLOC_MAX_PAIRS pairs
 * are found, *count receives the full count and the call returns
 * CCH_E_CAPACITY without copying.  When the query's intermediate pairs
 * outgrow the buffers the scene was created with (cch_query_pairs would grow
 * them; this call cannot), the full count is not known: *count receives -1
 * and the call returns CCH_E_CAPACITY.  All calls share the array and it
 * keeps the previous call's contents; calls whose work overlaps on the GPU
 * (other host threads, other scenes on other streams) race on it and must be
 * serialised by the caller. */
#define CCH_NOALLOC_MAX_PAIRS 131072
cch_status cch_query_pairs_noalloc(cch_scene* s, const double* x, const double* x_ref, double D,
                                   int32_t want_candidates, uint64_t* keys, double* dist, int64_t cap,
                                   int64_t* count);

/* ---- pre-passes that produce the target x~ of a step ----------------------
 * Both run on the scene's own topology (a single scene), take and write
 * DEVICE arrays of n_verts x 3 float64 and synchronise the scene's stream.
 * They use the scene's working arrays, so they must not run while a step of
 * the same scene runs (calls on one scene are serialised by its stream and
 * by the one-thread-at-a-time rule above).
 *
 * Target of the globally injective normal flow (Sec. 7.4, Eq. normal flow):
 * y = x + (sign beta) n(x), n the area-weighted vertex normals (the
 * normalised sum of (b - a) x (c - a) over the incident triangles), followed
 * by iters (0..64) Jacobi steps y <- y + alpha Lap(y) of the cotangent
 * Laplacian with the mixed Voronoi areas of Meyer et al. (2003), the operator
 * taken on the current y.  x and y must not alias. */
cch_status cch_normal_flow_target(cch_scene* s, const double* x, double beta, double alpha, double sign,
                                  int32_t iters, double* y);

/* Friction by velocity filtering (Sec. 6.3) on the frictionless target y.
 * Every pair of a collision vertex p and a triangle t not containing it,
 * closer than reach at x (closest point by the triangle's Voronoi regions)
 * and with a vertex of positive inverse mass, is a contact with normal n
 * from the closest point to p.  With u the relative target displacement of
 * p against the closest point and pen = sep - (d + n.u): if pen > 0, the
 * relative correction pen n - min(mu pen, |u_t|) u_t/|u_t| is shared by
 * inverse mass (p: m_p^-1 / W, corner i: -w_i m_i^-1 / W, W = m_p^-1 +
 * sum w_i^2 m_i^-1) and each vertex moves by the mean of its corrections.
 * y_out receives the filtered target (it may alias y).  mu >= 0, reach > 0,
 * sep >= 0. */
cch_status cch_friction_filter(cch_scene* s, const double* x, const double* y, double* y_out, double mu,
                               double reach, double sep);

/* ---- profiling -----------------------------------------------------------
 * With profiling on, steps launch kernels directly (no CUDA graphs) and
 * record CUDA events on the scene's stream around each kernel group:
 * 0 BVH refit, 1 vertex-triangle query, 2 edge-edge query, 3 vertex-vertex
 * query, 4 distance refresh, 5 contact assembly, 6 sweep order (per-vertex
 * ranks), 7 backward sweeps (Gauss-Seidel or Jacobi), 8 forward step, 9 loop
 * control, 10 step set-up (inputs, BVH build), 11 output, 12 exact FP64 stage
 * of the search, 13 colouring of the contacts (Gauss-Seidel).
 * cch_set_profiling resets the accumulators;
 * cch_get_profile returns, per group, the summed milliseconds and the number
 * of timed launches (n entries). */
cch_status cch_set_profiling(cch_scene* s, int32_t on);
cch_status cch_get_profile(cch_scene* s, double* ms, int64_t* count, int32_t n);

/* ---- serving --------------------------------------------------------------
 * A server keeps scenes resident in HBM (topology, BVH, last state) and runs
 * a request loop on its own host thread: requests that arrive while others
 * are on the GPU join the running batch at the next launch boundary (when
 * memory and slots allow) and leave it when their own loop ends. */
cch_status cch_server_create(size_t hbm_budget_bytes, const cch_params* prm, int32_t max_active, void* cuda_stream,
                             cch_server** out);
/* Make a scene resident; CCH_E_BUDGET when it would exceed the budget. */
cch_status cch_server_add_scene(cch_server* sv, const cch_topology* topo, int32_t* scene_id);
/* The same, with the scene's own physical parameters (the fields that
 * cch_create_batch_params takes per scene; the rest from the server's).
 * scene_prm is copied; an invalid one returns CCH_E_INVALID_ARG. */
cch_status cch_server_add_scene_params(cch_server* sv, const cch_topology* topo, const cch_params* scene_prm,
                                       int32_t* scene_id);
/* Queue one step of a resident scene; pointers are device pointers that must
 * stay valid until the request completes. */
cch_status cch_server_submit(cch_server* sv, int32_t scene_id, const double* x_t, const double* x_tilde,
                             double* x_next, uint64_t* ticket);
/* Block until the request completes; latency_ms = submit to completion. */
cch_status cch_server_wait(cch_server* sv, uint64_t ticket, cch_step_stats* stats, double* latency_ms);
cch_status cch_server_destroy(cch_server* sv);

#ifdef __cplusplus
}
#endif
#endif

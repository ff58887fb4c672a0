/*
 * silg.h - C ABI of the sparse-inverse local-global simulator (B300, sm_103a).
 *
 * Implements the per-iteration local-global solve of Zeng et al., "Fast But Accurate: A
 * Real-Time Hyperelastic Simulator with Robust Frictional Contact":
 *   - implicit Euler as minimisation (Sec. 3.1, Eq. 1), solved by local-global
 *     iterations (Sec. 3.3, Eqs. 5-6, Alg. 1);
 *   - the global step applied as products with the sparse inverse S of the Cholesky
 *     factor, A^-1 = S^T S (Sec. 4.2, Theorem 1, Eqs. 7-8, Alg. 2);
 *   - frictional contact by a Fischer-Burmeister non-smooth Newton step inside every
 *     iteration (Sec. 5.2, Eqs. 14-23; App. B.2), with split non-smooth indicators and the
 *     Delassus operator W = H S^T S H^T formed once per frame (Sec. 5.3, Eqs. 24-27) and
 *     its diagonal as complementarity preconditioner (Sec. 5.4, Eq. 28), in the order of
 *     Alg. 4 (Sec. 6).
 *
 * Conventions
 *   - Every function returns an int status: SIM_OK (0) or a negative SIM_E* code; no
 *     exception crosses the ABI. sim_strerror() names a code.
 *   - Host inputs are FP64 / int32, always copied; the library never keeps a caller
 *     pointer. Output buffers are caller-owned host memory unless a parameter says
 *     "device".
 *   - Vertex arrays are n_verts x 3, row-major (x, y, z per vertex), in the caller's
 *     vertex numbering.
 *   - A handle owns all its device memory and one CUDA stream (or uses the caller's
 *     stream, see sim_options.cuda_stream). A handle is not thread-safe.
 *   - GPU work is asynchronous: sim_step() only enqueues; errors raised on the device
 *     (capacity overflow, non-finite state, bounded-wait timeout) are reported by the next
 *     call that synchronises (sim_synchronize, sim_get_state, sim_get_stats, ...).
 */
#ifndef SILG_H
#define SILG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define SIM_OK          0
#define SIM_EINVAL     (-1)  /* invalid argument (bad index, size, material, geometry)   */
#define SIM_ENOMEM     (-2)  /* host or device allocation failed                        */
#define SIM_ENOTSPD    (-3)  /* the system matrix A is not positive definite             */
#define SIM_ECUDA      (-4)  /* a CUDA runtime call failed (no device, launch error)     */
#define SIM_ECAPACITY  (-5)  /* more contacts in a frame than sim_options.contact_capacity */
#define SIM_ETIMEOUT   (-6)  /* a bounded device-side wait gave up                       */
#define SIM_ENONFINITE (-7)  /* a NaN or Inf appeared in the state                       */
#define SIM_ENOTSUP    (-8)  /* option combination not supported                        */

/* ---- enumerations ------------------------------------------------------------------ */
enum { SIM_MODEL_ARAP = 0,      /* PD as-rigid-as-possible: SO(3) indicator (Eq. 5)      */
       SIM_MODEL_COROT = 1,     /* co-rotational: mu||F-R||^2 + lam/2 tr^2(R^T F - I)     */
       SIM_MODEL_SNH = 2 };     /* stable Neo-Hookean (Smith, de Goes, Kim 2018)           */
enum { SIM_OBST_PLANE = 0,      /* p: point on plane, axis: unit outward normal           */
       SIM_OBST_CYLINDER = 1 }; /* infinite cylinder: p on axis, axis unit, radius        */
enum { SIM_S_FP32 = 0,          /* S stored in FP32                                       */
       SIM_S_BF16 = 1 };        /* S stored in BF16, FP32 accumulation                     */
enum { SIM_NCP_FB = 0,          /* Fischer-Burmeister complementarity functions (App. B.2) */
       SIM_NCP_MINMAP = 1 };    /* minimum-map functions (App. B.1)                       */
enum { SIM_LOCAL_PD = 0,        /* the local step of Eq. 5 (projective dynamics)          */
       SIM_LOCAL_ADMM = 1 };    /* ADMM-PD: scaled dual variables per element, zero at each
                                   frame start; the local step projects G q + u, the global
                                   step reads z - u; ARAP elements use mu |F - R|^2        */
enum { SIM_GLOBAL_SPARSE_INVERSE = 0, /* the global step x = S^T S b (Eq. 8)            */
       SIM_GLOBAL_JACOBI = 1 }; /* jacobi_sweeps Jacobi sweeps on A x = b from the current
                                   iterate: the incomplete solve the paper compares against
                                   (Sec. 8); scenes without obstacles or anchors only    */
enum { SIM_PRECOND_DELASSUS = 0,/* r_n = h^2 W_jj, r_f = h W_jj from the Delassus operator
                                   (Eq. 28)                                               */
       SIM_PRECOND_MASS = 1 };  /* r_n = h^2 [H M^-1 H^T]_jj, r_f = h [H M^-1 H^T]_jj: the
                                   mass-inverse alternative of Sec. 5.4 (h^2/m_v, h/m_v)   */

/* ---- inputs ------------------------------------------------------------------------- */
typedef struct {
  int32_t n_verts;
  int32_t n_tets;
  const double* rest_pos;      /* n_verts x 3, rest positions X                           */
  const int32_t* tets;         /* n_tets x 4 vertex ids, positively oriented at rest      */
  const int32_t* tet_material; /* n_tets material indices, or NULL for material 0         */
  const int32_t* pinned;       /* n_pinned vertex ids (Dirichlet), or NULL                */
  int32_t n_pinned;
  double handle_vel[3];        /* velocity of every pinned vertex (m/s)                   */
  /* Triangle (membrane) elements of a sheet: F = [x1 - x0, x2 - x0] D_m^-1 (3 x 2) with D_m
   * the rest edges in the triangle's plane, volume = area x thickness, weight 2 mu V; ARAP
   * (closest orthonormal columns) or co-rotational (SIM_MODEL_SNH: SIM_EINVAL), the plain
   * local step only (SIM_LOCAL_ADMM with triangles: SIM_EINVAL). n_tets may be 0 when
   * n_tris > 0. Bending: k_b/2 sum over interior vertices of |L x|^2 / A (L the rest
   * cotangent Laplacian, A the mixed Voronoi area), a constant term of the system matrix;
   * the rest sheet is taken as flat (zero rest curvature). */
  const int32_t* tris;         /* n_tris x 3 vertex ids, or NULL                           */
  const int32_t* tri_material; /* n_tris material indices, or NULL for material 0         */
  int32_t n_tris;
  double thickness;            /* of the sheet (m); > 0 when n_tris > 0                    */
  double bending;              /* k_b (N m) >= 0                                          */
} sim_mesh;

typedef struct {
  int32_t model;               /* SIM_MODEL_*                                              */
  double E, nu, rho;           /* Young's modulus (Pa), Poisson ratio, density (kg/m^3)   */
} sim_material;

typedef struct {
  int32_t kind;                /* SIM_OBST_*                                               */
  double p[3];
  double axis[3];
  double radius;
  double mu;                   /* Coulomb friction coefficient                             */
  double vel[3];               /* surface velocity of the obstacle (0 for fixed)          */
} sim_obstacle;

typedef struct {
  int32_t n_iters;             /* local-global iterations per frame (default 5)           */
  int32_t n_cr_iters;          /* conjugate-residual iterations per solve (default 10)    */
  int32_t s_precision;         /* SIM_S_FP32 (default) or SIM_S_BF16                      */
  int32_t refine;              /* BF16 only: residual correction x += S~^T S~ (b - A~ x),
                                  the residual summed in FP64 from the FP32 iterate, after
                                  the global step of the last iteration of
                                  each frame (1, default), of every iteration (2), or never
                                  (0). Each correction costs one A~ product and two more
                                  profile products. Other values: SIM_EINVAL.            */
  int32_t contact_capacity;    /* max contacts per frame (default 4096)                   */
  int32_t device;              /* CUDA device ordinal (default 0)                          */
  double gravity[3];           /* default (0, 0, -9.81)                                    */
  double contact_margin;       /* contact when gap < margin; <= 0: half the mean edge     */
  uint64_t spin_limit;         /* polls of a device-side wait (the CR kernel's bulk copy of
                                  its Delassus rows into shared memory) before it gives up,
                                  falls back to global memory and reports SIM_ETIMEOUT at
                                  the next synchronisation (0: 2^22)                      */
  void* cuda_stream;           /* cudaStream_t to run on, or NULL for a private stream    */
  int32_t n_host_threads;      /* threads for the host precompute (0: all cores)          */
  int32_t autotune;            /* 1: time the profile products' launch configurations at
                                  creation and keep the fastest (sim_get_tuning); 0
                                  (default): the fixed configuration; 2: the fixed grid
                                  with the products in their bulk-copy form (S~ rows moved
                                  into shared memory by cp.async.bulk)                   */
  int32_t ncp;                 /* SIM_NCP_FB (default) or SIM_NCP_MINMAP: the functions
                                  that drive the iteration. The residual (sim_stats) is one
                                  measure for every choice: min(delta_n, r_n lambda_n) and
                                  h phi_f with the FB E_f, r from the Delassus diagonal. */
  int32_t precond;             /* SIM_PRECOND_DELASSUS (default) or SIM_PRECOND_MASS      */
  double residual_tol;         /* > 0: sim_step with n_iters <= 0 iterates until the
                                  residual R_k (sim_stats) is <= residual_tol, at least one
                                  update and at most max_iters, decided on the device (a
                                  CUDA graph while-node); 0 (default): n_iters <= 0 means
                                  the option's n_iters. Negative or NaN: SIM_EINVAL.     */
  int32_t max_iters;           /* cap of those iterations, 1..63 (default 40)             */
  int32_t local_solver;        /* SIM_LOCAL_PD (default) or SIM_LOCAL_ADMM                */
  int32_t global_solver;       /* SIM_GLOBAL_SPARSE_INVERSE (default) or SIM_GLOBAL_JACOBI  */
  int32_t jacobi_sweeps;       /* sweeps per global step with SIM_GLOBAL_JACOBI, 1..1000
                                  (default 1: the single sweep of Sec. 8's baseline)     */
  int32_t phase_marks;         /* 1 (default): event nodes around every phase of every
                                  iteration (sim_get_phase_times itemises them); 0: only
                                  around the frame's once-per-frame phases, the iterations
                                  reported as SIM_PHASE_ITERATIONS (each event node costs a
                                  few microseconds: 6% of a star frame, 13% of a 6^3 cube's) */
  /* Device memory of the simulator's buffers (all of them; not the page-locked host
   * staging, not a network's or the allocation-free solve's): dev_alloc(bytes, alloc_ctx)
   * must return memory on opts->device aligned to 256 bytes, or NULL (sim_create then
   * returns SIM_ENOMEM); dev_free(ptr, alloc_ctx) releases it, in sim_destroy or when
   * creation fails. Both NULL (default): cudaMalloc / cudaFree. Only one of them set:
   * SIM_EINVAL. The calls happen inside sim_create / sim_create_batch and sim_destroy. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  int32_t cr_exchanges;        /* cluster exchanges per conjugate-residual iteration: 2
                                  (default) one for the product's input and one for the dot
                                  products, the iteration as written; 1 one exchange (the
                                  vertex images of r and Ap advanced by the iteration's own
                                  recurrences) for scenes without contacts between bodies
                                  (with them: 2). Equal in exact arithmetic; in FP32 the
                                  one-exchange form can end an order of magnitude further
                                  from the FP64 iteration on ill-conditioned systems, and
                                  its vertex vectors (64 bytes per contact vertex of a scene
                                  in shared memory) must fit, else SIM_ECAPACITY. Other
                                  values: SIM_EINVAL.                                    */
  int32_t cr_sync;             /* how the CTAs of a constraint-solve cluster exchange their
                                  data in the two-exchange form: 0 (default) point to point,
                                  stores into the other CTAs' shared memory that count their
                                  bytes on the receiver's barrier (st.async, mbarrier), each
                                  CTA waiting only for its own data; 1 a cluster-wide barrier
                                  after each exchange. Same results bit for bit. Scenes with
                                  contacts between bodies always use 1. Other values:
                                  SIM_EINVAL.                                            */
  int32_t s_build;             /* where a simulator builds S~ = L~^-1 P from the host's
                                  FP64 Cholesky factor: 1 (default) on the device in FP64
                                  (one warp per column along its elimination-tree path; the
                                  same FP64 values as the host loop), 0 on the host (all
                                  cores). Meshes whose elimination tree is too deep for the
                                  device kernel's shared memory are built on the host. The
                                  host-only plan (sim_plan_create) always builds on the
                                  host. Other values: SIM_EINVAL.                        */
  int32_t delassus_reuse;      /* 1 (default): a frame whose contact vertices are the
                                  previous frame's (the same sorted list) keeps Y and W~ =
                                  Y^T Y instead of building them again: both depend on that
                                  list only (S is constant; the Delassus reuse across steps
                                  that Sec. 5.3 and Sec. 6 point to). The result is
                                  bit-identical. sim_set_state, sim_set_checkpoint and a new
                                  start mode or portfolio forget the list. 0: always build. */
} sim_options;

/* Launch configuration of the two profile products (z = S g, x = S^T y), chosen by the
 * autotuner or fixed. */
typedef struct {
  int32_t tuned;               /* 1 if the autotuner ran                                   */
  int32_t candidates;          /* configurations timed per product                        */
  int32_t pass1_ctas, pass2_ctas;       /* CTAs of each product's launch                  */
  int32_t pass1_unroll, pass2_unroll;   /* tiles in flight per warp: 1 the format's default,
                                           0 half, 2 twice (one resident CTA per SM); 3:
                                           bulk copies into a ring of shared-memory stages
                                           (a producer warp, eight consumer warps)       */
  double pass1_balance, pass2_balance;  /* cost of an empty tile position relative to a
                                           stored value when the tiles are split over CTAs */
  double pass1_us, pass2_us;            /* median launch time of the choice (tuned only)   */
  double pass1_default_us, pass2_default_us; /* ... of the fixed configuration           */
} sim_tuning;

/* Per-frame statistics of the most recent sim_step. */
#define SIM_MAX_RESIDUALS 64
typedef struct {
  int64_t frame;               /* frames advanced since creation or sim_set_state        */
  int32_t n_contacts;          /* contacts detected in the last frame                    */
  int32_t n_contact_verts;     /* distinct contact vertices (order of W~)                */
  int32_t n_iters;             /* iterations run in the last frame                       */
  int32_t n_residuals;         /* n_iters + 1 residuals follow                           */
  double residual[SIM_MAX_RESIDUALS]; /* R_k = max_j max(|min(dn, r_n ln)|, h|phi_f|)/L */
  double max_penetration;      /* max over contacts of -delta_n at the end of the frame  */
  int32_t kernels_per_frame;   /* kernel launches in one frame of the last n_iters        */
  int32_t delassus_reused;     /* 1 if the last frame kept the previous frame's Y and W~  */
  int64_t delassus_reuse_frames; /* frames that did so since creation                    */
} sim_stats;

/* Phases of a frame timed by event nodes inside the frame's CUDA graph (milliseconds,
 * summed over the iterations of the most recent frame); the paper reports the same split
 * (Tab. 3: Schur., Local, Global, Assem., Cst. Solve, Corr.). */
enum { SIM_PHASE_COLLIDE = 0,   /* prediction and collision detection (App. A.1)         */
       SIM_PHASE_DELASSUS = 1,  /* W~ = Y^T Y and preconditioner (Eqs. 27-28)            */
       SIM_PHASE_LOCAL = 2,     /* local step per tetrahedron (Eq. 5), beside the FB
                                   evaluation of the contacts (two graph branches; with a
                                   cold start the first local step runs beside collision
                                   and Delassus work)                                     */
       SIM_PHASE_ASSEMBLE = 3,  /* right-hand side (Eq. 19)                                */
       SIM_PHASE_SPMV1 = 4,     /* z = S g (first profile product, Eq. 8): the product     */
       SIM_PHASE_SOLVE = 5,     /* J A^-1 g, conjugate residual, S J^T dlambda (Alg. 4)   */
       SIM_PHASE_SPMV2 = 6,     /* q = S^T y (second profile product): the product         */
       SIM_PHASE_INTEGRATE = 7, /* final residual and integration                         */
       SIM_PHASE_REDUCE = 8,    /* fixed-order sums of both products' partial sums (and a
                                   BF16 residual correction)                              */
       SIM_PHASE_WARMSTART = 9, /* warm-start features, guess and its acceptance          */
       SIM_PHASE_ITERATIONS = 10, /* a frame to a tolerance or without phase_marks: all its
                                  iterations (phases 2-6 and 8 are then 0; integration
                                  includes the final evaluation). 0 otherwise.           */
       SIM_NUM_PHASES = 11 };

/* Sizes of the precomputed structure (Theorem 1 profile of S). */
typedef struct {
  int32_t n_verts, n_free, n_tets;
  int64_t nnz_A;               /* non-zeros of the per-vertex matrix A~ (A = A~ (x) I3)   */
  int64_t nnz_L;               /* non-zeros of its Cholesky factor                       */
  int64_t nnz_S;               /* entries of S~ = L~^-1 in its row profile              */
  int64_t stored_S;            /* stored entries including alignment padding            */
  int32_t etree_max_depth;
  double etree_mean_depth;
  int32_t n_roots;
  double precompute_seconds;   /* host precompute, wall clock (with S~ when built there)  */
  double s_build_seconds;      /* the build of S~ = L~^-1 P alone: host loop, or device
                                  kernel (Sec. 4.2) with its uploads, wall clock         */
  int32_t s_built_on_device;   /* 1 if S~ was built on the device (sim_options.s_build)   */
} sim_plan_info;

typedef struct sim_s sim_t;
typedef struct sim_plan_s sim_plan_t;

const char* sim_strerror(int status);
void sim_default_options(sim_options* opts);

/*
 * Host-only precompute (no GPU needed). Builds per-element data, lumped masses, the
 * per-vertex system matrix A~ = M~ + h^2 sum_i w_i G~_i^T G~_i over the free vertices
 * (Eq. 6; A = A~ (x) I3 because G acts identically on x, y, z), a nested-dissection
 * ordering P, the elimination tree in postorder, the FP64 Cholesky factor
 * P A~ P^T = L~ L~^T and S~ = L~^-1 P stored as a row profile: row i covers exactly the
 * columns of its elimination subtree, the contiguous range [fd(i), i] (Theorem 1).
 * Errors: SIM_EINVAL (bad mesh), SIM_ENOTSPD, SIM_ENOMEM.
 */
int sim_plan_create(const sim_mesh* mesh, const sim_material* mats, int32_t n_mat, double h,
                    const sim_options* opts, sim_plan_t** out);
void sim_plan_destroy(sim_plan_t* plan);
int sim_plan_get_info(const sim_plan_t* plan, sim_plan_info* info);
/* order[k] = caller vertex id of internal free row k (n_free entries); parent[k] = etree
 * parent of row k (-1 for roots); first_desc[k] = fd(k). Any pointer may be NULL. */
int sim_plan_get_ordering(const sim_plan_t* plan, int32_t* order, int32_t* parent,
                          int32_t* first_desc);
/* x = A^-1 b on the host in FP64 through the two profile products x = S^T (S b) (Eq. 8).
 * b, x: n_verts x 3 in caller numbering; pinned rows of b are ignored, of x set to 0. */
int sim_plan_apply_inverse_host(const sim_plan_t* plan, const double* b, double* x);

/*
 * Create a simulator on one GPU for the implicit-Euler problem of Sec. 3.1 (Eq. 1: the
 * mesh, its materials, the obstacles and the step h): runs the host precompute (the
 * system matrix of Eq. 6, its Cholesky factor and S = L^-1 P, Sec. 4.2 and Theorem 1: the
 * one-time first line of Alg. 4), uploads everything, and prepares the per-frame CUDA graph.
 * opts may be NULL (defaults). Positions start at the rest shape with zero velocity
 * (sim_set_state to change). All inputs are copied. Errors: SIM_EINVAL, SIM_ENOTSPD,
 * SIM_ENOMEM, SIM_ECUDA.
 */
int sim_create(const sim_mesh* mesh, const sim_material* mats, int32_t n_mat,
               const sim_obstacle* obstacles, int32_t n_obs, double h,
               const sim_options* opts, sim_t** out);

/* An anchor: a bilateral constraint (the b rows of J with compliance E_b, App. A.1 and
 * App. B) tying a free vertex to a moving target by the three rows e_x, e_y, e_z of
 *   phi_b = q_v - p(t) + compliance * lambda_b = 0,
 * always active. p(t) = target + vel * t is the target at the end of the frame, t counted
 * from the simulator's creation or the last sim_set_state. Rows enter the constraint solve
 * like normal rows (compliance / h^2 in the Schur system); they count in the residual with
 * max |phi_b| / L, appear among the contacts (sim_get_contacts) with obstacle id = the
 * simulator's obstacle count + the anchor's index over all scenes, and in n_contacts.
 * vertex: a free (not pinned) vertex of its scene, at most one anchor per vertex;
 * compliance >= 0 (m/N; 0: a hard constraint).
 * paired = 1 ties the vertex to another vertex instead (App. A.1's two-vertex bilateral
 * rows, e.g. a cable): the rows of
 *   phi_b = (q_v - q_partner) - p(t) + compliance * lambda_b = 0,
 * p(t) the target offset; the impulse acts on the vertex and, opposite, on the partner (a
 * free vertex of the same scene other than the vertex; it may be the partner of several
 * anchors). paired = 0 (zero-initialised): the target form above, partner ignored.
 * Anything else: SIM_EINVAL at creation. */
typedef struct {
  int32_t vertex;
  double target[3];
  double vel[3];
  double compliance;
  int32_t paired;
  int32_t partner;
} sim_anchor;

/* One independent scene of a batch: its mesh, its materials (tet_material indexes this
 * list), its obstacles (they act on this scene's vertices only), its contact margin
 * (<= 0: half the scene's mean edge; opts->contact_margin is not used by a batch) and its
 * anchors (may be NULL with n_anchors = 0).
 *
 * body_contact = 1: contact between the scene's bodies, the connected components of its
 * tetrahedra (App. A.1's contact map with both sides moving). The surface triangles are
 * the element faces that belong to one tetrahedron, oriented outward (at rest) and
 * numbered in the order of their sorted vertex triples. Each frame, every free vertex of a
 * surface triangle is matched with the nearest surface triangle of another body whose
 * corners are all free (closest point p, Euclidean distance; the lower number on a tie),
 * at the predicted positions. The gap g is signed by the triangle's plane where p is
 * inside the triangle; at an edge or a corner the vertex counts as outside (g = |x - p|).
 * It is a contact when -2 margin < g < margin, with normal n = (x - p) / g (the triangle's
 * normal when x = p), rows (n, f1, f2), the map x_v - sum_k w_k x_k (w: p's barycentric
 * weights; a corner with w_k = 0 drops out), d = 0 and friction coefficient body_mu. One
 * such contact per vertex at most, after its obstacles and anchor; sim_get_contacts lists
 * it with obstacle id = n_obstacles + n_anchors (of the whole simulator) + the triangle's
 * number (numbers run over the scenes with body contact, scene by scene). Triangle corners
 * become contact vertices: W~ covers them (Eq. 27 with the map's weights). Not with
 * SIM_GLOBAL_JACOBI. body_contact = 0: none (body_mu unused). */
typedef struct {
  sim_mesh mesh;
  const sim_material* materials;
  int32_t n_materials;
  const sim_obstacle* obstacles;
  int32_t n_obstacles;
  double contact_margin;
  const sim_anchor* anchors;
  int32_t n_anchors;
  int32_t body_contact;
  double body_mu;
} sim_scene;

/*
 * Many independent scenes of uneven size in one simulator: every kernel of a frame runs
 * once over all scenes (no per-scene launches). Vertices (and tets) are numbered scene
 * after scene: scene s's vertex v is vertex sum_{s'<s} n_verts(s') + v of every state,
 * contact and Delassus accessor. The system matrix is block diagonal (one elimination
 * forest, ordered scene by scene), the Delassus operator is stored as one block per scene
 * and each scene's constraint solve runs in its own thread-block cluster with its own
 * scalars, so a scene's frame is the frame it would have alone (up to the rounding of its
 * reordered sums). Errors as sim_create; n_scenes < 1 or a NULL list: SIM_EINVAL.
 */
int sim_create_batch(const sim_scene* scenes, int32_t n_scenes, double h,
                     const sim_options* opts, sim_t** out);
/* Per-scene residuals of the last frame: out[s * (n_iters + 1) + k] for scene s, iteration
 * k (the same measure as sim_stats.residual, over the scene's contacts; 0 without contacts).
 * capacity: doubles available in out. */
int sim_get_scene_residuals(sim_t* sim, int32_t capacity, double* out);
/* The products' launch configuration (tuned or fixed). */
int sim_get_tuning(const sim_t* sim, sim_tuning* out);
/* Release a simulator (waits for its stream; frees every device buffer through the
 * allocator it was created with). NULL is ignored. The paper's method keeps no state beyond
 * the precompute and the frame state (Alg. 4), all of it owned by the handle. */
void sim_destroy(sim_t* sim);

/* One frame of Alg. 4 (Sec. 6): prediction s~ (Eq. 1), collision and linearisation
 * (App. A.1), Delassus operator and preconditioner (Eqs. 27-28), then local steps (Eq. 5),
 * Fischer-Burmeister evaluation (App. B.2), constrained global steps through S (Eqs. 19-23,
 * Eq. 8) and integration, with n_iters local-global iterations (n_iters <= 0: the option's
 * n_iters, or, if sim_options.residual_tol > 0, iterations until R_k <= residual_tol: at
 * least 1 and at most max_iters, the stopping decision taken on the device; sim_stats
 * reports the count). Asynchronous on the handle's stream. */
int sim_step(sim_t* sim, int32_t n_iters);
/* Wait for the handle's stream; returns the first device-side error, if any. */
int sim_synchronize(sim_t* sim);

/* Copy the state out (synchronises): the positions q_{t+h} and velocities
 * v_{t+h} = (q_{t+h} - q_t) / h of the last frame (the integration line of Alg. 4), its
 * contact impulses lambda (Eq. 23a; per contact the n, f1, f2 components in N, in the order
 * sim_get_contacts lists them, `capacity` rows; the count goes to *n_contacts, and may exceed
 * capacity) and its statistics (as sim_get_stats). q, v: n_verts x 3. Every output pointer
 * may be NULL; lambda needs capacity > 0. */
int sim_get_state(sim_t* sim, double* q, double* v, int32_t capacity, double* lambda,
                  int32_t* n_contacts, sim_stats* stats);
/* Replace the state (positions, velocities; pinned vertices included) from which the next
 * frame starts (q_t, v_t of Alg. 4). Resets the frame counter and the anchors' time, and
 * forgets the previous frame's contacts: the next frame starts like a first frame in every
 * warm-start mode. To resume exactly, contacts included, use sim_set_checkpoint. */
int sim_set_state(sim_t* sim, const double* q, const double* v);
/* Checkpoint and restore of everything a later frame depends on: q_t, v_t, the frame
 * counter, the anchors' current targets and the previous frame's contact record that the
 * warm starts read (per vertex: contact, obstacle, world impulse D^T lambda, normal move). A
 * restored simulator continues bit for bit as the saved one would in every start mode (cold,
 * learned, previous-frame, portfolio). The paper has no counterpart (its method holds no
 * state across frames but q and v).
 * sim_get_checkpoint: *bytes receives the size (buf may be NULL to ask for it only); with
 * buf, capacity >= that size (else SIM_ECAPACITY). Synchronises.
 * sim_set_checkpoint: bytes must be that size and the checkpoint must come from a simulator
 * with the same scenes (a signature of every input is checked), else SIM_EINVAL. */
int sim_get_checkpoint(sim_t* sim, void* buf, size_t capacity, size_t* bytes);
int sim_set_checkpoint(sim_t* sim, const void* buf, size_t bytes);
int sim_get_stats(sim_t* sim, sim_stats* stats);
/* Contacts of the last frame, ordered by (caller vertex id, obstacle index): vertex,
 * obstacle, lambda (n, f1, f2 components, N), frame rows (n, f1, f2: 9 doubles). Arrays of
 * `capacity` entries; *n_out receives the count (which may exceed capacity). */
int sim_get_contacts(sim_t* sim, int32_t capacity, int32_t* vertex, int32_t* obstacle,
                     double* lambda, double* frame, int32_t* n_out);

/* Sizes of the simulator's precomputed structure (same fields as sim_plan_get_info). */
int sim_get_plan_info(const sim_t* sim, sim_plan_info* info);
/* The simulator's internal row order (Sec. 4.2: the nested-dissection order in postorder of
 * its elimination forest, Theorem 1), as sim_plan_get_ordering gives it for a plan, for one
 * scene or a whole batch (vertex ids in the batch numbering of sim_create_batch; a batch's
 * rows run scene by scene). n_free entries each (sim_get_plan_info); NULL skips an array. */
int sim_get_ordering(const sim_t* sim, int32_t* order, int32_t* parent, int32_t* first_desc);

/* Per-phase device time of the most recent frame (synchronises). ms: SIM_NUM_PHASES. */
int sim_get_phase_times(sim_t* sim, double* ms);

/* ---- component entry points (parity and profiling) ------------------------------- */
/* x = A^-1 b with the device profile products (Eq. 8). b, x as in the host variant. With
 * a BF16 profile and refine > 0, one residual correction follows (see sim_options).
 * SIM_ETIMEOUT if a wait of the products' bulk-copy form ran out (x is then not written). */
int sim_apply_inverse(sim_t* sim, const double* b, double* x);
/* Local step (Eq. 5) on the device for positions q (n_verts x 3): p (n_tets x 9,
 * row-major F-shaped projections, caller tet order). */
int sim_local_project(sim_t* sim, const double* q, double* p);
/* Delassus operator of the last frame over distinct contact vertices: W~ (n_cv x n_cv,
 * row-major) with W_jk = W~(v_j, v_k) D_j D_k^T (Eq. 27); cv_vertex receives the caller
 * vertex ids. Arrays hold `capacity` vertices; *n_out receives n_cv. */
int sim_get_delassus(sim_t* sim, int32_t capacity, double* Wtilde, int32_t* cv_vertex,
                     int32_t* n_out);

/* ---- learned warm start (not from the paper) ----------------------------------------
 * A small network predicts, per contact, the initial impulse lambda^0 and a normal
 * displacement guess from SIM_MLP_FEATURES features. The paper starts every frame from
 * lambda = 0; the network is an addition, trained on frames the plain method solved, with
 * the cold start kept as the fallback. Layout of the flat FP32 parameter vector
 * (SIM_MLP_PARAMS values): W1 (16 x 128, row = input; rows 11..15 multiply zero padding),
 * b1 (128), W2 (128 x 128), b2, W3 (128 x 128), b3, W4 (128 x 8, columns 4..7 unused), b4 (8);
 * hidden units use GELU(x) = x Phi(x). The device computes with BF16 weights and
 * activations and FP32 accumulation (tensor cores). */
#define SIM_MLP_FEATURES 11
#define SIM_MLP_OUTPUTS 4
#define SIM_MLP_PARAMS 36232
typedef struct sim_mlp_s sim_mlp_t;
/* A network on `device` with zero parameters; max_batch bounds the rows of one gradient. */
int sim_mlp_create(int32_t device, int32_t max_batch, sim_mlp_t** out);
void sim_mlp_destroy(sim_mlp_t* net);
/* Which tensor-core instructions run the network's inference (sim_mlp_forward, and a
 * simulator's learned start, which takes the choice with the network in sim_set_warmstart):
 * SIM_MLP_MMA_SYNC (default) warp-level mma.sync, each warp carrying 16 rows; SIM_MLP_TCGEN05
 * the 5th-generation tensor cores, one CTA of 128 rows per tcgen05.mma chain with its FP32
 * accumulators in tensor memory. Both take BF16 weights and activations with FP32
 * accumulation. Training always uses mma.sync. Other values: SIM_EINVAL. */
enum { SIM_MLP_MMA_SYNC = 0, SIM_MLP_TCGEN05 = 1 };
int sim_mlp_set_tensor_cores(sim_mlp_t* net, int32_t kind);
/* Weights uniform in +-sqrt(6 / (fan_in + fan_out)) from a splitmix64 stream, biases 0. */
int sim_mlp_init(sim_mlp_t* net, uint64_t seed);
int sim_mlp_set_params(sim_mlp_t* net, const float* theta);   /* also resets Adam's moments */
int sim_mlp_get_params(const sim_mlp_t* net, float* theta);
/* Y (rows x SIM_MLP_OUTPUTS) = net(X (rows x SIM_MLP_FEATURES)); host arrays. */
int sim_mlp_forward(sim_mlp_t* net, const float* X, int32_t rows, float* Y);
/* Gradient (SIM_MLP_PARAMS) and value of L = 1/(2 rows) sum (Y - T)^2 over the outputs;
 * rows <= max_batch (else SIM_ECAPACITY). grad or loss may be NULL. */
int sim_mlp_gradient(sim_mlp_t* net, const float* X, const float* T, int32_t rows, float* grad,
                     float* loss);
/* Adam (beta 0.9 / 0.999, eps 1e-8) on minibatches of `batch` rows of a fresh seeded
 * permutation each epoch; epoch_loss (epochs values, or NULL) receives the mean batch loss. */
int sim_mlp_train(sim_mlp_t* net, const float* X, const float* T, int32_t rows, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, float* epoch_loss);
/* Start of each frame: mode 0 cold (lambda = 0, q = s~; the paper's start, the default),
 * 1 the network's guess (net's current parameters are copied; same device), 2 the previous
 * frame's impulse and move at the same vertex and obstacle. A guess is kept for a scene only
 * if the residual of its impulses at k = 0 (at the position they predict) is below the cold
 * start's. */
int sim_set_warmstart(sim_t* sim, const sim_mlp_t* net, int32_t mode);
/* Gains of the network's outputs in the learned start (not from the paper): lambda^0 =
 * (previous impulse + g x predicted change) x scale with g = persist for a contact that had
 * an impulse at the same vertex and obstacle in the previous frame and g = fresh for a new
 * one; the predicted change of the normal move from the previous frame's is scaled by move.
 * 0 leaves that part at the previous frame's value, so 0, 0, 0 is the previous-frame start
 * (mode 2; the network is then not run); 1, 1, 1 (the default) is the network as trained.
 * accept in (0, 1]: the learned guess is kept when its residual at k = 0 is below accept
 * times the cold start's (1, the default: any improvement). Chosen, for example, on
 * validation frames by time to a residual tolerance. Gains non-negative and finite, accept
 * in (0, 1], else SIM_EINVAL. Synchronises the handle's stream. */
int sim_set_warmstart_gains(sim_t* sim, float persist, float fresh, float move, float accept);
/* Load a trained warm-start network and switch the learned start on (mode 1 of
 * sim_set_warmstart): weights is the flat FP32 parameter vector in the layout above
 * (SIM_MLP_PARAMS values, as sim_mlp_get_params writes it), bytes = 4 * SIM_MLP_PARAMS.
 * The simulator keeps its own copy. Errors: SIM_EINVAL (size, non-finite value). */
int sim_load_warmstart(sim_t* sim, const void* weights, size_t bytes);
/* Portfolio start (not from the paper): the simulator's scenes (sim_create_batch) are groups
 * of `copies` identical copies of a scene, consecutive (scenes g * copies .. g * copies +
 * copies - 1 form group g). Copy 0 of each group always runs the cold start; the other
 * copies take the start set with sim_set_warmstart. After each frame every copy of a group
 * continues from the copy whose final residual is the lowest (ties: the lowest copy):
 * positions, velocities and the previous-frame contact data the features read. The copies
 * run side by side in the same launches, so a group costs about one scene's latency.
 * copies = 1 turns it off (the default). Synchronises the handle's stream; frame graphs are
 * rebuilt. Errors: SIM_EINVAL (copies < 1, a scene count that is not a multiple of copies,
 * copies that differ in any input: mesh, materials, pins, handle, obstacles, margin). */
int sim_set_portfolio(sim_t* sim, int32_t copies);
/* Switch sim_options.phase_marks for the next frames (0 or 1, else SIM_EINVAL); both frame
 * graphs stay cached. */
int sim_set_phase_marks(sim_t* sim, int32_t on);
/* Training samples of the last frame, one per contact (device order): X (n x
 * SIM_MLP_FEATURES) the features at the frame's start -- gap / margin, normal (3), relative
 * velocity h / margin (3), the previous frame's impulse at the same vertex and obstacle in
 * this frame's basis / scale (3, or 0), m_v W~_vv -- where scale = margin / (h^2 W~_vv); T
 * (n x 4) what the network should output: the frame's final impulse / scale minus features
 * 7..9, and the change of the vertex's move along the normal over the frame from the previous
 * frame's move at the same vertex and obstacle (0 if none) / margin. The learned start uses
 * lambda^0 = (features 7..9 + gain x output 0..2) scale and translates the scene by the mean
 * over its contact vertices of (previous move + gain x output 3 x margin) x normal (see
 * sim_set_warmstart_gains), kept within one margin of the
 * translation h^2 sum_j D_j^T lambda_j^0 / (the scene's free mass) that the impulses give
 * it. *n_out receives the count; arrays hold `capacity` rows. */
int sim_get_warmstart_samples(sim_t* sim, int32_t capacity, float* X, float* T, int32_t* n_out);

/*
 * x = A^-1 g through the two profile products, for callers that cannot allocate device
 * memory at the time of the call: real-time loops that forbid cudaMalloc (it may
 * synchronise the device and its latency is unbounded), code running while another
 * component captures the stream into a CUDA graph, or embedders whose device memory is
 * all handed out by their own pool. The paper has no counterpart; it is a packaging of
 * the global step (the same kernels as sim_apply_inverse). It always reads the FP32
 * profile, which the device holds in either s_precision mode, and applies no correction.
 *
 * g, x: device pointers to n_free x 3 FP32 row-major arrays in the solver's internal row
 * order (row k is caller vertex order[k] of sim_get_ordering; pinned vertices have no row).
 * stream: a cudaStream_t, or NULL for the legacy stream. The work runs on the simulator's
 * device; the calling thread's current device is the same after the call as before it.
 * The call only enqueues work and returns; it calls no allocator. Its scratch (at most
 * 16 MiB: the padded copy of g, z = S g and the partial sums of both products) is one
 * static device array that every GPU loading the library holds until the process exits;
 * meshes whose scratch would exceed it get SIM_ECAPACITY. The first call on a device
 * looks up that array's device address, so make the first call before any stream
 * capture. Every call shares the array and overwrites all of it that it reads; calls that
 * overlap on the GPU (for example on two streams, or from two handles on one device) race.
 * Errors: SIM_EINVAL (null argument), SIM_ECAPACITY, SIM_ECUDA (a failed launch of this
 * call, or a sticky device error). A launch error that an earlier call of this library left
 * pending on the thread is cleared at entry, not reported here.
 */
int sim_apply_inverse_noalloc(const sim_t* sim, const float* g, float* x, void* stream);

/*
 * A diagnostic of the frame's structure (not from the paper): the device time per phase
 * boundary of a chain of n_phases small phases on `device`, run (a) as one kernel per phase in
 * a CUDA graph with programmatic dependent launch (how the frame graph chains the steps of an
 * iteration) and (b) as one cooperative kernel whose phases are separated by a software grid
 * barrier (how a persistent kernel per iteration would separate them), each with
 * ctas_per_sm CTAs of 256 threads per SM; medians over 20 runs, microseconds per boundary.
 * The barrier's wait is bounded: SIM_ETIMEOUT if it gave up (the numbers are then not
 * meaningful). Allocates and frees its own small buffers. Errors: SIM_EINVAL (n_phases
 * outside 2..4096, ctas_per_sm outside 1..8, null outputs), SIM_ENOTSUP (no cooperative
 * launch, or that many CTAs cannot be resident), SIM_ECUDA.
 */
int sim_measure_phase_boundaries(int32_t device, int32_t n_phases, int32_t ctas_per_sm,
                                 double* graph_us, double* barrier_us);

#ifdef __cplusplus
}
#endif
#endif /* SILG_H */

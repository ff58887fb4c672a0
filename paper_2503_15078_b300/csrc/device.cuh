// Device data layout and kernel launchers of the sparse-inverse local-global solver
// (internal header, sm_103a).
//
// Numbering: internal vertex ids put the free vertices first, in the nested-dissection
// postorder of the elimination tree (rows of S~), then the pinned vertices. Per-vertex
// state is FP64 AoS (x, y, z); the vectors the profile products read and write are FP32
// SoA of length n_pad (zero padded).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "devguard.hpp"
#include "mlp.cuh"
#include "plan.hpp"

namespace silg {

// First instruction of a kernel that may be launched with programmatic dependent launch:
// blocks until the grids it depends on have completed and their writes are visible (a
// no-op for a kernel launched without it), then allows its own dependent grid to launch.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // and let the next grid be launched now: its blocks are scheduled as this grid's leave
  // and wait (above) until this grid has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Two FP32 values in one 64-bit register pair, for the packed FMA (lo in bits 0-31).
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) |
         ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2lo(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2hi(unsigned long long v) {
  return __uint_as_float((unsigned)(v >> 32));
}
// d = a * b + c, lane-wise on two FP32 values (each rounded as one fmaf)
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// kernel<<<grid, block, smem, s>>>(args...), with programmatic stream serialisation when
// pdl is set
template <class Kernel, class... Args>
inline cudaError_t launch_k(bool pdl, Kernel kernel, unsigned grid, unsigned block, size_t smem,
                            cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace silg

namespace silg {

constexpr int kWarps = 8;                     // warps per CTA of the profile products
constexpr int kRowsPerWarp = kRowGroup / kWarps;
constexpr int kMaxIters = SIM_MAX_RESIDUALS - 1;

// device error word bits
constexpr int kErrCapacity = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrYCapacity = 8;

// counters[]: per-frame sizes decided on the device
enum { kCntContacts = 0, kCntCv = 1, kCntU = 2, kCntY = 3, kCntYC = 4, kNumCounters = 8 };

struct ObstDev {
  int kind;
  int pad;
  double p[3], a[3], radius, mu, vel[3];
};

struct MatDev {
  int model;
  float mu, lam, alpha;
};

struct DevSim {
  // sizes
  int n, n_all, n_tets, n_pad, n_obs, n_mat;
  int cap, cap_y, n_cr;
  int ncp, precond;  // SIM_NCP_*, SIM_PRECOND_*
  // ADMM-PD (SIM_LOCAL_ADMM): scaled duals per element, 9 FP32 values stored k * n_tets + t,
  // zeroed at every frame start (null with the plain local step)
  int admm;
  float* tet_u;
  // SIM_GLOBAL_JACOBI: sweeps per global step (0: the sparse-inverse solve) and the second
  // buffer of the sweeps (3 n_all)
  int jacobi_sweeps;
  float* dq_alt;
  // iterating to a tolerance (sim_options.residual_tol > 0, sim_step with n_iters <= 0): the
  // device counts the finished global updates and a CUDA graph while-node repeats the
  // iteration until R_k <= res_tol or max_iters updates
  int* iter_k;
  double res_tol;
  int max_iters;
  int n_rg, n_ct;
  double h;
  float h2f;        // h^2 in FP32
  double grav[3];
  // scenes (one for sim_create): vertices are ordered scene by scene
  int n_scenes;
  const int* vert_scene;      // n_all (internal numbering)
  const int* scene_vfirst;    // n_scenes + 1: first internal free vertex of each scene
  const int* obst_scene;      // n_obs: the scene an obstacle acts on
  const int* scene_ofirst;    // n_scenes + 1: each scene's obstacles are [first, next first)
  // anchors (bilateral constraints): contact slots with obstacle id n_obs + a, rows e_x,
  // e_y, e_z; the slot keeps the target in ct_dn (x) and ct_df (y, z), the compliance in
  // ct_mu
  int n_anc;
  int* anc_of;                // n: the anchor of a free vertex, or -1
  double* anc_pos;            // 3 n_anc: the target at the end of the current frame
  const double* anc_pos0;     // 3 n_anc: the target at time 0
  const double* anc_vel;      // 3 n_anc
  const double* anc_e;        // n_anc: compliance
  const int* anc_partner;     // n_anc: the partner of a two-vertex row (internal id), or -1
  const int* anc_ptri;        // n_anc: its one-corner map entry in btri, or -1
  int n_pairs;                // anchors with a partner
  int map_on;                 // contact maps beyond one vertex (bodies or pairs)
  const double* scene_margin; // contact margin
  const double* scene_Lref;   // rest bounding-box diagonal (residual scale)
  const double* scene_hvel;   // 3 per scene: velocity of the scene's pinned vertices
  const double* scene_mass;   // the scene's free mass
  // per frame, from the contact lists (k_scene_ranges): contact vertices [sc_cvb[s],
  // sc_cvb[s+1]) and contacts [sc_jb[s], sc_jb[s+1]) of scene s; its W~ block (row-major,
  // ld sc_ld[s]) at sc_wtoff[s]; its first 64 x 64 W~ tile in the tile list
  int* sc_cvb;
  int* sc_jb;
  int* sc_ld;
  long long* sc_wtoff;
  int* sc_tileoff;
  double* resid_scene;        // n_scenes x (kMaxIters + 1)
  // warm start (not from the paper): 0 cold (lambda = 0, q = s~), 1 learned, 2 the previous
  // frame's impulses
  int ws_mode;
  // portfolio (not from the paper): scenes form groups of pf_copies identical copies; copy 0
  // of a group runs the cold start, the others the warm start, and at the frame's end every
  // copy continues from the copy with the lowest final residual (1: off)
  int pf_copies;
  MlpDev ws_net;              // BF16 weights (w_t) and the parameter vector (biases)
  // gains of the network's outputs in the learned start: the impulse change of a contact
  // that had an impulse at the same vertex and obstacle in the previous frame, the impulse
  // of a new contact, the normal move (1, 1, 1 by default)
  float ws_gain[4];   // learned start: impulse gains (persisting, new), move gain, and the
                      // acceptance ratio (a guess is kept below ratio x the cold residual)
  float* ws_feat;             // cap x kMlpIn: features at the frame start
  float* ws_out;              // cap x kMlpOut: network outputs
  double* ws_scale;           // cap: impulse scale margin / (h^2 W~_vv)
  double* ws_lam0;            // cap x 3: the guess (contact frame)
  double* ws_move;            // cap: the guessed move of the contact's vertex along its normal
  double* ws_pmove;           // cap: the previous frame's move along the normal at the same
                              // vertex and obstacle, at the frame's start (0: none)
  double* ws_shift;           // 6 per scene: the impulse translation and the applied one
  double* ws_res;             // 2 per scene: residual of the guess, of the cold start
  double* ws_rg;              // cap: the guess's residual at each contact (k = 0)
  double* ws_rc;              // cap: the cold start's residual at each contact (k = 0)
  float* ws_target;           // cap x 4: the frame's final impulse / scale, normal move / margin
  int* prev_valid;            // n: the vertex had a contact in the previous frame
  int* prev_obst;             // n: its obstacle
  double* prev_force;         // 3 n: its impulse in world coordinates, D^T lambda
  double* prev_move;          // n: its move along the normal over the frame (q - s~) . n

  // per vertex (internal numbering, n_all)
  double* q_t;      // 3 n_all
  double* v_t;      // 3 n_all
  double* q_ref;    // 3 n_all: q_t for free vertices, prescribed positions for pinned
  double* s_tilde;  // 3 n_all
  float* dq;        // 3 n_all: q^k - q_ref (FP32)
  float* qr_hi;     // 3 n_all: q_ref as an unevaluated FP32 sum hi + lo (edge vectors
  float* qr_lo;     //          of the local step are formed from it in FP32)
  double* mass;     // n_all
  const int* depth; // n (etree depth of each free row)
  const int* parent;
  const int* first_desc;

  // per element (caller order, internal vertex ids)
  const int4* tet_v;
  const float* tet_dminv;  // [9][n_tets]
  const float* tet_w;      // PD weight
  const float* tet_vol;
  const int* tet_mat;
  const MatDev* mats;
  float4* contrib;         // h^2 w (p - F_ref) g_a per element corner, stored at the
                           // corner's incidence slot (vertex-major)
  // triangle (membrane) elements
  int n_tris;
  const int4* tri_v;       // internal vertex ids (w unused)
  const float* tri_dminv;  // 4 x n_tris (k * n_tris + t): D_m^-1 row-major 2 x 2
  const float* tri_w;
  const float* tri_vol;
  const int* tri_mat;
  // bending: rows of K = sum k_b L^T diag(interior / A) L for the free vertices (internal
  // numbering, columns over all vertices), and the per-frame force -h^2 K q_ref
  const int* bend_ptr;     // n + 1, or null without bending
  const int* bend_idx;
  const double* bend_val;
  float* bend_f;           // 3 n
  const int* inc_ptr;      // n + 1: incidences of free vertex i
  const int* inc_idx;      // entries 4 t + a
  const int* inc_slot;     // 4 n_tets + 3 n_tris: the corner's position in the incidence
                           // lists (-1: pinned), where contrib holds its contribution

  // S~ profile (FP32 values, or BF16 bit patterns when s_bf16 is set)
  const float* S;
  const unsigned short* Sb;
  int s_bf16;
  int refine;       // BF16 residual correction: 0 none, 1 last iteration, 2 every iteration
  // A~ over the free vertices (CSR, internal numbering, FP64): the residual of a solve
  const int* A_ptr;
  const int* A_idx;
  const double* A_val;
  float* gsave;     // 3 n_pad SoA: right-hand side of the residual-correction solve
  const long long* rowbase;
  const int* lo;
  const int* hi;
  // balanced tile streams of the two products (StreamSchedule on the host)
  const int2* s1_tiles;   // (row group, column tile)
  const int* s1_cta;      // s1_grid + 1
  const int* s1_seg_base; // s1_grid
  const int* s1_seg_first;// n_rg + 1
  const int2* s2_tiles;   // (column tile, row group)
  const int* s2_cta;
  const int* s2_seg_base;
  const int* s2_seg_first;// n_ct + 1
  const int* s1_col_first;  // s1_grid + 1: the CTA's distinct column tiles in s1_cols
  const int* s1_cols;
  const int* s1_col_slot;   // per pass-1 tile: position of its column tile in that list
  int s1_max_cols;
  int s1_grid, s2_grid, n_seg1, n_seg2;
  int s1_unroll, s2_unroll;  // tiles in flight per warp: 1 the format's, 0 half, 2 twice;
                             // kUnrollBulk: bulk copies into a ring of shared-memory stages
  int n_sm;         // persistent-kernel grid size
  int* scan_part;   // scratch of the two-pass scans (tile sums and offsets)
  // Delassus reuse across frames: W~ = Y^T Y and Y depend only on the list of contact
  // vertices (S~ is constant), so a frame whose list equals the previous frame's keeps them.
  // dl_state[0]: 1 when the current frame reuses them; [1]: the previous frame's
  // contact-vertex count (-1: none to compare with); [2]: frames that reused them.
  int dl_reuse_on;
  int* dl_state;
  int* dl_prev_cv;  // cap: the previous frame's contact vertices
  int ytz_warp;     // Y^T z with a warp per contact vertex (short ancestor paths) instead
                    // of a CTA per contact vertex
  const float* zero;  // kTileW zeros: the load target of lanes outside a row's range
  float* p1_part;   // [n_seg1][3][kRowGroup]
  float* p2_part;   // [n_seg2][3][kTileW]

  // vectors (SoA, n_pad per component)
  float* gvec;
  float* zvec;
  float* xout;      // 3 n (AoS) result of the transpose pass for apply_inverse

  // obstacles
  const ObstDev* obst;
  // contact between bodies (connected components of a scene's tetrahedra): a vertex
  // against the nearest surface triangle of another body, the map x_v - sum_k w_k x_k
  int bc_on;               // some scene has it (every array below is null otherwise)
  int n_bodies;
  const int* vert_body;    // n: body of a free surface vertex, -1 otherwise
  const int4* btri;        // surface triangles with free corners, grouped by body: internal
                           // corner ids, w = the triangle's number
  const int* body_toff;    // n_bodies + 1
  const int* scene_bfirst; // n_scenes + 1
  const double* scene_bmu; // n_scenes: friction coefficient between bodies
  double* body_box;        // 6 per body: bounds of its triangles' corners at s~
  int n_btri;
  float* chunk_box;        // 6 per run of kTriChunk consecutive triangles: their bounds
  float* tri_box;          // 6 per triangle: its bounds (both rounded outward to FP32)
  float* super_box;        // 6 per run of kTriSuper triangles (kTriSuper / kTriChunk runs)
  int* bc_tri;             // n: the vertex's matched triangle (index into btri) or -1
  double* bc_w;            // 3 n: barycentric weights of the closest point
  double* bc_n;            // 3 n: contact normal
  int* x_cnt;              // n: corner terms at free vertex i (contacts whose triangle has
  int* x_fill;             //    it as a corner with a non-zero weight)
  int* x_off;              // n + 1
  int* x_list;             // 3 cap: corner terms 3 j + k, per vertex ascending
  int* ct_tri;             // cap: index into btri, -1 for other contacts
  double* ct_bw;           // 3 cap: the corners' weights w_k (0: no term)
  int* ct_tcv;             // 3 cap: the corners' contact-vertex indices (-1: no term)

  // contacts (capacity cap), sorted by internal vertex then obstacle
  int* counters;    // kNumCounters
  int* ct_cnt;      // n: contacts of free vertex i
  int* ct_off;      // n + 1
  int* cv_flag;     // n
  int* cv_off;      // n + 1
  int* ct_vert;     // cap
  int* ct_obst;
  int* ct_cv;       // contact -> contact-vertex index
  double* ct_D;     // 9 cap: rows n, f1, f2
  double* ct_dn;    // cap
  double* ct_df;    // 2 cap
  double* ct_mu;    // cap
  double* ct_r;     // 4 cap: r_n, r_f of the iteration, then r_n, r_f of the Delassus
                    // diagonal (the residual's; the same unless SIM_PRECOND_MASS)
  double* ct_lam;   // 3 cap
  double* ct_force; // 3 cap: D^T (Omega lambda)
  float* ct_omega;  // 3 cap
  float* ct_ecal;   // 3 cap: E_n / h^2, E_f / h, E_f / h
  float* ct_Df;     // 9 cap: D in FP32
  double* ct_hv;    // 3 cap: h-vector shifted by J q_ref
  float* ct_rhs;    // 3 cap: Schur right-hand side
  int* cv_vert;     // cap: internal vertex of contact vertex c (ascending)
  int* cv_first;    // cap: first contact of contact vertex c
  int* cv_nct;      // cap
  float* uvec;      // 3 cap: per contact vertex D^T Omega dlambda
  float* svec;      // 3 cap: (Y^T z) per contact vertex
  // ancestors of contact vertices (U) and Y = S~ columns at contact vertices
  int* u_flag;      // n
  int* u_off;       // n + 1
  int* u_list;      // n
  int* row_clo;     // n: first contact vertex in the subtree of row a (row indexed)
  int* row_len;     // n: contact vertices in the subtree of row a
  int* u_clo;       // n: the same, compacted over U
  int* u_len;       // n
  int* y_ptr;       // n + 1
  float* y_val;     // cap_y
  int* yc_len;      // cap
  int* yc_ptr;      // cap + 1
  float* yc_val;    // cap_y
  int* yc_row;      // cap_y
  float* wt;        // cap x cap (W~, row-major with ld = n_cv)
  int* kb_lo;       // n / 32 + 1: union of the contact-vertex intervals of 32 rows of U
  int* kb_hi;
  float* wt_part;   // partial 64 x 64 tiles of W~
  int wt_grid;      // CTAs of the W~ product
  int cr_R;         // CTAs per CR cluster (one cluster per scene)
  int cr_single;    // 1: one cluster exchange per CR iteration (k_cr1); 0: two (k_cr)
  int cr_sync;      // k_cr's exchanges: 0 point-to-point (st.async + mbarrier), 1 cluster barriers
  int* cr_split;    // per scene 2 (kCrMaxRanks + 1): first contact vertex (scene-local) and
                    // first contact (global) of each rank
  unsigned long long spin_limit;  // polls of a device-side wait before it reports a timeout
  // launch the straight-line kernels of an iteration with programmatic dependent launch
  // (the next kernel's launch overlaps the tail of the one before; it waits for that one's
  // completion at its first instruction). Host-side switch, set while capturing a
  // production frame graph, whose kernels are not separated by event nodes.
  int pdl;
  // diagnostics
  double* resid;    // kMaxIters + 1
  double* max_pen;
  int* err;
  // local-projection debug output
  float* p_out;     // 9 n_tets
};

// ---- launchers (all asynchronous on stream s) ----------------------------------------
void launch_frame_begin(const DevSim& d, cudaStream_t s);
void launch_collide(const DevSim& d, cudaStream_t s);
void launch_delassus(const DevSim& d, cudaStream_t s);
// W~ work items: at most kWtMaxSplit K-splits per 64 x 64 tile; partial tiles for
// wt_items_max(cap, grid) items
constexpr int kWtMaxSplit = 16;
constexpr int kCrMaxRanks = 16;
constexpr int kTriChunk = 16;   // surface triangles per bounding box of the body search
constexpr int kTriSuper = 256;  // ... and per bounding box of the level above
constexpr int kUnrollBulk = 3;
constexpr int kMaxStagedCols = 32;  // column tiles of g staged per pass-1 CTA (96 KB)
inline long long wt_items_max(int cap, int grid) {
  long long best = 0;
  for (int nb = 1; nb <= (cap + 63) / 64; ++nb) {
    long long nt = (long long)nb * (nb + 1) / 2;
    long long S = (grid + nt - 1) / nt;
    if (S < 1) S = 1;
    if (S > kWtMaxSplit) S = kWtMaxSplit;
    if (nt * S > best) best = nt * S;
  }
  return best;
}
void launch_local(const DevSim& d, cudaStream_t s, bool debug_p);
// k < 0: the iteration index is read from d.iter_k (frames that iterate to a tolerance)
void launch_contact_eval(const DevSim& d, cudaStream_t s, int k, bool final_eval);
// frames that iterate to a tolerance: count one more finished update; set the while-node's
// condition (continue while k < max_iters, R_k > res_tol and no device error); clear the
// residual entries of the current k (before a final correction re-evaluates them)
void launch_iter_advance(const DevSim& d, cudaStream_t s);
void launch_iter_decide(const DevSim& d, cudaStream_t s, cudaGraphConditionalHandle h);
void launch_iter_clear(const DevSim& d, cudaStream_t s);
void launch_rhs(const DevSim& d, cudaStream_t s);
// the Jacobi global step: d.jacobi_sweeps sweeps dq <- dq + D^-1 (g - A~ dq), result in d.dq
void launch_jacobi(const DevSim& d, cudaStream_t s);
// z = S~ g: the product (partial sums) and the fixed-order reduction into zvec
void launch_pass1(const DevSim& d, cudaStream_t s);
void launch_reduce1(const DevSim& d, cudaStream_t s);
// x = S~^T y: the product and the reduction, which writes dq or xout or adds into them
enum { kOutDq = 0, kOutX = 1, kOutAddDq = 2, kOutAddX = 3 };
void launch_pass2(const DevSim& d, cudaStream_t s);
void launch_reduce2(const DevSim& d, cudaStream_t s, int out_mode);
inline void launch_solve(const DevSim& d, cudaStream_t s, int out_mode) {
  launch_pass1(d, s);
  launch_reduce1(d, s);
  launch_pass2(d, s);
  launch_reduce2(d, s, out_mode);
}
// residual of a global solve into gsave: gsave - A xout (kResApply), g - A dq (kResFrame),
// g + h^2 J^T dlambda - A dq (kResFrameContact)
enum { kResApply = 0, kResFrame = 1, kResFrameContact = 2 };
void launch_residual(const DevSim& d, cudaStream_t s, int mode);
void launch_ytz(const DevSim& d, cudaStream_t s);
int launch_cr(const DevSim& d, cudaStream_t s, int cluster);
void launch_yu(const DevSim& d, cudaStream_t s);
void launch_integrate(const DevSim& d, cudaStream_t s);
// warm start: features of the frame's contacts (always, for training data); the guess and
// its acceptance (modes 1, 2); the record of the frame's impulses and targets at its end
void launch_ws_features(const DevSim& d, cudaStream_t s);
void launch_ws_start(const DevSim& d, cudaStream_t s);
void launch_ws_record(const DevSim& d, cudaStream_t s);
int ws_kernels(const DevSim& d);   // launches of launch_ws_start
// portfolio: every copy of a group takes the state of the copy with the lowest final
// residual after a K-iteration frame (one launch)
// (K < 0: read from d.iter_k)
void launch_pf_sync(const DevSim& d, cudaStream_t s, int K);
// exclusive scan of n ints (or of min(*n_dev, n)): one CTA, or with `scratch`
// (scan_scratch_ints(n) ints) and n above 65,536 one CTA per 4,096-element tile in three
// launches (scan_launches(n))
// skip: when non-null and *skip != 0 on the device, the launches do nothing
void launch_scan(const int* in, int* out, int n, const int* n_dev, int* total, cudaStream_t s,
                 int* scratch = nullptr, const int* skip = nullptr);
int scan_launches(int n);
int scan_scratch_ints(int n);
int cr_setup(int n_scenes, int max_cv, int max_ct, int* cluster_out, size_t* smem_out);
// S~ built on the device in FP64 from the host's factor L~ (k_sbuild.cu)
struct SinvBuildArgs {
  int nf;
  const long long* Lp;      // nf + 1: column starts of L~ (diagonal first)
  const int* Ldd;           // per entry: depth(column) - depth(row), 0 on the diagonal
  const double* Lx;
  const int* parent;
  const int* depth;
  const long long* rowbase; // S~ profile: offset of column lo of each row
  const int* lo;
  int max_depth;
  int* next_col;            // work counter (1 int)
  float* S;                 // stored values, zero-initialised
  unsigned short* Sb;       // BF16 copy, or null
};
bool sinv_build_fits(int max_depth);
int launch_sinv_build(const SinvBuildArgs& a, cudaStream_t s);
void sinv_build_depth_steps(const Plan& p, std::vector<int>* ldd);
int sinv_setup();

}  // namespace silg

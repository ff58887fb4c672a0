// Host-side precompute of the sparse-inverse local-global solver (internal header).
//
// Everything here runs once per mesh on the CPU in FP64 (and integer arithmetic for the
// ordering and symbolic phases): per-element rest data, lumped masses, the per-vertex
// system matrix A~ (Eq. 6 with A = A~ (x) I3), a nested-dissection ordering, the
// postordered elimination tree, the Cholesky factor L~ and the sparse inverse
// S~ = L~^-1 P in row-profile form (Theorem 1), plus the tile schedule the device
// products use.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "silg.h"

namespace silg {

// Row-profile alignment (values): every stored row starts at a column multiple of
// kAlign and its length is a multiple of kAlign, so 16-byte vector loads of FP32 (4) and
// BF16 (8) values stay aligned.
constexpr int kAlign = 8;
// Device tile shape of the two profile products: kRowGroup rows x kTileW columns.
constexpr int kRowGroup = 32;
constexpr int kTileW = 256;

struct MatParams {
  int model;
  double mu_le, lam_le;   // Lame parameters of linear elasticity
  double mu, lam, alpha;  // parameters of the element energy (SNH re-parameterised)
  double rho;
};

struct Plan {
  // ---- copied input ---------------------------------------------------------------
  int n_verts = 0, n_tets = 0;
  double h = 0;
  std::vector<double> X;          // n_verts x 3 (caller numbering)
  std::vector<int32_t> tets;      // n_tets x 4 (caller numbering)
  std::vector<int32_t> tet_mat;   // n_tets
  std::vector<MatParams> mats;
  std::vector<uint8_t> pinned;    // n_verts flags
  double handle_vel[3] = {0, 0, 0};
  int n_scenes = 1;
  std::vector<int32_t> vertex_scene;  // scene of each vertex (caller numbering)
  std::vector<int32_t> scene_vfirst;  // n_scenes + 1: scene boundaries, internal free ids

  // ---- triangle (membrane) elements and bending ------------------------------------
  int n_tris = 0;
  std::vector<int32_t> tris;      // n_tris x 3 (caller numbering)
  std::vector<int32_t> tri_mat;
  std::vector<double> tri_dminv;  // 4 per triangle: D_m^-1, row-major 2 x 2
  std::vector<double> tri_vol;    // area x thickness
  std::vector<double> tri_weight; // 2 mu_LE V
  // K = sum k_b L^T diag(interior / A) L (caller numbering, CSR over all vertices, symmetric)
  std::vector<int64_t> Kp;
  std::vector<int32_t> Ki;
  std::vector<double> Kx;

  // ---- per element (caller tet order) ----------------------------------------------
  std::vector<double> Dm_inv;     // 9 per tet, row-major
  std::vector<double> vol;        // rest volume V_i
  std::vector<double> weight;     // PD weight w_i = 2 mu_LE V_i
  std::vector<double> mass;       // lumped vertex mass (caller numbering)
  double mean_edge = 0;

  // ---- numbering ------------------------------------------------------------------
  int n_free = 0;
  std::vector<int32_t> order;     // internal free row k -> caller vertex id
  std::vector<int32_t> internal;  // caller vertex id -> internal id (free: k, pinned: n_free + j)
  std::vector<int32_t> pinned_ids;// internal pinned j -> caller vertex id

  // ---- elimination tree (postordered; internal free numbering) ----------------------
  std::vector<int32_t> parent, first_desc, depth;

  // ---- A~ over free vertices (CSR, internal numbering, full symmetric pattern) -------
  std::vector<int64_t> Ap;
  std::vector<int32_t> Ai;
  std::vector<double> Ax;

  // ---- L~ (CSC, diagonal first in each column) -----------------------------------
  std::vector<int64_t> Lp;
  std::vector<int32_t> Li;
  std::vector<double> Lx;

  // ---- S~ row profile --------------------------------------------------------------
  int n_pad = 0;                  // vector length: n_free rounded up to kTileW
  std::vector<int32_t> lo, hi;    // stored column range [lo, hi) of each row
  std::vector<int64_t> rowbase;   // offset of column lo of each row (n_free + 1 entries)
  std::vector<double> S;          // stored values (zeros outside [fd(i), i])
  int64_t nnz_S = 0;

  // ---- tiles of the device products ------------------------------------------------
  // Tiles of kRowGroup rows x kTileW columns that hold stored values. tiles1: (row group,
  // column tile, values) ordered by row group, then column tile (pass 1, z = S g);
  // tiles2: (column tile, row group, values) ordered by column tile, then row group
  // (pass 2, x = S^T y).
  int n_rg = 0, n_ct = 0;
  std::vector<int32_t> tiles1, tiles2;

  // ---- statistics -----------------------------------------------------------------
  int64_t nnz_A = 0, nnz_L = 0;
  int max_depth = 0, n_roots = 0;
  double mean_depth = 0, seconds = 0;
  double s_seconds = 0;           // the build of S~ (host loop, or device kernel incl. uploads)
  int s_on_device = 0;            // 1: S~ was built on the device
};

// Build the plan. Returns SIM_OK or an error code; *err receives a message.
// vertex_scene (optional): scene of each vertex, non-decreasing; the ordering is computed
// scene by scene so that every scene's free vertices are contiguous.
// tri_thickness (per triangle) and vert_bending (per vertex) override the mesh's single
// thickness and bending (a batch's scenes each have their own)
// build_S = false leaves S empty (the profile's shape -- lo, hi, rowbase -- is built): a
// simulator then builds the values on the device, or with build_sinv_host.
int build_plan(const sim_mesh* mesh, const sim_material* mats, int n_mat, double h,
               int n_threads, Plan* plan, std::string* err,
               const int32_t* vertex_scene = nullptr, int n_scenes = 1,
               const double* tri_thickness = nullptr, const double* vert_bending = nullptr,
               bool build_S = true);
// S~ = L~^-1 P on the host (FP64), into plan->S.
void build_sinv_host(Plan& p, int n_threads);

// Device work split of one product: CTA c streams tiles [cta_first[c], cta_first[c+1])
// of the pass's tile order, split so that every CTA has about the same cost; each run of
// tiles with the same key (row group in pass 1, column tile in pass 2) inside a CTA writes
// one partial-sum slot, seg_base[c] being the CTA's first; the slots of key k are
// [seg_first[k], seg_first[k+1]).
struct StreamSchedule {
  std::vector<int32_t> tiles;      // 2 per tile: key, other coordinate
  // pass 1: the distinct column tiles of each CTA's range (cta_cols[cta_col_first[c] ..
  // cta_col_first[c+1])), the position of each tile's column tile in that list, and the
  // longest list
  std::vector<int32_t> cta_col_first, cta_cols, tile_col_slot;
  int max_cols = 0;
  std::vector<int32_t> cta_first;  // grid + 1
  std::vector<int32_t> seg_base;   // grid
  std::vector<int32_t> seg_first;  // keys + 1
  int n_seg = 0;
};
void build_stream_schedule(const Plan& p, bool pass2, int grid, double zero_cost,
                           StreamSchedule* out);

// x = S^T (S b) on the host in FP64, internal free numbering, b and x of n_free x 3.
void apply_inverse_internal(const Plan& p, const double* b, double* x);

}  // namespace silg

// Host-side precompute: rest data, A~, nested dissection, elimination tree, Cholesky,
// sparse inverse S~ = L~^-1 P in row-profile form, and the device tile schedule.
#include "plan.hpp"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <cmath>
#include <numeric>
#include <thread>

namespace silg {
namespace {

constexpr int kLeaf = 48;  // nested-dissection leaf size

inline double det3(const double* m) {
  return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
         m[2] * (m[3] * m[7] - m[4] * m[6]);
}

inline void inv3(const double* m, double* o) {
  double d = det3(m);
  o[0] = (m[4] * m[8] - m[5] * m[7]) / d;
  o[1] = (m[2] * m[7] - m[1] * m[8]) / d;
  o[2] = (m[1] * m[5] - m[2] * m[4]) / d;
  o[3] = (m[5] * m[6] - m[3] * m[8]) / d;
  o[4] = (m[0] * m[8] - m[2] * m[6]) / d;
  o[5] = (m[2] * m[3] - m[0] * m[5]) / d;
  o[6] = (m[3] * m[7] - m[4] * m[6]) / d;
  o[7] = (m[1] * m[6] - m[0] * m[7]) / d;
  o[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

// Geometric nested dissection over a graph given in CSR (adj_p, adj_i) with vertex
// coordinates xyz: split the vertex set at the median of its longest bounding-box axis;
// the separator is the set of right-side vertices adjacent to the left side, so the two
// remaining halves are disconnected. Order: left, right, separator (recursively).
struct Dissector {
  const std::vector<int64_t>& adj_p;
  const std::vector<int32_t>& adj_i;
  const double* xyz;
  std::vector<int32_t> stamp;
  int32_t next_stamp = 1;
  std::vector<int32_t> out;

  Dissector(const std::vector<int64_t>& p, const std::vector<int32_t>& i, const double* x,
            int n)
      : adj_p(p), adj_i(i), xyz(x), stamp(n, 0) {}

  void run(std::vector<int32_t> S) {
    if ((int)S.size() <= kLeaf) {
      out.insert(out.end(), S.begin(), S.end());
      return;
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int v : S)
      for (int r = 0; r < 3; ++r) {
        mn[r] = std::min(mn[r], xyz[3 * v + r]);
        mx[r] = std::max(mx[r], xyz[3 * v + r]);
      }
    int ax = 0;
    for (int r = 1; r < 3; ++r)
      if (mx[r] - mn[r] > mx[ax] - mn[ax]) ax = r;
    std::sort(S.begin(), S.end(), [&](int a, int b) {
      double ca = xyz[3 * a + ax], cb = xyz[3 * b + ax];
      return ca < cb || (ca == cb && a < b);
    });
    double med = xyz[3 * S[S.size() / 2] + ax];
    size_t cut = 0;
    while (cut < S.size() && xyz[3 * S[cut] + ax] < med) ++cut;
    if (cut == 0) cut = S.size() / 2;  // degenerate coordinates: split by rank
    std::vector<int32_t> L(S.begin(), S.begin() + cut), R;
    int32_t st = next_stamp++;
    for (int v : L) stamp[v] = st;
    std::vector<int32_t> sep;
    for (size_t k = cut; k < S.size(); ++k) {
      int v = S[k];
      bool touches = false;
      for (int64_t e = adj_p[v]; e < adj_p[v + 1] && !touches; ++e)
        touches = stamp[adj_i[e]] == st;
      (touches ? sep : R).push_back(v);
    }
    run(std::move(L));
    run(std::move(R));
    out.insert(out.end(), sep.begin(), sep.end());
  }
};

}  // namespace

// S~ = L~^-1 P on the host in FP64, column by column over elimination-tree ancestors
// (Alg. 2, Theorem 1), multithreaded over columns.
void build_sinv_host(Plan& p, int n_threads) {
  const auto t0 = std::chrono::steady_clock::now();
  const int nf = p.n_free;
  p.S.assign(p.rowbase[nf], 0.0);
  {
    int nt = n_threads > 0 ? n_threads : (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt, 256));
    std::atomic<int> next_col(0);
    auto worker = [&]() {
      std::vector<double> x(nf, 0.0);
      std::vector<int32_t> path;
      for (;;) {
        int j0 = next_col.fetch_add(16);
        if (j0 >= nf) break;
        for (int j = j0; j < std::min(nf, j0 + 16); ++j) {
          path.clear();
          for (int a = j; a != -1; a = p.parent[a]) path.push_back(a);
          x[j] = 1.0;
          for (int a : path) {
            double xa = x[a] / p.Lx[p.Lp[a]];
            x[a] = xa;
            for (int64_t q = p.Lp[a] + 1; q < p.Lp[a + 1]; ++q) x[p.Li[q]] -= p.Lx[q] * xa;
          }
          for (int a : path) {
            p.S[p.rowbase[a] + (j - p.lo[a])] = x[a];
            x[a] = 0.0;
          }
        }
      }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(worker);
    for (auto& t : th) t.join();
  }
  p.s_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  p.s_on_device = 0;
}

int build_plan(const sim_mesh* mesh, const sim_material* mats, int n_mat, double h,
               int n_threads, Plan* P, std::string* err, const int32_t* vertex_scene,
               int n_scenes, const double* tri_thickness, const double* vert_bending,
               bool build_S) {
  auto t0 = std::chrono::steady_clock::now();
  Plan& p = *P;
  if (!mesh || !mesh->rest_pos || mesh->n_verts <= 0 || mesh->n_tets < 0 || mesh->n_tris < 0 ||
      mesh->n_tets + mesh->n_tris <= 0 || (mesh->n_tets > 0 && !mesh->tets) ||
      (mesh->n_tris > 0 && !mesh->tris) || !mats || n_mat <= 0 || !(h > 0) ||
      !std::isfinite(h)) {
    *err = "null or empty mesh / materials, or non-positive h";
    return SIM_EINVAL;
  }
  const int n = mesh->n_verts, T = mesh->n_tets, Nt = mesh->n_tris;
  p.n_verts = n;
  p.n_tets = T;
  p.n_tris = Nt;
  p.h = h;
  p.X.assign(mesh->rest_pos, mesh->rest_pos + 3 * (size_t)n);
  if (T > 0) p.tets.assign(mesh->tets, mesh->tets + 4 * (size_t)T);
  if (Nt > 0) p.tris.assign(mesh->tris, mesh->tris + 3 * (size_t)Nt);
  p.tri_mat.assign(Nt, 0);
  if (Nt > 0 && mesh->tri_material) p.tri_mat.assign(mesh->tri_material, mesh->tri_material + Nt);
  p.tet_mat.assign(T, 0);
  if (mesh->tet_material) p.tet_mat.assign(mesh->tet_material, mesh->tet_material + T);
  for (int r = 0; r < 3; ++r) p.handle_vel[r] = mesh->handle_vel[r];
  p.n_scenes = std::max(1, n_scenes);
  p.vertex_scene.assign(n, 0);
  if (vertex_scene) {
    for (int v = 0; v < n; ++v) {
      if (vertex_scene[v] < 0 || vertex_scene[v] >= p.n_scenes ||
          (v > 0 && vertex_scene[v] < vertex_scene[v - 1])) {
        *err = "vertex scene ids must be non-decreasing and below the scene count";
        return SIM_EINVAL;
      }
      p.vertex_scene[v] = vertex_scene[v];
    }
  }
  for (double x : p.X)
    if (!std::isfinite(x)) {
      *err = "non-finite rest position";
      return SIM_EINVAL;
    }
  for (int m = 0; m < n_mat; ++m) {
    const sim_material& M = mats[m];
    if (M.model < SIM_MODEL_ARAP || M.model > SIM_MODEL_SNH || !(M.E > 0) ||
        !(M.nu >= 0 && M.nu < 0.5) || !(M.rho > 0)) {
      *err = "invalid material " + std::to_string(m);
      return SIM_EINVAL;
    }
    MatParams mp;
    mp.model = M.model;
    mp.rho = M.rho;
    mp.mu_le = M.E / (2 * (1 + M.nu));
    mp.lam_le = M.E * M.nu / ((1 + M.nu) * (1 - 2 * M.nu));
    if (M.model == SIM_MODEL_SNH) {
      mp.mu = 4.0 / 3.0 * mp.mu_le;
      mp.lam = mp.lam_le + 5.0 / 6.0 * mp.mu_le;
      mp.alpha = 1.0 + 0.75 * mp.mu / mp.lam;
    } else {
      mp.mu = mp.mu_le;
      mp.lam = mp.lam_le;
      mp.alpha = 0.0;
    }
    p.mats.push_back(mp);
  }
  p.pinned.assign(n, 0);
  if (mesh->n_pinned < 0 || (mesh->n_pinned > 0 && !mesh->pinned)) {
    *err = "bad pinned list";
    return SIM_EINVAL;
  }
  for (int k = 0; k < mesh->n_pinned; ++k) {
    int v = mesh->pinned[k];
    if (v < 0 || v >= n) {
      *err = "pinned vertex out of range";
      return SIM_EINVAL;
    }
    p.pinned[v] = 1;
  }
  // ---- per element ----------------------------------------------------------------
  p.Dm_inv.resize(9 * (size_t)T);
  p.vol.resize(T);
  p.weight.resize(T);
  p.mass.assign(n, 0.0);
  double edge_sum = 0;
  for (int t = 0; t < T; ++t) {
    const int32_t* v = &p.tets[4 * (size_t)t];
    for (int a = 0; a < 4; ++a)
      if (v[a] < 0 || v[a] >= n) {
        *err = "tet index out of range";
        return SIM_EINVAL;
      }
    if (p.tet_mat[t] < 0 || p.tet_mat[t] >= n_mat) {
      *err = "tet material out of range";
      return SIM_EINVAL;
    }
    double Dm[9];
    for (int a = 1; a < 4; ++a)
      for (int r = 0; r < 3; ++r) Dm[3 * r + (a - 1)] = p.X[3 * v[a] + r] - p.X[3 * v[0] + r];
    double d = det3(Dm);
    if (!(d > 0)) {
      *err = "inverted or degenerate rest tetrahedron " + std::to_string(t);
      return SIM_EINVAL;
    }
    inv3(Dm, &p.Dm_inv[9 * (size_t)t]);
    p.vol[t] = d / 6.0;
    const MatParams& mp = p.mats[p.tet_mat[t]];
    p.weight[t] = 2.0 * mp.mu_le * p.vol[t];
    for (int a = 0; a < 4; ++a) p.mass[v[a]] += mp.rho * p.vol[t] / 4.0;
    for (int a = 1; a < 4; ++a)
      edge_sum += std::sqrt(Dm[a - 1] * Dm[a - 1] + Dm[3 + a - 1] * Dm[3 + a - 1] +
                            Dm[6 + a - 1] * Dm[6 + a - 1]);
  }
  // ---- triangles: in-plane rest edges, area x thickness, mass -----------------------
  p.tri_dminv.resize(4 * (size_t)Nt);
  p.tri_vol.resize(Nt);
  p.tri_weight.resize(Nt);
  for (int t = 0; t < Nt; ++t) {
    const int32_t* v = &p.tris[3 * (size_t)t];
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= n) {
        *err = "triangle index out of range";
        return SIM_EINVAL;
      }
    if (p.tri_mat[t] < 0 || p.tri_mat[t] >= n_mat ||
        p.mats[p.tri_mat[t]].model == SIM_MODEL_SNH) {
      *err = "triangle material out of range, or stable Neo-Hookean (membranes: ARAP or "
             "co-rotational)";
      return SIM_EINVAL;
    }
    const double th = tri_thickness ? tri_thickness[t] : mesh->thickness;
    if (!(th > 0) || !std::isfinite(th)) {
      *err = "a triangle sheet needs a positive thickness";
      return SIM_EINVAL;
    }
    double e1[3], e2[3], nr[3];
    for (int r = 0; r < 3; ++r) {
      e1[r] = p.X[3 * v[1] + r] - p.X[3 * v[0] + r];
      e2[r] = p.X[3 * v[2] + r] - p.X[3 * v[0] + r];
    }
    nr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    const double nn = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    if (!(l1 > 0) || !(nn > 0)) {
      *err = "degenerate rest triangle " + std::to_string(t);
      return SIM_EINVAL;
    }
    // rest frame: a1 along e1, a2 = n x a1; D_m = [[l1, e2.a1], [0, e2.a2]]
    double a1[3], a2[3];
    for (int r = 0; r < 3; ++r) a1[r] = e1[r] / l1;
    a2[0] = (nr[1] * a1[2] - nr[2] * a1[1]) / nn;
    a2[1] = (nr[2] * a1[0] - nr[0] * a1[2]) / nn;
    a2[2] = (nr[0] * a1[1] - nr[1] * a1[0]) / nn;
    const double d00 = l1, d01 = e2[0] * a1[0] + e2[1] * a1[1] + e2[2] * a1[2];
    const double d11 = e2[0] * a2[0] + e2[1] * a2[1] + e2[2] * a2[2];
    double* Mi = &p.tri_dminv[4 * (size_t)t];
    Mi[0] = 1.0 / d00;
    Mi[1] = -d01 / (d00 * d11);
    Mi[2] = 0.0;
    Mi[3] = 1.0 / d11;
    p.tri_vol[t] = 0.5 * nn * th;
    const MatParams& mp = p.mats[p.tri_mat[t]];
    p.tri_weight[t] = 2.0 * mp.mu_le * p.tri_vol[t];
    for (int a = 0; a < 3; ++a) p.mass[v[a]] += mp.rho * p.tri_vol[t] / 3.0;
    edge_sum += l1 + std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
  }
  p.mean_edge = edge_sum / (3.0 * T + 2.0 * Nt);
  // ---- bending: K = sum k_b L^T diag(interior / A) L ----------------------------------
  {
    // cotangent weights per edge, mixed Voronoi areas, boundary edges (one triangle)
    std::map<std::pair<int, int>, std::pair<double, int>> edge;   // (w_ij, triangles)
    std::vector<double> area(n, 0.0);
    bool any = false;
    for (int t = 0; t < Nt; ++t) {
      const int32_t* v = &p.tris[3 * (size_t)t];
      double P[3][3], cot[3];
      for (int a = 0; a < 3; ++a)
        for (int r = 0; r < 3; ++r) P[a][r] = p.X[3 * v[a] + r];
      for (int k = 0; k < 3; ++k) {
        // the angle at corner k, between the edges to the two others
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        double u[3], w[3], c[3];
        for (int r = 0; r < 3; ++r) {
          u[r] = P[a][r] - P[k][r];
          w[r] = P[b][r] - P[k][r];
        }
        c[0] = u[1] * w[2] - u[2] * w[1];
        c[1] = u[2] * w[0] - u[0] * w[2];
        c[2] = u[0] * w[1] - u[1] * w[0];
        cot[k] = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) /
                 std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        auto key = std::make_pair(std::min(v[a], v[b]), std::max(v[a], v[b]));
        auto& e = edge[key];
        e.first += 0.5 * cot[k];
        e.second += 1;
      }
      const double ar = p.tri_vol[t] / (tri_thickness ? tri_thickness[t] : mesh->thickness);
      const bool obtuse = cot[0] < 0 || cot[1] < 0 || cot[2] < 0;
      for (int k = 0; k < 3; ++k) {
        if (obtuse) {
          area[v[k]] += cot[k] < 0 ? ar / 2 : ar / 4;
        } else {
          const int a = (k + 1) % 3, b = (k + 2) % 3;
          double lb = 0, la = 0;
          for (int r = 0; r < 3; ++r) {
            lb += (P[b][r] - P[k][r]) * (P[b][r] - P[k][r]);
            la += (P[a][r] - P[k][r]) * (P[a][r] - P[k][r]);
          }
          area[v[k]] += (lb * cot[a] + la * cot[b]) / 8.0;
        }
      }
    }
    std::vector<char> boundary(n, 0);
    for (auto& e : edge)
      if (e.second.second == 1) boundary[e.first.first] = boundary[e.first.second] = 1;
    // rows of L (L_ii = sum w, L_ij = -w), then K = L^T diag(c) L with c = k_b / A at
    // interior sheet vertices
    std::vector<std::vector<std::pair<int32_t, double>>> Lr(n);
    for (auto& e : edge) {
      const int i = e.first.first, j = e.first.second;
      const double w = e.second.first;
      Lr[i].push_back({i, w});
      Lr[i].push_back({j, -w});
      Lr[j].push_back({j, w});
      Lr[j].push_back({i, -w});
    }
    std::vector<std::map<int32_t, double>> K(n);
    for (int i = 0; i < n; ++i) {
      const double kb = vert_bending ? vert_bending[i] : mesh->bending;
      if (!(kb >= 0) || !std::isfinite(kb)) {
        *err = "bending stiffness must be finite and non-negative";
        return SIM_EINVAL;
      }
      if (kb == 0 || boundary[i] || !(area[i] > 0) || Lr[i].empty()) continue;
      std::map<int32_t, double> row;   // row i of L, merged
      for (auto& e : Lr[i]) row[e.first] += e.second;
      const double c = kb / area[i];
      for (auto& a : row)
        for (auto& b : row) K[a.first][b.first] += c * a.second * b.second;
      any = true;
    }
    p.Kp.assign(n + 1, 0);
    p.Ki.clear();
    p.Kx.clear();
    if (any)
      for (int i = 0; i < n; ++i) {
        for (auto& e : K[i]) {
          p.Ki.push_back(e.first);
          p.Kx.push_back(e.second);
        }
        p.Kp[i + 1] = (int64_t)p.Ki.size();
      }
  }
  for (int v = 0; v < n; ++v)
    if (!(p.mass[v] > 0)) {
      *err = "vertex " + std::to_string(v) + " belongs to no element";
      return SIM_EINVAL;
    }
  // ---- free vertices and their graph ---------------------------------------------
  std::vector<int32_t> free_ids, free_of(n, -1);
  for (int v = 0; v < n; ++v)
    if (!p.pinned[v]) {
      free_of[v] = (int)free_ids.size();
      free_ids.push_back(v);
    }
  const int nf = (int)free_ids.size();
  p.n_free = nf;
  if (nf == 0) {
    *err = "every vertex is pinned";
    return SIM_EINVAL;
  }
  std::vector<std::vector<int32_t>> nb(nf);
  for (int t = 0; t < T; ++t) {
    const int32_t* v = &p.tets[4 * (size_t)t];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        if (a != b && free_of[v[a]] >= 0 && free_of[v[b]] >= 0)
          nb[free_of[v[a]]].push_back(free_of[v[b]]);
  }
  for (int t = 0; t < Nt; ++t) {
    const int32_t* v = &p.tris[3 * (size_t)t];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (a != b && free_of[v[a]] >= 0 && free_of[v[b]] >= 0)
          nb[free_of[v[a]]].push_back(free_of[v[b]]);
  }
  if (!p.Kx.empty())
    for (int i = 0; i < n; ++i)
      for (int64_t e = p.Kp[i]; e < p.Kp[i + 1]; ++e) {
        const int j = p.Ki[e];
        if (i != j && free_of[i] >= 0 && free_of[j] >= 0) nb[free_of[i]].push_back(free_of[j]);
      }
  std::vector<int64_t> gp(nf + 1, 0);
  std::vector<int32_t> gi;
  for (int f = 0; f < nf; ++f) {
    auto& L = nb[f];
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    gp[f + 1] = gp[f] + (int64_t)L.size();
    gi.insert(gi.end(), L.begin(), L.end());
  }
  // ---- nested dissection ------------------------------------------------------------
  std::vector<double> fxyz(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f)
    for (int r = 0; r < 3; ++r) fxyz[3 * f + r] = p.X[3 * free_ids[f] + r];
  Dissector D(gp, gi, fxyz.data(), nf);
  {
    // scene by scene (scenes share no element, so each is ordered on its own and the
    // elimination forest keeps them apart and in scene order)
    std::vector<std::vector<int32_t>> by_scene(p.n_scenes);
    for (int f = 0; f < nf; ++f) by_scene[p.vertex_scene[free_ids[f]]].push_back(f);
    for (auto& S : by_scene)
      if (!S.empty()) D.run(std::move(S));
  }
  std::vector<int32_t>& nd = D.out;  // nd[k] = free index at position k
  std::vector<int32_t> nd_inv(nf);
  for (int k = 0; k < nf; ++k) nd_inv[nd[k]] = k;
  // ---- elimination tree of the ND-ordered matrix (ancestor walk with compression) ----
  std::vector<int32_t> par(nf, -1), anc(nf, -1);
  for (int k = 0; k < nf; ++k) {
    int f = nd[k];
    for (int64_t e = gp[f]; e < gp[f + 1]; ++e) {
      int i = nd_inv[gi[e]];
      while (i != -1 && i < k) {
        int nx = anc[i];
        anc[i] = k;
        if (nx == -1) par[i] = k;
        i = nx;
      }
    }
  }
  // ---- postorder --------------------------------------------------------------------
  std::vector<int32_t> head(nf, -1), nxt(nf, -1), post;
  post.reserve(nf);
  for (int j = nf - 1; j >= 0; --j)
    if (par[j] >= 0) {
      nxt[j] = head[par[j]];
      head[par[j]] = j;
    }
  {
    std::vector<int32_t> stack;
    for (int r = 0; r < nf; ++r) {
      if (par[r] != -1) continue;
      stack.push_back(r);
      while (!stack.empty()) {
        int v = stack.back();
        int c = head[v];
        if (c == -1) {
          stack.pop_back();
          post.push_back(v);
        } else {
          head[v] = nxt[c];
          stack.push_back(c);
        }
      }
    }
  }
  // final internal order: internal k -> ND position post[k] -> free index -> caller id
  std::vector<int32_t> pos_of(nf);
  for (int k = 0; k < nf; ++k) pos_of[post[k]] = k;
  p.order.resize(nf);
  p.parent.assign(nf, -1);
  for (int k = 0; k < nf; ++k) {
    p.order[k] = free_ids[nd[post[k]]];
    int pp = par[post[k]];
    p.parent[k] = pp < 0 ? -1 : pos_of[pp];
  }
  p.internal.assign(n, -1);
  for (int k = 0; k < nf; ++k) p.internal[p.order[k]] = k;
  // scene boundaries in the internal free numbering
  p.scene_vfirst.assign(p.n_scenes + 1, nf);
  for (int k = nf - 1; k >= 0; --k) p.scene_vfirst[p.vertex_scene[p.order[k]]] = k;
  for (int sc = p.n_scenes - 1; sc >= 0; --sc)
    p.scene_vfirst[sc] = std::min(p.scene_vfirst[sc], p.scene_vfirst[sc + 1]);
  for (int k = 1; k < nf; ++k)
    if (p.vertex_scene[p.order[k]] < p.vertex_scene[p.order[k - 1]]) {
      *err = "internal: scenes are not contiguous in the elimination order";
      return SIM_EINVAL;
    }
  for (int v = 0; v < n; ++v)
    if (p.pinned[v]) {
      p.internal[v] = nf + (int)p.pinned_ids.size();
      p.pinned_ids.push_back(v);
    }
  // subtree sizes, first descendants, depths
  std::vector<int32_t> sub(nf, 1);
  for (int k = 0; k < nf; ++k)
    if (p.parent[k] >= 0) sub[p.parent[k]] += sub[k];
  p.first_desc.resize(nf);
  p.depth.assign(nf, 1);
  for (int k = 0; k < nf; ++k) p.first_desc[k] = k - sub[k] + 1;
  for (int k = nf - 1; k >= 0; --k)
    if (p.parent[k] >= 0) p.depth[k] = p.depth[p.parent[k]] + 1;
  p.max_depth = 0;
  double dsum = 0;
  p.n_roots = 0;
  for (int k = 0; k < nf; ++k) {
    p.max_depth = std::max(p.max_depth, p.depth[k]);
    dsum += p.depth[k];
    p.n_roots += p.parent[k] < 0;
  }
  p.mean_depth = dsum / nf;
  // ---- A~ over free vertices in internal numbering ----------------------------------
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(nf);
    for (int k = 0; k < nf; ++k) rows[k].push_back({k, p.mass[p.order[k]]});
    for (int t = 0; t < T; ++t) {
      const int32_t* v = &p.tets[4 * (size_t)t];
      const double* Mi = &p.Dm_inv[9 * (size_t)t];
      double g[4][3];
      for (int c = 0; c < 3; ++c) {
        g[1][c] = Mi[0 * 3 + c];
        g[2][c] = Mi[1 * 3 + c];
        g[3][c] = Mi[2 * 3 + c];
        g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
      }
      double s = h * h * p.weight[t];
      for (int a = 0; a < 4; ++a) {
        int ia = p.internal[v[a]];
        if (ia >= nf) continue;
        for (int b = 0; b < 4; ++b) {
          int ib = p.internal[v[b]];
          if (ib >= nf) continue;
          double k = s * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
          rows[ia].push_back({ib, k});
        }
      }
    }
    for (int t = 0; t < Nt; ++t) {
      const int32_t* v = &p.tris[3 * (size_t)t];
      const double* Mi = &p.tri_dminv[4 * (size_t)t];
      double g[3][2];
      for (int c = 0; c < 2; ++c) {
        g[1][c] = Mi[c];
        g[2][c] = Mi[2 + c];
        g[0][c] = -(g[1][c] + g[2][c]);
      }
      const double s = h * h * p.tri_weight[t];
      for (int a = 0; a < 3; ++a) {
        const int ia = p.internal[v[a]];
        if (ia >= nf) continue;
        for (int b = 0; b < 3; ++b) {
          const int ib = p.internal[v[b]];
          if (ib >= nf) continue;
          rows[ia].push_back({ib, s * (g[a][0] * g[b][0] + g[a][1] * g[b][1])});
        }
      }
    }
    if (!p.Kx.empty())
      for (int i = 0; i < n; ++i) {
        const int ii = p.internal[i];
        if (ii >= nf) continue;
        for (int64_t e = p.Kp[i]; e < p.Kp[i + 1]; ++e) {
          const int jj = p.internal[p.Ki[e]];
          if (jj < nf) rows[ii].push_back({jj, h * h * p.Kx[e]});
        }
      }
    p.Ap.assign(nf + 1, 0);
    p.Ai.clear();
    p.Ax.clear();
    for (int k = 0; k < nf; ++k) {
      auto& R = rows[k];
      std::sort(R.begin(), R.end(),
                [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                  return a.first < b.first;
                });
      int32_t last = -1;
      for (auto& e : R) {
        if (e.first == last) {
          p.Ax.back() += e.second;
        } else {
          p.Ai.push_back(e.first);
          p.Ax.push_back(e.second);
          last = e.first;
        }
      }
      p.Ap[k + 1] = (int64_t)p.Ai.size();
      std::vector<std::pair<int32_t, double>>().swap(R);
    }
    p.nnz_A = p.Ap[nf];
  }
  // ---- symbolic: column counts from the row subtrees ----------------------------------
  std::vector<int32_t> mark(nf, -1), colcount(nf, 1);
  for (int k = 0; k < nf; ++k) {
    mark[k] = k;
    for (int64_t e = p.Ap[k]; e < p.Ap[k + 1]; ++e) {
      int j = p.Ai[e];
      while (j < k && mark[j] != k) {
        mark[j] = k;
        ++colcount[j];
        j = p.parent[j];
        if (j < 0) break;
      }
    }
  }
  p.Lp.assign(nf + 1, 0);
  for (int j = 0; j < nf; ++j) p.Lp[j + 1] = p.Lp[j] + colcount[j];
  p.nnz_L = p.Lp[nf];
  p.Li.assign(p.nnz_L, 0);
  p.Lx.assign(p.nnz_L, 0.0);
  // ---- numeric up-looking Cholesky ----------------------------------------------------
  {
    std::vector<double> x(nf, 0.0);
    std::vector<int64_t> fill(nf);
    for (int j = 0; j < nf; ++j) fill[j] = p.Lp[j] + 1;
    std::fill(mark.begin(), mark.end(), -1);
    std::vector<int32_t> pattern;
    for (int k = 0; k < nf; ++k) {
      pattern.clear();
      mark[k] = k;
      for (int64_t e = p.Ap[k]; e < p.Ap[k + 1]; ++e) {
        int j = p.Ai[e];
        if (j > k) continue;
        x[j] = p.Ax[e];
        while (j < k && mark[j] != k) {
          mark[j] = k;
          pattern.push_back(j);
          j = p.parent[j];
          if (j < 0) break;
        }
      }
      std::sort(pattern.begin(), pattern.end());
      double d = x[k];
      x[k] = 0.0;
      for (int j : pattern) {
        double lkj = x[j] / p.Lx[p.Lp[j]];
        x[j] = 0.0;
        for (int64_t q = p.Lp[j] + 1; q < fill[j]; ++q) x[p.Li[q]] -= p.Lx[q] * lkj;
        d -= lkj * lkj;
        p.Li[fill[j]] = k;
        p.Lx[fill[j]] = lkj;
        ++fill[j];
      }
      if (!(d > 0) || !std::isfinite(d)) {
        *err = "system matrix not positive definite at row " + std::to_string(k);
        return SIM_ENOTSPD;
      }
      p.Li[p.Lp[k]] = k;
      p.Lx[p.Lp[k]] = std::sqrt(d);
    }
  }
  // ---- row profile of S~ = L~^-1 ----------------------------------------------------------
  p.n_pad = (nf + kTileW - 1) / kTileW * kTileW;
  p.lo.resize(nf);
  p.hi.resize(nf);
  p.rowbase.assign(nf + 1, 0);
  p.nnz_S = 0;
  for (int i = 0; i < nf; ++i) {
    p.lo[i] = p.first_desc[i] / kAlign * kAlign;
    p.hi[i] = std::min(p.n_pad, (i + 1 + kAlign - 1) / kAlign * kAlign);
    p.rowbase[i + 1] = p.rowbase[i] + (p.hi[i] - p.lo[i]);
    p.nnz_S += i - p.first_desc[i] + 1;
  }
  if (build_S) build_sinv_host(p, n_threads);
  // ---- tiles of the device products ------------------------------------------------
  const int RG = kRowGroup, TW = kTileW;
  p.n_rg = (nf + RG - 1) / RG;
  p.n_ct = p.n_pad / TW;
  std::vector<std::vector<std::pair<int32_t, int32_t>>> tiles_of_ct(p.n_ct);  // (rg, values)
  p.tiles1.clear();
  for (int rg = 0; rg < p.n_rg; ++rg) {
    const int r0 = rg * RG, r1 = std::min(nf, r0 + RG);
    int cmin = p.n_pad, cmax = 0;
    for (int r = r0; r < r1; ++r) {
      cmin = std::min(cmin, p.lo[r]);
      cmax = std::max(cmax, p.hi[r]);
    }
    for (int ct = cmin / TW; ct < (cmax + TW - 1) / TW; ++ct) {
      int32_t w = 0;
      for (int r = r0; r < r1; ++r) {
        const int a = std::max(p.lo[r], ct * TW), b = std::min(p.hi[r], (ct + 1) * TW);
        if (b > a) w += b - a;
      }
      if (w == 0) continue;
      p.tiles1.insert(p.tiles1.end(), {rg, ct, w});
      tiles_of_ct[ct].push_back({rg, w});
    }
  }
  p.tiles2.clear();
  for (int ct = 0; ct < p.n_ct; ++ct)
    for (auto& e : tiles_of_ct[ct]) p.tiles2.insert(p.tiles2.end(), {ct, e.first, e.second});
  p.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SIM_OK;
}

void apply_inverse_internal(const Plan& p, const double* b, double* x) {
  const int nf = p.n_free;
  std::vector<double> z(3 * (size_t)nf, 0.0);
  for (int i = 0; i < nf; ++i) {
    double s0 = 0, s1 = 0, s2 = 0;
    const double* row = &p.S[p.rowbase[i]];
    int c1 = std::min(p.hi[i], nf);
    for (int c = p.lo[i]; c < c1; ++c) {
      double s = row[c - p.lo[i]];
      s0 += s * b[3 * c];
      s1 += s * b[3 * c + 1];
      s2 += s * b[3 * c + 2];
    }
    z[3 * i] = s0;
    z[3 * i + 1] = s1;
    z[3 * i + 2] = s2;
  }
  std::fill(x, x + 3 * (size_t)nf, 0.0);
  for (int i = 0; i < nf; ++i) {
    const double* row = &p.S[p.rowbase[i]];
    int c1 = std::min(p.hi[i], nf);
    for (int c = p.lo[i]; c < c1; ++c) {
      double s = row[c - p.lo[i]];
      x[3 * c] += s * z[3 * i];
      x[3 * c + 1] += s * z[3 * i + 1];
      x[3 * c + 2] += s * z[3 * i + 2];
    }
  }
}

void build_stream_schedule(const Plan& p, bool pass2, int grid, double zero_cost,
                           StreamSchedule* out) {
  const std::vector<int32_t>& T = pass2 ? p.tiles2 : p.tiles1;
  const int nt = (int)T.size() / 3;
  const int n_keys = pass2 ? p.n_ct : p.n_rg;
  grid = std::max(1, grid);
  // cost of a tile: its stored values plus a share of the loads issued for its empty
  // positions (those are served from the zero page in L1, not from memory)
  std::vector<double> pre(nt + 1, 0.0);
  for (int t = 0; t < nt; ++t)
    pre[t + 1] = pre[t] + T[3 * t + 2] + zero_cost * (kRowGroup * kTileW - T[3 * t + 2]);
  out->tiles.resize(2 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    out->tiles[2 * t] = T[3 * t];
    out->tiles[2 * t + 1] = T[3 * t + 1];
  }
  out->cta_first.assign(grid + 1, nt);
  int t = 0;
  for (int c = 0; c < grid; ++c) {
    const double target = pre[nt] * c / grid;
    while (t < nt && pre[t + 1] <= target) ++t;
    out->cta_first[c] = t;
  }
  out->cta_first[grid] = nt;
  for (int c = 1; c <= grid; ++c) out->cta_first[c] = std::max(out->cta_first[c], out->cta_first[c - 1]);
  // distinct second coordinates (pass 1: column tiles) of each CTA's range
  out->cta_col_first.assign(grid + 1, 0);
  out->cta_cols.clear();
  out->tile_col_slot.assign(nt, 0);
  out->max_cols = 0;
  for (int c = 0; c < grid; ++c) {
    out->cta_col_first[c] = (int)out->cta_cols.size();
    const int first = (int)out->cta_cols.size();
    for (int u = out->cta_first[c]; u < out->cta_first[c + 1]; ++u) {
      const int col = T[3 * u + 1];
      int pos = -1;
      for (int k = first; k < (int)out->cta_cols.size(); ++k)
        if (out->cta_cols[k] == col) pos = k - first;
      if (pos < 0) {
        pos = (int)out->cta_cols.size() - first;
        out->cta_cols.push_back(col);
      }
      out->tile_col_slot[u] = pos;
    }
    out->max_cols = std::max(out->max_cols, (int)out->cta_cols.size() - first);
  }
  out->cta_col_first[grid] = (int)out->cta_cols.size();
  // partial-sum slots: one per run of equal keys inside a CTA's range, numbered CTA by
  // CTA, so the slots of each key are contiguous and in a fixed order
  out->seg_base.assign(grid, 0);
  out->seg_first.assign(n_keys + 1, -1);
  int slot = 0;
  for (int c = 0; c < grid; ++c) {
    out->seg_base[c] = slot;
    int prev = -1;
    for (int u = out->cta_first[c]; u < out->cta_first[c + 1]; ++u) {
      const int key = T[3 * u];
      if (key != prev) {
        if (out->seg_first[key] < 0) out->seg_first[key] = slot;
        ++slot;
        prev = key;
      }
    }
  }
  out->n_seg = slot;
  out->seg_first[n_keys] = slot;
  for (int k = n_keys - 1; k >= 0; --k)
    if (out->seg_first[k] < 0) out->seg_first[k] = out->seg_first[k + 1];
}

}  // namespace silg

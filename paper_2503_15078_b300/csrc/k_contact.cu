// Contacts: detection and linearisation (App. A.1), the Delassus operator W = H S^T S H^T
// and its diagonal preconditioner (Sec. 5.3-5.4, Eqs. 27-28), the Fischer-Burmeister
// evaluation of indicators, compliances and NCP values (App. B.2, Eqs. 52-57; Eq. 19), the
// Schur right-hand side J A^-1 g (Alg. 4), the conjugate-residual solve (Sec. 6) and the
// correction S (J^T dlambda) that enters the second profile product.
//
// W has the per-vertex structure W_jk = W~(v_j, v_k) D_j D_k^T (A = A~ (x) I3, D_j the
// contact frame rows n, f1, f2), so only W~ = Y^T Y over the distinct contact vertices is
// formed, with Y = S~ restricted to the contact-vertex columns. Column v of S~ is non-zero
// exactly on the ancestors of v (Theorem 1), so Y lives on U = the union of those
// ancestors; in postorder, row a of Y is non-zero on the contiguous run of contact
// vertices inside a's subtree [fd(a), a].
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "fb.cuh"

namespace cg = cooperative_groups;

namespace silg {
namespace {

constexpr int kCrThreads = 256;

// W~ is stored row-major with its leading dimension padded to a multiple of 4 floats
// (zero padding), so rows can be read with 16-byte vector loads.
__host__ __device__ __forceinline__ int wt_ld(int ncv) { return (ncv + 3) & ~3; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


__device__ void tangent_frame(const double* n, double* f1, double* f2) {
  int k = 0;
  if (fabs(n[1]) < fabs(n[k])) k = 1;
  if (fabs(n[2]) < fabs(n[k])) k = 2;
  double e[3] = {0, 0, 0};
  e[k] = 1.0;
  double en = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
  double t[3] = {e[0] - en * n[0], e[1] - en * n[1], e[2] - en * n[2]};
  double inv = 1.0 / sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  f1[0] = t[0] * inv;
  f1[1] = t[1] * inv;
  f1[2] = t[2] * inv;
  f2[0] = n[1] * f1[2] - n[2] * f1[1];
  f2[1] = n[2] * f1[0] - n[0] * f1[2];
  f2[2] = n[0] * f1[1] - n[1] * f1[0];
}

// signed distance, outward normal and closest surface point of x to an obstacle
__device__ double obst_query(const ObstDev& o, const double* x, double* n, double* ph) {
  if (o.kind == SIM_OBST_PLANE) {
    double phi = o.a[0] * (x[0] - o.p[0]) + o.a[1] * (x[1] - o.p[1]) + o.a[2] * (x[2] - o.p[2]);
    for (int r = 0; r < 3; ++r) {
      n[r] = o.a[r];
      ph[r] = x[r] - phi * o.a[r];
    }
    return phi;
  }
  double dd[3] = {x[0] - o.p[0], x[1] - o.p[1], x[2] - o.p[2]};
  double axial = dd[0] * o.a[0] + dd[1] * o.a[1] + dd[2] * o.a[2];
  double rad[3] = {dd[0] - axial * o.a[0], dd[1] - axial * o.a[1], dd[2] - axial * o.a[2]};
  double rho = sqrt(rad[0] * rad[0] + rad[1] * rad[1] + rad[2] * rad[2]);
  if (rho == 0.0) {
    double f2[3];
    tangent_frame(o.a, n, f2);
  } else {
    for (int r = 0; r < 3; ++r) n[r] = rad[r] / rho;
  }
  for (int r = 0; r < 3; ++r) ph[r] = o.p[r] + axial * o.a[r] + o.radius * n[r];
  return rho - o.radius;
}

// Signed distance in FP32 as a conservative filter: pairs clearly farther than the margin
// are rejected without FP64 work; every pair within kPrefilterSlack of the margin is
// decided by the FP64 query, exactly as in FP64 arithmetic throughout.
constexpr float kPrefilterSlack = 1e-3f;
__device__ __forceinline__ bool maybe_contact(const ObstDev& o, const double* x, double margin) {
  const float px = (float)(x[0] - o.p[0]), py = (float)(x[1] - o.p[1]), pz = (float)(x[2] - o.p[2]);
  const float ax = (float)o.a[0], ay = (float)o.a[1], az = (float)o.a[2];
  float phi;
  if (o.kind == SIM_OBST_PLANE) {
    phi = ax * px + ay * py + az * pz;
  } else {
    const float axial = ax * px + ay * py + az * pz;
    const float rx = px - axial * ax, ry = py - axial * ay, rz = pz - axial * az;
    phi = sqrtf(rx * rx + ry * ry + rz * rz) - (float)o.radius;
  }
  const float scale = fabsf(px) + fabsf(py) + fabsf(pz) + (float)o.radius + (float)fabs(margin);
  return phi < (float)margin + kPrefilterSlack * scale;
}

// Closest point of the triangle abc to x by the Voronoi-region method (Ericson, Real-Time
// Collision Detection, Sec. 5.1.5): the corner regions, then the edge regions, else the
// interior. Writes the barycentric weights w (exact zeros away from the corner or edge
// found); returns whether the point lies inside the triangle (all weights positive).
__device__ bool tri_closest(const double* x, const double* a, const double* b, const double* c,
                            double* w) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int r = 0; r < 3; ++r) {
    ab[r] = b[r] - a[r];
    ac[r] = c[r] - a[r];
    ap[r] = x[r] - a[r];
    bp[r] = x[r] - b[r];
    cp[r] = x[r] - c[r];
  }
  auto dot = [](const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
  w[0] = w[1] = w[2] = 0.0;
  const double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) { w[0] = 1.0; return false; }
  const double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) { w[1] = 1.0; return false; }
  const double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double t = d1 / (d1 - d3);
    w[0] = 1.0 - t;
    w[1] = t;
    return false;
  }
  const double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) { w[2] = 1.0; return false; }
  const double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double t = d2 / (d2 - d6);
    w[0] = 1.0 - t;
    w[2] = t;
    return false;
  }
  const double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && d4 - d3 >= 0.0 && d5 - d6 >= 0.0) {
    const double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    w[1] = 1.0 - t;
    w[2] = t;
    return false;
  }
  const double inv = 1.0 / (va + vb + vc);
  w[0] = va * inv;
  w[1] = vb * inv;
  w[2] = vc * inv;
  return true;
}

__device__ __forceinline__ void load3(const double* src, int v, double* o) {
  o[0] = src[3 * v];
  o[1] = src[3 * v + 1];
  o[2] = src[3 * v + 2];
}

// bounds of every body's triangle corners at the predicted positions (one CTA per body)
constexpr int kBoxThreads = 128;
__global__ void __launch_bounds__(kBoxThreads) k_body_box(DevSim d) {
  const int b = blockIdx.x;
  __shared__ double red[6][kBoxThreads];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int t = d.body_toff[b] + threadIdx.x; t < d.body_toff[b + 1]; t += blockDim.x) {
    const int4 tv = d.btri[t];
    const int cs[3] = {tv.x, tv.y, tv.z};
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) {
        const double v = d.s_tilde[3 * cs[k] + r];
        lo[r] = fmin(lo[r], v);
        hi[r] = fmax(hi[r], v);
      }
  }
  for (int r = 0; r < 3; ++r) {
    red[r][threadIdx.x] = lo[r];
    red[3 + r][threadIdx.x] = hi[r];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int r = 0; r < 3; ++r) {
        red[r][threadIdx.x] = fmin(red[r][threadIdx.x], red[r][threadIdx.x + w]);
        red[3 + r][threadIdx.x] = fmax(red[3 + r][threadIdx.x], red[3 + r][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) d.body_box[6 * b + threadIdx.x] = red[threadIdx.x][0];
}

// bounds of every triangle and of every run of kTriChunk consecutive triangles, in FP32
// rounded outward (runs may straddle two bodies: the bounds then cover both parts, still a
// bound for either). One warp per run, a lane per triangle.
__global__ void k_chunk_box(DevSim d) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int t = c * kTriChunk + lane;
  const bool own = lane < kTriChunk && t < d.n_btri;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  if (own) {
    const int4 tv = d.btri[t];
    const int cs[3] = {tv.x, tv.y, tv.z};
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) {
        const double v = d.s_tilde[3 * cs[k] + r];
        lo[r] = fminf(lo[r], __double2float_rd(v));
        hi[r] = fmaxf(hi[r], __double2float_ru(v));
      }
    for (int r = 0; r < 3; ++r) {
      d.tri_box[6 * t + r] = lo[r];
      d.tri_box[6 * t + 3 + r] = hi[r];
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int r = 0; r < 3; ++r) {
      lo[r] = fminf(lo[r], __shfl_xor_sync(0xffffffffu, lo[r], o));
      hi[r] = fmaxf(hi[r], __shfl_xor_sync(0xffffffffu, hi[r], o));
    }
  if (lane < 6 && c * kTriChunk < d.n_btri) d.chunk_box[6 * c + lane] = lane < 3 ? lo[lane] : hi[lane - 3];
}

// bounds of every run of kTriSuper triangles from its runs' bounds (one thread per run)
__global__ void k_super_box(DevSim d) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = u * (kTriSuper / kTriChunk);
  const int c1 = min(c0 + kTriSuper / kTriChunk, (d.n_btri + kTriChunk - 1) / kTriChunk);
  if (c0 >= c1) return;
  float b[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
  for (int c = c0; c < c1; ++c)
    for (int r = 0; r < 3; ++r) {
      b[r] = fminf(b[r], d.chunk_box[6 * c + r]);
      b[3 + r] = fmaxf(b[3 + r], d.chunk_box[6 * c + 3 + r]);
    }
  for (int r = 0; r < 6; ++r) d.super_box[6 * u + r] = b[r];
}

__device__ __forceinline__ bool far_from(const float* box, const float* x, float lim) {
  return x[0] < box[0] - lim || x[1] < box[1] - lim || x[2] < box[2] - lim ||
         x[0] > box[3] + lim || x[1] > box[4] + lim || x[2] > box[5] + lim;
}

// The body contact of free vertex i, if any (bc_tri, bc_w, bc_n): the nearest surface
// triangle of another body of its scene (distance to the closest point, then the
// triangle's number), accepted when its gap g lies in (-2 margin, margin). Only triangles
// within 2 margins can be accepted, so bodies and triangles farther than that (bounds
// padded by a relative 1e-6) are skipped without changing the choice.
__device__ bool body_match(const DevSim& d, int i, const double* x, double margin) {
  const int vb = d.vert_body[i];
  d.bc_tri[i] = -1;
  if (vb < 0) return false;
  const int sc = d.vert_scene[i];
  // the culling runs in FP32 on bounds rounded outward, with the limit padded by a relative
  // 1e-5 (far above FP32 rounding of x and of the subtraction): it only ever keeps more
  const double ax = fabs(x[0]) + fabs(x[1]) + fabs(x[2]);
  const float lim = __double2float_ru(2.0 * margin * (1.0 + 1e-5) + 1e-5 * ax);
  const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
  double best_d = 1e300, bw[3] = {0.0, 0.0, 0.0};
  int best = -1, best_id = 0;
  bool best_in = false;
  for (int b = d.scene_bfirst[sc]; b < d.scene_bfirst[sc + 1]; ++b) {
    if (b == vb) continue;
    const double* bx = d.body_box + 6 * b;
    const float bxf[6] = {__double2float_rd(bx[0]), __double2float_rd(bx[1]),
                          __double2float_rd(bx[2]), __double2float_ru(bx[3]),
                          __double2float_ru(bx[4]), __double2float_ru(bx[5])};
    if (far_from(bxf, xf, lim)) continue;
    const int te = d.body_toff[b + 1];
    for (int t = d.body_toff[b]; t < te; ++t) {
      // skip the rest of a run of triangles whose bounds are farther than the limit: first
      // the runs of kTriSuper, then those of kTriChunk
      if ((t == d.body_toff[b] || t % kTriSuper == 0) &&
          far_from(d.super_box + 6 * (t / kTriSuper), xf, lim)) {
        t = min(te, (t / kTriSuper + 1) * kTriSuper) - 1;
        continue;
      }
      if ((t == d.body_toff[b] || t % kTriChunk == 0) &&
          far_from(d.chunk_box + 6 * (t / kTriChunk), xf, lim)) {
        t = min(te, (t / kTriChunk + 1) * kTriChunk) - 1;
        continue;
      }
      if (far_from(d.tri_box + 6 * t, xf, lim)) continue;
      const int4 tv = d.btri[t];
      double a[3], bb[3], c[3];
      load3(d.s_tilde, tv.x, a);
      load3(d.s_tilde, tv.y, bb);
      load3(d.s_tilde, tv.z, c);
      double w[3];
      const bool in = tri_closest(x, a, bb, c, w);
      double e[3];
      for (int r = 0; r < 3; ++r) e[r] = x[r] - (w[0] * a[r] + w[1] * bb[r] + w[2] * c[r]);
      const double dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      if (dist < best_d || (dist == best_d && tv.w < best_id)) {
        best_d = dist;
        best = t;
        best_id = tv.w;
        best_in = in;
        for (int k = 0; k < 3; ++k) bw[k] = w[k];
      }
    }
  }
  if (best < 0) return false;
  const int4 tv = d.btri[best];
  double a[3], bb[3], c[3];
  load3(d.s_tilde, tv.x, a);
  load3(d.s_tilde, tv.y, bb);
  load3(d.s_tilde, tv.z, c);
  double e1[3], e2[3], m[3], e[3];
  for (int r = 0; r < 3; ++r) {
    e1[r] = bb[r] - a[r];
    e2[r] = c[r] - a[r];
    e[r] = x[r] - (bw[0] * a[r] + bw[1] * bb[r] + bw[2] * c[r]);
  }
  m[0] = e1[1] * e2[2] - e1[2] * e2[1];
  m[1] = e1[2] * e2[0] - e1[0] * e2[2];
  m[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int r = 0; r < 3; ++r) m[r] /= mn;
  const double g = best_in ? m[0] * e[0] + m[1] * e[1] + m[2] * e[2] : best_d;
  if (!(g > -2.0 * margin && g < margin)) return false;
  for (int r = 0; r < 3; ++r) {
    d.bc_n[3 * i + r] = best_d > 0.0 ? e[r] / g : m[r];
    d.bc_w[3 * i + r] = bw[r];
  }
  d.bc_tri[i] = best;
  return true;
}

__global__ void k_collide_count(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double x[3] = {d.s_tilde[3 * i], d.s_tilde[3 * i + 1], d.s_tilde[3 * i + 2]};
  const int sc = d.vert_scene[i];
  const double margin = d.scene_margin[sc];
  int cnt = 0;
  for (int o = 0; o < d.n_obs; ++o) {
    if (d.obst_scene[o] != sc || !maybe_contact(d.obst[o], x, margin)) continue;
    double nn[3], ph[3];
    if (obst_query(d.obst[o], x, nn, ph) < margin) ++cnt;
  }
  if (d.n_anc > 0 && d.anc_of[i] >= 0) ++cnt;   // its anchor: one more slot, after the obstacles
  if (d.map_on) {
    d.x_cnt[i] = 0;
    d.x_fill[i] = 0;
  }
  // its contact with another body: one more slot, after the anchor
  if (d.bc_on && body_match(d, i, x, margin)) ++cnt;
  d.ct_cnt[i] = cnt;
  d.cv_flag[i] = cnt > 0;
}

// a matched triangle's corners (non-zero weights) become contact vertices and count one
// corner term each
__global__ void k_corner_flag(DevSim d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  // the partner of a two-vertex anchor row at i: a contact vertex with one corner term
  const int a = d.n_anc > 0 ? d.anc_of[i] : -1;
  if (a >= 0 && d.anc_partner[a] >= 0) {
    d.cv_flag[d.anc_partner[a]] = 1;
    atomicAdd(d.x_cnt + d.anc_partner[a], 1);
  }
  if (!d.bc_on) return;
  const int t = d.bc_tri[i];
  if (t < 0) return;
  const int4 tv = d.btri[t];
  const int cs[3] = {tv.x, tv.y, tv.z};
  for (int k = 0; k < 3; ++k)
    if (d.bc_w[3 * i + k] != 0.0) {
      d.cv_flag[cs[k]] = 1;
      atomicAdd(d.x_cnt + cs[k], 1);
    }
}

// each vertex's corner terms in ascending order (the fill order above is not fixed)
__global__ void k_corner_sort(DevSim d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const int b = d.x_off[i], e = min(d.x_off[i + 1], 3 * d.cap);
  for (int p = b + 1; p < e; ++p) {
    const int key = d.x_list[p];
    int q = p - 1;
    while (q >= b && d.x_list[q] > key) {
      d.x_list[q + 1] = d.x_list[q];
      --q;
    }
    d.x_list[q + 1] = key;
  }
}

__global__ void k_collide_write(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (d.ct_off[d.n] > d.cap || d.cv_off[d.n] > d.cap)) atomicOr(d.err, kErrCapacity);
  if (i >= d.n || (d.ct_cnt[i] == 0 && !d.cv_flag[i])) return;
  double x[3] = {d.s_tilde[3 * i], d.s_tilde[3 * i + 1], d.s_tilde[3 * i + 2]};
  int j = d.ct_off[i];
  const int cv = d.cv_off[i];
  if (cv < d.cap) {
    d.cv_vert[cv] = i;
    d.cv_first[cv] = j;
    d.cv_nct[cv] = d.ct_cnt[i];
  }
  const int sc = d.vert_scene[i];
  const double margin = d.scene_margin[sc];
  for (int o = 0; o < d.n_obs; ++o) {
    const ObstDev& ob = d.obst[o];
    if (d.obst_scene[o] != sc || !maybe_contact(ob, x, margin)) continue;
    double n[3], ph[3];
    if (!(obst_query(ob, x, n, ph) < margin)) continue;
    if (j < d.cap) {
      double f1[3], f2[3];
      tangent_frame(n, f1, f2);
      for (int r = 0; r < 3; ++r) {
        d.ct_D[9 * j + r] = n[r];
        d.ct_D[9 * j + 3 + r] = f1[r];
        d.ct_D[9 * j + 6 + r] = f2[r];
      }
      d.ct_vert[j] = i;
      d.ct_obst[j] = o;
      d.ct_cv[j] = cv;
      if (d.map_on) d.ct_tri[j] = -1;
      d.ct_dn[j] = n[0] * ph[0] + n[1] * ph[1] + n[2] * ph[2];
      d.ct_df[2 * j] = f1[0] * ob.vel[0] + f1[1] * ob.vel[1] + f1[2] * ob.vel[2];
      d.ct_df[2 * j + 1] = f2[0] * ob.vel[0] + f2[1] * ob.vel[1] + f2[2] * ob.vel[2];
      d.ct_mu[j] = ob.mu;
    }
    ++j;
  }
  const int a = d.n_anc > 0 ? d.anc_of[i] : -1;
  const int pb = a >= 0 ? d.anc_partner[a] : -1;   // the partner of a two-vertex row
  if (a >= 0 && j < d.cap) {
    // the anchor's slot: rows e_x, e_y, e_z; the target (or target offset, at the frame's
    // end) in ct_dn and ct_df; the compliance in ct_mu
    for (int r = 0; r < 9; ++r) d.ct_D[9 * j + r] = (r % 4 == 0) ? 1.0 : 0.0;
    d.ct_vert[j] = i;
    d.ct_obst[j] = d.n_obs + a;
    d.ct_cv[j] = cv;
    d.ct_dn[j] = d.anc_pos[3 * a];
    d.ct_df[2 * j] = d.anc_pos[3 * a + 1];
    d.ct_df[2 * j + 1] = d.anc_pos[3 * a + 2];
    d.ct_mu[j] = d.anc_e[a];
    if (d.map_on) d.ct_tri[j] = -1;
    if (pb >= 0) {
      // a two-vertex row: the map x_i - 1 x_partner (a one-corner map entry, weight 1)
      d.ct_tri[j] = d.anc_ptri[a];
      d.ct_bw[3 * j] = 1.0;
      d.ct_bw[3 * j + 1] = d.ct_bw[3 * j + 2] = 0.0;
      const int cc = d.cv_off[pb];
      d.ct_tcv[3 * j] = cc < d.cap ? cc : -1;
      d.ct_tcv[3 * j + 1] = d.ct_tcv[3 * j + 2] = -1;
      const int pos = d.x_off[pb] + atomicAdd(d.x_fill + pb, 1);
      if (pos < 3 * d.cap) d.x_list[pos] = 3 * j;
    }
  } else if (a >= 0 && pb >= 0) {
    // beyond the capacity (the frame reports SIM_ECAPACITY): the counted corner term is
    // filled with -1, which every reader skips
    const int pos = d.x_off[pb] + atomicAdd(d.x_fill + pb, 1);
    if (pos < 3 * d.cap) d.x_list[pos] = -1;
  }
  if (a >= 0) ++j;
  const int t = d.bc_on ? d.bc_tri[i] : -1;
  if (t >= 0 && j >= d.cap) {
    // beyond the capacity (the frame reports SIM_ECAPACITY): its counted corner terms are
    // filled with -1, which every reader skips
    for (int k = 0; k < 3; ++k) {
      if (d.bc_w[3 * i + k] == 0.0) continue;
      const int4 tv = d.btri[t];
      const int ck = k == 0 ? tv.x : (k == 1 ? tv.y : tv.z);
      const int pos = d.x_off[ck] + atomicAdd(d.x_fill + ck, 1);
      if (pos < 3 * d.cap) d.x_list[pos] = -1;
    }
  }
  if (t >= 0 && j < d.cap) {
    // the contact with another body: rows (n, f1, f2), the map x_i - sum_k w_k x_k, d = 0;
    // the id -1 - the triangle's number; each corner with a non-zero weight gets a term
    double n[3], f1[3], f2[3];
    for (int r = 0; r < 3; ++r) n[r] = d.bc_n[3 * i + r];
    tangent_frame(n, f1, f2);
    for (int r = 0; r < 3; ++r) {
      d.ct_D[9 * j + r] = n[r];
      d.ct_D[9 * j + 3 + r] = f1[r];
      d.ct_D[9 * j + 6 + r] = f2[r];
    }
    const int4 tv = d.btri[t];
    d.ct_vert[j] = i;
    d.ct_obst[j] = -1 - tv.w;
    d.ct_cv[j] = cv;
    d.ct_dn[j] = 0.0;
    d.ct_df[2 * j] = d.ct_df[2 * j + 1] = 0.0;
    d.ct_mu[j] = d.scene_bmu[sc];
    d.ct_tri[j] = t;
    const int cs[3] = {tv.x, tv.y, tv.z};
    for (int k = 0; k < 3; ++k) {
      const double w = d.bc_w[3 * i + k];
      d.ct_bw[3 * j + k] = w;
      d.ct_tcv[3 * j + k] = -1;
      if (w == 0.0) continue;
      const int cc = d.cv_off[cs[k]];
      if (cc < d.cap) d.ct_tcv[3 * j + k] = cc;
      const int pos = d.x_off[cs[k]] + atomicAdd(d.x_fill + cs[k], 1);
      if (pos < 3 * d.cap) d.x_list[pos] = 3 * j + k;
    }
  }
}

// single-CTA exclusive scan: out[k] = sum in[0..k), out[len] = total; *total = total. The
// length is n_static, or the device count *n_dev capped at n_static (the arrays' size).
// The array is walked in coalesced tiles of 4 x blockDim elements (each thread scans four
// consecutive values), with the running total carried from tile to tile.
// one tile of 4 x blockDim elements from `base`, exclusive, starting from `carry`; returns
// the tile's sum
__device__ __forceinline__ int scan_tile(const int* in, int* out, int n, int base, int carry,
                                         int* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int idx = base + 4 * tid;
  int v0 = idx < n ? in[idx] : 0, v1 = idx + 1 < n ? in[idx + 1] : 0;
  int v2 = idx + 2 < n ? in[idx + 2] : 0, v3 = idx + 3 < n ? in[idx + 3] : 0;
  const int sum4 = v0 + v1 + v2 + v3;
  int incl = sum4;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int run = carry + (wid > 0 ? wsum[wid - 1] : 0) + incl - sum4;
  if (idx < n) out[idx] = run;
  run += v0;
  if (idx + 1 < n) out[idx + 1] = run;
  run += v1;
  if (idx + 2 < n) out[idx + 2] = run;
  run += v2;
  if (idx + 3 < n) out[idx + 3] = run;
  const int tile_sum = wsum[31];
  __syncthreads();
  return tile_sum;
}

__device__ __forceinline__ int scan_len(int n_static, const int* n_dev) {
  const int n = n_dev ? min(*n_dev, n_static) : n_static;
  return n < 0 ? 0 : n;
}

__global__ void __launch_bounds__(1024) k_scan(const int* in, int* out, int n_static,
                                               const int* n_dev, int* total, const int* skip) {
  if (skip && *skip) return;
  __shared__ int wsum[32];
  const int n = scan_len(n_static, n_dev);
  int carry = 0;
  for (int base = 0; base < n; base += 4 * blockDim.x)
    carry += scan_tile(in, out, n, base, carry, wsum);
  if (threadIdx.x == 0) {
    out[n] = carry;
    if (total) *total = carry;
  }
}

// Long arrays in two passes, one CTA per tile: the tiles' sums, their scan (k_scan on
// them), then every tile scanned from its offset.
constexpr int kScanTile = 4096;     // elements per tile: 1024 threads x 4
constexpr int kScanSplit = 65536;   // arrays longer than this take the two-pass scan
__global__ void __launch_bounds__(1024) k_scan_tiles(const int* in, int n_static,
                                                     const int* n_dev, int* part,
                                                     const int* skip) {
  if (skip && *skip) return;
  __shared__ int wsum[32];
  const int n = scan_len(n_static, n_dev);
  const int idx = blockIdx.x * kScanTile + 4 * threadIdx.x;
  int v = 0;
  for (int q = 0; q < 4; ++q) v += idx + q < n ? in[idx + q] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) part[blockIdx.x] = w;
  }
}
__global__ void __launch_bounds__(1024) k_scan_fin(const int* in, int* out, int n_static,
                                                   const int* n_dev, const int* part_off,
                                                   int n_tiles, int* total, const int* skip) {
  if (skip && *skip) return;
  __shared__ int wsum[32];
  const int n = scan_len(n_static, n_dev);
  const int base = blockIdx.x * kScanTile;
  if (base < n) scan_tile(in, out, n, base, part_off[blockIdx.x], wsum);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[n] = part_off[n_tiles];
    if (total) *total = part_off[n_tiles];
  }
}

__device__ __forceinline__ int lower_bound_i(const int* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Whether this frame's contact vertices are the previous frame's (same count, same sorted
// list): then Y and W~ = Y^T Y, functions of that list alone, are kept, and the kernels that
// build them return at once. Not after an error, nor when the previous list is unknown
// (creation, sim_set_state, a new start mode). One CTA; records the list for the next frame.
__global__ void __launch_bounds__(1024) k_dl_check(DevSim d) {
  __shared__ int differs;
  const int ncv_raw = d.counters[kCntCv], ncv = min(ncv_raw, d.cap);
  const int prev = d.dl_state[1];
  if (threadIdx.x == 0)
    differs = !d.dl_reuse_on || prev < 0 || prev != ncv_raw || ncv_raw > d.cap || *d.err != 0;
  __syncthreads();
  if (!differs)
    for (int i = threadIdx.x; i < ncv; i += blockDim.x)
      if (d.cv_vert[i] != d.dl_prev_cv[i]) differs = 1;
  __syncthreads();
  for (int i = threadIdx.x; i < ncv; i += blockDim.x) d.dl_prev_cv[i] = d.cv_vert[i];
  if (threadIdx.x == 0) {
    d.dl_state[0] = !differs;
    d.dl_state[1] = ncv_raw <= d.cap ? ncv_raw : -1;
    d.dl_state[2] += !differs;
  }
}

// rows of U: a is an ancestor of some contact vertex iff its subtree [fd(a), a] holds one
__global__ void k_u_flag(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.n) return;
  int ncv = min(d.counters[kCntCv], d.cap);
  int clo = lower_bound_i(d.cv_vert, ncv, d.first_desc[a]);
  int chi = lower_bound_i(d.cv_vert, ncv, a + 1);
  d.u_flag[a] = chi > clo;
  d.row_clo[a] = clo;
  d.row_len[a] = chi - clo;
}

__global__ void k_u_compact(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.n || !d.u_flag[a]) return;
  int idx = d.u_off[a];
  d.u_list[idx] = a;
  d.u_clo[idx] = d.row_clo[a];
  d.u_len[idx] = d.row_len[a];
}

__global__ void k_yc_len(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int ncv = min(d.counters[kCntCv], d.cap);
  if (c >= ncv) return;
  d.yc_len[c] = d.depth[d.cv_vert[c]];
}

// Y rows (row-major over U) and Y columns (contact vertex major, bottom-up along the
// ancestor path) gathered from the S~ profile.
__global__ void k_y_gather(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  const int lane = threadIdx.x & 31, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nU = d.counters[kCntU];
  if (d.y_ptr[nU] > d.cap_y || d.yc_ptr[min(d.counters[kCntCv], d.cap)] > d.cap_y) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(d.err, kErrYCapacity);
    return;
  }
  // warps walk the rows of U with a grid stride (the grid is sized for the SMs)
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nU; w += nwarps) {
    const int a = d.u_list[w];
    const int clo = d.u_clo[w], len = d.u_len[w];
    const float* srow = d.S + (d.rowbase[a] - d.lo[a]);
    const int base = d.y_ptr[w];
    const int da = d.depth[a];
    for (int k = lane; k < len; k += 32) {
      const int c = clo + k;
      const int v = d.cv_vert[c];
      const float val = srow[v];
      d.y_val[base + k] = val;
      const int pos = d.yc_ptr[c] + d.depth[v] - da;
      d.yc_val[pos] = val;
      d.yc_row[pos] = a;
    }
  }
}

// W~ = Y^T Y (FP32) as a block-sparse product. Y has one row per ancestor row a of a
// contact vertex (the set U, in elimination-tree postorder) and is non-zero only on the
// contact vertices of a's subtree, a contiguous interval [clo_a, clo_a + len_a). Rows are
// taken in blocks of kWtKB; a block contributes to the output tile (I, J) only if the
// union of its rows' intervals meets both column blocks, so the lower-level blocks of the
// tree drop out of every off-diagonal tile. Work items are (lower-triangle tile, K split):
// the split count S is chosen on the device from the contact-vertex count so that there
// are about as many items as resident CTAs; each item sums its share of the tile's
// contributing row blocks into a partial tile, and k_wt_reduce adds the S partials in a
// fixed order (deterministic) and writes both triangles and the zero padding.
constexpr int kWtT = 64;         // output tile
constexpr int kWtKB = 32;        // rows of Y per block
constexpr int kWtThreads = 128;  // 8 x 4 outputs per thread
constexpr int kWtList = 1024;    // row blocks staged per round

// K splits for ntiles tiles so that there are about `target` work items
__device__ __forceinline__ int wt_splits(int ntiles, int target) {
  return ntiles > 0 ? min(kWtMaxSplit, max(1, (target + ntiles - 1) / ntiles)) : 1;
}

// tile t of the list of every scene's lower-triangle tiles -> scene, block row I, column J
__device__ __forceinline__ int tile_scene(const DevSim& d, int t) {
  int lo = 0, hi = d.n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.sc_tileoff[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void tri_decode(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// Per-scene ranges of the contact lists (contacts and contact vertices are sorted by
// internal vertex, and vertices are ordered scene by scene), the scenes' W~ blocks and
// their tiles. One CTA; the scans over scenes are serial.
__global__ void k_scene_ranges(DevSim d) {
  const int ncv = min(d.counters[kCntCv], d.cap), c = min(d.counters[kCntContacts], d.cap);
  for (int sc = threadIdx.x; sc <= d.n_scenes; sc += blockDim.x) {
    const int cvb = lower_bound_i(d.cv_vert, ncv, d.scene_vfirst[sc]);
    d.sc_cvb[sc] = cvb;
    d.sc_jb[sc] = cvb < ncv ? min(d.cv_first[cvb], c) : c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long off = 0;
    int toff = 0;
    for (int sc = 0; sc < d.n_scenes; ++sc) {
      const int nv = d.sc_cvb[sc + 1] - d.sc_cvb[sc], ld = wt_ld(nv), nb = (nv + kWtT - 1) / kWtT;
      d.sc_ld[sc] = ld;
      d.sc_wtoff[sc] = off;
      d.sc_tileoff[sc] = toff;
      off += (long long)nv * ld;
      toff += nb * (nb + 1) / 2;
    }
    d.sc_wtoff[d.n_scenes] = off;
    d.sc_tileoff[d.n_scenes] = toff;
  }
}

// union of the contact-vertex intervals of each block of kWtKB rows of U
__global__ void k_wt_blocks(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  const int kb = blockIdx.x * blockDim.x + threadIdx.x;
  const int nU = d.counters[kCntU];
  if (kb * kWtKB >= nU) return;
  int lo = 1 << 30, hi = -1;
  for (int u = kb * kWtKB; u < min(nU, (kb + 1) * kWtKB); ++u) {
    lo = min(lo, d.u_clo[u]);
    hi = max(hi, d.u_clo[u] + d.u_len[u]);
  }
  d.kb_lo[kb] = lo;
  d.kb_hi[kb] = hi;
}

__global__ void __launch_bounds__(kWtThreads) k_wt_items(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  const int ncv = min(d.counters[kCntCv], d.cap);
  const int nU = d.counters[kCntU];
  if (ncv == 0 || nU == 0 || d.y_ptr[nU] > d.cap_y) return;
  const int ntiles = d.sc_tileoff[d.n_scenes], S = wt_splits(ntiles, d.wt_grid);
  const int nitems = ntiles * S;
  const int nkb = (nU + kWtKB - 1) / kWtKB;
  __shared__ __align__(16) float As[kWtKB][kWtT];
  __shared__ __align__(16) float Bs[kWtKB][kWtT];
  __shared__ int kbl[kWtList];
  __shared__ int list_n;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ty = t >> 4, tx = t & 15;  // outputs rows 8 ty .. +7, columns 4 tx .. +3
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item / S, sp = item - tile * S;
    const int sc = tile_scene(d, tile);
    int I, J;
    tri_decode(tile - d.sc_tileoff[sc], I, J);
    // global contact-vertex ranges of the tile's rows and columns
    const int cvb = d.sc_cvb[sc], cve = d.sc_cvb[sc + 1];
    const int a0 = cvb + I * kWtT, b0 = cvb + J * kWtT;
    const int a1 = min(a0 + kWtT, cve), b1 = min(b0 + kWtT, cve);
    const bool diag = I == J;
    // contributing row blocks, counted by every warp alike (uniform across the CTA)
    int cnt = 0;
    for (int g0 = 0; g0 < nkb; g0 += 32) {
      const int kb = g0 + lane;
      const bool v = kb < nkb && d.kb_lo[kb] < a1 && d.kb_hi[kb] > a0 && d.kb_lo[kb] < b1 &&
                     d.kb_hi[kb] > b0;
      cnt += __popc(__ballot_sync(0xffffffffu, v));
    }
    const int r_begin = (int)((long long)sp * cnt / S), r_end = (int)((long long)(sp + 1) * cnt / S);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    int scan_g0 = 0, rank = 0;  // scan state, meaningful in warp 0
    while (true) {
      __syncthreads();
      if (warp == 0) {
        int m = 0;
        while (scan_g0 < nkb && m <= kWtList - 32 && rank < r_end) {
          const int kb = scan_g0 + lane;
          const bool v = kb < nkb && d.kb_lo[kb] < a1 && d.kb_hi[kb] > a0 && d.kb_lo[kb] < b1 &&
                         d.kb_hi[kb] > b0;
          const unsigned mask = __ballot_sync(0xffffffffu, v);
          const int myrank = rank + __popc(mask & ((1u << lane) - 1u));
          const bool take = v && myrank >= r_begin && myrank < r_end;
          const unsigned tmask = __ballot_sync(0xffffffffu, take);
          if (take) kbl[m + __popc(tmask & ((1u << lane) - 1u))] = kb;
          m += __popc(tmask);
          rank += __popc(mask);
          scan_g0 += 32;
        }
        if (lane == 0) list_n = m;
      }
      __syncthreads();
      const int m = list_n;
      if (m == 0) break;
      for (int li = 0; li < m; ++li) {
        const int r0 = kbl[li] * kWtKB;
        // stage the block: warp w loads rows 8w .. 8w+7, lanes cover 64 columns
        float pa[8][2], pb[8][2];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int u = r0 + 8 * warp + k;
          int clo = 0, len = 0, base = 0;
          if (u < nU) {
            clo = d.u_clo[u];
            len = d.u_len[u];
            base = d.y_ptr[u];
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            const int ca = a0 + c - clo, cb = b0 + c - clo;
            pa[k][h] = (ca >= 0 && ca < len) ? d.y_val[base + ca] : 0.f;
            pb[k][h] = (!diag && cb >= 0 && cb < len) ? d.y_val[base + cb] : 0.f;
          }
        }
        __syncthreads();  // previous block's products are done
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            As[8 * warp + k][lane + 32 * h] = pa[k][h];
            Bs[8 * warp + k][lane + 32 * h] = pb[k][h];
          }
        __syncthreads();
        const float(*Bsrc)[kWtT] = diag ? As : Bs;
#pragma unroll 8
        for (int k = 0; k < kWtKB; ++k) {
          const float4 x0 = *reinterpret_cast<const float4*>(&As[k][8 * ty]);
          const float4 x1 = *reinterpret_cast<const float4*>(&As[k][8 * ty + 4]);
          const float4 y = *reinterpret_cast<const float4*>(&Bsrc[k][4 * tx]);
          const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          const float bv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
      }
    }
    float* out = d.wt_part + (size_t)item * kWtT * kWtT;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      *reinterpret_cast<float4*>(out + (8 * ty + i) * kWtT + 4 * tx) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

__global__ void k_wt_reduce(DevSim d) {
  if (*d.dl_state) return;   // Y and W~ kept from the previous frame
  const int ncv = min(d.counters[kCntCv], d.cap);
  const int nU = d.counters[kCntU];
  if (ncv == 0 || nU == 0 || d.y_ptr[nU] > d.cap_y) return;
  const int ntiles = d.sc_tileoff[d.n_scenes], S = wt_splits(ntiles, d.wt_grid);
  const long long total = (long long)ntiles * kWtT * kWtT;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int tile = (int)(e / (kWtT * kWtT)), el = (int)(e % (kWtT * kWtT));
    const int sc = tile_scene(d, tile);
    int I, J;
    tri_decode(tile - d.sc_tileoff[sc], I, J);
    // scene-local row and column of the scene's block
    const int nv = d.sc_cvb[sc + 1] - d.sc_cvb[sc], ld = d.sc_ld[sc];
    float* W = d.wt + d.sc_wtoff[sc];
    const int ra = I * kWtT + el / kWtT, cb = J * kWtT + el % kWtT;
    if (ra < nv && cb < nv) {
      float sum = 0.f;
      const float* p = d.wt_part + (size_t)tile * S * kWtT * kWtT + el;
      for (int sp = 0; sp < S; ++sp) sum += p[(size_t)sp * kWtT * kWtT];
      W[(size_t)ra * ld + cb] = sum;
      W[(size_t)cb * ld + ra] = sum;
    } else if (ra >= nv && ra < ld && cb < nv) {
      W[(size_t)cb * ld + ra] = 0.f;   // zero padding of the last column group
    } else if (cb >= nv && cb < ld && ra < nv) {
      W[(size_t)ra * ld + cb] = 0.f;
    }
  }
}

// Split of a scene's contact vertices over its CR cluster's ranks, balanced by contacts:
// rank r owns the scene's contact vertices [cv_split(r), cv_split(r + 1)) (global ids).
__device__ int cv_split(const DevSim& d, int r, int R, int cvb, int cve, int jb, int je) {
  if (r >= R) return cve;
  const long long target = jb + (long long)r * (je - jb) / R;
  int lo = cvb, hi = cve;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (d.cv_first[mid] < target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_precond(DevSim d) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = min(d.counters[kCntContacts], d.cap);
  if (blockIdx.x == 0) {
    const int R = d.cr_R, per = 2 * (kCrMaxRanks + 1);
    for (int e = threadIdx.x; e < d.n_scenes * (R + 1); e += blockDim.x) {
      const int sc = e / (R + 1), r = e % (R + 1);
      const int cvb = d.sc_cvb[sc], cve = d.sc_cvb[sc + 1];
      const int jb = d.sc_jb[sc], je = d.sc_jb[sc + 1];
      const int cv = cv_split(d, r, R, cvb, cve, jb, je);
      d.cr_split[sc * per + r] = cv - cvb;
      d.cr_split[sc * per + kCrMaxRanks + 1 + r] = cv < cve ? min(d.cv_first[cv], je) : je;
    }
  }
  if (j >= c) return;
  const int ncv = min(d.counters[kCntCv], d.cap);
  const int cv = d.ct_cv[j];
  double w = 0.0;
  // the contact's terms: its vertex (weight 1) and, for a contact with another body, the
  // triangle's corners (weights -w_k); W_jj = sum_pq c_p c_q W~_pq (the frame rows are
  // orthonormal), [H M^-1 H^T]_jj = sum_p c_p^2 / m_p
  int tc[4] = {cv, -1, -1, -1};
  double tw[4] = {1.0, 0.0, 0.0, 0.0};
  int tv[4] = {d.ct_vert[j], 0, 0, 0};
  if (d.map_on && d.ct_tri[j] >= 0) {
    const int4 t = d.btri[d.ct_tri[j]];
    const int cs[3] = {t.x, t.y, t.z};
    for (int k = 0; k < 3; ++k) {
      tc[1 + k] = d.ct_tcv[3 * j + k];
      tw[1 + k] = -d.ct_bw[3 * j + k];
      tv[1 + k] = cs[k];
    }
  }
  double wm = 0.0;
  const int sc = d.vert_scene[d.ct_vert[j]];
  const float* Wb = d.wt + d.sc_wtoff[sc];
  const int ld = d.sc_ld[sc], cvb = d.sc_cvb[sc];
  for (int p = 0; p < 4; ++p) {
    if (tc[p] < 0 || tc[p] >= ncv) continue;
    wm += tw[p] * tw[p] / d.mass[tv[p]];
    for (int q = 0; q < 4; ++q)
      if (tc[q] >= 0 && tc[q] < ncv)
        w += tw[p] * tw[q] * (double)Wb[(size_t)(tc[p] - cvb) * ld + (tc[q] - cvb)];
  }
  // the residual's scale is always the Delassus diagonal (Eq. 28); the iteration's is that
  // or, with the mass-inverse preconditioner (Sec. 5.4), [H M^-1 H^T]_jj (1 / m_v for a
  // one-vertex contact with unit frame rows)
  const double wi = d.precond == SIM_PRECOND_MASS ? wm : w;
  d.ct_r[4 * j] = d.h * d.h * wi;
  d.ct_r[4 * j + 1] = d.h * wi;
  d.ct_r[4 * j + 2] = d.h * d.h * w;
  d.ct_r[4 * j + 3] = d.h * w;
  for (int r = 0; r < 3; ++r) d.ct_lam[3 * j + r] = 0.0;
  for (int r = 0; r < 9; ++r) d.ct_Df[9 * j + r] = (float)d.ct_D[9 * j + r];
}

// Fischer-Burmeister terms at (q^k, lambda^k) for every contact (FP64).
__global__ void k_contact_eval(DevSim d, int k, int final_eval) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  if (k < 0) k = *d.iter_k;
  const int v = d.ct_vert[j];
  const double h = d.h;
  double D[9];
  for (int r = 0; r < 9; ++r) D[r] = d.ct_D[9 * j + r];
  double dqv[3], q[3];
  contact_dq(d, j, dqv);
  contact_q(d, j, nullptr, q);
  const double lamv[3] = {d.ct_lam[3 * j], d.ct_lam[3 * j + 1], d.ct_lam[3 * j + 2]};
  const int sc = d.vert_scene[v];
  const FbTerms fb = fb_terms(d, j, q, lamv, d.scene_Lref[sc]);
  if (fb.bilateral) {
    // an anchor: three position-level rows, always active (App. B, bilateral items)
    atomic_max_nonneg(&d.resid[k], fb.res);
    atomic_max_nonneg(&d.resid_scene[sc * (kMaxIters + 1) + k], fb.res);
    if (final_eval) return;
    const double phb[3] = {fb.phin, fb.phif0, fb.phif1};
    for (int r = 0; r < 3; ++r) {
      d.ct_force[3 * j + r] = D[r] * lamv[0] + D[3 + r] * lamv[1] + D[6 + r] * lamv[2];
      d.ct_omega[3 * j + r] = 1.f;
      d.ct_ecal[3 * j + r] = (float)(fb.En / (h * h));
      const double Ddq = D[3 * r] * dqv[0] + D[3 * r + 1] * dqv[1] + D[3 * r + 2] * dqv[2];
      d.ct_hv[3 * j + r] = -phb[r] + Ddq;
    }
    return;
  }
  const double dn = fb.dn, phin = fb.phin, omn = fb.omn, En = fb.En;
  const double omf = fb.omf, Ef = fb.Ef, phif0 = fb.phif0, phif1 = fb.phif1;
  const double ln = lamv[0], lf0 = lamv[1], lf1 = lamv[2];
  const double res = fb.res;
  atomic_max_nonneg(&d.resid[k], res);
  atomic_max_nonneg(&d.resid_scene[sc * (kMaxIters + 1) + k], res);
  if (final_eval) {
    if (-dn > 0.0) atomic_max_nonneg(d.max_pen, -dn);
    return;
  }
  const double om[3] = {omn, omf, omf};
  const double lam[3] = {ln, lf0, lf1};
  for (int r = 0; r < 3; ++r)
    d.ct_force[3 * j + r] = D[r] * om[0] * lam[0] + D[3 + r] * om[1] * lam[1] + D[6 + r] * om[2] * lam[2];
  d.ct_omega[3 * j] = (float)omn;
  d.ct_omega[3 * j + 1] = (float)omf;
  d.ct_omega[3 * j + 2] = (float)omf;
  d.ct_ecal[3 * j] = (float)(En / (h * h));
  d.ct_ecal[3 * j + 1] = (float)(Ef / h);
  d.ct_ecal[3 * j + 2] = (float)(Ef / h);
  const double phi[3] = {phin, h * phif0, h * phif1};
  for (int r = 0; r < 3; ++r) {
    const double Ddq = D[3 * r] * dqv[0] + D[3 * r + 1] * dqv[1] + D[3 * r + 2] * dqv[2];
    d.ct_hv[3 * j + r] = -phi[r] + om[r] * Ddq;
  }
}

// (Y^T z) per contact vertex, then the Schur right-hand side h^-2 (h - J A^-1 g) per
// contact. One 128-thread CTA per contact vertex strides along its ancestor path and the
// partial sums are combined in a fixed order.
constexpr int kYtzThreads = 128;
__global__ void __launch_bounds__(kYtzThreads) k_ytz(DevSim d) {
  pdl_wait();
  const int ncv = min(d.counters[kCntCv], d.cap);
  if (d.yc_ptr[ncv] > d.cap_y) return;   // uniform over the grid
  __shared__ float part[3][kYtzThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double ih2 = 1.0 / (d.h * d.h);
  // CTAs walk the contact vertices with a grid stride (the grid is sized for the SMs, not
  // for the capacity); every thread of a CTA runs the same iterations
  for (int c = blockIdx.x; c < ncv; c += gridDim.x) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    const int k1 = d.yc_ptr[c + 1];
#pragma unroll 4
    for (int k = d.yc_ptr[c] + threadIdx.x; k < k1; k += kYtzThreads) {
      const float y = d.yc_val[k];
      const int a = d.yc_row[k];
      s0 += y * d.zvec[a];
      s1 += y * d.zvec[d.n_pad + a];
      s2 += y * d.zvec[2 * d.n_pad + a];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
      part[0][wid] = s0;
      part[1][wid] = s1;
      part[2][wid] = s2;
    }
    __syncthreads();
    if (wid == 0) {
      s0 = s1 = s2 = 0.f;
      for (int w = 0; w < kYtzThreads / 32; ++w) {
        s0 += part[0][w];
        s1 += part[1][w];
        s2 += part[2][w];
      }
      if (d.map_on && lane == 0) {
        d.svec[3 * c] = s0;
        d.svec[3 * c + 1] = s1;
        d.svec[3 * c + 2] = s2;
      }
      const int j0 = d.cv_first[c], j1 = min(j0 + d.cv_nct[c], d.cap);
      for (int j = j0 + lane; j < j1; j += 32) {
        if (d.map_on && d.ct_tri[j] >= 0) continue;   // k_body_rhs
        for (int r = 0; r < 3; ++r) {
          const float* Dr = d.ct_Df + 9 * j + 3 * r;
          const float jag = d.ct_omega[3 * j + r] * (Dr[0] * s0 + Dr[1] * s1 + Dr[2] * s2);
          d.ct_rhs[3 * j + r] = (float)((d.ct_hv[3 * j + r] - (double)jag) * ih2);
        }
      }
    }
    __syncthreads();   // part[] is reused by the next contact vertex
  }
}

// The same with one warp per contact vertex (no block barriers; more vertices in flight),
// for meshes whose ancestor paths are short (many small scenes).
__global__ void k_ytz_warp(DevSim d) {
  pdl_wait();
  const int ncv = min(d.counters[kCntCv], d.cap);
  if (d.yc_ptr[ncv] > d.cap_y) return;   // uniform over the grid
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const double ih2 = 1.0 / (d.h * d.h);
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncv; c += nwarps) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    const int k1 = d.yc_ptr[c + 1];
#pragma unroll 4
    for (int k = d.yc_ptr[c] + lane; k < k1; k += 32) {
      const float y = d.yc_val[k];
      const int a = d.yc_row[k];
      s0 += y * d.zvec[a];
      s1 += y * d.zvec[d.n_pad + a];
      s2 += y * d.zvec[2 * d.n_pad + a];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (d.map_on && lane == 0) {
      d.svec[3 * c] = s0;
      d.svec[3 * c + 1] = s1;
      d.svec[3 * c + 2] = s2;
    }
    const int j0 = d.cv_first[c], j1 = min(j0 + d.cv_nct[c], d.cap);
    for (int j = j0 + lane; j < j1; j += 32) {
      if (d.map_on && d.ct_tri[j] >= 0) continue;   // k_body_rhs
      for (int r = 0; r < 3; ++r) {
        const float* Dr = d.ct_Df + 9 * j + 3 * r;
        const float jag = d.ct_omega[3 * j + r] * (Dr[0] * s0 + Dr[1] * s1 + Dr[2] * s2);
        d.ct_rhs[3 * j + r] = (float)((d.ct_hv[3 * j + r] - (double)jag) * ih2);
      }
    }
  }
}

// the Schur right-hand side of the contacts with another body, whose J A^-1 g combines
// (Y^T z) of the vertex and the triangle's corners with the map's weights
__global__ void k_body_rhs(DevSim d) {
  pdl_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = min(d.counters[kCntContacts], d.cap);
  const int ncv = min(d.counters[kCntCv], d.cap);
  if (j >= c || d.ct_tri[j] < 0 || d.yc_ptr[ncv] > d.cap_y) return;
  const double ih2 = 1.0 / (d.h * d.h);
  const int cv = d.ct_cv[j];
  if (cv >= ncv) return;   // beyond the capacity: the frame reports SIM_ECAPACITY
  float s[3] = {d.svec[3 * cv], d.svec[3 * cv + 1], d.svec[3 * cv + 2]};
  for (int k = 0; k < 3; ++k) {
    const int t = d.ct_tcv[3 * j + k];
    if (t < 0) continue;
    const float w = (float)d.ct_bw[3 * j + k];
    for (int r = 0; r < 3; ++r) s[r] -= w * d.svec[3 * t + r];
  }
  for (int r = 0; r < 3; ++r) {
    const float* Dr = d.ct_Df + 9 * j + 3 * r;
    const float jag = d.ct_omega[3 * j + r] * (Dr[0] * s[0] + Dr[1] * s[1] + Dr[2] * s[2]);
    d.ct_rhs[3 * j + r] = (float)((d.ct_hv[3 * j + r] - (double)jag) * ih2);
  }
}

// y = z + h^2 Y u, in place on z (rows of U only)
__global__ void k_yu(DevSim d) {
  pdl_wait();
  const int lane = threadIdx.x & 31, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nU = d.counters[kCntU];
  if (d.y_ptr[nU] > d.cap_y) return;
  const float h2 = (float)(d.h * d.h);
  // warps walk the rows of U with a grid stride (the grid is sized for the SMs)
  for (int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < nU; idx += nwarps) {
    const int clo = d.u_clo[idx], len = d.u_len[idx], base = d.y_ptr[idx];
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll 4
    for (int k = lane; k < len; k += 32) {
      const float y = d.y_val[base + k];
      const float* u = d.uvec + 3 * (clo + k);
      t0 += y * u[0];
      t1 += y * u[1];
      t2 += y * u[2];
    }
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if (lane == 0) {
      const int a = d.u_list[idx];
      d.zvec[a] += h2 * t0;
      d.zvec[d.n_pad + a] += h2 * t1;
      d.zvec[2 * d.n_pad + a] += h2 * t2;
    }
  }
}

// ---- conjugate residual in one thread-block cluster -----------------------------------
// Every CTA owns a contiguous range of contact vertices (and their contacts). The operator
// K = Omega W Omega + E is applied through W~: u_c = sum_{j at c} D_j^T (omega_j * v_j),
// w = W~ u, (K v)_j = omega_j * (D_j w_{c(j)}) + E_j * v_j. Owned slices of u are exchanged
// through distributed shared memory; dot products are reduced per CTA and then over the
// cluster in rank order, so every CTA holds the same scalars and the result is
// deterministic.
constexpr unsigned kBulkChunk = 32768;  // bytes per bulk-copy instruction

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// wait for phase `parity` of an mbarrier, at most `limit` polls (0: a default of 2^22);
// false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit) {
  if (limit == 0) limit = 1ull << 22;
  for (unsigned long long i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Point-to-point exchange between the CTAs of a cluster: 16-byte stores into another CTA's
// shared memory (st.async) that count their bytes on that CTA's mbarrier, which its threads
// wait on (cluster-scope acquire) instead of a cluster-wide barrier.
__device__ __forceinline__ unsigned mapa_u32(unsigned addr, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async_v4(unsigned remote_addr, float4 v, unsigned remote_bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::
          "r"(remote_addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(remote_bar) : "memory");
}
__device__ __forceinline__ void st_async_f32(unsigned remote_addr, float v, unsigned remote_bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(remote_addr),
      "f"(v), "r"(remote_bar) : "memory");
}
// this CTA's arrival on its barrier for the current phase, expecting `bytes` from the stores
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cluster.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes) : "memory");
}
// wait for phase `parity` with cluster-scope acquire (the stores of other CTAs become
// visible), at most `limit` polls (0: 2^22); false on timeout
__device__ __forceinline__ bool mbar_wait_cluster(unsigned bar, unsigned parity,
                                                  unsigned long long limit) {
  if (limit == 0) limit = 1ull << 22;
  for (unsigned long long i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct CrLayout {
  int R, rank, c, ncv, cv0, cv1, j0, j1;
};

// Row products of the constraint solves: lane l of a warp takes the column pairs
// (2l, 2l + 1) + 64 m of the vertex vector; a warp multiplies four rows of W~ at a time with
// 8-byte loads and packed FP32 FMAs and reduces the twelve row sums over the warp with a
// butterfly of 16 shuffles.
constexpr int kCrPairs = 16;     // column pairs per lane of the packed row product: rows up to
                                 // 1024 wide (wider ones take the float4 path)
constexpr int kCrDotSlots = kCrMaxRanks * (kCrThreads / 32);   // (rank, warp) partials

// Sum each of v[0..11] over the warp; afterwards lanes 2i and 2i + 1 hold the total of v[i]
// in v[0]. Butterfly halving: at each step a lane keeps half of its values and adds the
// partner's copy of that half.
__device__ __forceinline__ float warp_sum12(float (&v)[16], int lane) {
#pragma unroll
  for (int i = 12; i < 16; ++i) v[i] = 0.f;
#pragma unroll
  for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float keep = up ? v[i + n / 2] : v[i];
      const float send = up ? v[i] : v[i + n / 2];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__global__ void __launch_bounds__(kCrThreads, 1) k_cr(DevSim d, int smem_bytes) {
  pdl_wait();
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cl = cg::this_cluster();
  CrLayout L;
  L.R = (int)cl.num_blocks();
  L.rank = (int)cl.block_rank();
  // this cluster's scene: its contacts and contact vertices (global ids cvb.., jb..)
  const int scene = blockIdx.x / L.R;
  const int cvb = d.sc_cvb[scene], jb = d.sc_jb[scene];
  L.c = d.sc_jb[scene + 1] - jb;
  L.ncv = d.sc_cvb[scene + 1] - cvb;
  // every CTA reads the same counters, so this exit is taken by all or by none
  if (L.c == 0 || L.ncv == 0) return;
  // split of the contact vertices over the cluster ranks, computed once per CTA
  __shared__ int split_cv[kCrMaxRanks + 1], split_j[kCrMaxRanks + 1];
  if (threadIdx.x <= L.R) {
    const int* sp = d.cr_split + scene * 2 * (kCrMaxRanks + 1);
    split_cv[threadIdx.x] = sp[threadIdx.x];
    split_j[threadIdx.x] = sp[kCrMaxRanks + 1 + threadIdx.x];
  }
  __syncthreads();
  L.cv0 = split_cv[L.rank];
  L.cv1 = split_cv[L.rank + 1];
  L.j0 = split_j[L.rank];
  L.j1 = max(split_j[L.rank + 1], L.j0);
  const int nj = L.j1 - L.j0, nv = L.cv1 - L.cv0;
  int nj_max = 0, nv_max = 0;
  for (int r = 0; r < L.R; ++r) {
    nj_max = max(nj_max, max(0, split_j[r + 1] - split_j[r]));
    nv_max = max(nv_max, split_cv[r + 1] - split_cv[r]);
  }
  // shared layout (identical offsets in every CTA for the parts written remotely):
  //   dots[kCrDotSlots] float4  per-(rank, warp) partial dot products (written by every rank)
  //   usx, usy, usz[ldw] float  u for all contact vertices, one array per component (each
  //                             rank writes its own range everywhere)
  const int ldw = d.sc_ld[scene];
  const float* wblk = d.wt + d.sc_wtoff[scene];  // the scene's W~ block, row-major
  // With contacts between bodies (a contact's map also reaches the corners of a triangle,
  // whose contact vertices may belong to another rank) two more exchanges per product:
  //   tall[c] float4   D_j^T (omega_j v_j) of every contact of the scene
  //   wall[ldw] float4 (W~ u) of every contact vertex of the scene
  const bool gen = d.map_on != 0;
  float4* dots = reinterpret_cast<float4*>(sm);          // kCrDotSlots float4
  float* usx = reinterpret_cast<float*>(dots + kCrDotSlots);   // ldw floats each
  float* usy = usx + ldw;
  float* usz = usy + ldw;
  float4* tall = reinterpret_cast<float4*>(usz + ldw);  // c float4 (gen); ldw % 4 == 0
  float4* wall = tall + (gen ? L.c : 0);                 // ldw float4 (gen)
  float4* uloc = wall + (gen ? ldw : 0);                 // nv_max float4 (own slice)
  float* wloc = reinterpret_cast<float*>(uloc + nv_max); // 3 nv
  float* vx = wloc + 3 * nv_max;      // per owned contact: x, r, p, Ar, Ap (3 each)
  float* vr = vx + 3 * nj_max;
  float* vp = vr + 3 * nj_max;
  float* vAr = vp + 3 * nj_max;
  float* vAp = vAr + 3 * nj_max;
  float* Df = vAp + 3 * nj_max;       // 9 nj
  float* om = Df + 9 * nj_max;        // 3 nj
  float* ec = om + 3 * nj_max;        // 3 nj
  int* cvf = reinterpret_cast<int*>(ec + 3 * nj_max);   // owned cv: first local contact
  int* cvn = cvf + nv_max;                              // owned cv: contact count
  int* ctl = cvn + nv_max;                              // owned contact: local cv index
  int* tcl = ctl + nj_max;                              // owned contact: its corners' scene
                                                        // cv indices, -1: none (gen, 3 nj)
  float* twl = reinterpret_cast<float*>(tcl + (gen ? 3 * nj_max : 0));   // their weights
  // the owned rows of W~ that fit (16-byte aligned, one bulk copy); the rest are read from
  // global memory
  float* wrows = sm + ((((twl + (gen ? 3 * nj_max : 0)) - sm) + 3) & ~size_t(3));
  const size_t used = (size_t)(wrows - sm) * sizeof(float);
  __shared__ __align__(8) unsigned long long wbar;
  if (used > (size_t)smem_bytes) {   // uniform: depends only on cluster-wide maxima
    if (threadIdx.x == 0 && L.rank == 0) atomicOr(d.err, kErrCapacity);
    cl.sync();
    return;
  }
  int rows_sm = (int)min((size_t)nv, ((size_t)smem_bytes - used) / ((size_t)ldw * sizeof(float)));
  if (threadIdx.x == 0 && rows_sm > 0) {
    // rows are contiguous in W~ (row-major, ld a multiple of 4 floats): 16-byte aligned
    // source and destination, sizes multiples of 16 bytes
    const unsigned bar = smem_u32(&wbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned long long bytes = (unsigned long long)rows_sm * ldw * sizeof(float);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((unsigned)bytes) : "memory");
    const char* src = reinterpret_cast<const char*>(wblk + (size_t)L.cv0 * ldw);
    const unsigned dst = smem_u32(wrows);
    for (unsigned long long off = 0; off < bytes; off += kBulkChunk) {
      const unsigned sz = (unsigned)min((unsigned long long)kBulkChunk, bytes - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst + (unsigned)off), "l"(src + off), "r"(sz), "r"(bar) : "memory");
    }
  }
  // point-to-point exchanges (sim_options.cr_sync = 0) for scenes without contacts between
  // bodies; the byte count of one phase must stay below the mbarrier's 2^20 limit
  const bool async_x = d.cr_sync == 0 && !gen && L.ncv < 65536;
  __shared__ __align__(8) unsigned long long xbar[2];   // [0]: u slices, [1]: dot products
  if (threadIdx.x == 0 && async_x) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&xbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&xbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  unsigned ph_u = 0, ph_d = 0;
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    const int j = L.j0 + e / 3;
    vx[e] = 0.f;
    vr[e] = d.ct_rhs[3 * j + e % 3];
    om[e] = d.ct_omega[3 * j + e % 3];
    ec[e] = d.ct_ecal[3 * j + e % 3];
  }
  for (int e = threadIdx.x; e < 9 * nj; e += blockDim.x) Df[e] = d.ct_Df[9 * L.j0 + e];
  for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
    const int jf = max(0, d.cv_first[cvb + L.cv0 + cvl] - L.j0);
    cvf[cvl] = jf;
    cvn[cvl] = max(0, min(nj, jf + d.cv_nct[cvb + L.cv0 + cvl]) - jf);
  }
  for (int jl = threadIdx.x; jl < nj; jl += blockDim.x)
    ctl[jl] = min(max(d.ct_cv[L.j0 + jl] - cvb - L.cv0, 0), max(nv - 1, 0));
  if (gen)
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      const int j = L.j0 + e / 3, t = d.ct_tri[j] >= 0 ? d.ct_tcv[3 * j + e % 3] : -1;
      tcl[e] = t >= cvb && t < cvb + L.ncv ? t - cvb : -1;
      twl[e] = t >= 0 ? (float)d.ct_bw[3 * j + e % 3] : 0.f;
    }
  for (int e = L.ncv + threadIdx.x; e < ldw; e += blockDim.x) usx[e] = usy[e] = usz[e] = 0.f;
  __syncthreads();
  const bool w_copy = rows_sm > 0;
  bool w_late = false;
  if (w_copy && !mbar_wait(smem_u32(&wbar), 0, d.spin_limit)) {
    // the copy did not complete in time: report it and read every row from global memory
    if (threadIdx.x == 0) atomicOr(d.err, kErrTimeout);
    rows_sm = 0;
    w_late = true;
  }
  __syncthreads();
  // every CTA of the cluster must be running before shared memory is written remotely
  cl.sync();

  // Kv = K v for the owned contacts; v must be complete in shared memory on entry
  // u = sum over the terms at each owned contact vertex of the terms' weights times
  // D_j^T (omega_j v_j): its own contacts (weight 1, contiguous) and, with contacts between
  // bodies, the corner terms (-w_k, ascending contact order) read from tall
  auto vertex_u = [&](const float* v, int cvl) {
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    const int jb0 = cvf[cvl], je0 = jb0 + cvn[cvl];
    if (!gen) {
      for (int jl = jb0; jl < je0; ++jl) {
        const float* D = Df + 9 * jl;
        const float a0 = om[3 * jl] * v[3 * jl], a1 = om[3 * jl + 1] * v[3 * jl + 1],
                    a2 = om[3 * jl + 2] * v[3 * jl + 2];
        u0 += D[0] * a0 + D[3] * a1 + D[6] * a2;
        u1 += D[1] * a0 + D[4] * a1 + D[7] * a2;
        u2 += D[2] * a0 + D[5] * a1 + D[8] * a2;
      }
      return make_float4(u0, u1, u2, 0.f);
    }
    for (int jl = jb0; jl < je0; ++jl) {
      const float4 t = tall[L.j0 - jb + jl];
      u0 += t.x;
      u1 += t.y;
      u2 += t.z;
    }
    const int vtx = d.cv_vert[cvb + L.cv0 + cvl];
    const int xe = min(d.x_off[vtx + 1], 3 * d.cap);
    for (int e = d.x_off[vtx]; e < xe; ++e) {
      const int tk = d.x_list[e], jg = tk / 3 - jb;
      if (tk < 0 || jg < 0 || jg >= L.c) continue;
      const float w = (float)d.ct_bw[tk];
      const float4 t = tall[jg];
      u0 -= w * t.x;
      u1 -= w * t.y;
      u2 -= w * t.z;
    }
    return make_float4(u0, u1, u2, 0.f);
  };
  // tall <- D_j^T (omega_j v_j) of the owned contacts, in every rank
  auto publish_t = [&](const float* v) {
    for (int e = threadIdx.x; e < L.R * nj; e += blockDim.x) {
      const int r = e / nj, jl = e - r * nj;
      const float* D = Df + 9 * jl;
      const float a0 = om[3 * jl] * v[3 * jl], a1 = om[3 * jl + 1] * v[3 * jl + 1],
                  a2 = om[3 * jl + 2] * v[3 * jl + 2];
      cl.map_shared_rank(tall, r)[L.j0 - jb + jl] =
          make_float4(D[0] * a0 + D[3] * a1 + D[6] * a2, D[1] * a0 + D[4] * a1 + D[7] * a2,
                      D[2] * a0 + D[5] * a1 + D[8] * a2, 0.f);
    }
    cl.sync();
  };
  auto apply = [&](const float* v, float* Kv) {
    if (gen) publish_t(v);
    // this phase brings every contact vertex's u (12 bytes each) from its owner
    if (async_x) {
      // the thread that computes an owned vertex's u stores it into every rank (itself
      // included), counted on that rank's barrier (measured faster than staging u and
      // spreading the stores over all threads after a block barrier)
      if (threadIdx.x == 0) mbar_expect(smem_u32(&xbar[0]), (unsigned)L.ncv * 12u);
      const unsigned ub = smem_u32(usx + L.cv0), bb = smem_u32(&xbar[0]);
      const unsigned cstride = 4u * (unsigned)ldw;   // bytes between the component arrays
      for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
        const float4 u = vertex_u(v, cvl);
        for (int r = 0; r < L.R; ++r) {
          const unsigned ra = mapa_u32(ub + 4u * (unsigned)cvl, r), rb = mapa_u32(bb, r);
          st_async_f32(ra, u.x, rb);
          st_async_f32(ra + cstride, u.y, rb);
          st_async_f32(ra + 2u * cstride, u.z, rb);
        }
      }
      if (!mbar_wait_cluster(smem_u32(&xbar[0]), ph_u & 1u, d.spin_limit) && threadIdx.x == 0)
        atomicOr(d.err, kErrTimeout);
      ++ph_u;
    } else {
      for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) uloc[cvl] = vertex_u(v, cvl);
      __syncthreads();
      // one 16-byte remote store per (rank, owned vertex), spread over all threads
      for (int e = threadIdx.x; e < L.R * nv; e += blockDim.x) {
        const int r = e / nv, cvl = e - r * nv;
        const float4 u = uloc[cvl];
        cl.map_shared_rank(usx, r)[L.cv0 + cvl] = u.x;
        cl.map_shared_rank(usy, r)[L.cv0 + cvl] = u.y;
        cl.map_shared_rank(usz, r)[L.cv0 + cvl] = u.z;
      }
      cl.sync();   // every rank's slice of u is now in every CTA
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int ng = ldw / 4;
    auto wrow_ptr = [&](int row) {
      return reinterpret_cast<const float4*>(
          row < rows_sm ? wrows + (size_t)row * ldw : wblk + (size_t)(L.cv0 + row) * ldw);
    };
    if (ldw <= 64 * kCrPairs) {
      // lane l takes the column pairs (2l, 2l + 1) + 64 m; a warp multiplies four rows of W~
      // at a time with 8-byte loads of W~ and of each component of u (one conflict-free load
      // each) and packed FP32 FMAs (fma.rn.f32x2: two independent round-to-nearest FMAs),
      // and reduces the twelve row sums over the warp with a butterfly of 16 shuffles. The
      // loop over the pairs stays rolled (measured faster than the fully unrolled form with
      // u held in registers: less code per iteration of the solve)
      auto rows4 = [&](int r_begin, int r_end, auto row_ptr) {
        for (int row = r_begin + 4 * warp; row < r_end; row += 4 * nw) {
          const int nr = min(4, r_end - row);
          const float* w[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) w[k] = row_ptr(min(row + k, r_end - 1));
          unsigned long long acc[4][3];
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0ull;
#pragma unroll 2
          for (int col = 2 * lane; col < ldw; col += 64) {
            const unsigned long long ux = *reinterpret_cast<const unsigned long long*>(usx + col);
            const unsigned long long uy = *reinterpret_cast<const unsigned long long*>(usy + col);
            const unsigned long long uz = *reinterpret_cast<const unsigned long long*>(usz + col);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float2 p = *reinterpret_cast<const float2*>(w[k] + col);
              const unsigned long long pp = f2pack(p.x, p.y);
              acc[k][0] = ffma2(pp, ux, acc[k][0]);
              acc[k][1] = ffma2(pp, uy, acc[k][1]);
              acc[k][2] = ffma2(pp, uz, acc[k][2]);
            }
          }
          float v[16];
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) v[3 * k + q] = f2lo(acc[k][q]) + f2hi(acc[k][q]);
          const float tot = warp_sum12(v, lane);
          const int idx = lane >> 1;
          if (!(lane & 1) && idx < 3 * nr) wloc[3 * row + idx] = tot;
        }
      };
      // rows held in shared memory are read through a shared-memory pointer (shared-memory
      // loads, not generic ones); the rest through a global one
      const int n_sm_rows = min(rows_sm, nv);
      rows4(0, n_sm_rows, [&](int r) { return static_cast<const float*>(wrows + (size_t)r * ldw); });
      rows4(n_sm_rows, nv, [&](int r) { return wblk + (size_t)(L.cv0 + r) * ldw; });
    } else {
    // four rows per warp at a time, so the shuffle reductions of the rows overlap
    for (int row0 = 4 * warp; row0 < nv; row0 += 4 * nw) {
      float acc[4][3] = {};
      const int nrow = min(4, nv - row0);
      const float4* wrow[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) wrow[k] = wrow_ptr(min(row0 + k, nv - 1));
#pragma unroll 2
      for (int g4 = lane; g4 < ng; g4 += 32) {
        // the four vertices 4 g4 .. 4 g4 + 3, one component per load
        const float4 X = reinterpret_cast<const float4*>(usx)[g4],
                     Y = reinterpret_cast<const float4*>(usy)[g4],
                     Z = reinterpret_cast<const float4*>(usz)[g4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k < nrow) {
            const float4 w = wrow[k][g4];
            acc[k][0] += w.x * X.x + w.y * X.y + w.z * X.z + w.w * X.w;
            acc[k][1] += w.x * Y.x + w.y * Y.y + w.z * Y.z + w.w * Y.w;
            acc[k][2] += w.x * Z.x + w.y * Z.y + w.z * Z.z + w.w * Z.w;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[k][q] = warp_sum(acc[k][q]);
      if (lane < 3 * nrow) {
        const int k = lane / 3, q = lane % 3;
        float val = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int qq = 0; qq < 3; ++qq)
            if (kk == k && qq == q) val = acc[kk][qq];
        wloc[3 * (row0 + k) + q] = val;
      }
    }
    }
    __syncthreads();
    if (gen) {
      // every rank's W~ u, then the map's combination at each owned contact
      for (int e = threadIdx.x; e < L.R * nv; e += blockDim.x) {
        const int r = e / nv, cvl = e - r * nv;
        cl.map_shared_rank(wall, r)[L.cv0 + cvl] =
            make_float4(wloc[3 * cvl], wloc[3 * cvl + 1], wloc[3 * cvl + 2], 0.f);
      }
      cl.sync();
      for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
        const int jl = e / 3, r = e % 3;
        const float4 w0 = wall[L.cv0 + ctl[jl]];
        float wx = w0.x, wy = w0.y, wz = w0.z;
        for (int k = 0; k < 3; ++k) {
          const int t = tcl[3 * jl + k];
          if (t < 0) continue;
          const float c = twl[3 * jl + k];
          const float4 q = wall[t];
          wx -= c * q.x;
          wy -= c * q.y;
          wz -= c * q.z;
        }
        const float* D = Df + 9 * jl + 3 * r;
        Kv[e] = om[e] * (D[0] * wx + D[1] * wy + D[2] * wz) + ec[e] * v[e];
      }
      return;
    }
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      const int jl = e / 3, r = e % 3;
      const int cvl = ctl[jl];
      const float* D = Df + 9 * jl + 3 * r;
      const float dw = D[0] * wloc[3 * cvl] + D[1] * wloc[3 * cvl + 1] + D[2] * wloc[3 * cvl + 2];
      Kv[e] = om[e] * dw + ec[e] * v[e];
    }
  };
  // cluster-wide sums of three values: per warp (butterfly), then every warp's partial goes
  // to slot (rank, warp) of every CTA in one exchange, and every warp adds all R x 8 slots
  // in the same order (lane l: slots l, l + 32, ...; then the butterfly). Every warp of
  // every CTA holds identical scalars (deterministic), with no block barrier.
  auto exchange = [&](float& a, float& b, float& c) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int nslot = L.R * nw;
    if (async_x) {
      // this phase brings one float4 from every (rank, warp)
      if (threadIdx.x == 0) mbar_expect(smem_u32(&xbar[1]), (unsigned)nslot * 16u);
      if (lane < L.R)
        st_async_v4(mapa_u32(smem_u32(dots + L.rank * nw + wid), lane), make_float4(a, b, c, 0.f),
                    mapa_u32(smem_u32(&xbar[1]), lane));
      if (!mbar_wait_cluster(smem_u32(&xbar[1]), ph_d & 1u, d.spin_limit) && threadIdx.x == 0)
        atomicOr(d.err, kErrTimeout);
      ++ph_d;
    } else {
      if (lane < L.R) cl.map_shared_rank(dots, lane)[L.rank * nw + wid] = make_float4(a, b, c, 0.f);
      cl.sync();
    }
    float ta = 0.f, tb = 0.f, tc = 0.f;
    for (int q = lane; q < nslot; q += 32) {
      const float4 t = dots[q];
      ta += t.x;
      tb += t.y;
      tc += t.z;
    }
    a = warp_sum(ta);
    b = warp_sum(tb);
    c = warp_sum(tc);
  };

  // r = rhs, x = 0, p = r, Ap = Ar
  apply(vr, vAr);
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    vp[e] = vr[e];
    vAp[e] = vAr[e];
    s1 += vr[e] * vAr[e];
    s2 += vAr[e] * vAr[e];
  }
  exchange(s1, s2, s3);
  float rAr = s1, ApAp = s2;
  for (int it = 0; it < d.n_cr; ++it) {
    if (!(ApAp > 0.f)) break;
    const float alpha = rAr / ApAp;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vx[e] += alpha * vp[e];
      vr[e] -= alpha * vAp[e];
    }
    __syncthreads();
    apply(vr, vAr);
    s1 = s2 = s3 = 0.f;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      s1 += vr[e] * vAr[e];
      s2 += vAr[e] * vAr[e];
      s3 += vAr[e] * vAp[e];
    }
    exchange(s1, s2, s3);
    const float rAr_new = s1, ArAr = s2, ArAp = s3;
    const float beta = rAr != 0.f ? rAr_new / rAr : 0.f;
    ApAp = ArAr + 2.f * beta * ArAp + beta * beta * ApAp;
    rAr = rAr_new;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vp[e] = vr[e] + beta * vp[e];
      vAp[e] = vAr[e] + beta * vAp[e];
    }
  }
  __syncthreads();
  // lambda += dlambda; u = D^T (omega * dlambda) per owned contact vertex
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) d.ct_lam[3 * L.j0 + e] += (double)vx[e];
  if (gen) publish_t(vx);
  for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
    const int cv = cvb + L.cv0 + cvl;
    const float4 u = vertex_u(vx, cvl);
    d.uvec[3 * cv] = u.x;
    d.uvec[3 * cv + 1] = u.y;
    d.uvec[3 * cv + 2] = u.z;
  }
  // a copy that timed out may still be in flight: give it another bounded wait before the
  // shared memory is released
  if (w_late) mbar_wait(smem_u32(&wbar), 0, d.spin_limit);
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}


// ---- conjugate residual with one cluster exchange per iteration --------------------------
// The iteration of k_cr (unpreconditioned CR from x = 0, n_cr iterations, (Ap, Ap) expanded
// from (Ar, Ar), (Ar, Ap) and beta), for scenes without contacts between bodies, rearranged
// so that each iteration needs one exchange between the CTAs instead of two. K = B^T W~ B + E
// with B v = sum over a vertex's contacts of D_j^T (omega_j v_j). Every CTA keeps the
// vertex-space images y_r = B r and y_Ap = B Ap of the whole scene and advances them with
// the iteration's own recurrences (r -= alpha Ap gives y_r -= alpha y_Ap; Ap = Ar + beta Ap
// gives y_Ap = B Ar + beta y_Ap); W~ y_r is a full product every iteration. The only data
// an iteration needs from the other CTAs are then their partial dot products and the B Ar of
// their contact vertices, which travel together. The final x = dlambda and its B x are
// computed directly (not from the recurrences). In FP32 the recurrences carry rounding
// from one iteration to the next: on ill-conditioned systems the result can be an order of
// magnitude further from the FP64 iteration than k_cr's, so this form is an option.
// The constraint solve with one cluster exchange per CR iteration (sim_options.cr_exchanges
// = 1; scenes without contacts between bodies). Owned W~ rows that do not fit in shared
// memory are read from L2; a layout that does not fit at all reports SIM_ECAPACITY.
__global__ void __launch_bounds__(kCrThreads, 1) k_cr1(DevSim d, int smem_bytes) {
  pdl_wait();
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int scene = blockIdx.x / R;
  const int cvb = d.sc_cvb[scene], jb = d.sc_jb[scene];
  const int c = d.sc_jb[scene + 1] - jb, ncv = d.sc_cvb[scene + 1] - cvb;
  // every CTA reads the same counters, so this exit is taken by all or by none
  if (c == 0 || ncv == 0) return;
  __shared__ int split_cv[kCrMaxRanks + 1], split_j[kCrMaxRanks + 1];
  if (threadIdx.x <= R) {
    const int* sp = d.cr_split + scene * 2 * (kCrMaxRanks + 1);
    split_cv[threadIdx.x] = sp[threadIdx.x];
    split_j[threadIdx.x] = sp[kCrMaxRanks + 1 + threadIdx.x];
  }
  __syncthreads();
  const int cv0 = split_cv[rank], cv1 = split_cv[rank + 1];
  const int j0 = split_j[rank], j1 = max(split_j[rank + 1], j0);
  const int nj = j1 - j0, nv = cv1 - cv0;
  int nj_max = 0, nv_max = 0;
  for (int r = 0; r < R; ++r) {
    nj_max = max(nj_max, max(0, split_j[r + 1] - split_j[r]));
    nv_max = max(nv_max, split_cv[r + 1] - split_cv[r]);
  }
  const int ldw = d.sc_ld[scene];
  const float* wblk = d.wt + d.sc_wtoff[scene];
  // shared layout (identical offsets in every CTA for the parts written remotely):
  //   dots[2][16] float4   per-rank partial dot products (two exchange buffers)
  //   yr[ldw], yap[ldw]     B r and B Ap of every contact vertex of the scene
  //   yar[2][ldw]           B Ar of every contact vertex (two exchange buffers)
  float4* dots = reinterpret_cast<float4*>(sm);
  float4* yr = dots + 32;
  float4* yap = yr + ldw;
  float4* yar = yap + ldw;
  float* wloc = reinterpret_cast<float*>(yar + 2 * ldw);   // 3 nv: (W~ y_r) of owned rows
  float* vx = wloc + 3 * nv_max;   // per owned contact (3 each): x, r, p, Ar, Ap
  float* vr = vx + 3 * nj_max;
  float* vp = vr + 3 * nj_max;
  float* vAr = vp + 3 * nj_max;
  float* vAp = vAr + 3 * nj_max;
  float* Df = vAp + 3 * nj_max;    // 9 nj
  float* om = Df + 9 * nj_max;     // 3 nj
  float* ec = om + 3 * nj_max;     // 3 nj
  int* cvf = reinterpret_cast<int*>(ec + 3 * nj_max);   // owned cv: first local contact
  int* cvn = cvf + nv_max;                              // owned cv: contact count
  int* ctl = cvn + nv_max;                              // owned contact: local cv index
  float* wrows = sm + ((((reinterpret_cast<float*>(ctl + nj_max)) - sm) + 3) & ~size_t(3));
  const size_t used = (size_t)(wrows - sm) * sizeof(float);
  __shared__ __align__(8) unsigned long long wbar;
  if (used > (size_t)smem_bytes) {   // uniform: depends only on cluster-wide maxima
    if (threadIdx.x == 0 && rank == 0) atomicOr(d.err, kErrCapacity);
    cl.sync();
    return;
  }
  int rows_sm = (int)min((size_t)nv, ((size_t)smem_bytes - used) / ((size_t)ldw * sizeof(float)));
  if (threadIdx.x == 0 && rows_sm > 0) {
    // owned rows are contiguous in W~ (row-major, ld a multiple of 4 floats): 16-byte
    // aligned source and destination, sizes multiples of 16 bytes
    const unsigned bar = smem_u32(&wbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned long long bytes = (unsigned long long)rows_sm * ldw * sizeof(float);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((unsigned)bytes) : "memory");
    const char* src = reinterpret_cast<const char*>(wblk + (size_t)cv0 * ldw);
    const unsigned dst = smem_u32(wrows);
    for (unsigned long long off = 0; off < bytes; off += kBulkChunk) {
      const unsigned sz = (unsigned)min((unsigned long long)kBulkChunk, bytes - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst + (unsigned)off), "l"(src + off), "r"(sz), "r"(bar) : "memory");
    }
  }
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    const int j = j0 + e / 3;
    vx[e] = 0.f;
    vr[e] = d.ct_rhs[3 * j + e % 3];
    om[e] = d.ct_omega[3 * j + e % 3];
    ec[e] = d.ct_ecal[3 * j + e % 3];
  }
  for (int e = threadIdx.x; e < 9 * nj; e += blockDim.x) Df[e] = d.ct_Df[9 * j0 + e];
  for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
    const int jf = max(0, d.cv_first[cvb + cv0 + cvl] - j0);
    cvf[cvl] = jf;
    cvn[cvl] = max(0, min(nj, jf + d.cv_nct[cvb + cv0 + cvl]) - jf);
  }
  for (int jl = threadIdx.x; jl < nj; jl += blockDim.x)
    ctl[jl] = min(max(d.ct_cv[j0 + jl] - cvb - cv0, 0), max(nv - 1, 0));
  // the padding columns [ncv, ldw) multiply zero entries of W~: keep them zero (finite) in
  // the four contiguous vectors yr, yap, yar[0], yar[1]
  if (ldw > ncv)
    for (int e = threadIdx.x; e < 4 * (ldw - ncv); e += blockDim.x)
      yr[(e / (ldw - ncv)) * ldw + ncv + e % (ldw - ncv)] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  bool w_late = false;
  if (rows_sm > 0 && !mbar_wait(smem_u32(&wbar), 0, d.spin_limit)) {
    // the copy did not complete in time: report it and read every row from global memory
    if (threadIdx.x == 0) atomicOr(d.err, kErrTimeout);
    rows_sm = 0;
    w_late = true;
  }
  __syncthreads();
  // every CTA of the cluster must be running before shared memory is written remotely
  cl.sync();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // B v at owned contact vertex cvl: sum over its contacts of D_j^T (omega_j v_j)
  auto vertex_b = [&](const float* v, int cvl) {
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    const int jb0 = cvf[cvl], je0 = jb0 + cvn[cvl];
    for (int jl = jb0; jl < je0; ++jl) {
      const float* D = Df + 9 * jl;
      const float a0 = om[3 * jl] * v[3 * jl], a1 = om[3 * jl + 1] * v[3 * jl + 1],
                  a2 = om[3 * jl + 2] * v[3 * jl + 2];
      u0 += D[0] * a0 + D[3] * a1 + D[6] * a2;
      u1 += D[1] * a0 + D[4] * a1 + D[7] * a2;
      u2 += D[2] * a0 + D[5] * a1 + D[8] * a2;
    }
    return make_float4(u0, u1, u2, 0.f);
  };
  // B v of the owned vertices into `buf` of every CTA (one 16-byte remote store per
  // (rank, vertex), spread over all threads); v must be complete in shared memory
  auto publish = [&](const float* v, float4* buf) {
    for (int e = threadIdx.x; e < R * nv; e += blockDim.x) {
      const int r = e / nv, cvl = e - r * nv;
      cl.map_shared_rank(buf, r)[cv0 + cvl] = vertex_b(v, cvl);
    }
  };
  // wloc = W~ y_r over the owned rows
  auto product = [&]() {
    if (ldw <= 64 * kCrPairs) {
      unsigned long long ux[kCrPairs], uy[kCrPairs], uz[kCrPairs];
#pragma unroll
      for (int m = 0; m < kCrPairs; ++m) {
        const int col = 2 * lane + 64 * m;
        const float4 a = col < ldw ? yr[col] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = col < ldw ? yr[col + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        ux[m] = f2pack(a.x, b.x);
        uy[m] = f2pack(a.y, b.y);
        uz[m] = f2pack(a.z, b.z);
      }
      auto rows4 = [&](int r_begin, int r_end, auto row_ptr) {
        for (int row = r_begin + 4 * warp; row < r_end; row += 4 * nw) {
          const int nr = min(4, r_end - row);
          const float* w[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) w[k] = row_ptr(min(row + k, r_end - 1));
          unsigned long long acc[4][3];
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0ull;
#pragma unroll
          for (int m = 0; m < kCrPairs; ++m) {
            const int col = 2 * lane + 64 * m;
            if (col < ldw) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float2 p = *reinterpret_cast<const float2*>(w[k] + col);
                const unsigned long long pp = f2pack(p.x, p.y);
                acc[k][0] = ffma2(pp, ux[m], acc[k][0]);
                acc[k][1] = ffma2(pp, uy[m], acc[k][1]);
                acc[k][2] = ffma2(pp, uz[m], acc[k][2]);
              }
            }
          }
          float v[16];
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) v[3 * k + q] = f2lo(acc[k][q]) + f2hi(acc[k][q]);
          const float tot = warp_sum12(v, lane);
          const int idx = lane >> 1;
          if (!(lane & 1) && idx < 3 * nr) wloc[3 * row + idx] = tot;
        }
      };
      const int n_sm = min(rows_sm, nv);
      rows4(0, n_sm, [&](int r) { return static_cast<const float*>(wrows + (size_t)r * ldw); });
      rows4(n_sm, nv, [&](int r) { return wblk + (size_t)(cv0 + r) * ldw; });
    } else {
      // wide rows: four rows per warp at a time, 16-byte loads of W~ and y_r
      const int ng = ldw / 4;
      for (int row0 = 4 * warp; row0 < nv; row0 += 4 * nw) {
        float acc[4][3] = {};
        const int nrow = min(4, nv - row0);
        const float4* wrow[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = min(row0 + k, nv - 1);
          wrow[k] = reinterpret_cast<const float4*>(row < rows_sm ? wrows + (size_t)row * ldw
                                                                  : wblk + (size_t)(cv0 + row) * ldw);
        }
        for (int g4 = lane; g4 < ng; g4 += 32) {
          const float4 a = yr[4 * g4], b = yr[4 * g4 + 1], cc = yr[4 * g4 + 2], e = yr[4 * g4 + 3];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 w = wrow[k][g4];
            acc[k][0] += w.x * a.x + w.y * b.x + w.z * cc.x + w.w * e.x;
            acc[k][1] += w.x * a.y + w.y * b.y + w.z * cc.y + w.w * e.y;
            acc[k][2] += w.x * a.z + w.y * b.z + w.z * cc.z + w.w * e.z;
          }
        }
        float v[16];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int q = 0; q < 3; ++q) v[3 * k + q] = acc[k][q];
        const float tot = warp_sum12(v, lane);
        const int idx = lane >> 1;
        if (!(lane & 1) && idx < 3 * nrow) wloc[3 * row0 + idx] = tot;
      }
    }
  };
  // Ar = omega D (W~ y_r) + E r over the owned contacts, with the partial dot products
  // (r, Ar), (Ar, Ar), (Ar, Ap) of this CTA
  auto apply_dots = [&](float& s1, float& s2, float& s3) {
    s1 = s2 = s3 = 0.f;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      const int jl = e / 3, r = e % 3;
      const int cvl = ctl[jl];
      const float* D = Df + 9 * jl + 3 * r;
      const float dw = D[0] * wloc[3 * cvl] + D[1] * wloc[3 * cvl + 1] + D[2] * wloc[3 * cvl + 2];
      const float ar = om[e] * dw + ec[e] * vr[e];
      vAr[e] = ar;
      s1 += vr[e] * ar;
      s2 += ar * ar;
      s3 += ar * vAp[e];
    }
  };
  // reduce three values over the CTA (per warp, then warp 0 in warp order) and send them to
  // slot `rank` of dots buffer `buf` in every CTA; ends with the CTA's shared writes visible
  __shared__ float wpart[3][32];
  auto send_dots = [&](float a, float b, float cc, int buf) {
    a = warp_sum(a);
    b = warp_sum(b);
    cc = warp_sum(cc);
    if (lane == 0) {
      wpart[0][warp] = a;
      wpart[1][warp] = b;
      wpart[2][warp] = cc;
    }
    __syncthreads();
    if (warp == 0) {
      a = warp_sum(lane < nw ? wpart[0][lane] : 0.f);
      b = warp_sum(lane < nw ? wpart[1][lane] : 0.f);
      cc = warp_sum(lane < nw ? wpart[2][lane] : 0.f);
      if (lane < R) cl.map_shared_rank(dots + 16 * buf, lane)[rank] = make_float4(a, b, cc, 0.f);
    }
  };
  // the cluster-wide sums: every thread adds the ranks' partials in rank order, so every CTA
  // holds identical scalars (deterministic)
  auto gather_dots = [&](int buf) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = 0; r < R; ++r) {
      const float4 q = dots[16 * buf + r];
      t.x += q.x;
      t.y += q.y;
      t.z += q.z;
    }
    return t;
  };

  // r = rhs, x = 0: y_r = B r everywhere, then Ar = K r, p = r, Ap = Ar, y_Ap = B Ar
  publish(vr, yr);
  cl.sync();
  product();
  __syncthreads();
  float s1, s2, s3;
  apply_dots(s1, s2, s3);
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    vp[e] = vr[e];
    vAp[e] = vAr[e];
  }
  send_dots(s1, s2, 0.f, 0);
  publish(vAr, yar);
  cl.sync();
  float4 t = gather_dots(0);
  float rAr = t.x, ApAp = t.y;
  for (int i = threadIdx.x; i < ncv; i += blockDim.x) yap[i] = yar[i];
  __syncthreads();
  for (int it = 0; it < d.n_cr; ++it) {
    if (!(ApAp > 0.f)) break;   // identical scalars everywhere: a uniform exit
    const float alpha = rAr / ApAp;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vx[e] += alpha * vp[e];
      vr[e] -= alpha * vAp[e];
    }
    if (it == d.n_cr - 1) break;   // x is final; the last update needs no product
    for (int i = threadIdx.x; i < ncv; i += blockDim.x) {
      const float4 a = yr[i], b = yap[i];
      yr[i] = make_float4(a.x - alpha * b.x, a.y - alpha * b.y, a.z - alpha * b.z, 0.f);
    }
    __syncthreads();
    product();
    __syncthreads();
    apply_dots(s1, s2, s3);
    const int buf = (it + 1) & 1;
    send_dots(s1, s2, s3, buf);    // its barrier also publishes Ar within the CTA
    publish(vAr, yar + buf * ldw);
    cl.sync();
    t = gather_dots(buf);
    const float beta = rAr != 0.f ? t.x / rAr : 0.f;
    ApAp = t.y + 2.f * beta * t.z + beta * beta * ApAp;
    rAr = t.x;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vp[e] = vr[e] + beta * vp[e];
      vAp[e] = vAr[e] + beta * vAp[e];
    }
    const float4* yb = yar + buf * ldw;
    for (int i = threadIdx.x; i < ncv; i += blockDim.x) {
      const float4 a = yb[i], b = yap[i];
      yap[i] = make_float4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z, 0.f);
    }
    __syncthreads();
  }
  __syncthreads();
  // lambda += dlambda; u = B dlambda per owned contact vertex
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) d.ct_lam[3 * j0 + e] += (double)vx[e];
  for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
    const int cv = cvb + cv0 + cvl;
    const float4 u = vertex_b(vx, cvl);
    d.uvec[3 * cv] = u.x;
    d.uvec[3 * cv + 1] = u.y;
    d.uvec[3 * cv + 2] = u.z;
  }
  // a copy that timed out may still be in flight: give it another bounded wait before the
  // shared memory is released
  if (w_late) mbar_wait(smem_u32(&wbar), 0, d.spin_limit);
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

}  // namespace

void launch_scan(const int* in, int* out, int n, const int* n_dev, int* total, cudaStream_t s,
                 int* scratch, const int* skip) {
  if (!scratch || n <= kScanSplit) {
    k_scan<<<1, 1024, 0, s>>>(in, out, n, n_dev, total, skip);
    return;
  }
  // scratch: n_tiles tile sums, then their n_tiles + 1 offsets
  const int nt = (n + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<nt, 1024, 0, s>>>(in, n, n_dev, scratch, skip);
  k_scan<<<1, 1024, 0, s>>>(scratch, scratch + nt, nt, nullptr, nullptr, skip);
  k_scan_fin<<<nt, 1024, 0, s>>>(in, out, n, n_dev, scratch + nt, nt, total, skip);
}

int scan_launches(int n) { return n > kScanSplit ? 3 : 1; }
int scan_scratch_ints(int n) { return 2 * ((n + kScanTile - 1) / kScanTile) + 2; }

void launch_collide(const DevSim& d, cudaStream_t s) {
  const int g = (d.n + 63) / 64;
  if (d.bc_on) {
    k_body_box<<<d.n_bodies, kBoxThreads, 0, s>>>(d);
    k_chunk_box<<<((d.n_btri / kTriChunk + 1) * 32 + 127) / 128, 128, 0, s>>>(d);
    k_super_box<<<(d.n_btri / kTriSuper + 1 + 127) / 128, 128, 0, s>>>(d);
  }
  k_collide_count<<<g, 64, 0, s>>>(d);
  if (d.map_on) {
    k_corner_flag<<<(d.n + 255) / 256, 256, 0, s>>>(d);
    launch_scan(d.x_cnt, d.x_off, d.n, nullptr, nullptr, s, d.scan_part);
  }
  launch_scan(d.ct_cnt, d.ct_off, d.n, nullptr, d.counters + kCntContacts, s, d.scan_part);
  launch_scan(d.cv_flag, d.cv_off, d.n, nullptr, d.counters + kCntCv, s, d.scan_part);
  k_collide_write<<<g, 64, 0, s>>>(d);
  if (d.map_on) k_corner_sort<<<(d.n + 255) / 256, 256, 0, s>>>(d);
}

void launch_delassus(const DevSim& d, cudaStream_t s) {
  const int g = (d.n + 255) / 256;
  k_dl_check<<<1, 1024, 0, s>>>(d);
  const int* skip = d.dl_state;
  k_u_flag<<<g, 256, 0, s>>>(d);
  launch_scan(d.u_flag, d.u_off, d.n, nullptr, d.counters + kCntU, s, d.scan_part, skip);
  k_u_compact<<<g, 256, 0, s>>>(d);
  launch_scan(d.u_len, d.y_ptr, d.n, d.counters + kCntU, d.counters + kCntY, s, d.scan_part, skip);
  k_yc_len<<<(d.cap + 255) / 256, 256, 0, s>>>(d);
  launch_scan(d.yc_len, d.yc_ptr, d.cap, d.counters + kCntCv, d.counters + kCntYC, s, d.scan_part,
              skip);
  k_y_gather<<<std::min((d.n * 32 + 255) / 256, 8 * d.n_sm), 256, 0, s>>>(d);
  k_scene_ranges<<<1, 256, 0, s>>>(d);
  k_wt_blocks<<<(d.n / kWtKB + 1 + 127) / 128, 128, 0, s>>>(d);
  k_wt_items<<<d.wt_grid, kWtThreads, 0, s>>>(d);
  k_wt_reduce<<<2 * d.n_sm, 256, 0, s>>>(d);
  k_precond<<<(d.cap + 255) / 256, 256, 0, s>>>(d);
}

void launch_contact_eval(const DevSim& d, cudaStream_t s, int k, bool final_eval) {
  // FP64-heavy and short: small CTAs spread the contacts over many SMs
  k_contact_eval<<<(d.cap + 31) / 32, 32, 0, s>>>(d, k, final_eval ? 1 : 0);
}

namespace {

__global__ void k_iter_advance(DevSim d) {
  if (threadIdx.x == 0) *d.iter_k += 1;
}

// one thread: whether the while-node runs another iteration. It always terminates the loop
// at max_iters (<= kMaxIters) finished updates, whatever the residuals hold. The residual
// is the worst scene's; with a portfolio, a group counts with its best copy.
__global__ void k_iter_decide(DevSim d, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const int k = *d.iter_k;
  double r = d.resid[k];
  if (d.pf_copies > 1) {
    r = 0.0;
    for (int g0 = 0; g0 < d.n_scenes; g0 += d.pf_copies) {
      double best = INFINITY;
      for (int c = 0; c < d.pf_copies; ++c)
        best = fmin(best, d.resid_scene[(g0 + c) * (kMaxIters + 1) + k]);
      r = fmax(r, best);
    }
  }
  const bool more = k < d.max_iters && !(r <= d.res_tol) && *d.err == 0;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_iter_clear(DevSim d) {
  const int k = *d.iter_k;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.resid[k] = 0.0;
  for (int sc = threadIdx.x; sc < d.n_scenes; sc += blockDim.x)
    d.resid_scene[sc * (kMaxIters + 1) + k] = 0.0;
}

}  // namespace

void launch_iter_advance(const DevSim& d, cudaStream_t s) { k_iter_advance<<<1, 32, 0, s>>>(d); }

void launch_iter_decide(const DevSim& d, cudaStream_t s, cudaGraphConditionalHandle h) {
  k_iter_decide<<<1, 32, 0, s>>>(d, h);
}

void launch_iter_clear(const DevSim& d, cudaStream_t s) { k_iter_clear<<<1, 256, 0, s>>>(d); }

void launch_ytz(const DevSim& d, cudaStream_t s) {
  if (d.ytz_warp)
    launch_k(d.pdl, k_ytz_warp, std::min((d.cap + 7) / 8, 8 * d.n_sm), 256, 0, s, d);
  else
    launch_k(d.pdl, k_ytz, std::min(d.cap, 8 * d.n_sm), kYtzThreads, 0, s, d);
  if (d.map_on) launch_k(d.pdl, k_body_rhs, (d.cap + 127) / 128, 128, 0, s, d);
}

void launch_yu(const DevSim& d, cudaStream_t s) {
  launch_k(d.pdl, k_yu, std::min((d.n * 32 + 255) / 256, 8 * d.n_sm), 256, 0, s, d);
}

static size_t g_cr_smem = 0;

// Cluster size of the CR kernel: the largest R (16, 8, 4, 2, 1) such that one cluster per
// scene can be resident at once, then halved while a rank's share of the largest scene
// still fits in three quarters of a CTA's shared memory (its W~ rows for max_cv contact
// vertices and its contacts' vectors for max_ct contacts): a small scene's solve is then
// not spread over CTAs that mostly exchange. R = 1 when not even one cluster fits a wave.
int cr_setup(int n_scenes, int max_cv, int max_ct, int* cluster_out, size_t* smem_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t smem = (size_t)optin - 1024;  // leave room for static shared memory
  if (cudaFuncSetAttribute(k_cr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_cr1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SIM_ECUDA;
  cudaFuncSetAttribute(k_cr, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_cr1, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  int chosen = 0;
  for (int R : {16, 8, 4, 2, 1}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R);
    cfg.blockDim = dim3(kCrThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_cr, &cfg) == cudaSuccess &&
        (nclusters >= n_scenes || (R == 1 && nclusters > 0))) {
      chosen = R;
      break;
    }
    cudaGetLastError();
  }
  if (!chosen) return SIM_ECUDA;
  auto fits = [&](int R) {
    const size_t rows = (size_t)(max_cv + R - 1) / R, ld = (size_t)((max_cv + 3) & ~3);
    const size_t cts = (size_t)(max_ct + R - 1) / R;
    // W~ rows, u per component, per-vertex and per-contact vectors, dot slots and slack
    const size_t bytes = rows * ld * 4 + ld * 12 + rows * 48 + cts * 160 + 8192;
    return bytes <= smem * 3 / 4;
  };
  while (chosen > 1 && fits(chosen / 2)) chosen /= 2;
  g_cr_smem = smem;
  *cluster_out = chosen;
  *smem_out = smem;
  return SIM_OK;
}

int launch_cr(const DevSim& d, cudaStream_t s, int cluster) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * d.n_scenes);
  cfg.blockDim = dim3(kCrThreads);
  cfg.dynamicSmemBytes = g_cr_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = d.pdl ? 2 : 1;
  // one exchange per CR iteration when asked for and the scene has no contacts between
  // bodies; the two-exchange form otherwise
  const bool one = d.cr_single && !d.map_on;
  return cudaLaunchKernelEx(&cfg, one ? k_cr1 : k_cr, d, (int)g_cr_smem) == cudaSuccess ? SIM_OK
                                                                                       : SIM_ECUDA;
}

}  // namespace silg

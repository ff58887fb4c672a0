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

#include "device.cuh"

namespace cg = cooperative_groups;

namespace silg {
namespace {

constexpr int kCrThreads = 512;
constexpr double kTinyRel = 1e-12;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
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

__global__ void k_collide_count(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double x[3] = {d.s_tilde[3 * i], d.s_tilde[3 * i + 1], d.s_tilde[3 * i + 2]};
  int cnt = 0;
  for (int o = 0; o < d.n_obs; ++o) {
    double nn[3], ph[3];
    if (obst_query(d.obst[o], x, nn, ph) < d.margin) ++cnt;
  }
  d.ct_cnt[i] = cnt;
  d.cv_flag[i] = cnt > 0;
}

__global__ void k_collide_write(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && d.ct_off[d.n] > d.cap) atomicOr(d.err, kErrCapacity);
  if (i >= d.n || d.ct_cnt[i] == 0) return;
  double x[3] = {d.s_tilde[3 * i], d.s_tilde[3 * i + 1], d.s_tilde[3 * i + 2]};
  int j = d.ct_off[i];
  const int cv = d.cv_off[i];
  if (cv < d.cap) {
    d.cv_vert[cv] = i;
    d.cv_first[cv] = j;
    d.cv_nct[cv] = d.ct_cnt[i];
  }
  for (int o = 0; o < d.n_obs; ++o) {
    const ObstDev& ob = d.obst[o];
    double n[3], ph[3];
    if (!(obst_query(ob, x, n, ph) < d.margin)) continue;
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
      d.ct_dn[j] = n[0] * ph[0] + n[1] * ph[1] + n[2] * ph[2];
      d.ct_df[2 * j] = f1[0] * ob.vel[0] + f1[1] * ob.vel[1] + f1[2] * ob.vel[2];
      d.ct_df[2 * j + 1] = f2[0] * ob.vel[0] + f2[1] * ob.vel[1] + f2[2] * ob.vel[2];
      d.ct_mu[j] = ob.mu;
    }
    ++j;
  }
}

// single-CTA exclusive scan: out[k] = sum in[0..k), out[len] = total; *total = total
__global__ void __launch_bounds__(1024) k_scan(const int* in, int* out, int n_static,
                                               const int* n_dev, int* total) {
  __shared__ int wsum[32];
  int n = n_dev ? *n_dev : n_static;
  if (n < 0) n = 0;
  const int T = blockDim.x, tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int start = min(n, tid * per), end = min(n, start + per);
  int local = 0;
  for (int k = start; k < end; ++k) local += in[k];
  const int lane = tid & 31, wid = tid >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = (lane < T / 32) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  int run = incl - local + (wid > 0 ? wsum[wid - 1] : 0);
  for (int k = start; k < end; ++k) {
    int v = in[k];
    out[k] = run;
    run += v;
  }
  if (tid == 0) {
    int tot = wsum[31];
    out[n] = tot;
    if (total) *total = tot;
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

// rows of U: a is an ancestor of some contact vertex iff its subtree [fd(a), a] holds one
__global__ void k_u_flag(DevSim d) {
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
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.n || !d.u_flag[a]) return;
  int idx = d.u_off[a];
  d.u_list[idx] = a;
  d.u_clo[idx] = d.row_clo[a];
  d.u_len[idx] = d.row_len[a];
}

__global__ void k_yc_len(DevSim d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int ncv = min(d.counters[kCntCv], d.cap);
  if (c >= ncv) return;
  d.yc_len[c] = d.depth[d.cv_vert[c]];
}

// Y rows (row-major over U) and Y columns (contact vertex major, bottom-up along the
// ancestor path) gathered from the S~ profile.
__global__ void k_y_gather(DevSim d) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nU = d.counters[kCntU];
  if (warp >= nU) return;
  if (d.y_ptr[nU] > d.cap_y || d.yc_ptr[min(d.counters[kCntCv], d.cap)] > d.cap_y) {
    if (warp == 0 && lane == 0) atomicOr(d.err, kErrYCapacity);
    return;
  }
  const int a = d.u_list[warp];
  const int clo = d.u_clo[warp], len = d.u_len[warp];
  const float* srow = d.S + (d.rowbase[a] - d.lo[a]);
  const int base = d.y_ptr[warp];
  const int da = d.depth[a];
  for (int k = lane; k < len; k += 32) {
    const int c = clo + k;
    const int v = d.cv_vert[c];
    float val = srow[v];
    d.y_val[base + k] = val;
    const int pos = d.yc_ptr[c] + d.depth[v] - da;
    d.yc_val[pos] = val;
    d.yc_row[pos] = a;
  }
}

// W~ = Y^T Y, 64 x 64 output tiles of the lower triangle (mirrored), FP32. A row of Y
// touches the tile only if its contact-vertex range meets both column blocks; the CTA
// first compacts those rows (ranges are nested subtree intervals, so most rows below
// the top separators drop out for off-diagonal tiles), then accumulates 16 rows at a time.
constexpr int kWT = 64;
constexpr int kWTRows = 4096;   // compacted rows per chunk
__global__ void __launch_bounds__(256) k_wtilde(DevSim d) {
  const int ncv = min(d.counters[kCntCv], d.cap);
  const int ta = blockIdx.x, tb = blockIdx.y;
  if (tb > ta || ta * kWT >= ncv) return;
  const int nU = d.counters[kCntU];
  if (d.y_ptr[nU] > d.cap_y) return;
  __shared__ float As[16][kWT + 4], Bs[16][kWT + 4];
  __shared__ int rows[kWTRows];
  __shared__ int nrows;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  const int a0 = ta * kWT, b0 = tb * kWT;
  const int a1 = min(a0 + kWT, ncv), b1 = min(b0 + kWT, ncv);
  for (int chunk0 = 0; chunk0 < nU; chunk0 += kWTRows) {
    __syncthreads();
    if (threadIdx.x == 0) nrows = 0;
    __syncthreads();
    // deterministic compaction: ballot within warps, then warps in order
    const int chunk1 = min(nU, chunk0 + kWTRows);
    for (int base = chunk0; base < chunk1; base += blockDim.x) {
      const int u = base + threadIdx.x;
      bool keep = false;
      if (u < chunk1) {
        const int clo = d.u_clo[u], chi = clo + d.u_len[u];
        keep = clo < a1 && chi > a0 && clo < b1 && chi > b0;
      }
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      __shared__ int wcount[8];
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      if (lane == 0) wcount[wid] = __popc(ball);
      __syncthreads();
      int off = nrows;
      for (int w = 0; w < wid; ++w) off += wcount[w];
      if (keep) rows[off + __popc(ball & ((1u << lane) - 1))] = u;
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += wcount[w];
        nrows += t;
      }
      __syncthreads();
    }
    const int nr = nrows;
    for (int r0 = 0; r0 < nr; r0 += 16) {
      __syncthreads();
      for (int e = threadIdx.x; e < 16 * kWT; e += 256) {
        const int rl = e / kWT, cl = e % kWT;
        float va = 0.f, vb = 0.f;
        if (r0 + rl < nr) {
          const int u = rows[r0 + rl];
          const int clo = d.u_clo[u], len = d.u_len[u], base = d.y_ptr[u];
          const int ca = a0 + cl - clo, cb = b0 + cl - clo;
          if (ca >= 0 && ca < len) va = d.y_val[base + ca];
          if (cb >= 0 && cb < len) vb = d.y_val[base + cb];
        }
        As[rl][cl] = va;
        Bs[rl][cl] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = As[k][ty * 4 + q];
          bv[q] = Bs[k][tx * 4 + q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int ra = a0 + ty * 4 + p, cb = b0 + tx * 4 + q;
      if (ra < ncv && cb < ncv) {
        d.wt[(size_t)ra * ncv + cb] = acc[p][q];
        d.wt[(size_t)cb * ncv + ra] = acc[p][q];
      }
    }
}

__global__ void k_precond(DevSim d) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  int ncv = min(d.counters[kCntCv], d.cap);
  int cv = d.ct_cv[j];
  double w = (cv < ncv) ? (double)d.wt[(size_t)cv * ncv + cv] : 0.0;
  d.ct_r[2 * j] = d.h * d.h * w;
  d.ct_r[2 * j + 1] = d.h * w;
  for (int r = 0; r < 3; ++r) d.ct_lam[3 * j + r] = 0.0;
  for (int r = 0; r < 9; ++r) d.ct_Df[9 * j + r] = (float)d.ct_D[9 * j + r];
}

// Fischer-Burmeister terms at (q^k, lambda^k) for every contact (FP64).
__global__ void k_contact_eval(DevSim d, int k, int final_eval) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  const int v = d.ct_vert[j];
  const double h = d.h;
  double D[9];
  for (int r = 0; r < 9; ++r) D[r] = d.ct_D[9 * j + r];
  double dqv[3], q[3], qt[3];
  for (int r = 0; r < 3; ++r) {
    dqv[r] = (double)d.dq[3 * v + r];
    q[r] = d.q_ref[3 * v + r] + dqv[r];
    qt[r] = d.q_t[3 * v + r];
  }
  const double dn = D[0] * q[0] + D[1] * q[1] + D[2] * q[2] - d.ct_dn[j];
  double vf[2];
  for (int a = 0; a < 2; ++a) {
    const double* f = D + 3 + 3 * a;
    vf[a] = ((f[0] * (q[0] - qt[0]) + f[1] * (q[1] - qt[1]) + f[2] * (q[2] - qt[2])) -
             h * d.ct_df[2 * j + a]) / h;
  }
  const double ln = d.ct_lam[3 * j], lf0 = d.ct_lam[3 * j + 1], lf1 = d.ct_lam[3 * j + 2];
  const double rn = d.ct_r[2 * j], rf = d.ct_r[2 * j + 1], mu = d.ct_mu[j];
  // normal row (Eqs. 52-54)
  const double rho = sqrt(dn * dn + rn * rn * ln * ln);
  const double phin = dn + rn * ln - rho;
  double omn, En;
  if (rho == 0.0) {
    omn = 1.0;
    En = 0.0;
  } else {
    omn = 1.0 - dn / rho;
    En = (1.0 - rn * ln / rho) * rn;
  }
  // friction rows (Eqs. 55-57)
  double omf, Ef, phif0, phif1;
  if (ln <= 0.0 || mu <= 0.0) {
    omf = 0.0;
    Ef = 1.0;
    phif0 = lf0;
    phif1 = lf1;
  } else {
    const double a = sqrt(vf[0] * vf[0] + vf[1] * vf[1]);
    const double lf = sqrt(lf0 * lf0 + lf1 * lf1);
    const double s = mu * ln - lf;
    const double root = sqrt(a * a + rf * rf * s * s);
    const double num = root - rf * s;
    const double den = a + mu * rf * ln - root;
    const double scale = a + mu * rf * ln + rf * fabs(s);
    if (num <= kTinyRel * scale)
      Ef = 0.0;
    else if (den <= kTinyRel * scale)
      Ef = (a + rf * (lf - mu * ln)) / (mu * ln);
    else
      Ef = num / den * rf;
    omf = 1.0;
    phif0 = vf[0] + Ef * lf0;
    phif1 = vf[1] + Ef * lf1;
  }
  const double res = fmax(fabs(fmin(dn, rn * ln)), h * sqrt(phif0 * phif0 + phif1 * phif1)) / d.L_ref;
  atomic_max_nonneg(&d.resid[k], res);
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

// (Y^T z) per contact vertex, then the Schur right-hand side h^-2 (h - J A^-1 g) per contact
__global__ void k_ytz(DevSim d) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int ncv = min(d.counters[kCntCv], d.cap);
  if (c >= ncv) return;
  if (d.yc_ptr[ncv] > d.cap_y) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
  for (int k = d.yc_ptr[c] + lane; k < d.yc_ptr[c + 1]; k += 32) {
    const float y = d.yc_val[k];
    const int a = d.yc_row[k];
    s0 += y * d.zvec[a];
    s1 += y * d.zvec[d.n_pad + a];
    s2 += y * d.zvec[2 * d.n_pad + a];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  const double ih2 = 1.0 / (d.h * d.h);
  const int j0 = d.cv_first[c], j1 = min(j0 + d.cv_nct[c], d.cap);
  for (int j = j0 + lane; j < j1; j += 32) {
    for (int r = 0; r < 3; ++r) {
      const float* Dr = d.ct_Df + 9 * j + 3 * r;
      float jag = d.ct_omega[3 * j + r] * (Dr[0] * s0 + Dr[1] * s1 + Dr[2] * s2);
      d.ct_rhs[3 * j + r] = (float)((d.ct_hv[3 * j + r] - (double)jag) * ih2);
    }
  }
}

// y = z + h^2 Y u, in place on z (rows of U only)
__global__ void k_yu(DevSim d) {
  const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nU = d.counters[kCntU];
  if (idx >= nU || d.y_ptr[nU] > d.cap_y) return;
  const int clo = d.u_clo[idx], len = d.u_len[idx], base = d.y_ptr[idx];
  float t0 = 0.f, t1 = 0.f, t2 = 0.f;
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
    const float h2 = (float)(d.h * d.h);
    d.zvec[a] += h2 * t0;
    d.zvec[d.n_pad + a] += h2 * t1;
    d.zvec[2 * d.n_pad + a] += h2 * t2;
  }
}

// ---- conjugate residual in one thread-block cluster -----------------------------------
// Every CTA owns a contiguous range of contact vertices (and their contacts). The operator
// K = Omega W Omega + E is applied through W~: u_c = sum_{j at c} D_j^T (omega_j * v_j),
// w = W~ u, (K v)_j = omega_j * (D_j w_{c(j)}) + E_j * v_j. Owned slices of u are exchanged
// through distributed shared memory; dot products are reduced per CTA and then over the
// cluster in rank order, so every CTA holds the same scalars and the result is
// deterministic.
struct CrLayout {
  int R, rank, c, ncv, cv0, cv1, j0, j1;
};

__device__ int cv_split(const DevSim& d, int r, int R, int c, int ncv) {
  if (r >= R) return ncv;
  long long target = (long long)r * c / R;
  int lo = 0, hi = ncv;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (d.cv_first[mid] < target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ float block_sum(float v, float* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  float t = 0.f;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? scratch[lane] : 0.f;
    t = warp_sum(t);
  }
  return t;  // valid in warp 0
}

__global__ void __launch_bounds__(kCrThreads) k_cr(DevSim d, int smem_bytes) {
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cl = cg::this_cluster();
  CrLayout L;
  L.R = (int)cl.num_blocks();
  L.rank = (int)cl.block_rank();
  L.c = min(d.counters[kCntContacts], d.cap);
  L.ncv = min(d.counters[kCntCv], d.cap);
  // every CTA reads the same counters, so this exit is taken by all or by none
  if (L.c == 0 || L.ncv == 0) return;
  // split of the contact vertices over the cluster ranks, computed once per CTA
  __shared__ int split_cv[17], split_j[17];
  if (threadIdx.x <= L.R) {
    const int r = threadIdx.x;
    const int cv = cv_split(d, r, L.R, L.c, L.ncv);
    split_cv[r] = cv;
    split_j[r] = cv < L.ncv ? min(d.cv_first[cv], L.c) : L.c;
  }
  __syncthreads();
  L.cv0 = split_cv[L.rank];
  L.cv1 = split_cv[L.rank + 1];
  L.j0 = split_j[L.rank];
  L.j1 = max(split_j[L.rank + 1], L.j0);
  const int nj = L.j1 - L.j0, nv = L.cv1 - L.cv0;
  // the largest owned slice over the cluster decides, identically in every CTA, whether
  // the per-contact vectors fit in shared memory
  int nj_max = 0, nv_max = 0;
  for (int r = 0; r < L.R; ++r) {
    nj_max = max(nj_max, max(0, split_j[r + 1] - split_j[r]));
    nv_max = max(nv_max, split_cv[r + 1] - split_cv[r]);
  }
  // shared layout (same offsets in every CTA for the exchanged parts)
  float* dots = sm;                   // 8 floats, exchanged
  float* scratch = sm + 8;            // 32 floats
  float* uall = sm + 64;              // 3 ncv, own range exchanged
  float* wloc = uall + 3 * L.ncv;     // 3 nv
  float* vx = wloc + 3 * nv;          // per owned contact: x, r, p, Ar, Ap, rhs (3 each)
  float* vr = vx + 3 * nj;
  float* vp = vr + 3 * nj;
  float* vAr = vp + 3 * nj;
  float* vAp = vAr + 3 * nj;
  float* Df = vAp + 3 * nj;           // 9 nj
  float* om = Df + 9 * nj;            // 3 nj
  float* ec = om + 3 * nj;            // 3 nj
  float* wrows = ec + 3 * nj;         // nv x ncv if it fits
  const size_t used = (size_t)(wrows - sm) * sizeof(float);
  const size_t used_max = (size_t)(64 + 3 * L.ncv + 3 * nv_max + 30 * nj_max) * sizeof(float);
  const bool w_in_smem = used + (size_t)nv * L.ncv * sizeof(float) <= (size_t)smem_bytes;
  const float* wsrc = w_in_smem ? wrows : d.wt + (size_t)L.cv0 * L.ncv;
  if (used_max > (size_t)smem_bytes) {
    if (threadIdx.x == 0 && L.rank == 0) atomicOr(d.err, kErrCapacity);
    cl.sync();
    return;
  }
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    const int j = L.j0 + e / 3;
    vx[e] = 0.f;
    vr[e] = d.ct_rhs[3 * j + e % 3];
    om[e] = d.ct_omega[3 * j + e % 3];
    ec[e] = d.ct_ecal[3 * j + e % 3];
  }
  for (int e = threadIdx.x; e < 9 * nj; e += blockDim.x) Df[e] = d.ct_Df[9 * L.j0 + e];
  if (w_in_smem) {
    const float4* src = reinterpret_cast<const float4*>(d.wt + (size_t)L.cv0 * L.ncv);
    const size_t total = (size_t)nv * L.ncv;
    if ((((size_t)L.cv0 * L.ncv) & 3) == 0 && (reinterpret_cast<size_t>(wrows) & 15) == 0) {
      for (size_t e = threadIdx.x; e < total / 4; e += blockDim.x)
        reinterpret_cast<float4*>(wrows)[e] = src[e];
      for (size_t e = (total / 4) * 4 + threadIdx.x; e < total; e += blockDim.x)
        wrows[e] = d.wt[(size_t)L.cv0 * L.ncv + e];
    } else {
      for (size_t e = threadIdx.x; e < total; e += blockDim.x)
        wrows[e] = d.wt[(size_t)L.cv0 * L.ncv + e];
    }
  }
  __syncthreads();

  // K v -> Kv for the owned contacts
  auto apply = [&](const float* v, float* Kv) {
    for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
      const int cv = L.cv0 + cvl;
      float u0 = 0.f, u1 = 0.f, u2 = 0.f;
      const int jb = max(0, d.cv_first[cv] - L.j0), je = min(nj, jb + d.cv_nct[cv]);
      for (int jl = jb; jl < je; ++jl) {
        const float* D = Df + 9 * jl;
        float a0 = om[3 * jl] * v[3 * jl], a1 = om[3 * jl + 1] * v[3 * jl + 1],
              a2 = om[3 * jl + 2] * v[3 * jl + 2];
        u0 += D[0] * a0 + D[3] * a1 + D[6] * a2;
        u1 += D[1] * a0 + D[4] * a1 + D[7] * a2;
        u2 += D[2] * a0 + D[5] * a1 + D[8] * a2;
      }
      uall[3 * cv] = u0;
      uall[3 * cv + 1] = u1;
      uall[3 * cv + 2] = u2;
    }
    cl.sync();
    for (int r = 0; r < L.R; ++r) {
      if (r == L.rank) continue;
      const int a0 = split_cv[r], a1 = split_cv[r + 1];
      const float* src = cl.map_shared_rank(uall, r);
      for (int e = 3 * a0 + threadIdx.x; e < 3 * a1; e += blockDim.x) uall[e] = src[e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int cvl = warp; cvl < nv; cvl += nw) {
      const float* wr = wsrc + (size_t)cvl * L.ncv;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int k = lane; k < L.ncv; k += 32) {
        const float w = wr[k];
        s0 += w * uall[3 * k];
        s1 += w * uall[3 * k + 1];
        s2 += w * uall[3 * k + 2];
      }
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      if (lane == 0) {
        wloc[3 * cvl] = s0;
        wloc[3 * cvl + 1] = s1;
        wloc[3 * cvl + 2] = s2;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      const int jl = e / 3, r = e % 3;
      const int cvl = min(max(d.ct_cv[L.j0 + jl] - L.cv0, 0), max(nv - 1, 0));
      const float* D = Df + 9 * jl + 3 * r;
      const float dw = D[0] * wloc[3 * cvl] + D[1] * wloc[3 * cvl + 1] + D[2] * wloc[3 * cvl + 2];
      Kv[e] = om[e] * dw + ec[e] * v[e];
    }
    __syncthreads();
  };
  // cluster-wide sums of up to 3 values, identical in every CTA
  __shared__ float red_out[4];
  auto exchange = [&](float a, float b, float c3, int nvals) {
    float sa = block_sum(a, scratch);
    float sb = nvals > 1 ? block_sum(b, scratch) : 0.f;
    float sc = nvals > 2 ? block_sum(c3, scratch) : 0.f;
    if (threadIdx.x == 0) {
      dots[0] = sa;
      dots[1] = sb;
      dots[2] = sc;
    }
    cl.sync();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      float t[3] = {0.f, 0.f, 0.f};
      if (lane < L.R) {
        const float* src = cl.map_shared_rank(dots, lane);
        t[0] = src[0];
        t[1] = src[1];
        t[2] = src[2];
      }
      for (int q = 0; q < 3; ++q) {
        float v = warp_sum(t[q]);
        if (lane == 0) red_out[q] = v;
      }
    }
    __syncthreads();
  };

  // r = rhs, x = 0, p = r, Ap = Ar
  apply(vr, vAr);
  float pa = 0.f, pb = 0.f;
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
    vp[e] = vr[e];
    vAp[e] = vAr[e];
    pa += vr[e] * vAr[e];
    pb += vAr[e] * vAr[e];
  }
  exchange(pa, pb, 0.f, 2);
  float rAr = red_out[0], ApAp = red_out[1];
  for (int it = 0; it < d.n_cr; ++it) {
    if (!(ApAp > 0.f)) break;
    const float alpha = rAr / ApAp;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vx[e] += alpha * vp[e];
      vr[e] -= alpha * vAp[e];
    }
    __syncthreads();
    apply(vr, vAr);
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      s1 += vr[e] * vAr[e];
      s2 += vAr[e] * vAr[e];
      s3 += vAr[e] * vAp[e];
    }
    exchange(s1, s2, s3, 3);
    const float rAr_new = red_out[0], ArAr = red_out[1], ArAp = red_out[2];
    const float beta = rAr != 0.f ? rAr_new / rAr : 0.f;
    ApAp = ArAr + 2.f * beta * ArAp + beta * beta * ApAp;
    rAr = rAr_new;
    for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) {
      vp[e] = vr[e] + beta * vp[e];
      vAp[e] = vAr[e] + beta * vAp[e];
    }
    __syncthreads();
  }
  // lambda += dlambda; u = D^T (omega * dlambda) per owned contact vertex
  for (int e = threadIdx.x; e < 3 * nj; e += blockDim.x) d.ct_lam[3 * L.j0 + e] += (double)vx[e];
  for (int cvl = threadIdx.x; cvl < nv; cvl += blockDim.x) {
    const int cv = L.cv0 + cvl;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    const int jb = max(0, d.cv_first[cv] - L.j0), je = min(nj, jb + d.cv_nct[cv]);
    for (int jl = jb; jl < je; ++jl) {
      const float* D = Df + 9 * jl;
      float a0 = om[3 * jl] * vx[3 * jl], a1 = om[3 * jl + 1] * vx[3 * jl + 1],
            a2 = om[3 * jl + 2] * vx[3 * jl + 2];
      u0 += D[0] * a0 + D[3] * a1 + D[6] * a2;
      u1 += D[1] * a0 + D[4] * a1 + D[7] * a2;
      u2 += D[2] * a0 + D[5] * a1 + D[8] * a2;
    }
    d.uvec[3 * cv] = u0;
    d.uvec[3 * cv + 1] = u1;
    d.uvec[3 * cv + 2] = u2;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace

void launch_scan(const int* in, int* out, int n, const int* n_dev, int* total, cudaStream_t s) {
  k_scan<<<1, 1024, 0, s>>>(in, out, n, n_dev, total);
}

void launch_collide(const DevSim& d, cudaStream_t s) {
  const int g = (d.n + 255) / 256;
  k_collide_count<<<g, 256, 0, s>>>(d);
  launch_scan(d.ct_cnt, d.ct_off, d.n, nullptr, d.counters + kCntContacts, s);
  launch_scan(d.cv_flag, d.cv_off, d.n, nullptr, d.counters + kCntCv, s);
  k_collide_write<<<g, 256, 0, s>>>(d);
}

void launch_delassus(const DevSim& d, cudaStream_t s, int wt_tiles) {
  const int g = (d.n + 255) / 256;
  k_u_flag<<<g, 256, 0, s>>>(d);
  launch_scan(d.u_flag, d.u_off, d.n, nullptr, d.counters + kCntU, s);
  k_u_compact<<<g, 256, 0, s>>>(d);
  launch_scan(d.u_len, d.y_ptr, 0, d.counters + kCntU, d.counters + kCntY, s);
  k_yc_len<<<(d.cap + 255) / 256, 256, 0, s>>>(d);
  launch_scan(d.yc_len, d.yc_ptr, 0, d.counters + kCntCv, d.counters + kCntYC, s);
  k_y_gather<<<(d.n * 32 + 255) / 256, 256, 0, s>>>(d);
  dim3 grid(wt_tiles, wt_tiles);
  k_wtilde<<<grid, 256, 0, s>>>(d);
  k_precond<<<(d.cap + 255) / 256, 256, 0, s>>>(d);
}

void launch_contact_eval(const DevSim& d, cudaStream_t s, int k, bool final_eval) {
  k_contact_eval<<<(d.cap + 127) / 128, 128, 0, s>>>(d, k, final_eval ? 1 : 0);
}

void launch_ytz(const DevSim& d, cudaStream_t s) {
  k_ytz<<<(d.cap * 32 + 255) / 256, 256, 0, s>>>(d);
}

void launch_yu(const DevSim& d, cudaStream_t s) {
  k_yu<<<(d.n * 32 + 255) / 256, 256, 0, s>>>(d);
}

static size_t g_cr_smem = 0;

int cr_setup(int* cluster_out, size_t* smem_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t smem = (size_t)optin - 1024;  // leave room for static shared memory
  if (cudaFuncSetAttribute(k_cr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SIM_ECUDA;
  cudaFuncSetAttribute(k_cr, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_cr, &cfg) == cudaSuccess && nclusters > 0) {
      chosen = R;
      break;
    }
    cudaGetLastError();
  }
  if (!chosen) return SIM_ECUDA;
  g_cr_smem = smem;
  *cluster_out = chosen;
  *smem_out = smem;
  return SIM_OK;
}

int launch_cr(const DevSim& d, cudaStream_t s, int cluster) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kCrThreads);
  cfg.dynamicSmemBytes = g_cr_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cr, d, (int)g_cr_smem) == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

}  // namespace silg

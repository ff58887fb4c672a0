// Local step (Eq. 5) per tetrahedron, right-hand-side assembly (Eq. 6), frame start
// (prediction, Eq. 1) and integration (Alg. 4, last two lines).
//
// The local step forms F = D_s D_m^-1 from the frame's reference positions plus the
// iterate's FP32 displacement, computes the signed SVD by one-sided Jacobi rotations
// (Hestenes 1958; 3x3 columns orthogonalised pairwise, quadratic convergence), and
// projects the singular values per material:
//   ARAP          sigma_hat = (1, 1, 1)                     (PD indicator of SO(3))
//   co-rotational closed form of a linear 3x3 system in sigma
//   stable NH     Newton in sigma-space with backtracking (<= 20 steps, FP32)
// The frame's reference positions are kept as two FP32 words (hi + lo), so edge vectors
// x_a - x_0 are formed in FP32 as (hi_a - hi_0) + (lo_a - lo_0) without FP64 arithmetic.
// It then writes h^2 w_i (p_i - F_ref) g_a for the four corners a, where F_ref is the
// deformation gradient of the frame's reference state q_ref; the RHS is assembled in
// displacement form b - A q_ref, so the global solve yields q - q_ref directly.
#include <cuda_runtime.h>

#include "device.cuh"

namespace silg {
namespace {

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One-sided Jacobi SVD of a 3x3 matrix (row-major F): F = U diag(s) V^T with U, V
// rotations and the smallest |s| negative when det F < 0.
__device__ void svd3(const float* F, float* U, float* s, float* V) {
  float a[3][3], v[3][3];  // a[col][row], v[col][row]
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      a[c][r] = F[3 * r + c];
      v[c][r] = (r == c) ? 1.f : 0.f;
    }
  for (int sweep = 0; sweep < 10; ++sweep) {
    bool rotated = false;
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
      const int p = pr == 2 ? 1 : 0;
      const int q = pr == 0 ? 1 : 2;
      float al = dot3(a[p], a[p]), be = dot3(a[q], a[q]), ga = dot3(a[p], a[q]);
      if (!(fabsf(ga) > 1e-7f * sqrtf(al * be))) continue;
      rotated = true;
      float zeta = (be - al) / (2.f * ga);
      float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
      float c = 1.f / sqrtf(1.f + t * t);
      float sn = c * t;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        float ap = a[p][r], aq = a[q][r];
        a[p][r] = c * ap - sn * aq;
        a[q][r] = sn * ap + c * aq;
        float vp = v[p][r], vq = v[q][r];
        v[p][r] = c * vp - sn * vq;
        v[q][r] = sn * vp + c * vq;
      }
    }
    if (!rotated) break;
  }
  float sg[3], u[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sg[c] = sqrtf(dot3(a[c], a[c]));
    float inv = sg[c] > 0.f ? 1.f / sg[c] : 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) u[c][r] = a[c][r] * inv;
  }
  int kmin = 0;
  if (sg[1] < sg[kmin]) kmin = 1;
  if (sg[2] < sg[kmin]) kmin = 2;
  float smax = fmaxf(sg[0], fmaxf(sg[1], sg[2]));
  float detF = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
               F[2] * (F[3] * F[7] - F[4] * F[6]);
  if (sg[kmin] <= 1e-6f * smax) {
    // (nearly) rank deficient: complete U to a right-handed frame
    const int i = (kmin + 1) % 3, j = (kmin + 2) % 3;
    u[kmin][0] = u[i][1] * u[j][2] - u[i][2] * u[j][1];
    u[kmin][1] = u[i][2] * u[j][0] - u[i][0] * u[j][2];
    u[kmin][2] = u[i][0] * u[j][1] - u[i][1] * u[j][0];
    if (detF < 0.f) sg[kmin] = -sg[kmin];
  } else {
    float du = u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
               u[1][0] * (u[0][1] * u[2][2] - u[0][2] * u[2][1]) +
               u[2][0] * (u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    if (du < 0.f) {
      sg[kmin] = -sg[kmin];
#pragma unroll
      for (int r = 0; r < 3; ++r) u[kmin][r] = -u[kmin][r];
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s[c] = sg[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      U[3 * r + c] = u[c][r];
      V[3 * r + c] = v[c][r];
    }
  }
}

__device__ float snh_objective(const float* x, const float* s, float w, float V, float mu,
                               float lam, float alpha) {
  float d0 = x[0] - s[0], d1 = x[1] - s[1], d2 = x[2] - s[2];
  float ic = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  float J = x[0] * x[1] * x[2];
  float psi = 0.5f * mu * (ic - 3.f) + 0.5f * lam * (J - alpha) * (J - alpha) -
              0.5f * mu * logf(ic + 1.f);
  return 0.5f * w * (d0 * d0 + d1 * d1 + d2 * d2) + V * psi;
}

// argmin_x w/2 |x - s|^2 + V psi_SNH(x) by Newton with Armijo backtracking.
__device__ void snh_sigma(const float* s, float w, float V, float mu, float lam, float alpha,
                          float* x) {
  x[0] = s[0];
  x[1] = s[1];
  x[2] = s[2];
  const float scale = w + V * (mu + lam);
  for (int it = 0; it < 20; ++it) {
    float ic = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    float J = x[0] * x[1] * x[2];
    float dJ[3] = {x[1] * x[2], x[0] * x[2], x[0] * x[1]};
    float ic1 = ic + 1.f;
    float g[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      g[i] = w * (x[i] - s[i]) + V * (mu * x[i] + lam * (J - alpha) * dJ[i] - mu * x[i] / ic1);
    float xm = fmaxf(1.f, fmaxf(fabsf(x[0]), fmaxf(fabsf(x[1]), fabsf(x[2]))));
    float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn <= 1e-6f * scale * xm) break;
    float H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float d2J = (i == j) ? 0.f : x[3 - i - j];
        float eye = (i == j) ? 1.f : 0.f;
        H[i][j] = w * eye + V * (mu * eye + lam * (dJ[i] * dJ[j] + (J - alpha) * d2J) -
                                 mu * (eye / ic1 - 2.f * x[i] * x[j] / (ic1 * ic1)));
      }
    // Cholesky with an increasing diagonal shift until positive definite
    float L00 = 0, L10 = 0, L11 = 0, L20 = 0, L21 = 0, L22 = 0;
    float tau = 0.f;
    bool ok = false;
    for (int attempt = 0; attempt < 12 && !ok; ++attempt) {
      float a00 = H[0][0] + tau, a11 = H[1][1] + tau, a22 = H[2][2] + tau;
      ok = false;
      if (a00 > 1e-12f * scale) {
        L00 = sqrtf(a00);
        L10 = H[1][0] / L00;
        L20 = H[2][0] / L00;
        float t11 = a11 - L10 * L10;
        if (t11 > 1e-12f * scale) {
          L11 = sqrtf(t11);
          L21 = (H[2][1] - L20 * L10) / L11;
          float t22 = a22 - L20 * L20 - L21 * L21;
          if (t22 > 1e-12f * scale) {
            L22 = sqrtf(t22);
            ok = true;
          }
        }
      }
      tau = tau > 0.f ? 4.f * tau : 1e-4f * scale;
    }
    if (!ok) break;
    float y0 = -g[0] / L00;
    float y1 = (-g[1] - L10 * y0) / L11;
    float y2 = (-g[2] - L20 * y0 - L21 * y1) / L22;
    float d[3];
    d[2] = y2 / L22;
    d[1] = (y1 - L21 * d[2]) / L11;
    d[0] = (y0 - L10 * d[1] - L20 * d[2]) / L00;
    float f0 = snh_objective(x, s, w, V, mu, lam, alpha);
    float slope = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
    float t = 1.f;
    float xc[3];
    for (int ls = 0; ls < 24; ++ls) {
      xc[0] = x[0] + t * d[0];
      xc[1] = x[1] + t * d[1];
      xc[2] = x[2] + t * d[2];
      float f1 = snh_objective(xc, s, w, V, mu, lam, alpha);
      if (f1 <= f0 + 1e-4f * t * slope + 4e-7f * fabsf(f0)) break;
      t *= 0.5f;
    }
    float step = t * fmaxf(fabsf(d[0]), fmaxf(fabsf(d[1]), fabsf(d[2])));
    x[0] = xc[0];
    x[1] = xc[1];
    x[2] = xc[2];
    if (step <= 1e-7f * xm) break;
  }
}

__device__ void project_tet(const float* F, int model, float w, float V, float mu, float lam,
                            float alpha, float* p) {
  float U[9], s[3], Vm[9], sh[3];
  svd3(F, U, s, Vm);
  if (model == SIM_MODEL_COROT) {
    float a = w + 2.f * mu * V, c = lam * V;
    float k = 2.f * mu * V + 3.f * lam * V;
    float r0 = w * s[0] + k, r1 = w * s[1] + k, r2 = w * s[2] + k;
    float S = (r0 + r1 + r2) / (a + 3.f * c);
    sh[0] = (r0 - c * S) / a;
    sh[1] = (r1 - c * S) / a;
    sh[2] = (r2 - c * S) / a;
  } else if (model == SIM_MODEL_SNH) {
    snh_sigma(s, w, V, mu, lam, alpha, sh);
  } else {
    sh[0] = sh[1] = sh[2] = 1.f;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      p[3 * r + c] = U[3 * r + 0] * sh[0] * Vm[3 * c + 0] + U[3 * r + 1] * sh[1] * Vm[3 * c + 1] +
                     U[3 * r + 2] * sh[2] * Vm[3 * c + 2];
}

__device__ __forceinline__ void split_ref(const DevSim& d, int i, int r, double q) {
  const float hi = (float)q;
  d.qr_hi[3 * i + r] = hi;
  d.qr_lo[3 * i + r] = (float)(q - (double)hi);
}

__global__ void k_frame_begin(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_all) return;
  const double h = d.h;
  if (i < d.n && d.n_anc > 0) {
    // the vertex's anchor target moves to the end of this frame
    const int a = d.anc_of[i];
    if (a >= 0)
      for (int r = 0; r < 3; ++r) d.anc_pos[3 * a + r] += h * d.anc_vel[3 * a + r];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double qt = d.q_t[3 * i + r];
    if (i < d.n) {
      double st = qt + h * d.v_t[3 * i + r] + h * h * d.grav[r];
      d.s_tilde[3 * i + r] = st;
      d.q_ref[3 * i + r] = qt;
      d.dq[3 * i + r] = (float)(st - qt);
      split_ref(d, i, r, qt);
    } else {
      double qp = qt + h * d.scene_hvel[3 * d.vert_scene[i] + r];
      d.s_tilde[3 * i + r] = qp;
      d.q_ref[3 * i + r] = qp;
      d.dq[3 * i + r] = 0.f;
      split_ref(d, i, r, qp);
    }
  }
}

// q_ref -> (hi, lo) for callers that set q_ref directly (component entry points)
__global__ void k_split_ref(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_all) return;
#pragma unroll
  for (int r = 0; r < 3; ++r) split_ref(d, i, r, d.q_ref[3 * i + r]);
}

template <bool kDebug>
__global__ void __launch_bounds__(128) k_local(DevSim d) {
  pdl_wait();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tets) return;
  const int T = d.n_tets;
  int4 vi = d.tet_v[t];
  int vv[4] = {vi.x, vi.y, vi.z, vi.w};
  float Mi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Mi[k] = d.tet_dminv[k * T + t];
  float g[4][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[1][c] = Mi[c];
    g[2][c] = Mi[3 + c];
    g[3][c] = Mi[6 + c];
    g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  }
  float h0[3], l0[3], dq0[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    h0[r] = d.qr_hi[3 * vv[0] + r];
    l0[r] = d.qr_lo[3 * vv[0] + r];
    dq0[r] = d.dq[3 * vv[0] + r];
  }
  float Fr[9], F[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Fr[k] = F[k] = 0.f;
#pragma unroll
  for (int a = 1; a < 4; ++a) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float er = (d.qr_hi[3 * vv[a] + r] - h0[r]) + (d.qr_lo[3 * vv[a] + r] - l0[r]);
      float ed = d.dq[3 * vv[a] + r] - dq0[r];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Fr[3 * r + c] += er * g[a][c];
        F[3 * r + c] += (er + ed) * g[a][c];
      }
    }
  }
  const MatDev m = d.mats[d.tet_mat[t]];
  const float w = d.tet_w[t], V = d.tet_vol[t];
  float p[9];
  if (d.admm && !kDebug) {
    // ADMM-PD: z = prox at F + u (ARAP as mu |F - R|^2: co-rotational with lambda = 0),
    // u += F - z, and the global step reads z - u
    float y[9], u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      u[k] = d.tet_u[(size_t)k * T + t];
      y[k] = F[k] + u[k];
    }
    const bool arap = m.model == SIM_MODEL_ARAP;
    project_tet(y, arap ? SIM_MODEL_COROT : m.model, w, V, m.mu, arap ? 0.f : m.lam, m.alpha, p);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float un = u[k] + F[k] - p[k];
      d.tet_u[(size_t)k * T + t] = un;
      p[k] -= un;
    }
  } else {
    project_tet(F, m.model, w, V, m.mu, m.lam, m.alpha, p);
  }
  if (kDebug) {
#pragma unroll
    for (int k = 0; k < 9; ++k) d.p_out[9 * t + k] = p[k];
    return;
  }
  const float s = d.h2f * w;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float o[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      o[r] = s * ((p[3 * r] - Fr[3 * r]) * g[a][0] + (p[3 * r + 1] - Fr[3 * r + 1]) * g[a][1] +
                  (p[3 * r + 2] - Fr[3 * r + 2]) * g[a][2]);
    const int sl = d.inc_slot[4 * t + a];
    if (sl >= 0) d.contrib[sl] = make_float4(o[0], o[1], o[2], 0.f);
  }
}

// The local step of a triangle (membrane) element: F = [x1 - x0, x2 - x0] D_m^-1 (3 x 2),
// p = U diag(sigma_hat) V^T over the thin SVD, written as p = F V diag(sigma_hat / sigma) V^T
// with V and sigma^2 the eigenpairs of the 2 x 2 F^T F (a Jacobi rotation). ARAP:
// sigma_hat = 1 (the closest matrix with orthonormal columns); co-rotational: the closed-form
// minimiser of w/2 |x - sigma|^2 + V (mu |x - 1|^2 + lam/2 (sum x - 2)^2). Corner a's
// contribution h^2 w (p - F_ref) g_a goes to the incidence slot of element entry
// 4 n_tets + 3 t + a.
__global__ void __launch_bounds__(128) k_local_tri(DevSim d) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tris) return;
  const int Nt = d.n_tris;
  const int4 vi = d.tri_v[t];
  const int vv[3] = {vi.x, vi.y, vi.z};
  const float M0 = d.tri_dminv[t], M1 = d.tri_dminv[Nt + t], M2 = d.tri_dminv[2 * Nt + t],
              M3 = d.tri_dminv[3 * Nt + t];
  float g[3][2];
  g[1][0] = M0;
  g[1][1] = M1;
  g[2][0] = M2;
  g[2][1] = M3;
  g[0][0] = -(M0 + M2);
  g[0][1] = -(M1 + M3);
  float h0[3], l0[3], dq0[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    h0[r] = d.qr_hi[3 * vv[0] + r];
    l0[r] = d.qr_lo[3 * vv[0] + r];
    dq0[r] = d.dq[3 * vv[0] + r];
  }
  float Fr[6], F[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) Fr[k] = F[k] = 0.f;
#pragma unroll
  for (int a = 1; a < 3; ++a) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float er = (d.qr_hi[3 * vv[a] + r] - h0[r]) + (d.qr_lo[3 * vv[a] + r] - l0[r]);
      const float ed = d.dq[3 * vv[a] + r] - dq0[r];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        Fr[2 * r + c] += er * g[a][c];
        F[2 * r + c] += (er + ed) * g[a][c];
      }
    }
  }
  // C = F^T F and its eigenpairs
  const float c00 = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
  const float c01 = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
  const float c11 = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
  const float th = 0.5f * atan2f(2.f * c01, c00 - c11);
  const float cs = cosf(th), sn = sinf(th);
  const float mid = 0.5f * (c00 + c11), rad = sqrtf(0.25f * (c00 - c11) * (c00 - c11) + c01 * c01);
  const float s0 = sqrtf(fmaxf(mid + rad, 0.f)), s1 = sqrtf(fmaxf(mid - rad, 0.f));
  const MatDev m = d.mats[d.tri_mat[t]];
  const float w = d.tri_w[t], V = d.tri_vol[t];
  float x0 = 1.f, x1 = 1.f;
  if (m.model == SIM_MODEL_COROT) {
    const float a = w + 2.f * m.mu * V, c = m.lam * V;
    const float k = 2.f * m.mu * V + 2.f * m.lam * V;
    const float r0 = w * s0 + k, r1 = w * s1 + k;
    const float S = (r0 + r1) / (a + 2.f * c);
    x0 = (r0 - c * S) / a;
    x1 = (r1 - c * S) / a;
  }
  // p = F M with M = V diag(x / s) V^T (the eigenvectors (cs, sn) and (-sn, cs)); a
  // collapsed direction keeps its ratio finite
  const float k0 = x0 / fmaxf(s0, 1e-12f), k1 = x1 / fmaxf(s1, 1e-12f);
  const float m00 = k0 * cs * cs + k1 * sn * sn, m11 = k0 * sn * sn + k1 * cs * cs;
  const float m01 = (k0 - k1) * cs * sn;
  float p[6];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    p[2 * r] = F[2 * r] * m00 + F[2 * r + 1] * m01;
    p[2 * r + 1] = F[2 * r] * m01 + F[2 * r + 1] * m11;
  }
  const float sc = d.h2f * w;
  const size_t base = 4 * (size_t)d.n_tets + 3 * (size_t)t;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float o[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      o[r] = sc * ((p[2 * r] - Fr[2 * r]) * g[a][0] + (p[2 * r + 1] - Fr[2 * r + 1]) * g[a][1]);
    const int sl = d.inc_slot[base + a];
    if (sl >= 0) d.contrib[sl] = make_float4(o[0], o[1], o[2], 0.f);
  }
}

// The bending term's part of b - A q_ref, -h^2 K q_ref for every free vertex (the rest
// curvature is zero, so the term has no projection); once per frame, after q_ref is set.
__global__ void k_bend_force(DevSim d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double f[3] = {0.0, 0.0, 0.0};
  for (int e = d.bend_ptr[i]; e < d.bend_ptr[i + 1]; ++e) {
    const double k = d.bend_val[e];
    const int j = d.bend_idx[e];
#pragma unroll
    for (int r = 0; r < 3; ++r) f[r] += k * d.q_ref[3 * j + r];
  }
  const double h2 = d.h * d.h;
#pragma unroll
  for (int r = 0; r < 3; ++r) d.bend_f[3 * i + r] = (float)(-h2 * f[r]);
}

// b_i - (A q_ref)_i + h^2 (J^T lambda)_i for every free vertex i, written as the FP32 SoA
// vector g of the first profile product.
// b_i = M_i (s~_i - q_ref_i) + sum of the vertex's element contributions + h^2 (contact
// forces), for the free vertex i. kRhsLanes lanes share a vertex: each sums a strided part of
// its incidence list, the parts meet in a fixed shuffle tree (deterministic), so the
// dependent gathers of one thread shrink by that factor.
constexpr int kRhsLanes = 8;
__global__ void k_rhs(DevSim d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / kRhsLanes, sub = t % kRhsLanes;
  // the grid is exactly n_pad * kRhsLanes threads (n_pad is a multiple of 256), so every
  // lane of a warp reaches the shuffles below
  float e[3] = {0.f, 0.f, 0.f};
  const int k0 = i < d.n ? d.inc_ptr[i] : 0, k1 = i < d.n ? d.inc_ptr[i + 1] : 0;
  for (int k = k0 + sub; k < k1; k += kRhsLanes) {
    const float4 c = d.contrib[k];   // the vertex's run of incidence slots
    e[0] += c.x;
    e[1] += c.y;
    e[2] += c.z;
  }
  const unsigned mask = 0xffffffffu;
#pragma unroll
  for (int o = kRhsLanes / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < 3; ++r) e[r] += __shfl_xor_sync(mask, e[r], o, kRhsLanes);
  if (sub != 0) return;
  if (i >= d.n) {
    d.gvec[i] = d.gvec[d.n_pad + i] = d.gvec[2 * d.n_pad + i] = 0.f;
    return;
  }
  const double m = d.mass[i];
  double b[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) b[r] = m * (d.s_tilde[3 * i + r] - d.q_ref[3 * i + r]);
  const double h2 = d.h * d.h;
  const int nc = d.ct_cnt[i];
  if (nc > 0) {
    const int j0 = d.ct_off[i];
    for (int j = j0; j < j0 + nc && j < d.cap; ++j)
#pragma unroll
      for (int r = 0; r < 3; ++r) b[r] += h2 * d.ct_force[3 * j + r];
  }
  if (d.map_on) {
    // the vertex as a corner of other bodies' contacts (or the partner of a two-vertex
    // anchor row): -w_k of their force
    const int xe = min(d.x_off[i + 1], 3 * d.cap);
    for (int e = d.x_off[i]; e < xe; ++e) {
      const int tk = d.x_list[e];
      if (tk < 0) continue;   // a contact beyond the capacity
      const double w = d.ct_bw[tk];
#pragma unroll
      for (int r = 0; r < 3; ++r) b[r] -= h2 * w * d.ct_force[3 * (tk / 3) + r];
    }
  }
  if (d.bend_f)
#pragma unroll
    for (int r = 0; r < 3; ++r) e[r] += d.bend_f[3 * i + r];
#pragma unroll
  for (int r = 0; r < 3; ++r) d.gvec[r * d.n_pad + i] = (float)(b[r] + (double)e[r]);
}

__global__ void k_integrate(DevSim d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_all) return;
  bool bad = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double qn = d.q_ref[3 * i + r] + (double)d.dq[3 * i + r];
    double vn = (qn - d.q_t[3 * i + r]) / d.h;
    bad |= !isfinite(qn) || !isfinite(vn);
    d.q_t[3 * i + r] = qn;
    d.v_t[3 * i + r] = vn;
  }
  if (bad) atomicOr(d.err, kErrNonFinite);
}

}  // namespace

void launch_frame_begin(const DevSim& d, cudaStream_t s) {
  k_frame_begin<<<(d.n_all + 255) / 256, 256, 0, s>>>(d);
  if (d.bend_ptr) k_bend_force<<<(d.n + 255) / 256, 256, 0, s>>>(d);
}

void launch_local(const DevSim& d, cudaStream_t s, bool debug_p) {
  int grid = (d.n_tets + 127) / 128;
  if (debug_p) {
    k_split_ref<<<(d.n_all + 255) / 256, 256, 0, s>>>(d);
    if (grid > 0) k_local<true><<<grid, 128, 0, s>>>(d);
  } else {
    if (grid > 0) launch_k(d.pdl, k_local<false>, grid, 128, 0, s, d);
    if (d.n_tris > 0) launch_k(d.pdl, k_local_tri, (d.n_tris + 127) / 128, 128, 0, s, d);
  }
}

void launch_rhs(const DevSim& d, cudaStream_t s) {
  k_rhs<<<(d.n_pad * kRhsLanes + 255) / 256, 256, 0, s>>>(d);
}

void launch_integrate(const DevSim& d, cudaStream_t s) {
  k_integrate<<<(d.n_all + 255) / 256, 256, 0, s>>>(d);
}

}  // namespace silg

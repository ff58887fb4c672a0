// Fischer-Burmeister terms of one contact (App. B.2), shared by the per-iteration contact
// evaluation and the warm start's choice between its guess and the cold start (FP64).
#pragma once

#include "device.cuh"

namespace silg {

constexpr double kFbTinyRel = 1e-12;

struct FbTerms {
  double dn;            // delta_n = n . q - d_n
  double vf[2];         // tangential velocity relative to the obstacle
  double phin, omn, En; // normal row (Eqs. 52-54)
  double phif0, phif1, omf, Ef;  // friction rows (Eqs. 55-57)
  double res;           // the residual measure max(|min(dn, r_n lambda_n)|, h |phi_f|) / L
};

// contact j at vertex position q (world) with impulses lam (n, f1, f2); L: residual scale
__device__ inline FbTerms fb_terms(const DevSim& d, int j, const double q[3], const double lam[3],
                                   double L) {
  FbTerms o;
  const int v = d.ct_vert[j];
  const double h = d.h;
  const double* D = d.ct_D + 9 * j;
  double qt[3];
  for (int r = 0; r < 3; ++r) qt[r] = d.q_t[3 * v + r];
  o.dn = D[0] * q[0] + D[1] * q[1] + D[2] * q[2] - d.ct_dn[j];
  for (int a = 0; a < 2; ++a) {
    const double* f = D + 3 + 3 * a;
    o.vf[a] = ((f[0] * (q[0] - qt[0]) + f[1] * (q[1] - qt[1]) + f[2] * (q[2] - qt[2])) -
               h * d.ct_df[2 * j + a]) / h;
  }
  const double ln = lam[0], lf0 = lam[1], lf1 = lam[2];
  const double rn = d.ct_r[2 * j], rf = d.ct_r[2 * j + 1], mu = d.ct_mu[j];
  const double dn = o.dn;
  const double rho = sqrt(dn * dn + rn * rn * ln * ln);
  o.phin = dn + rn * ln - rho;
  if (rho == 0.0) {
    o.omn = 1.0;
    o.En = 0.0;
  } else {
    o.omn = 1.0 - dn / rho;
    o.En = (1.0 - rn * ln / rho) * rn;
  }
  if (ln <= 0.0 || mu <= 0.0) {
    o.omf = 0.0;
    o.Ef = 1.0;
    o.phif0 = lf0;
    o.phif1 = lf1;
  } else {
    const double a = sqrt(o.vf[0] * o.vf[0] + o.vf[1] * o.vf[1]);
    const double lf = sqrt(lf0 * lf0 + lf1 * lf1);
    const double s = mu * ln - lf;
    const double root = sqrt(a * a + rf * rf * s * s);
    const double num = root - rf * s;
    const double den = a + mu * rf * ln - root;
    const double scale = a + mu * rf * ln + rf * fabs(s);
    if (num <= kFbTinyRel * scale)
      o.Ef = 0.0;
    else if (den <= kFbTinyRel * scale)
      o.Ef = (a + rf * (lf - mu * ln)) / (mu * ln);
    else
      o.Ef = num / den * rf;
    o.omf = 1.0;
    o.phif0 = o.vf[0] + o.Ef * lf0;
    o.phif1 = o.vf[1] + o.Ef * lf1;
  }
  o.res = fmax(fabs(fmin(dn, rn * ln)), h * sqrt(o.phif0 * o.phif0 + o.phif1 * o.phif1)) / L;
  return o;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace silg

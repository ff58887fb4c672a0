// Complementarity terms of one contact, shared by the per-iteration contact evaluation and
// the warm start's choice between its guess and the cold start (FP64): the
// Fischer-Burmeister functions (App. B.2) or the minimum map (App. B.1), and the residual
// measure, which is the same for both.
#pragma once

#include "device.cuh"

namespace silg {

constexpr double kFbTinyRel = 1e-12;
// Friction rows are active when the normal impulse is resolvable, r_n lambda_n > kActiveRel L
// (r_n from the Delassus diagonal, L the scene's length): App. B.1-B.2 write lambda_n > 0,
// but a normal impulse cancelled by the Newton step lands on rounding residues of either
// sign (about 1e-7 of the cancelled value in FP32), and a positive residue would switch on
// a friction compliance ~ |v_f| / (mu lambda_n) that swamps the constraint solve.
constexpr double kActiveRel = 1e-6;

struct FbTerms {
  double dn;            // delta_n = n . q - d_n
  double vf[2];         // tangential velocity relative to the obstacle
  double phin, omn, En; // normal row (Eqs. 52-54, or App. B.1)
  double phif0, phif1, omf, Ef;  // friction rows (Eqs. 55-57, or App. B.1)
  double res;           // the residual measure max(|min(dn, r_n lambda_n)|, h |phi_f|) / L
  bool bilateral;       // an anchor: phin, phif0, phif1 are its three position-level rows
                        // phi_b = q - p + e lambda, En = Ef = e, omn = omf = 1, res =
                        // max |phi_b| / L
};

// Normal and friction rows at gap dn, tangential velocity vf, impulses (ln, lf0, lf1) with
// preconditioner (rn, rf): Fischer-Burmeister (minmap = false) or minimum map; active: the
// friction activity decision.
__device__ inline void ncp_rows(bool minmap, double dn, const double vf[2], double ln,
                                double lf0, double lf1, double rn, double rf, double mu,
                                bool active, FbTerms& o) {
  if (minmap) {
    // min(delta_n, r_n lambda_n): the gap branch (ties included) or the impulse branch
    if (dn <= rn * ln) {
      o.phin = dn;
      o.omn = 1.0;
      o.En = 0.0;
    } else {
      o.phin = rn * ln;
      o.omn = 0.0;
      o.En = rn;
    }
  } else {
    const double rho = sqrt(dn * dn + rn * rn * ln * ln);
    o.phin = dn + rn * ln - rho;
    if (rho == 0.0) {
      o.omn = 1.0;
      o.En = 0.0;
    } else {
      o.omn = 1.0 - dn / rho;
      o.En = (1.0 - rn * ln / rho) * rn;
    }
  }
  if (!active || mu <= 0.0) {
    // inactive friction in both forms: phi_f = lambda_f drives the impulse to zero
    o.omf = 0.0;
    o.Ef = 1.0;
    o.phif0 = lf0;
    o.phif1 = lf1;
    return;
  }
  const double a = sqrt(vf[0] * vf[0] + vf[1] * vf[1]);
  const double lf = sqrt(lf0 * lf0 + lf1 * lf1);
  const double s = mu * ln - lf;
  if (minmap) {
    // stick while |v_f| <= r_f s, else the slip compliance (|v_f| - r_f s) / (mu lambda_n)
    o.Ef = a <= rf * s ? 0.0 : (a - rf * s) / (mu * ln);
  } else {
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
  }
  o.omf = 1.0;
  o.phif0 = vf[0] + o.Ef * lf0;
  o.phif1 = vf[1] + o.Ef * lf1;
}

// The map of contact j applied to a per-vertex field: f_v for a contact at one vertex,
// f_v - sum_k w_k f_k (the triangle's corners) for a contact with another body, and
// f_v - f_partner for a two-vertex anchor row (a one-corner map entry of weight 1).
template <typename Field>
__device__ inline void contact_map(const DevSim& d, int j, Field f, double o[3]) {
  const int v = d.ct_vert[j];
  for (int r = 0; r < 3; ++r) o[r] = f(v, r);
  if (!d.map_on || d.ct_tri[j] < 0) return;
  const int4 t = d.btri[d.ct_tri[j]];
  const int cs[3] = {t.x, t.y, t.z};
  for (int k = 0; k < 3; ++k) {
    const double w = d.ct_bw[3 * j + k];
    if (w != 0.0)
      for (int r = 0; r < 3; ++r) o[r] -= w * f(cs[k], r);
  }
}

// the map at the iterate q = q_ref + dq, and of dq alone; a common translation `shift` of
// the scene adds to a one-vertex contact only (the weights of a contact with another body
// sum to one, and a two-vertex row's map is a difference)
__device__ inline void contact_q(const DevSim& d, int j, const double* shift, double q[3]) {
  contact_map(d, j, [&](int v, int r) { return d.q_ref[3 * v + r] + (double)d.dq[3 * v + r]; }, q);
  if (shift && !(d.map_on && d.ct_tri[j] >= 0))
    for (int r = 0; r < 3; ++r) q[r] += shift[r];
}
__device__ inline void contact_dq(const DevSim& d, int j, double dq[3]) {
  contact_map(d, j, [&](int v, int r) { return (double)d.dq[3 * v + r]; }, dq);
}

// contact j at map position q (world) with impulses lam (n, f1, f2); L: residual scale
__device__ inline FbTerms fb_terms(const DevSim& d, int j, const double q[3], const double lam[3],
                                   double L) {
  FbTerms o;
  const int v = d.ct_vert[j];
  const double h = d.h;
  const double* D = d.ct_D + 9 * j;
  o.bilateral = d.ct_obst[j] >= d.n_obs;
  if (o.bilateral) {
    // rows e_x, e_y, e_z (D = I): phi_b = q - p + e lambda with the target p in ct_dn, ct_df
    const double e = d.ct_mu[j];
    const double p[3] = {d.ct_dn[j], d.ct_df[2 * j], d.ct_df[2 * j + 1]};
    double ph[3];
    for (int r = 0; r < 3; ++r)
      ph[r] = D[3 * r] * q[0] + D[3 * r + 1] * q[1] + D[3 * r + 2] * q[2] - p[r] + e * lam[r];
    o.dn = ph[0] - e * lam[0];
    o.vf[0] = o.vf[1] = 0.0;
    o.phin = ph[0];
    o.phif0 = ph[1];
    o.phif1 = ph[2];
    o.omn = o.omf = 1.0;
    o.En = o.Ef = e;
    o.res = fmax(fabs(ph[0]), fmax(fabs(ph[1]), fabs(ph[2]))) / L;
    return o;
  }
  double qt[3];
  contact_map(d, j, [&](int u, int r) { return d.q_t[3 * u + r]; }, qt);
  o.dn = D[0] * q[0] + D[1] * q[1] + D[2] * q[2] - d.ct_dn[j];
  for (int a = 0; a < 2; ++a) {
    const double* f = D + 3 + 3 * a;
    o.vf[a] = ((f[0] * (q[0] - qt[0]) + f[1] * (q[1] - qt[1]) + f[2] * (q[2] - qt[2])) -
               h * d.ct_df[2 * j + a]) / h;
  }
  const double ln = lam[0], lf0 = lam[1], lf1 = lam[2];
  const double mu = d.ct_mu[j];
  const double rn_m = d.ct_r[4 * j + 2];
  const bool active = rn_m * ln > kActiveRel * L;
  ncp_rows(d.ncp == SIM_NCP_MINMAP, o.dn, o.vf, ln, lf0, lf1, d.ct_r[4 * j], d.ct_r[4 * j + 1],
           mu, active, o);
  // the residual: min(delta_n, r_n lambda_n) and h phi_f with the Fischer-Burmeister E_f, r
  // from the Delassus diagonal, whichever functions and preconditioner drive the iteration
  double pf0 = o.phif0, pf1 = o.phif1;
  if (d.ncp != SIM_NCP_FB || d.precond != SIM_PRECOND_DELASSUS) {
    FbTerms m;
    ncp_rows(false, o.dn, o.vf, ln, lf0, lf1, rn_m, d.ct_r[4 * j + 3], mu, active, m);
    pf0 = m.phif0;
    pf1 = m.phif1;
  }
  o.res = fmax(fabs(fmin(o.dn, rn_m * ln)), h * sqrt(pf0 * pf0 + pf1 * pf1)) / L;
  return o;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace silg

// Warm start of a frame (an addition to the paper, whose frames start from lambda = 0 and
// q = s~): per contact, the impulse lambda^0 and a move of its vertex along the normal,
// predicted by the network from per-contact features (impulse and move as changes of the
// previous frame's) or taken from the previous frame's contact at the same vertex and
// obstacle; per scene, a translation from the moves (see k_ws_shift). The guess is kept
// only if the residual of its impulses (the frame's residual measure at k = 0, at the
// position those impulses predict) is below the cold start's; the decision is per scene.
//
// Features (dimensionless): gap at s~ / margin; the normal (3); the velocity relative to the
// obstacle times h / margin (3); the previous frame's impulse at the same vertex and
// obstacle, in this frame's contact basis / scale (3, or 0); m_v W~_vv in (0, 1] (how much
// of the vertex's inertia the rest of the body adds). The impulse scale margin / (h^2 W~_vv)
// is the impulse that moves the vertex by one margin.
#include <cuda_runtime.h>

#include "device.cuh"
#include "fb.cuh"

namespace silg {
namespace {

__device__ __forceinline__ double wt_diag(const DevSim& d, int j) {
  const int cv = d.ct_cv[j];
  // a contact vertex beyond the capacity (the frame reports SIM_ECAPACITY) has no row
  if (cv >= min(d.counters[kCntCv], d.cap)) return 0.0;
  const int sc = d.vert_scene[d.ct_vert[j]], l = cv - d.sc_cvb[sc];
  return (double)d.wt[d.sc_wtoff[sc] + (size_t)l * d.sc_ld[sc] + l];
}

__global__ void k_ws_features(DevSim d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  const int v = d.ct_vert[j], sc = d.vert_scene[v], o = d.ct_obst[j];
  const double* D = d.ct_D + 9 * j;
  const double margin = d.scene_margin[sc], h = d.h;
  const double w = fmax(wt_diag(d, j), 1e-300);
  const double scale = margin / (h * h * w);
  float* f = d.ws_feat + (size_t)j * kMlpIn;
  if (o < 0 || o >= d.n_obs) {
    // an anchor: not guessed (its impulse starts at 0), no features. A contact with another
    // body: only the previous frame's impulse at the same vertex and triangle (features
    // 7..9); the network, trained on obstacle contacts, does not see it
    for (int r = 0; r < kMlpIn; ++r) f[r] = 0.f;
    d.ws_pmove[j] = 0.0;
    if (o < 0 && d.prev_valid[v] && d.prev_obst[v] == o)
      for (int r = 0; r < 3; ++r)
        f[7 + r] = (float)((D[3 * r] * d.prev_force[3 * v] + D[3 * r + 1] * d.prev_force[3 * v + 1] +
                            D[3 * r + 2] * d.prev_force[3 * v + 2]) / scale);
    d.ws_scale[j] = scale;
    return;
  }
  double st[3];
  for (int r = 0; r < 3; ++r) st[r] = d.s_tilde[3 * v + r];
  f[0] = (float)((D[0] * st[0] + D[1] * st[1] + D[2] * st[2] - d.ct_dn[j]) / margin);
  for (int r = 0; r < 3; ++r) f[1 + r] = (float)D[r];
  // relative velocity: the vertex's v_t minus the obstacle's surface velocity
  for (int r = 0; r < 3; ++r) {
    const double u = d.ct_df[2 * j] * D[3 + r] + d.ct_df[2 * j + 1] * D[6 + r];  // tangential part
    f[4 + r] = (float)(h * (d.v_t[3 * v + r] - u) / margin);
  }
  double lp[3] = {0.0, 0.0, 0.0};
  const bool persists = d.prev_valid[v] && d.prev_obst[v] == o;
  if (persists)
    for (int r = 0; r < 3; ++r)
      lp[r] = D[3 * r] * d.prev_force[3 * v] + D[3 * r + 1] * d.prev_force[3 * v + 1] +
              D[3 * r + 2] * d.prev_force[3 * v + 2];
  d.ws_pmove[j] = persists ? d.prev_move[v] : 0.0;
  for (int r = 0; r < 3; ++r) f[7 + r] = (float)(lp[r] / scale);
  f[10] = (float)(d.mass[v] * w);
  for (int r = kMlpNF; r < kMlpIn; ++r) f[r] = 0.f;
  d.ws_scale[j] = scale;
}

// the guess of contact j: its impulse (admissible: lambda_n >= 0, |lambda_f| <= mu
// lambda_n) and the move of its vertex along the normal
__device__ void ws_guess(const DevSim& d, int j) {
  const int v = d.ct_vert[j], sc = d.vert_scene[v];
  if (d.ct_obst[j] >= d.n_obs) {   // anchors start from lambda = 0
    for (int r = 0; r < 3; ++r) d.ws_lam0[3 * j + r] = 0.0;
    d.ws_move[j] = 0.0;
    return;
  }
  const double scale = d.ws_scale[j], mu = d.ct_mu[j], margin = d.scene_margin[sc];
  double lam[3] = {0.0, 0.0, 0.0}, move = 0.0;
  if (d.ct_obst[j] < 0) {
    // a contact with another body, in either mode: its previous impulse, no move
    const float* f = d.ws_feat + (size_t)j * kMlpIn;
    for (int r = 0; r < 3; ++r) lam[r] = (double)f[7 + r] * scale;
  } else if (d.ws_mode == 1) {
    // the network predicts the changes from the previous frame's impulse (features 7..9)
    // and move at the same vertex and obstacle, each scaled by its gain: the impulse's by
    // the contact's class (persisting or new), the move's by the move gain. With all gains
    // 0 the guess is the previous frame's (mode 2).
    const float* y = d.ws_out + (size_t)j * kMlpOut;
    const float* f = d.ws_feat + (size_t)j * kMlpIn;
    const bool persists = d.prev_valid[v] && d.prev_obst[v] == d.ct_obst[j];
    const double g = persists ? d.ws_gain[0] : d.ws_gain[1];
    // an output with gain 0 is not read (the network is not run when all gains are 0)
    for (int r = 0; r < 3; ++r)
      lam[r] = ((double)f[7 + r] + (g > 0.0 ? g * (double)y[r] : 0.0)) * scale;
    move = d.ws_pmove[j] + (d.ws_gain[2] > 0.f ? (double)d.ws_gain[2] * (double)y[3] * margin : 0.0);
  } else {
    const float* f = d.ws_feat + (size_t)j * kMlpIn;
    for (int r = 0; r < 3; ++r) lam[r] = (double)f[7 + r] * scale;
    move = d.ws_pmove[j];
  }
  lam[0] = fmax(lam[0], 0.0);
  const double lf = sqrt(lam[1] * lam[1] + lam[2] * lam[2]), cap = mu * lam[0];
  if (lf > cap) {
    const double s = lf > 0.0 ? cap / lf : 0.0;
    lam[1] *= s;
    lam[2] *= s;
  }
  for (int r = 0; r < 3; ++r) d.ws_lam0[3 * j + r] = lam[r];
  d.ws_move[j] = move;
}

// strictly better than the cold start (an empty guess is the cold start and is not taken);
// copy 0 of a portfolio group always runs cold
__device__ __forceinline__ bool ws_accepted(const DevSim& d, int sc, double r_guess,
                                            double r_cold) {
  if (d.pf_copies > 1 && sc % d.pf_copies == 0) return false;
  // the learned start may ask for a margin (ratio < 1); the others take any improvement
  return r_guess < (d.ws_mode == 1 ? (double)d.ws_gain[3] : 1.0) * r_cold;
}

constexpr int kWsThreads = 256;
constexpr int kWsContactThreads = 32;   // per-contact kernels: their FP64 work spreads over SMs

// The warm start of every scene, in the order of its steps:
//  1. per contact (k_ws_contact): the guess (ws_guess) and the residual of the cold start
//     (s~, lambda = 0) at that contact;
//  2. per scene (k_ws_shift): two translations, summed in a fixed order. The impulse
//     translation h^2 sum_j D_j^T lambda_j^0 / M is what the guessed impulses give the
//     scene's free mass over one step (an impulse guess that holds a resting body up also
//     lifts its predicted position by the sag of gravity); it judges the impulse guess. The
//     move translation is the mean over the scene's contact vertices of their guessed move
//     along the normal; the scene is moved by it, kept within one contact margin of the
//     impulse translation;
//  3. per contact (k_ws_resid): the residual of the guess (translated scene, guessed
//     impulses) at that contact;
//  4. per scene (k_ws_apply): the residuals at k = 0 of the guess and of the cold start, max
//     over the scene's contacts; if the guess is kept, its impulses and the translation of
//     the scene's free vertices.
__global__ void k_ws_contact(DevSim d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  ws_guess(d, j);
  const int sc = d.vert_scene[d.ct_vert[j]];
  const double zero[3] = {0.0, 0.0, 0.0};
  double q0[3];
  contact_q(d, j, nullptr, q0);
  d.ws_rc[j] = fb_terms(d, j, q0, zero, d.scene_Lref[sc]).res;
}

__global__ void __launch_bounds__(kWsThreads) k_ws_shift(DevSim d) {
  const int sc = blockIdx.x;
  const int jb = d.sc_jb[sc], je = d.sc_jb[sc + 1];
  __shared__ double part[6][kWsThreads];
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
    if (d.ct_obst[j] < 0) continue;   // contacts between bodies are internal forces
    const double* D = d.ct_D + 9 * j;
    const double* l = d.ws_lam0 + 3 * j;
    for (int r = 0; r < 3; ++r) t[r] += D[r] * l[0] + D[3 + r] * l[1] + D[6 + r] * l[2];
    if (d.ct_cv[j] < d.cap && d.cv_first[d.ct_cv[j]] == j)
      for (int r = 0; r < 3; ++r) t[3 + r] += d.ws_move[j] * D[r];
  }
  for (int r = 0; r < 6; ++r) part[r][threadIdx.x] = t[r];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int r = 0; r < 6; ++r) part[r][threadIdx.x] += part[r][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int ncv = d.sc_cvb[sc + 1] - d.sc_cvb[sc];
    double imp[3], dev[3], dn = 0.0;
    for (int r = 0; r < 3; ++r) {
      imp[r] = d.h * d.h * part[r][0] / d.scene_mass[sc];
      dev[r] = (ncv > 0 ? part[3 + r][0] / ncv : 0.0) - imp[r];
      dn += dev[r] * dev[r];
    }
    dn = sqrt(dn);
    const double lim = d.scene_margin[sc], f = dn > lim ? lim / dn : 1.0;
    for (int r = 0; r < 3; ++r) {
      d.ws_shift[6 * sc + r] = imp[r];                  // judges the impulses
      d.ws_shift[6 * sc + 3 + r] = imp[r] + f * dev[r];  // applied
    }
  }
}

__global__ void k_ws_resid(DevSim d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  const int sc = d.vert_scene[d.ct_vert[j]];
  double q[3], lam[3];
  contact_q(d, j, d.ws_shift + 6 * sc, q);
  for (int r = 0; r < 3; ++r) lam[r] = d.ws_lam0[3 * j + r];
  d.ws_rg[j] = fb_terms(d, j, q, lam, d.scene_Lref[sc]).res;
}

__global__ void __launch_bounds__(kWsThreads) k_ws_apply(DevSim d) {
  const int sc = blockIdx.x;
  const int jb = d.sc_jb[sc], je = d.sc_jb[sc + 1];
  __shared__ double part[2][kWsThreads];
  __shared__ int keep;
  double rg = 0.0, rc = 0.0;
  for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
    rg = fmax(rg, d.ws_rg[j]);
    rc = fmax(rc, d.ws_rc[j]);
  }
  part[0][threadIdx.x] = rg;
  part[1][threadIdx.x] = rc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      part[0][threadIdx.x] = fmax(part[0][threadIdx.x], part[0][threadIdx.x + w]);
      part[1][threadIdx.x] = fmax(part[1][threadIdx.x], part[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d.ws_res[2 * sc] = part[0][0];
    d.ws_res[2 * sc + 1] = part[1][0];
    keep = ws_accepted(d, sc, part[0][0], part[1][0]) ? 1 : 0;
  }
  __syncthreads();
  if (!keep) return;
  for (int j = jb + threadIdx.x; j < je; j += blockDim.x)
    for (int r = 0; r < 3; ++r) d.ct_lam[3 * j + r] = d.ws_lam0[3 * j + r];
  const double* shift = d.ws_shift + 6 * sc;
  const float s0 = (float)shift[3], s1 = (float)shift[4], s2 = (float)shift[5];
  for (int v = d.scene_vfirst[sc] + threadIdx.x; v < d.scene_vfirst[sc + 1]; v += blockDim.x) {
    d.dq[3 * v] += s0;
    d.dq[3 * v + 1] += s1;
    d.dq[3 * v + 2] += s2;
  }
}

__global__ void k_ws_clear(DevSim d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n) d.prev_valid[v] = 0;
}

// the frame's final impulses (for the next frame's features) and the training targets
__global__ void k_ws_record(DevSim d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = min(d.counters[kCntContacts], d.cap);
  if (j >= c) return;
  const int v = d.ct_vert[j], sc = d.vert_scene[v];
  const double* D = d.ct_D + 9 * j;
  const double* lam = d.ct_lam + 3 * j;
  double mv = 0.0;
  for (int r = 0; r < 3; ++r)
    mv += D[r] * (d.q_ref[3 * v + r] + (double)d.dq[3 * v + r] - d.s_tilde[3 * v + r]);
  if (d.ct_cv[j] < d.cap && d.cv_first[d.ct_cv[j]] == j && d.ct_obst[j] < d.n_obs) {
    d.prev_valid[v] = 1;
    d.prev_obst[v] = d.ct_obst[j];
    d.prev_move[v] = mv;
    for (int r = 0; r < 3; ++r)
      d.prev_force[3 * v + r] = D[r] * lam[0] + D[3 + r] * lam[1] + D[6 + r] * lam[2];
  }
  // targets of the network: the changes from the previous frame's impulse (the features
  // 7..9 seen at this frame's start), over the scale, and from its normal move at the same
  // vertex and obstacle, over the margin
  const double scale = d.ws_scale[j];
  const float* f = d.ws_feat + (size_t)j * kMlpIn;
  float* t = d.ws_target + 4 * (size_t)j;
  for (int r = 0; r < 3; ++r) t[r] = (float)(lam[r] / scale - (double)f[7 + r]);
  t[3] = (float)((mv - d.ws_pmove[j]) / d.scene_margin[sc]);
}

// Portfolio: a free vertex of a copy that did not win takes its counterpart's state in the
// winning copy (lowest final residual, non-finite counted as infinite, ties to the lowest
// copy): positions, velocities and the previous-frame contact data of the features. The
// winner's vertices are only read.
__global__ void k_pf_sync(DevSim d, int K) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  if (K < 0) K = *d.iter_k;
  const int sc = d.vert_scene[v], C = d.pf_copies, g0 = sc - sc % C;
  int best = g0;
  double rb = INFINITY;
  for (int c = 0; c < C; ++c) {
    const double r = d.resid_scene[(size_t)(g0 + c) * (kMaxIters + 1) + K];
    if (isfinite(r) && r < rb) {
      rb = r;
      best = g0 + c;
    }
  }
  if (best == sc) return;
  const int w = v - d.scene_vfirst[sc] + d.scene_vfirst[best];
  for (int r = 0; r < 3; ++r) {
    d.q_t[3 * v + r] = d.q_t[3 * w + r];
    d.v_t[3 * v + r] = d.v_t[3 * w + r];
    d.prev_force[3 * v + r] = d.prev_force[3 * w + r];
  }
  // the same obstacle of this copy (copies list their obstacles in the same order); a
  // contact with another body (negative id: the triangles are numbered over all scenes)
  // is not carried over
  d.prev_valid[v] = d.prev_obst[w] < 0 ? 0 : d.prev_valid[w];
  d.prev_obst[v] = d.prev_obst[w] - d.scene_ofirst[best] + d.scene_ofirst[sc];
  d.prev_move[v] = d.prev_move[w];
}

}  // namespace

void launch_pf_sync(const DevSim& d, cudaStream_t s, int K) {
  k_pf_sync<<<(d.n + 255) / 256, 256, 0, s>>>(d, K);
}

void launch_ws_features(const DevSim& d, cudaStream_t s) {
  // FP64 per contact: small CTAs spread it over the SMs
  k_ws_features<<<(d.cap + kWsContactThreads - 1) / kWsContactThreads, kWsContactThreads, 0, s>>>(d);
}

int ws_kernels(const DevSim& d) {
  const bool net = d.ws_mode == 1 && (d.ws_gain[0] > 0.f || d.ws_gain[1] > 0.f || d.ws_gain[2] > 0.f);
  return d.ws_mode == 0 ? 0 : (net ? 5 : 4);
}

void launch_ws_start(const DevSim& d, cudaStream_t s) {
  if (d.ws_mode == 0) return;
  if (d.ws_mode == 1 && (d.ws_gain[0] > 0.f || d.ws_gain[1] > 0.f || d.ws_gain[2] > 0.f))
    mlp_launch_infer_dev(d.ws_net, d.ws_feat, d.counters + kCntContacts, d.cap, d.ws_out, s);
  const int gc = (d.cap + kWsContactThreads - 1) / kWsContactThreads;
  k_ws_contact<<<gc, kWsContactThreads, 0, s>>>(d);
  k_ws_shift<<<d.n_scenes, kWsThreads, 0, s>>>(d);
  k_ws_resid<<<gc, kWsContactThreads, 0, s>>>(d);
  k_ws_apply<<<d.n_scenes, kWsThreads, 0, s>>>(d);
}

void launch_ws_record(const DevSim& d, cudaStream_t s) {
  k_ws_clear<<<(d.n + 255) / 256, 256, 0, s>>>(d);
  k_ws_record<<<(d.cap + 127) / 128, 128, 0, s>>>(d);
}

}  // namespace silg

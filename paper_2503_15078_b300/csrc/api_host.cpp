// C ABI: status strings, default options and the host-only plan entry points.
#include <cstring>
#include <new>
#include <string>

#include "plan.hpp"
#include "silg.h"

struct sim_plan_s {
  silg::Plan plan;
};

extern "C" {

const char* sim_strerror(int status) {
  switch (status) {
    case SIM_OK: return "ok";
    case SIM_EINVAL: return "invalid argument";
    case SIM_ENOMEM: return "out of memory";
    case SIM_ENOTSPD: return "system matrix not positive definite";
    case SIM_ECUDA: return "CUDA error";
    case SIM_ECAPACITY: return "contact capacity exceeded";
    case SIM_ETIMEOUT: return "device-side wait timed out";
    case SIM_ENONFINITE: return "non-finite value in the state";
    case SIM_ENOTSUP: return "unsupported option";
    default: return "unknown status";
  }
}

void sim_default_options(sim_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_iters = 5;
  o->n_cr_iters = 10;
  o->s_precision = SIM_S_FP32;
  o->refine = 1;
  o->contact_capacity = 4096;
  o->device = 0;
  o->gravity[2] = -9.81;
  o->contact_margin = 0.0;
  o->spin_limit = 0;
  o->cuda_stream = nullptr;
  o->n_host_threads = 0;
  o->autotune = 0;
  o->ncp = SIM_NCP_FB;
  o->precond = SIM_PRECOND_DELASSUS;
  o->residual_tol = 0.0;
  o->max_iters = 40;
  o->local_solver = SIM_LOCAL_PD;
  o->global_solver = SIM_GLOBAL_SPARSE_INVERSE;
  o->jacobi_sweeps = 1;
  o->phase_marks = 1;
  o->cr_exchanges = 2;
  o->s_build = 1;
  o->delassus_reuse = 1;
}

int sim_plan_create(const sim_mesh* mesh, const sim_material* mats, int32_t n_mat, double h,
                    const sim_options* opts, sim_plan_t** out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  sim_options def;
  sim_default_options(&def);
  if (!opts) opts = &def;
  sim_plan_s* p = new (std::nothrow) sim_plan_s();
  if (!p) return SIM_ENOMEM;
  std::string err;
  int st;
  try {
    st = silg::build_plan(mesh, mats, n_mat, h, opts->n_host_threads, &p->plan, &err);
  } catch (const std::bad_alloc&) {
    st = SIM_ENOMEM;
  } catch (...) {
    st = SIM_EINVAL;
  }
  if (st != SIM_OK) {
    delete p;
    return st;
  }
  *out = p;
  return SIM_OK;
}

void sim_plan_destroy(sim_plan_t* p) { delete p; }

void silg_fill_plan_info(const silg::Plan& p, sim_plan_info* info);

int sim_plan_get_info(const sim_plan_t* pp, sim_plan_info* info) {
  if (!pp || !info) return SIM_EINVAL;
  silg_fill_plan_info(pp->plan, info);
  return SIM_OK;
}

void silg_fill_plan_info(const silg::Plan& p, sim_plan_info* info) {
  info->n_verts = p.n_verts;
  info->n_free = p.n_free;
  info->n_tets = p.n_tets;
  info->nnz_A = p.nnz_A;
  info->nnz_L = p.nnz_L;
  info->nnz_S = p.nnz_S;
  info->stored_S = p.rowbase.empty() ? 0 : (int64_t)p.rowbase.back();
  info->etree_max_depth = p.max_depth;
  info->etree_mean_depth = p.mean_depth;
  info->n_roots = p.n_roots;
  info->precompute_seconds = p.seconds;
  info->s_build_seconds = p.s_seconds;
  info->s_built_on_device = p.s_on_device;
}

int sim_plan_get_ordering(const sim_plan_t* pp, int32_t* order, int32_t* parent,
                          int32_t* first_desc) {
  if (!pp) return SIM_EINVAL;
  const silg::Plan& p = pp->plan;
  if (order) std::memcpy(order, p.order.data(), sizeof(int32_t) * p.n_free);
  if (parent) std::memcpy(parent, p.parent.data(), sizeof(int32_t) * p.n_free);
  if (first_desc) std::memcpy(first_desc, p.first_desc.data(), sizeof(int32_t) * p.n_free);
  return SIM_OK;
}

int sim_plan_apply_inverse_host(const sim_plan_t* pp, const double* b, double* x) {
  if (!pp || !b || !x) return SIM_EINVAL;
  const silg::Plan& p = pp->plan;
  const int nf = p.n_free;
  std::vector<double> bi(3 * (size_t)nf), xi(3 * (size_t)nf);
  for (int k = 0; k < nf; ++k)
    for (int r = 0; r < 3; ++r) bi[3 * k + r] = b[3 * (size_t)p.order[k] + r];
  silg::apply_inverse_internal(p, bi.data(), xi.data());
  std::memset(x, 0, sizeof(double) * 3 * (size_t)p.n_verts);
  for (int k = 0; k < nf; ++k)
    for (int r = 0; r < 3; ++r) x[3 * (size_t)p.order[k] + r] = xi[3 * k + r];
  return SIM_OK;
}

}  // extern "C"

// plan access for the device layer
const silg::Plan& silg_plan_of(const sim_plan_t* p) { return p->plan; }

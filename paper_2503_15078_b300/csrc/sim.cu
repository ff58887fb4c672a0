// C ABI of the simulator: creation (host precompute + upload), the per-frame CUDA graph
// of Alg. 4, state and diagnostic accessors, and the component entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdexcept>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "device.cuh"
#include "silg.h"

namespace {

using silg::DevSim;
using silg::Plan;

// event marks per iteration in the frame graph: after the local step, the assembly, the
// first product, its reduction, the constraint solve, the second product and its reduction
constexpr int kMarksPerIter = 7;

struct Graph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct sim_s {
  Plan plan;
  DevSim d{};
  int device = 0;
  cudaStream_t work = nullptr;    // private stream: captures and component calls
  cudaStream_t aux = nullptr;     // second branch of the frame graph (captured from work)
  cudaStream_t body = nullptr;    // capture of a while-node's body (frames to a tolerance)
  cudaStream_t body_aux = nullptr;// and its second branch
  std::vector<cudaEvent_t> fj;    // fork/join events of the frame graph's branches
  double* pinned = nullptr;       // page-locked staging of q and v (2 x 3 n_verts) for the
                                  // state accessors
  cudaStream_t launch = nullptr;  // where frames run (caller stream or work)
  int cluster = 1;
  size_t cr_smem = 0;
  int cr_vmax = 1, cr_cmax = 1;   // bounds of one scene's contact vertices and contacts
  int n_iters_default = 5;
  bool has_obstacles = false;
  std::map<int, Graph> graphs;
  std::vector<void*> allocs;
  void* (*dev_alloc)(size_t, void*) = nullptr;   // the caller's device allocator, if any
  void (*dev_free)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  int64_t frame = 0;
  int last_iters = 0;             // -1: a frame to a tolerance whose count is on the device
  bool last_to_tol = false;       // the most recent frame iterated to a tolerance
  bool phase_marks = true;        // event nodes around every phase of every iteration
  bool last_marks = true;         // ... in the most recent frame
  // phase events recorded by event nodes of the frame graph: [0] frame start,
  // [1] after collision, [2] after Delassus, [3] after the warm start, then kMarksPerIter
  // per iteration, then [end]
  std::vector<cudaEvent_t> ev;
  std::vector<uint64_t> scene_sig;  // per scene: hash of its inputs (portfolio copies check)
  std::vector<int32_t> tet_caller_order;
  sim_tuning tuning{};

  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    if (dev_alloc) {
      p = dev_alloc(count * sizeof(T), alloc_ctx);
      if (!p) throw std::bad_alloc();
      // the bulk copies into shared memory need 16-byte aligned sources; the contract is 256
      if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
        dev_free(p, alloc_ctx);
        throw std::invalid_argument("dev_alloc returned memory not aligned to 256 bytes");
      }
    } else if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
      throw std::bad_alloc();
    }
    allocs.push_back(p);
    cudaMemsetAsync(p, 0, count * sizeof(T), work);
    return static_cast<T*>(p);
  }
  // return one buffer to the allocator before destruction (temporaries of the creation)
  void release(void* p) {
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it == allocs.end()) return;
    if (dev_free)
      dev_free(p, alloc_ctx);
    else
      cudaFree(p);
    allocs.erase(it);
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, work);
    return p;
  }
  ~sim_s() {
    if (work) cudaStreamSynchronize(work);
    for (auto& kv : graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    for (void* p : allocs) {
      if (dev_free)
        dev_free(p, alloc_ctx);
      else
        cudaFree(p);
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : fj) cudaEventDestroy(e);
    if (pinned) cudaFreeHost(pinned);
    if (aux) cudaStreamDestroy(aux);
    if (body) cudaStreamDestroy(body);
    if (body_aux) cudaStreamDestroy(body_aux);
    if (work) cudaStreamDestroy(work);
  }
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SIM_OK;
  if (e == cudaErrorMemoryAllocation) return SIM_ENOMEM;
  return SIM_ECUDA;
}

int err_status(int bits) {
  if (bits & (silg::kErrCapacity | silg::kErrYCapacity)) return SIM_ECAPACITY;
  if (bits & silg::kErrNonFinite) return SIM_ENONFINITE;
  if (bits & silg::kErrTimeout) return SIM_ETIMEOUT;
  return SIM_OK;
}

// forget the previous frame's contact-vertex list: the next frame builds Y and W~ afresh
void delassus_forget(sim_s* s, cudaStream_t st) {
  cudaMemsetAsync(s->d.dl_state + 1, 0xff, sizeof(int), st);
}

int sync_and_check(sim_s* s) {
  cudaError_t e = cudaStreamSynchronize(s->launch);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->work);
  if (e != cudaSuccess) return cuda_status(e);
  int bits = 0;
  e = cudaMemcpy(&bits, s->d.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  return err_status(bits);
}

// iterations of a K-iteration frame that end with a residual correction (BF16 profile)
int refined_iters(const sim_s* s, int K) {
  if (!s->d.s_bf16 || s->d.refine <= 0 || s->d.jacobi_sweeps) return 0;
  return s->d.refine >= 2 ? K : 1;
}

// finished updates of the most recent frame (read from the device after a frame to a
// tolerance); -1 on a CUDA error
int frame_iters(sim_s* s) {
  if (s->last_iters >= 0) return s->last_iters;
  int k = 0;
  if (cudaStreamSynchronize(s->launch) != cudaSuccess ||
      cudaMemcpy(&k, s->d.iter_k, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -1;
  s->last_iters = k;
  return k;
}

// the extra launches of the two-pass scans of a frame with contacts: the n-length scans
// (contacts, contact vertices, corner terms with body contact, U flags, Y row lengths) and
// the capacity-length one (Y column lengths)
int scan_extra(const sim_s* s) {
  const int n = s->d.n, cap = s->d.cap;
  return (3 + (s->d.map_on ? 1 : 0) + 1) * (silg::scan_launches(n) - 1) +
         (silg::scan_launches(cap) - 1);
}

// local-step launches per iteration (tetrahedra, triangles) and per-frame extras (bending)
int local_kernels(const sim_s* s) { return (s->d.n_tets > 0) + (s->d.n_tris > 0); }

// launches of a frame to a tolerance that made K updates (enqueue_frame_to_tolerance)
int kernels_per_frame_to_tolerance(const sim_s* s, int K) {
  const bool c = s->has_obstacles;
  // contacts between bodies: 3 more collision launches (the body search); maps beyond one
  // vertex (bodies or two-vertex anchor rows): 3 more (corner terms) and one more per
  // constraint solve
  const int bc = s->d.bc_on ? 1 : 0, mp = s->d.map_on ? 1 : 0;
  const int scans = scan_extra(s);
  const int refine_body = s->d.s_bf16 && s->d.refine >= 2 && !s->d.jacobi_sweeps ? 5 : 0;
  const int refine_end = s->d.s_bf16 && s->d.refine == 1 && !s->d.jacobi_sweeps ? 6 : 0;
  const int global = s->d.jacobi_sweeps ? s->d.jacobi_sweeps : 2 + (c ? 3 + mp : 0) + 2;
  const int before = 1 + (s->d.bend_ptr != nullptr) +
                     (c ? 4 + 13 + 3 * bc + 3 * mp + scans + silg::ws_kernels(s->d) : 0) +
                     local_kernels(s) +
                     (c ? 1 : 0);
  const int body = 1 + global + refine_body + 1 + (c ? 1 : 0) + local_kernels(s) + 1;
  const int after = refine_end + (c ? 1 : 0) + 1 + (c && s->d.pf_copies > 1 ? 1 : 0);
  return before + K * body + after;
}

int kernels_per_frame(const sim_s* s, int K) {
  const bool c = s->has_obstacles;
  // per iteration: local, [contact eval], rhs, pass 1 + reduction, [Y^T z, CR, Y u],
  // pass 2 + reduction; a residual correction adds the residual and both passes
  const int bc = s->d.bc_on ? 1 : 0, mp = s->d.map_on ? 1 : 0;
  const int global = s->d.jacobi_sweeps ? s->d.jacobi_sweeps : 2 + (c ? 3 + mp : 0) + 2;
  return 1 + (s->d.bend_ptr != nullptr) + (c ? 4 + 13 + 3 * bc + 3 * mp + scan_extra(s) : 0) +
         K * (local_kernels(s) + (c ? 1 : 0) + 1 + global) + (c ? 1 : 0) + 1 +
         5 * refined_iters(s, K) + (c ? silg::ws_kernels(s->d) : 0) +
         (c && s->d.pf_copies > 1 ? 1 : 0);
}

void enqueue_frame(sim_s* s, int K, cudaStream_t st) {
  // the production graph (no event nodes between the kernels of an iteration) launches
  // the iteration's straight-line kernels with programmatic dependent launch
  DevSim dv = s->d;
  dv.pdl = s->phase_marks ? 0 : 1;
  const DevSim& d = dv;
  // external event-record nodes: observable from the host after each graph launch
  auto mark = [&](int i) { cudaEventRecordWithFlags(s->ev[i], st, cudaEventRecordExternal); };
  // per-iteration marks only with phase_marks (each event node costs a few microseconds)
  auto imark = [&](int i) {
    if (s->phase_marks) mark(i);
  };
  // two branches of the graph: work forked onto the aux stream and joined back
  int n_fj = 0;
  auto fork = [&]() {
    cudaEventRecord(s->fj[n_fj], st);
    cudaStreamWaitEvent(s->aux, s->fj[n_fj], 0);
    ++n_fj;
  };
  auto join = [&]() {
    cudaEventRecord(s->fj[n_fj], s->aux);
    cudaStreamWaitEvent(st, s->fj[n_fj], 0);
    ++n_fj;
  };
  mark(0);
  cudaMemsetAsync(d.resid, 0, sizeof(double) * (silg::kMaxIters + 1), st);
  cudaMemsetAsync(d.resid_scene, 0, sizeof(double) * (silg::kMaxIters + 1) * d.n_scenes, st);
  cudaMemsetAsync(d.max_pen, 0, sizeof(double), st);
  if (d.admm) cudaMemsetAsync(d.tet_u, 0, sizeof(float) * 9 * (size_t)d.n_tets, st);
  silg::launch_frame_begin(d, st);
  // the first local step needs only the prediction: with a cold start it runs beside the
  // collision and Delassus work (a warm start moves q^0, so then it waits)
  const bool early_local = s->has_obstacles && d.ws_mode == 0;
  if (early_local) {
    fork();
    silg::launch_local(d, s->aux, false);
  }
  if (s->has_obstacles) silg::launch_collide(d, st);
  mark(1);
  if (s->has_obstacles) silg::launch_delassus(d, st);
  mark(2);
  if (s->has_obstacles) {
    silg::launch_ws_features(d, st);
    silg::launch_ws_start(d, st);
  }
  mark(3);
  for (int k = 0; k < K; ++k) {
    const int e = 4 + kMarksPerIter * k;
    // the local step and the contact evaluation depend on the same iterate only: two
    // branches, joined before the right-hand side that needs both
    if (k == 0 && early_local) {
      silg::launch_contact_eval(d, st, k, false);
      join();
    } else if (s->has_obstacles) {
      fork();
      silg::launch_contact_eval(d, s->aux, k, false);
      silg::launch_local(d, st, false);
      join();
    } else {
      silg::launch_local(d, st, false);
    }
    imark(e);
    silg::launch_rhs(d, st);
    imark(e + 1);
    if (d.jacobi_sweeps) {
      // the incomplete global step of the comparison (timed as the first product's phase)
      silg::launch_jacobi(d, st);
      for (int m = 2; m <= 5; ++m) imark(e + m);
    } else {
    silg::launch_pass1(d, st);
    imark(e + 2);
    silg::launch_reduce1(d, st);
    imark(e + 3);
    if (s->has_obstacles) {
      silg::launch_ytz(d, st);
      silg::launch_cr(d, st, s->cluster);
      silg::launch_yu(d, st);
    }
    imark(e + 4);
    silg::launch_pass2(d, st);
    imark(e + 5);
    silg::launch_reduce2(d, st, silg::kOutDq);
    }
    if (k >= K - refined_iters(s, K)) {
      // BF16 profile: dq += S~^T S~ (rhs - A~ dq), the residual summed in FP64 and the
      // iteration's contact impulses held fixed
      silg::launch_residual(d, st, s->has_obstacles ? silg::kResFrameContact : silg::kResFrame);
      DevSim dr = d;
      dr.gvec = d.gsave;
      silg::launch_solve(dr, st, silg::kOutAddDq);
    }
    imark(e + 6);
  }
  if (!s->phase_marks) mark(4);   // the iterations as one phase
  if (s->has_obstacles) {
    silg::launch_contact_eval(d, st, K, true);
    silg::launch_ws_record(d, st);
  }
  silg::launch_integrate(d, st);
  if (s->has_obstacles && d.pf_copies > 1) silg::launch_pf_sync(d, st, K);
  mark(s->phase_marks ? 4 + kMarksPerIter * K : 5);
}

// A frame that iterates until the residual reaches sim_options.residual_tol (at least one
// update, at most max_iters): the same kernels as enqueue_frame, with the iterations in the
// body of a CUDA graph while-node. The body runs the rest of iteration k (right-hand side,
// products, constraint solve), counts the update on the device, evaluates the next iterate
// (contact terms beside the local step) and lets a one-thread kernel set the node's
// condition from R_{k+1}. Event nodes are not allowed in a conditional body, so phase
// marks stand only around the loop. Returns a CUDA error, or cudaSuccess.
cudaError_t enqueue_frame_to_tolerance(sim_s* s, cudaStream_t st) {
  DevSim dv = s->d;
  dv.pdl = 1;   // no event nodes inside the loop (see enqueue_frame)
  const DevSim& d = dv;
  auto mark = [&](int i) { cudaEventRecordWithFlags(s->ev[i], st, cudaEventRecordExternal); };
  int n_fj = 0;
  auto fork = [&](cudaStream_t from, cudaStream_t to) {
    cudaEventRecord(s->fj[n_fj], from);
    cudaStreamWaitEvent(to, s->fj[n_fj], 0);
    ++n_fj;
  };
  auto join = [&](cudaStream_t from, cudaStream_t to) { fork(from, to); };
  mark(0);
  cudaMemsetAsync(d.resid, 0, sizeof(double) * (silg::kMaxIters + 1), st);
  cudaMemsetAsync(d.resid_scene, 0, sizeof(double) * (silg::kMaxIters + 1) * d.n_scenes, st);
  cudaMemsetAsync(d.max_pen, 0, sizeof(double), st);
  cudaMemsetAsync(d.iter_k, 0, sizeof(int), st);
  if (d.admm) cudaMemsetAsync(d.tet_u, 0, sizeof(float) * 9 * (size_t)d.n_tets, st);
  silg::launch_frame_begin(d, st);
  const bool early_local = s->has_obstacles && d.ws_mode == 0;
  if (early_local) {
    fork(st, s->aux);
    silg::launch_local(d, s->aux, false);
  }
  if (s->has_obstacles) silg::launch_collide(d, st);
  mark(1);
  if (s->has_obstacles) silg::launch_delassus(d, st);
  mark(2);
  if (s->has_obstacles) {
    silg::launch_ws_features(d, st);
    silg::launch_ws_start(d, st);
  }
  mark(3);
  // the top of iteration 0
  if (early_local) {
    silg::launch_contact_eval(d, st, 0, false);
    join(s->aux, st);
  } else if (s->has_obstacles) {
    fork(st, s->aux);
    silg::launch_contact_eval(d, s->aux, 0, false);
    silg::launch_local(d, st, false);
    join(s->aux, st);
  } else {
    silg::launch_local(d, st, false);
  }
  // the while-node, its condition 1 at every launch (at least one update)
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t n_deps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &n_deps);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  e = cudaGraphAddNode(&loop, g, deps, nullptr, n_deps, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(st, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  {
    cudaStream_t b = s->body, ba = s->body_aux;
    e = cudaStreamBeginCaptureToGraph(b, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    silg::launch_rhs(d, b);
    if (d.jacobi_sweeps) {
      silg::launch_jacobi(d, b);
    } else {
      silg::launch_pass1(d, b);
      silg::launch_reduce1(d, b);
      if (s->has_obstacles) {
        silg::launch_ytz(d, b);
        silg::launch_cr(d, b, s->cluster);
        silg::launch_yu(d, b);
      }
      silg::launch_pass2(d, b);
      silg::launch_reduce2(d, b, silg::kOutDq);
    }
    if (d.s_bf16 && d.refine >= 2 && !d.jacobi_sweeps) {
      silg::launch_residual(d, b, s->has_obstacles ? silg::kResFrameContact : silg::kResFrame);
      DevSim dr = d;
      dr.gvec = d.gsave;
      silg::launch_solve(dr, b, silg::kOutAddDq);
    }
    silg::launch_iter_advance(d, b);
    if (s->has_obstacles) {
      fork(b, ba);
      silg::launch_contact_eval(d, ba, -1, false);
      silg::launch_local(d, b, false);
      join(ba, b);
    } else {
      silg::launch_local(d, b, false);
    }
    silg::launch_iter_decide(d, b, h);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(b, &captured);
    if (e != cudaSuccess) return e;
  }
  mark(4);
  if (d.s_bf16 && d.refine == 1 && !d.jacobi_sweeps) {
    // the correction after the last update; its residual entries are evaluated again
    silg::launch_iter_clear(d, st);
    silg::launch_residual(d, st, s->has_obstacles ? silg::kResFrameContact : silg::kResFrame);
    DevSim dr = d;
    dr.gvec = d.gsave;
    silg::launch_solve(dr, st, silg::kOutAddDq);
  }
  if (s->has_obstacles) {
    silg::launch_contact_eval(d, st, -1, true);
    silg::launch_ws_record(d, st);
  }
  silg::launch_integrate(d, st);
  if (s->has_obstacles && d.pf_copies > 1) silg::launch_pf_sync(d, st, -1);
  mark(5);
  return cudaGetLastError();
}

// frame graphs are cached per (iteration count, phase marks, warm-start mode); K = 0: to a
// tolerance
int get_graph(sim_s* s, int K, cudaGraphExec_t* out) {
  const int key = 8 * K + (K > 0 && s->phase_marks ? 4 : 0) + s->d.ws_mode;
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    *out = it->second.exec;
    return SIM_OK;
  }
  Graph g;
  cudaError_t e = cudaStreamBeginCapture(s->work, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  cudaError_t eq = cudaSuccess;
  if (K > 0)
    enqueue_frame(s, K, s->work);
  else
    eq = enqueue_frame_to_tolerance(s, s->work);
  e = cudaStreamEndCapture(s->work, &g.g);
  if (eq != cudaSuccess) {
    if (e == cudaSuccess) cudaGraphDestroy(g.g);
    return cuda_status(eq);
  }
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&g.exec, g.g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g.g);
    return cuda_status(e);
  }
  s->graphs[key] = g;
  *out = g.exec;
  return SIM_OK;
}

// Build and upload the balanced tile streams of the two profile products for the given
// grid sizes and zero-load cost; (re)allocates the partial-sum slots.
std::vector<int2> pairs(const std::vector<int32_t>& v) {
  std::vector<int2> o(v.size() / 2);
  for (size_t k = 0; k < o.size(); ++k) o[k] = make_int2(v[2 * k], v[2 * k + 1]);
  return o;
}

// Build and upload the balanced tile stream of one profile product for a grid size and a
// zero-load cost; (re)allocates its partial-sum slots.
int upload_schedule(sim_s* s, bool pass2, int grid, double zero_cost) {
  const Plan& p = s->plan;
  DevSim& d = s->d;
  silg::StreamSchedule sc;
  silg::build_stream_schedule(p, pass2, grid, zero_cost, &sc);
  if (!pass2) {
    // pass 1 stages the g slices of a CTA's column tiles in shared memory (3 KB each, at
    // most silg::kMaxStagedCols): more CTAs when a range has too many
    while (sc.max_cols > silg::kMaxStagedCols && grid < (1 << 20)) {
      grid *= 2;
      silg::build_stream_schedule(p, false, grid, zero_cost, &sc);
    }
    d.s1_tiles = s->upload(pairs(sc.tiles));
    d.s1_cta = s->upload(sc.cta_first);
    d.s1_seg_base = s->upload(sc.seg_base);
    d.s1_seg_first = s->upload(sc.seg_first);
    d.s1_col_first = s->upload(sc.cta_col_first);
    d.s1_cols = s->upload(sc.cta_cols);
    d.s1_col_slot = s->upload(sc.tile_col_slot);
    d.s1_max_cols = sc.max_cols;
    d.s1_grid = grid;
    d.n_seg1 = sc.n_seg;
    d.p1_part = s->alloc<float>((size_t)std::max(1, sc.n_seg) * 3 * silg::kRowGroup);
  } else {
    d.s2_tiles = s->upload(pairs(sc.tiles));
    d.s2_cta = s->upload(sc.cta_first);
    d.s2_seg_base = s->upload(sc.seg_base);
    d.s2_seg_first = s->upload(sc.seg_first);
    d.s2_grid = grid;
    d.n_seg2 = sc.n_seg;
    d.p2_part = s->alloc<float>((size_t)std::max(1, sc.n_seg) * 3 * silg::kTileW);
  }
  return SIM_OK;
}

// Launch configuration of the profile products before tuning: two CTAs per SM (the
// register limit of the kernels), tiles balanced by count, the format's tiles in flight.
constexpr int kDefaultCtasPerSm = 2;
constexpr double kDefaultBalance = 1.0;

// The autotuner of the two profile products. For each product it times every candidate
// launch configuration -- CTAs per SM (1 to 4; above the kernel's residency the grid runs
// in waves), the cost of an empty tile position relative to a stored value in the balanced
// split (1: equal tiles per CTA; 0.25: nearer equal bytes), and the tiles in flight per warp
// (the format's default, half, or twice with one resident CTA per SM) -- on the simulator's
// own matrix with CUDA events (median of 5 launches after 2 warm-up launches), and keeps
// the fastest.
int autotune_products(sim_s* s) {
  DevSim& d = s->d;
  cudaStream_t st = s->work;
  {
    // any right-hand side: the products' time does not depend on the values
    std::vector<float> g(3 * (size_t)d.n_pad, 0.f);
    uint32_t x = 12345u;
    for (int k = 0; k < d.n; ++k)
      for (int r = 0; r < 3; ++r) {
        x = x * 1664525u + 1013904223u;
        g[(size_t)r * d.n_pad + k] = (float)((x >> 8) * (1.0 / 16777216.0) - 0.5);
      }
    cudaMemcpyAsync(d.gvec, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    silg::launch_solve(d, st, silg::kOutX);   // zvec holds a valid z for pass 2
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SIM_ECUDA;
  const int ctas[] = {1, 2, 3, 4};
  const double balance[] = {1.0, 0.25};
  const int unroll[] = {1, 0, 2, silg::kUnrollBulk};
  sim_tuning& T = s->tuning;
  T = sim_tuning{};
  int status = SIM_OK;
  for (int pass = 0; pass < 2 && status == SIM_OK; ++pass) {
    double best = 1e300;
    int best_c = kDefaultCtasPerSm, best_u = 1;
    double best_b = kDefaultBalance, dflt = 0;
    int n_cand = 0;
    for (int c : ctas)
      for (double b : balance)
        for (int u : unroll) {
          upload_schedule(s, pass == 1, c * d.n_sm, b);
          (pass ? d.s2_unroll : d.s1_unroll) = u;
          auto launch = [&]() { pass ? silg::launch_pass2(d, st) : silg::launch_pass1(d, st); };
          for (int w = 0; w < 2; ++w) launch();
          std::vector<float> t(5);
          for (float& ms : t) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = SIM_ECUDA;
            cudaEventElapsedTime(&ms, e0, e1);
          }
          if (cudaGetLastError() != cudaSuccess) status = SIM_ECUDA;
          // a candidate whose waits ran out (bulk-copy form) is not a choice
          int err = 0;
          cudaMemcpy(&err, d.err, sizeof(int), cudaMemcpyDeviceToHost);
          if (err) cudaMemset(d.err, 0, sizeof(int));
          std::sort(t.begin(), t.end());
          const double us = err ? 1e300 : 1e3 * t[2];
          ++n_cand;
          if (c == kDefaultCtasPerSm && b == kDefaultBalance && u == 1) dflt = us;
          if (us < best) {
            best = us;
            best_c = c;
            best_b = b;
            best_u = u;
          }
        }
    upload_schedule(s, pass == 1, best_c * d.n_sm, best_b);
    (pass ? d.s2_unroll : d.s1_unroll) = best_u;
    if (pass == 0) {
      T.pass1_ctas = d.s1_grid;
      T.pass1_unroll = best_u;
      T.pass1_balance = best_b;
      T.pass1_us = best;
      T.pass1_default_us = dflt;
    } else {
      T.pass2_ctas = d.s2_grid;
      T.pass2_unroll = best_u;
      T.pass2_balance = best_b;
      T.pass2_us = best;
      T.pass2_default_us = dflt;
    }
    T.candidates = n_cand;
  }
  T.tuned = status == SIM_OK;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

// Per-scene inputs of the device arrays (one entry for sim_create).
struct SceneData {
  std::vector<sim_obstacle> obstacles;
  std::vector<int32_t> obstacle_scene;
  std::vector<double> margin, L_ref, hvel;  // hvel: 3 per scene
  std::vector<sim_anchor> anchors;          // vertex ids in the union's numbering
  // contact between bodies (union numbering): the first body of every scene (n_scenes + 1),
  // every body's surface triangles whose corners are all free (body_toff, n_bodies + 1;
  // corners and the triangle's number in btri), the body of every surface vertex (-1: none,
  // or a pinned vertex) and each scene's friction coefficient between bodies
  std::vector<int> scene_bfirst, body_toff, vert_body;
  std::vector<std::array<int, 4>> btri;
  std::vector<double> bmu;
};

// The connected components of a scene's tetrahedra (numbered in order of their smallest
// vertex id) and its surface triangles: faces of one element only, oriented so that
// (b - a) x (c - a) points away from the element at rest, rotated to start at the smallest
// id, in the order of their sorted vertex triples.
void scene_surface(const sim_mesh& m, std::vector<int>& comp,
                   std::vector<std::array<int, 3>>& tris) {
  const int nv = m.n_verts;
  std::vector<int> parent(nv);
  std::iota(parent.begin(), parent.end(), 0);
  auto root = [&](int a) {
    while (parent[a] != a) a = parent[a] = parent[parent[a]];
    return a;
  };
  for (int t = 0; t < m.n_tets; ++t) {
    const int32_t* v = m.tets + 4 * (size_t)t;
    int r0 = root(v[0]);
    for (int k = 1; k < 4; ++k) {
      const int r = root(v[k]);
      if (r != r0) {
        parent[std::max(r, r0)] = std::min(r, r0);
        r0 = std::min(r, r0);
      }
    }
  }
  comp.assign(nv, -1);
  std::vector<int> id(nv, -1);
  int nc = 0;
  for (int v = 0; v < nv; ++v) {
    const int r = root(v);
    if (id[r] < 0) id[r] = nc++;
    comp[v] = id[r];
  }
  struct Face { int cnt; std::array<int, 3> f; int opp; };
  std::map<std::array<int, 3>, Face> faces;
  for (int t = 0; t < m.n_tets; ++t) {
    const int32_t* v = m.tets + 4 * (size_t)t;
    for (int k = 0; k < 4; ++k) {
      std::array<int, 3> f;
      int q = 0;
      for (int i = 0; i < 4; ++i)
        if (i != k) f[q++] = v[i];
      std::array<int, 3> key = f;
      std::sort(key.begin(), key.end());
      auto it = faces.find(key);
      if (it == faces.end()) faces.emplace(key, Face{1, f, v[k]});
      else ++it->second.cnt;
    }
  }
  tris.clear();
  const double* X = m.rest_pos;
  for (const auto& kv : faces) {
    if (kv.second.cnt != 1) continue;
    int a = kv.second.f[0], b = kv.second.f[1], c = kv.second.f[2];
    const int dd = kv.second.opp;
    double e1[3], e2[3], e3[3];
    for (int r = 0; r < 3; ++r) {
      e1[r] = X[3 * b + r] - X[3 * a + r];
      e2[r] = X[3 * c + r] - X[3 * a + r];
      e3[r] = X[3 * dd + r] - X[3 * a + r];
    }
    const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                 nz = e1[0] * e2[1] - e1[1] * e2[0];
    if (nx * e3[0] + ny * e3[1] + nz * e3[2] > 0) std::swap(b, c);
    std::array<int, 3> tr = {a, b, c};
    const int i0 = (int)(std::min_element(tr.begin(), tr.end()) - tr.begin());
    tris.push_back({tr[i0], tr[(i0 + 1) % 3], tr[(i0 + 2) % 3]});
  }
}

int create_device(sim_s* s, const SceneData& sd, const sim_options* o) {
  const sim_obstacle* obstacles = sd.obstacles.data();
  const int n_obs = (int)sd.obstacles.size();
  Plan& p = s->plan;
  DevSim& d = s->d;
  const int n = p.n_free, n_all = p.n_verts, T = p.n_tets;
  d.n = n;
  d.n_all = n_all;
  d.n_tets = T;
  d.n_pad = p.n_pad;
  d.n_obs = n_obs;
  d.n_mat = (int)p.mats.size();
  d.cap = std::max(1, o->contact_capacity);
  d.n_cr = std::max(0, o->n_cr_iters);
  d.ncp = o->ncp;
  d.precond = o->precond;
  d.pf_copies = 1;
  d.res_tol = o->residual_tol;
  d.max_iters = o->max_iters;
  d.admm = o->local_solver == SIM_LOCAL_ADMM;
  d.tet_u = d.admm ? s->alloc<float>(9 * (size_t)T) : nullptr;
  d.jacobi_sweeps = o->global_solver == SIM_GLOBAL_JACOBI ? o->jacobi_sweeps : 0;
  d.dq_alt = d.jacobi_sweeps ? s->alloc<float>(3 * (size_t)n_all) : nullptr;
  if (d.jacobi_sweeps && (n_obs > 0 || !sd.anchors.empty())) return SIM_EINVAL;
  d.h = p.h;
  d.h2f = (float)(p.h * p.h);
  for (int r = 0; r < 3; ++r) d.grav[r] = o->gravity[r];
  // ---- scenes -------------------------------------------------------------------------
  d.n_scenes = p.n_scenes;
  {
    std::vector<int> vs(n_all);
    for (int v = 0; v < n_all; ++v) vs[p.internal[v]] = p.vertex_scene[v];
    d.vert_scene = s->upload(vs);
  }
  d.scene_vfirst = s->upload(p.scene_vfirst);
  d.obst_scene = s->upload(sd.obstacle_scene);
  {
    // anchors: per free internal vertex, its anchor (targets reset to time 0)
    const int na = (int)sd.anchors.size();
    d.n_anc = na;
    std::vector<int> of(std::max(1, n), -1);
    std::vector<double> pos(3 * (size_t)std::max(1, na)), vel(pos.size()), e(std::max(1, na));
    for (int a = 0; a < na; ++a) {
      const sim_anchor& an = sd.anchors[a];
      of[p.internal[an.vertex]] = a;
      for (int r = 0; r < 3; ++r) {
        pos[3 * a + r] = an.target[r];
        vel[3 * a + r] = an.vel[r];
      }
      e[a] = an.compliance;
    }
    // two-vertex rows: the partner's internal id per anchor (-1: a target anchor), and a
    // one-corner map entry per pair, appended after the bodies' surface triangles
    std::vector<int> partner(std::max(1, na), -1);
    for (int a = 0; a < na; ++a)
      if (sd.anchors[a].partner >= 0) partner[a] = p.internal[sd.anchors[a].partner];
    d.anc_partner = s->upload(partner);
    d.n_pairs = 0;
    for (int a = 0; a < na; ++a) d.n_pairs += partner[a] >= 0;
    d.anc_of = s->upload(of);
    d.anc_pos0 = s->upload(pos);
    d.anc_pos = s->upload(pos);
    d.anc_vel = s->upload(vel);
    d.anc_e = s->upload(e);
  }
  {
    // obstacles are listed scene by scene
    std::vector<int> of(p.n_scenes + 1, n_obs);
    for (int q = n_obs - 1; q >= 0; --q) of[sd.obstacle_scene[q]] = q;
    for (int sc = p.n_scenes - 1; sc >= 0; --sc) of[sc] = std::min(of[sc], of[sc + 1]);
    d.scene_ofirst = s->upload(of);
  }
  {
    // contact between bodies: per free vertex its body; per body its triangles (internal
    // corner ids, the triangle's number in w)
    const int nb = (int)sd.body_toff.size() - 1;
    d.n_bodies = nb;
    d.bc_on = nb > 0;
    // contact maps beyond one vertex: contacts between bodies and two-vertex anchor rows
    d.map_on = d.bc_on || d.n_pairs > 0;
    if (d.map_on && !d.bc_on) {
      // pairs only: their map entries, no bodies to search
      std::vector<int4> bt(std::max(1, d.n_pairs));
      std::vector<int> ptri(std::max(1, (int)sd.anchors.size()), -1);
      int k = 0;
      for (int a = 0; a < (int)sd.anchors.size(); ++a)
        if (sd.anchors[a].partner >= 0) {
          const int b = p.internal[sd.anchors[a].partner];
          bt[k] = make_int4(b, b, b, -1);
          ptri[a] = k++;
        }
      d.btri = s->upload(bt);
      d.anc_ptri = s->upload(ptri);
      d.n_btri = 0;
      d.x_cnt = s->alloc<int>(n);
      d.x_fill = s->alloc<int>(n);
      d.x_off = s->alloc<int>(n + 1);
      d.x_list = s->alloc<int>(3 * (size_t)d.cap);
      d.ct_tri = s->alloc<int>(d.cap);
      d.ct_bw = s->alloc<double>(3 * (size_t)d.cap);
      d.ct_tcv = s->alloc<int>(3 * (size_t)d.cap);
    }
    if (d.bc_on) {
      std::vector<int> vb(std::max(1, n), -1);
      for (int v = 0; v < n_all; ++v)
        if (p.internal[v] < n) vb[p.internal[v]] = sd.vert_body[v];
      d.vert_body = s->upload(vb);
      // the bodies' surface triangles, then one one-corner map entry per pair anchor
      std::vector<int4> bt(std::max<size_t>(1, sd.btri.size() + d.n_pairs));
      for (size_t t = 0; t < sd.btri.size(); ++t)
        bt[t] = make_int4(p.internal[sd.btri[t][0]], p.internal[sd.btri[t][1]],
                          p.internal[sd.btri[t][2]], sd.btri[t][3]);
      std::vector<int> ptri(std::max(1, (int)sd.anchors.size()), -1);
      int k = (int)sd.btri.size();
      for (int a = 0; a < (int)sd.anchors.size(); ++a)
        if (sd.anchors[a].partner >= 0) {
          const int b = p.internal[sd.anchors[a].partner];
          bt[k] = make_int4(b, b, b, -1);
          ptri[a] = k++;
        }
      d.btri = s->upload(bt);
      d.anc_ptri = s->upload(ptri);
      d.body_toff = s->upload(sd.body_toff);
      d.scene_bfirst = s->upload(sd.scene_bfirst);
      d.scene_bmu = s->upload(sd.bmu);
      d.body_box = s->alloc<double>(6 * (size_t)nb);
      d.n_btri = (int)sd.btri.size();
      d.chunk_box = s->alloc<float>(6 * (size_t)(d.n_btri / silg::kTriChunk + 1));
      d.tri_box = s->alloc<float>(6 * (size_t)std::max(1, d.n_btri));
      d.super_box = s->alloc<float>(6 * (size_t)(d.n_btri / silg::kTriSuper + 1));
      d.bc_tri = s->alloc<int>(n);
      d.bc_w = s->alloc<double>(3 * (size_t)n);
      d.bc_n = s->alloc<double>(3 * (size_t)n);
      d.x_cnt = s->alloc<int>(n);
      d.x_fill = s->alloc<int>(n);
      d.x_off = s->alloc<int>(n + 1);
      d.x_list = s->alloc<int>(3 * (size_t)d.cap);
      d.ct_tri = s->alloc<int>(d.cap);
      d.ct_bw = s->alloc<double>(3 * (size_t)d.cap);
      d.ct_tcv = s->alloc<int>(3 * (size_t)d.cap);
    }
  }
  d.scene_margin = s->upload(sd.margin);
  d.scene_Lref = s->upload(sd.L_ref);
  d.scene_hvel = s->upload(sd.hvel);
  {
    std::vector<double> sm(p.n_scenes, 0.0);
    for (int v = 0; v < n_all; ++v)
      if (!p.pinned[v]) sm[p.vertex_scene[v]] += p.mass[v];
    for (double& m : sm) m = m > 0 ? m : 1.0;
    d.scene_mass = s->upload(sm);
  }
  d.sc_cvb = s->alloc<int>(p.n_scenes + 1);
  d.sc_jb = s->alloc<int>(p.n_scenes + 1);
  d.sc_ld = s->alloc<int>(p.n_scenes);
  d.sc_wtoff = s->alloc<long long>(p.n_scenes + 1);
  d.sc_tileoff = s->alloc<int>(p.n_scenes + 1);
  d.resid_scene = s->alloc<double>((size_t)p.n_scenes * (silg::kMaxIters + 1));
  // ---- per vertex (internal numbering) ---------------------------------------------
  std::vector<double> mass(n_all), X(3 * (size_t)n_all);
  for (int v = 0; v < n_all; ++v) {
    int iv = p.internal[v];
    mass[iv] = p.mass[v];
    for (int r = 0; r < 3; ++r) X[3 * (size_t)iv + r] = p.X[3 * (size_t)v + r];
  }
  d.mass = s->upload(mass);
  d.q_t = s->upload(X);
  d.v_t = s->alloc<double>(3 * (size_t)n_all);
  d.q_ref = s->upload(X);
  d.s_tilde = s->upload(X);
  d.dq = s->alloc<float>(3 * (size_t)n_all);
  d.qr_hi = s->alloc<float>(3 * (size_t)n_all);
  d.qr_lo = s->alloc<float>(3 * (size_t)n_all);
  d.depth = s->upload(p.depth);
  d.parent = s->upload(p.parent);
  d.first_desc = s->upload(p.first_desc);
  // ---- per element ---------------------------------------------------------------
  std::vector<int4> tv(T);
  std::vector<float> dminv(9 * (size_t)T), tw(T), tvol(T);
  for (int t = 0; t < T; ++t) {
    const int32_t* v = &p.tets[4 * (size_t)t];
    tv[t] = make_int4(p.internal[v[0]], p.internal[v[1]], p.internal[v[2]], p.internal[v[3]]);
    for (int k = 0; k < 9; ++k) dminv[(size_t)k * T + t] = (float)p.Dm_inv[9 * (size_t)t + k];
    tw[t] = (float)p.weight[t];
    tvol[t] = (float)p.vol[t];
  }
  d.tet_v = s->upload(tv);
  d.tet_dminv = s->upload(dminv);
  d.tet_w = s->upload(tw);
  d.tet_vol = s->upload(tvol);
  d.tet_mat = s->upload(p.tet_mat);
  std::vector<silg::MatDev> md;
  for (auto& m : p.mats) md.push_back({m.model, (float)m.mu, (float)m.lam, (float)m.alpha});
  d.mats = s->upload(md);
  // triangles: element entries 4 n_tets + 3 t + a follow the tetrahedra's
  const int Nt = p.n_tris;
  d.n_tris = Nt;
  {
    std::vector<int4> trv(std::max(1, Nt));
    std::vector<float> tdm(4 * (size_t)std::max(1, Nt)), trw(std::max(1, Nt)),
        trvol(std::max(1, Nt));
    for (int t = 0; t < Nt; ++t) {
      const int32_t* v = &p.tris[3 * (size_t)t];
      trv[t] = make_int4(p.internal[v[0]], p.internal[v[1]], p.internal[v[2]], 0);
      for (int k = 0; k < 4; ++k) tdm[(size_t)k * Nt + t] = (float)p.tri_dminv[4 * (size_t)t + k];
      trw[t] = (float)p.tri_weight[t];
      trvol[t] = (float)p.tri_vol[t];
    }
    d.tri_v = s->upload(trv);
    d.tri_dminv = s->upload(tdm);
    d.tri_w = s->upload(trw);
    d.tri_vol = s->upload(trvol);
    d.tri_mat = s->upload(Nt ? p.tri_mat : std::vector<int32_t>(1, 0));
  }
  d.contrib = s->alloc<float4>(4 * (size_t)T + 3 * (size_t)Nt);
  {
    std::vector<int> cnt(n + 1, 0);
    for (int t = 0; t < T; ++t)
      for (int a = 0; a < 4; ++a) {
        int iv = p.internal[p.tets[4 * (size_t)t + a]];
        if (iv < n) ++cnt[iv + 1];
      }
    for (int t = 0; t < Nt; ++t)
      for (int a = 0; a < 3; ++a) {
        int iv = p.internal[p.tris[3 * (size_t)t + a]];
        if (iv < n) ++cnt[iv + 1];
      }
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int> idx(std::max(1, cnt[n])), fill(cnt.begin(), cnt.end() - 1);
    for (int t = 0; t < T; ++t)
      for (int a = 0; a < 4; ++a) {
        int iv = p.internal[p.tets[4 * (size_t)t + a]];
        if (iv < n) idx[fill[iv]++] = 4 * t + a;
      }
    for (int t = 0; t < Nt; ++t)
      for (int a = 0; a < 3; ++a) {
        int iv = p.internal[p.tris[3 * (size_t)t + a]];
        if (iv < n) idx[fill[iv]++] = 4 * T + 3 * t + a;
      }
    d.inc_ptr = s->upload(cnt);
    d.inc_idx = s->upload(idx);
    // where each element corner's contribution is stored: its place in its vertex's
    // incidence list (-1: a pinned vertex, not summed), so the right-hand side reads each
    // vertex's contributions as one contiguous run
    std::vector<int> slot(std::max<size_t>(1, 4 * (size_t)T + 3 * (size_t)Nt), -1);
    for (int k = 0; k < cnt[n]; ++k) slot[idx[k]] = k;
    d.inc_slot = s->upload(slot);
  }
  // bending rows of the free vertices in internal numbering
  d.bend_ptr = nullptr;
  d.bend_idx = nullptr;
  d.bend_val = nullptr;
  d.bend_f = nullptr;
  if (!p.Kx.empty()) {
    std::vector<int> bp(n + 1, 0), bi;
    std::vector<double> bv;
    std::vector<int> caller_of(n);
    for (int v = 0; v < n_all; ++v)
      if (p.internal[v] < n) caller_of[p.internal[v]] = v;
    for (int i = 0; i < n; ++i) {
      const int v = caller_of[i];
      for (int64_t e = p.Kp[v]; e < p.Kp[v + 1]; ++e) {
        bi.push_back(p.internal[p.Ki[e]]);
        bv.push_back(p.Kx[e]);
      }
      bp[i + 1] = (int)bi.size();
    }
    if (bi.empty()) {
      bi.push_back(0);
      bv.push_back(0.0);
    }
    d.bend_ptr = s->upload(bp);
    d.bend_idx = s->upload(bi);
    d.bend_val = s->upload(bv);
    d.bend_f = s->alloc<float>(3 * (size_t)n);
  }
  // ---- S~ profile and tile schedule ---------------------------------------------------
  {
    d.s_bf16 = o->s_precision == SIM_S_BF16;
    d.refine = std::max(0, std::min(2, o->refine));
    d.Sb = nullptr;
    std::vector<long long> rb(p.rowbase.begin(), p.rowbase.end());
    d.rowbase = s->upload(rb);
    d.lo = s->upload(p.lo);
    d.hi = s->upload(p.hi);
    // an elimination tree too deep for the device kernel's path vectors: the host builds S~
    if (p.S.empty() && !silg::sinv_build_fits(p.max_depth)) silg::build_sinv_host(p, o->n_host_threads);
    if (!p.S.empty()) {
      std::vector<float> Sf(p.S.size());
      for (size_t k = 0; k < p.S.size(); ++k) Sf[k] = (float)p.S[k];
      d.S = s->upload(Sf);
      if (d.s_bf16) {
        // round to nearest even from the FP32 value (finite inputs)
        std::vector<uint16_t> Sb(Sf.size());
        for (size_t k = 0; k < Sf.size(); ++k) {
          uint32_t u;
          std::memcpy(&u, &Sf[k], 4);
          u += 0x7fffu + ((u >> 16) & 1u);
          Sb[k] = (uint16_t)(u >> 16);
        }
        d.Sb = reinterpret_cast<const unsigned short*>(s->upload(Sb));
      }
    } else {
      // S~ = L~^-1 P on the device in FP64 from the host's factor (k_sbuild.cu); the factor
      // and the kernel's work counter are released once the values are in place
      const auto t0 = std::chrono::steady_clock::now();
      const size_t stored = (size_t)p.rowbase[p.n_free];
      float* Sd = s->alloc<float>(stored);
      unsigned short* Sbd = d.s_bf16 ? s->alloc<unsigned short>(stored) : nullptr;
      std::vector<long long> lp(p.Lp.begin(), p.Lp.end());
      std::vector<int> ldd;
      silg::sinv_build_depth_steps(p, &ldd);
      long long* Lp_d = s->upload(lp);
      int* Ldd_d = s->upload(ldd);
      double* Lx_d = s->upload(p.Lx);
      int* ctr = s->alloc<int>(1);
      silg::SinvBuildArgs a{p.n_free, Lp_d, Ldd_d, Lx_d, d.parent, d.depth, d.rowbase, d.lo,
                            p.max_depth, ctr, Sd, Sbd};
      int st = silg::launch_sinv_build(a, s->work);
      if (st != SIM_OK) return st;
      const cudaError_t e = cudaStreamSynchronize(s->work);
      if (e != cudaSuccess) return cuda_status(e);
      for (void* t : {static_cast<void*>(Lp_d), static_cast<void*>(Ldd_d),
                      static_cast<void*>(Lx_d), static_cast<void*>(ctr)})
        s->release(t);
      d.S = Sd;
      d.Sb = Sbd;
      p.s_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      p.s_on_device = 1;
    }
    // A~ over the free vertices (FP64) for residuals of the global solve
    std::vector<int> ap(p.Ap.begin(), p.Ap.end());
    d.A_ptr = s->upload(ap);
    d.A_idx = s->upload(p.Ai);
    d.A_val = s->upload(p.Ax);
    d.gsave = s->alloc<float>(3 * (size_t)p.n_pad);
    d.n_rg = p.n_rg;
    d.n_ct = p.n_ct;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    d.n_sm = std::max(1, nsm);
    d.zero = s->alloc<float>(silg::kTileW);
    d.s1_unroll = d.s2_unroll = 1;
    upload_schedule(s, false, kDefaultCtasPerSm * d.n_sm, kDefaultBalance);
    upload_schedule(s, true, kDefaultCtasPerSm * d.n_sm, kDefaultBalance);
  }
  d.gvec = s->alloc<float>(3 * (size_t)p.n_pad);
  d.zvec = s->alloc<float>(3 * (size_t)p.n_pad);
  d.xout = s->alloc<float>(3 * (size_t)n);
  // ---- obstacles and contacts --------------------------------------------------------
  std::vector<silg::ObstDev> ob(std::max(1, n_obs));
  for (int k = 0; k < n_obs; ++k) {
    const sim_obstacle& so = obstacles[k];
    if ((so.kind != SIM_OBST_PLANE && so.kind != SIM_OBST_CYLINDER) || !(so.mu >= 0) ||
        (so.kind == SIM_OBST_CYLINDER && !(so.radius > 0)))
      return SIM_EINVAL;
    double an = std::sqrt(so.axis[0] * so.axis[0] + so.axis[1] * so.axis[1] + so.axis[2] * so.axis[2]);
    if (!(an > 0)) return SIM_EINVAL;
    ob[k].kind = so.kind;
    for (int r = 0; r < 3; ++r) {
      ob[k].p[r] = so.p[r];
      ob[k].a[r] = so.axis[r] / an;
      ob[k].vel[r] = so.vel[r];
    }
    ob[k].radius = so.radius;
    ob[k].mu = so.mu;
  }
  d.obst = s->upload(ob);
  const int cap = d.cap;
  long long cap_y = (long long)cap * std::max(1, p.max_depth);
  cap_y = std::min<long long>(cap_y, 1LL << 27);
  d.cap_y = (int)cap_y;
  d.counters = s->alloc<int>(silg::kNumCounters);
  d.ct_cnt = s->alloc<int>(n);
  d.ct_off = s->alloc<int>(n + 1);
  d.cv_flag = s->alloc<int>(n);
  d.cv_off = s->alloc<int>(n + 1);
  d.ct_vert = s->alloc<int>(cap);
  d.ct_obst = s->alloc<int>(cap);
  d.ct_cv = s->alloc<int>(cap);
  d.ct_D = s->alloc<double>(9 * (size_t)cap);
  d.ct_dn = s->alloc<double>(cap);
  d.ct_df = s->alloc<double>(2 * (size_t)cap);
  d.ct_mu = s->alloc<double>(cap);
  d.ct_r = s->alloc<double>(4 * (size_t)cap);
  d.ct_lam = s->alloc<double>(3 * (size_t)cap);
  d.ct_force = s->alloc<double>(3 * (size_t)cap);
  d.ct_omega = s->alloc<float>(3 * (size_t)cap);
  d.ct_ecal = s->alloc<float>(3 * (size_t)cap);
  d.ct_Df = s->alloc<float>(9 * (size_t)cap);
  d.ct_hv = s->alloc<double>(3 * (size_t)cap);
  d.ct_rhs = s->alloc<float>(3 * (size_t)cap);
  d.cv_vert = s->alloc<int>(cap);
  d.cv_first = s->alloc<int>(cap);
  d.cv_nct = s->alloc<int>(cap);
  d.uvec = s->alloc<float>(3 * (size_t)cap);
  d.svec = s->alloc<float>(3 * (size_t)cap);
  d.u_flag = s->alloc<int>(n);
  d.u_off = s->alloc<int>(n + 1);
  d.u_list = s->alloc<int>(n);
  d.row_clo = s->alloc<int>(n);
  d.row_len = s->alloc<int>(n);
  d.u_clo = s->alloc<int>(n);
  d.u_len = s->alloc<int>(n);
  d.y_ptr = s->alloc<int>(n + 1);
  d.y_val = s->alloc<float>(cap_y);
  d.yc_len = s->alloc<int>(cap);
  d.yc_ptr = s->alloc<int>(cap + 1);
  d.yc_val = s->alloc<float>(cap_y);
  d.yc_row = s->alloc<int>(cap_y);
  // W~ holds one block per scene, nv_s x ld_s floats (ld_s = nv_s rounded up to 4), with
  // sum_s nv_s <= cap and nv_s <= V = min(cap, the largest scene's free vertex count)
  int vmax = 1;
  for (int sc = 0; sc < p.n_scenes; ++sc)
    vmax = std::max(vmax, p.scene_vfirst[sc + 1] - p.scene_vfirst[sc]);
  const int V = std::min(cap, vmax);
  d.wt = s->alloc<float>((size_t)cap * ((V + 3) & ~3));
  // contacts of one scene: at most one per vertex and obstacle, anchor and other body
  std::vector<int> obs_per_scene(p.n_scenes, 0);
  for (int o : sd.obstacle_scene)
    if (o >= 0 && o < p.n_scenes) ++obs_per_scene[o];
  const int omax = obs_per_scene.empty() ? 0
                                         : *std::max_element(obs_per_scene.begin(), obs_per_scene.end());
  s->cr_vmax = V;
  s->cr_cmax = (int)std::min<long long>(cap, (long long)V * (omax + 2));
  d.resid = s->alloc<double>(silg::kMaxIters + 1);
  d.max_pen = s->alloc<double>(1);
  d.iter_k = s->alloc<int>(1);
  d.err = s->alloc<int>(1);
  d.p_out = s->alloc<float>(9 * (size_t)T);
  s->has_obstacles = n_obs > 0 || !sd.anchors.empty() || d.bc_on;
  d.wt_grid = 4 * d.n_sm;
  d.scan_part = s->alloc<int>(silg::scan_scratch_ints(std::max(n, cap)));
  d.dl_reuse_on = o->delassus_reuse ? 1 : 0;
  d.dl_state = s->alloc<int>(4);
  d.dl_prev_cv = s->alloc<int>(cap);
  cudaMemsetAsync(d.dl_state + 1, 0xff, sizeof(int), s->work);   // no previous list yet
  // the path of a contact vertex in Y is its ancestor chain: a warp covers a short one
  d.ytz_warp = p.mean_depth < 600.0 ? 1 : 0;
  d.spin_limit = o->spin_limit;
  d.kb_lo = s->alloc<int>(n / 32 + 1);
  d.kb_hi = s->alloc<int>(n / 32 + 1);
  // work items of the W~ product: the bound for one scene of every contact vertex (each
  // scene may add one partly filled block row), or, smaller with many small scenes, the
  // tiles of blocks of at most ceil(V / 64) tile rows over at most cap / 64 + n_scenes + 1
  // tile rows in all, plus one grid of K splits
  {
    const long long one = silg::wt_items_max(cap + 64 * p.n_scenes, d.wt_grid);
    const long long nbm = (V + 63) / 64;
    const long long many = (cap / 64 + p.n_scenes + 1) * (nbm + 1) / 2 + 1 + d.wt_grid;
    d.wt_part = s->alloc<float>((size_t)std::min(one, many) * 64 * 64);
  }
  if (silg::sinv_setup() != SIM_OK) return SIM_ECUDA;
  s->ev.resize(5 + kMarksPerIter * silg::kMaxIters);
  for (auto& e : s->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return SIM_ECUDA;
  d.cr_split = s->alloc<int>((size_t)p.n_scenes * 2 * (silg::kCrMaxRanks + 1));
  // warm start
  d.ws_mode = 0;
  d.ws_net = silg::MlpDev{};
  d.ws_net.theta = s->alloc<float>(silg::kMlpParams);
  d.ws_net.w_t = s->alloc<__nv_bfloat16>(silg::kWTElems);
  d.ws_net.err = d.err;   // a tensor-core wait that gives up is the frame's SIM_ETIMEOUT
  d.ws_feat = s->alloc<float>((size_t)cap * silg::kMlpIn);
  d.ws_out = s->alloc<float>((size_t)cap * silg::kMlpOut);
  d.ws_scale = s->alloc<double>(cap);
  d.ws_pmove = s->alloc<double>(cap);
  d.ws_lam0 = s->alloc<double>(3 * (size_t)cap);
  d.ws_move = s->alloc<double>(cap);
  d.ws_shift = s->alloc<double>(6 * (size_t)p.n_scenes);
  d.ws_res = s->alloc<double>(2 * (size_t)p.n_scenes);
  d.ws_rg = s->alloc<double>(cap);
  d.ws_rc = s->alloc<double>(cap);
  d.ws_target = s->alloc<float>(4 * (size_t)cap);
  d.prev_valid = s->alloc<int>(n);
  d.prev_obst = s->alloc<int>(n);
  d.prev_force = s->alloc<double>(3 * (size_t)n);
  d.prev_move = s->alloc<double>(n);
  if (silg::mlp_setup() != 0) return SIM_ECUDA;
  if (s->has_obstacles) {
    int st = silg::cr_setup(p.n_scenes, s->cr_vmax, s->cr_cmax, &s->cluster, &s->cr_smem);
    if (st != SIM_OK) return st;
  }
  d.cr_R = s->cluster;
  d.ws_gain[0] = d.ws_gain[1] = d.ws_gain[2] = d.ws_gain[3] = 1.f;
  d.cr_single = o->cr_exchanges == 1 ? 1 : 0;
  d.cr_sync = o->cr_sync;
  if (o->autotune == 1) {
    int st = autotune_products(s);
    if (st != SIM_OK) return st;
  } else if (o->autotune == 2) {
    d.s1_unroll = d.s2_unroll = silg::kUnrollBulk;   // the fixed grid, bulk-copy products
  }
  cudaError_t e = cudaStreamSynchronize(s->work);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(cudaGetLastError());
}

template <class F>
int guarded(F f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return SIM_ENOMEM;
  } catch (...) {
    return SIM_EINVAL;
  }
}

}  // namespace

// Device view of a simulator (for entry points compiled in other files).
const silg::DevSim* silg_sim_devsim(const sim_t* s, int* device) {
  if (!s) return nullptr;
  if (device) *device = s->device;
  return &s->d;
}

extern "C" {

void silg_fill_plan_info(const silg::Plan& p, sim_plan_info* info);

int sim_get_plan_info(const sim_t* s, sim_plan_info* info) {
  if (!s || !info) return SIM_EINVAL;
  silg_fill_plan_info(s->plan, info);
  return SIM_OK;
}

int sim_get_ordering(const sim_t* s, int32_t* order, int32_t* parent, int32_t* first_desc) {
  if (!s) return SIM_EINVAL;
  const silg::Plan& p = s->plan;
  const size_t nf = (size_t)p.n_free;
  if (order) std::memcpy(order, p.order.data(), sizeof(int32_t) * nf);
  if (parent) std::memcpy(parent, p.parent.data(), sizeof(int32_t) * nf);
  if (first_desc) std::memcpy(first_desc, p.first_desc.data(), sizeof(int32_t) * nf);
  return SIM_OK;
}

namespace {

double mean_edge(const sim_mesh& m) {
  double sum = 0;
  long long cnt = 0;
  for (int t = 0; t < m.n_tets; ++t) {
    const int32_t* v = m.tets + 4 * (size_t)t;
    if (v[0] < 0 || v[0] >= m.n_verts) continue;
    for (int a = 1; a < 4; ++a) {
      if (v[a] < 0 || v[a] >= m.n_verts) continue;
      double e2 = 0;
      for (int r = 0; r < 3; ++r) {
        const double dx = m.rest_pos[3 * (size_t)v[a] + r] - m.rest_pos[3 * (size_t)v[0] + r];
        e2 += dx * dx;
      }
      sum += std::sqrt(e2);
      ++cnt;
    }
  }
  for (int t = 0; t < m.n_tris; ++t) {
    const int32_t* v = m.tris + 3 * (size_t)t;
    if (v[0] < 0 || v[0] >= m.n_verts) continue;
    for (int a = 1; a < 3; ++a) {
      if (v[a] < 0 || v[a] >= m.n_verts) continue;
      double e2 = 0;
      for (int r = 0; r < 3; ++r) {
        const double dx = m.rest_pos[3 * (size_t)v[a] + r] - m.rest_pos[3 * (size_t)v[0] + r];
        e2 += dx * dx;
      }
      sum += std::sqrt(e2);
      ++cnt;
    }
  }
  return cnt ? sum / cnt : 0.0;
}

double bbox_diagonal(const sim_mesh& m) {
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < m.n_verts; ++v)
    for (int r = 0; r < 3; ++r) {
      mn[r] = std::min(mn[r], m.rest_pos[3 * (size_t)v + r]);
      mx[r] = std::max(mx[r], m.rest_pos[3 * (size_t)v + r]);
    }
  double s2 = 0;
  for (int r = 0; r < 3; ++r) s2 += (mx[r] - mn[r]) * (mx[r] - mn[r]);
  return std::sqrt(s2);
}

int check_options(const sim_options* o) {
  if (o->n_iters < 0 || o->n_iters > silg::kMaxIters || o->n_cr_iters < 0 ||
      o->contact_capacity <= 0 || o->contact_capacity > (1 << 16))
    return SIM_EINVAL;
  if (o->s_precision != SIM_S_FP32 && o->s_precision != SIM_S_BF16) return SIM_EINVAL;
  if (o->refine < 0 || o->refine > 2) return SIM_EINVAL;
  if (o->ncp != SIM_NCP_FB && o->ncp != SIM_NCP_MINMAP) return SIM_EINVAL;
  if (o->local_solver != SIM_LOCAL_PD && o->local_solver != SIM_LOCAL_ADMM) return SIM_EINVAL;
  if (o->global_solver != SIM_GLOBAL_SPARSE_INVERSE && o->global_solver != SIM_GLOBAL_JACOBI)
    return SIM_EINVAL;
  if (o->global_solver == SIM_GLOBAL_JACOBI && (o->jacobi_sweeps < 1 || o->jacobi_sweeps > 1000))
    return SIM_EINVAL;
  if (!(o->residual_tol >= 0.0) || o->max_iters < 1 || o->max_iters > silg::kMaxIters)
    return SIM_EINVAL;
  if ((o->dev_alloc == nullptr) != (o->dev_free == nullptr)) return SIM_EINVAL;
  if (o->autotune < 0 || o->autotune > 2) return SIM_EINVAL;
  if (o->precond != SIM_PRECOND_DELASSUS && o->precond != SIM_PRECOND_MASS) return SIM_EINVAL;
  if (o->cr_exchanges != 1 && o->cr_exchanges != 2) return SIM_EINVAL;
  if (o->delassus_reuse != 0 && o->delassus_reuse != 1) return SIM_EINVAL;
  if (o->cr_sync != 0 && o->cr_sync != 1) return SIM_EINVAL;
  if (o->s_build != 0 && o->s_build != 1) return SIM_EINVAL;
  return SIM_OK;
}

// The union of the scenes: vertices, tets, materials and obstacles concatenated scene by
// scene; each scene keeps its margin, scale and handle velocity. margin_override > 0
// replaces every scene's margin (sim_create's option).
int create_common(const sim_scene* scenes, int n_scenes, double h, const sim_options* opts,
                  double margin_override, sim_t** out) {
  silg::DeviceGuard dg;   // creation selects the simulator's device; the caller's returns
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (!scenes || n_scenes < 1) return SIM_EINVAL;
  sim_options def;
  sim_default_options(&def);
  const sim_options* o = opts ? opts : &def;
  if (check_options(o) != SIM_OK) return SIM_EINVAL;
  long long nv_tot = 0, nt_tot = 0, np_tot = 0, ntr_tot = 0;
  for (int k = 0; k < n_scenes; ++k) {
    const sim_scene& sc = scenes[k];
    if (sc.mesh.n_verts <= 0 || sc.mesh.n_tets < 0 || sc.mesh.n_tris < 0 ||
        sc.mesh.n_tets + sc.mesh.n_tris <= 0 || !sc.mesh.rest_pos ||
        (sc.mesh.n_tets > 0 && !sc.mesh.tets) || (sc.mesh.n_tris > 0 && !sc.mesh.tris) ||
        (sc.mesh.n_tris > 0 && o->local_solver == SIM_LOCAL_ADMM) ||
        // the Jacobi comparison solves the contact-free system only
        (o->global_solver == SIM_GLOBAL_JACOBI &&
         (sc.n_obstacles > 0 || sc.n_anchors > 0 || sc.body_contact)) ||
        (sc.body_contact != 0 && sc.body_contact != 1) ||
        (sc.body_contact && !(std::isfinite(sc.body_mu) && sc.body_mu >= 0.0)) ||
        (sc.body_contact && sc.mesh.n_tets <= 0) ||
        !sc.materials || sc.n_materials <= 0 || sc.n_obstacles < 0 ||
        (sc.n_obstacles > 0 && !sc.obstacles) || sc.mesh.n_pinned < 0 ||
        (sc.mesh.n_pinned > 0 && !sc.mesh.pinned))
      return SIM_EINVAL;
    nv_tot += sc.mesh.n_verts;
    nt_tot += sc.mesh.n_tets;
    ntr_tot += sc.mesh.n_tris;
    np_tot += sc.mesh.n_pinned;
  }
  if (nv_tot >= (1LL << 31) || nt_tot >= (1LL << 29)) return SIM_EINVAL;
  sim_s* s = new (std::nothrow) sim_s();
  if (!s) return SIM_ENOMEM;
  s->phase_marks = o->phase_marks != 0;
  s->dev_alloc = o->dev_alloc;
  s->dev_free = o->dev_free;
  s->alloc_ctx = o->alloc_ctx;
  int st = guarded([&]() {
    std::vector<double> X;
    std::vector<int32_t> tets, tmat, pinned, vscene, tris, trmat;
    std::vector<double> trthick, vbend;
    std::vector<sim_material> mats;
    SceneData sd;
    X.reserve(3 * nv_tot);
    tets.reserve(4 * nt_tot);
    int voff = 0, btri_base = 0;
    for (int k = 0; k < n_scenes; ++k) {
      const sim_scene& sc = scenes[k];
      const sim_mesh& m = sc.mesh;
      const int moff = (int)mats.size();
      X.insert(X.end(), m.rest_pos, m.rest_pos + 3 * (size_t)m.n_verts);
      for (int t = 0; t < m.n_tets; ++t) {
        for (int a = 0; a < 4; ++a) {
          const int v = m.tets[4 * (size_t)t + a];
          tets.push_back(v >= 0 && v < m.n_verts ? v + voff : -1);
        }
        const int mt = m.tet_material ? m.tet_material[t] : 0;
        tmat.push_back(mt >= 0 && mt < sc.n_materials ? mt + moff : -1);
      }
      for (int t = 0; t < m.n_tris; ++t) {
        for (int a = 0; a < 3; ++a) {
          const int v = m.tris[3 * (size_t)t + a];
          tris.push_back(v >= 0 && v < m.n_verts ? v + voff : -1);
        }
        const int mt = m.tri_material ? m.tri_material[t] : 0;
        trmat.push_back(mt >= 0 && mt < sc.n_materials ? mt + moff : -1);
        trthick.push_back(m.thickness);
      }
      vbend.insert(vbend.end(), m.n_verts, m.bending);
      for (int q = 0; q < m.n_pinned; ++q)
        pinned.push_back(m.pinned[q] >= 0 && m.pinned[q] < m.n_verts ? m.pinned[q] + voff : -1);
      mats.insert(mats.end(), sc.materials, sc.materials + sc.n_materials);
      vscene.insert(vscene.end(), m.n_verts, k);
      for (int q = 0; q < sc.n_obstacles; ++q) {
        sd.obstacles.push_back(sc.obstacles[q]);
        sd.obstacle_scene.push_back(k);
      }
      if (sc.n_anchors < 0 || (sc.n_anchors > 0 && !sc.anchors)) return SIM_EINVAL;
      {
        std::vector<char> used(m.n_verts, 0);
        for (int q = 0; q < m.n_pinned; ++q)
          if (m.pinned[q] >= 0 && m.pinned[q] < m.n_verts) used[m.pinned[q]] = 1;
        for (int q = 0; q < sc.n_anchors; ++q) {
          sim_anchor a = sc.anchors[q];
          bool ok = a.vertex >= 0 && a.vertex < m.n_verts && used[a.vertex] != 1 &&
                    used[a.vertex] != 2 && std::isfinite(a.compliance) &&
                    a.compliance >= 0.0 && (a.paired == 0 || a.paired == 1);
          for (int r = 0; r < 3; ++r) ok = ok && std::isfinite(a.target[r]) && std::isfinite(a.vel[r]);
          // the partner of a pair: another free vertex of the same scene
          if (a.paired)
            ok = ok && a.partner >= 0 && a.partner < m.n_verts && a.partner != a.vertex &&
                 used[a.partner] != 1;
          if (!ok) return SIM_EINVAL;
          used[a.vertex] = 2;
          a.vertex += voff;
          if (a.paired) a.partner += voff;
          else a.partner = -1;
          sd.anchors.push_back(a);
        }
      }
      {
        // contact between the scene's bodies: components, surface, per-body triangle lists
        const int nb0 = (int)sd.body_toff.size();
        sd.scene_bfirst.push_back(nb0);
        sd.bmu.push_back(sc.body_contact ? sc.body_mu : 0.0);
        sd.vert_body.insert(sd.vert_body.end(), m.n_verts, -1);
        if (sc.body_contact) {
          for (size_t e = 0; e < 4 * (size_t)m.n_tets; ++e)
            if (m.tets[e] < 0 || m.tets[e] >= m.n_verts) return SIM_EINVAL;
          std::vector<int> comp;
          std::vector<std::array<int, 3>> st;
          scene_surface(m, comp, st);
          std::vector<char> pin(m.n_verts, 0);
          for (int q = 0; q < m.n_pinned; ++q)
            if (m.pinned[q] >= 0 && m.pinned[q] < m.n_verts) pin[m.pinned[q]] = 1;
          const int ncomp = m.n_verts > 0 ? *std::max_element(comp.begin(), comp.end()) + 1 : 0;
          std::vector<std::vector<std::array<int, 4>>> per(ncomp);
          for (size_t t = 0; t < st.size(); ++t) {
            bool free = true;
            for (int v : st[t]) {
              if (!pin[v]) sd.vert_body[voff + v] = nb0 + comp[v];
              free = free && !pin[v];
            }
            if (free)
              per[comp[st[t][0]]].push_back(
                  {st[t][0] + voff, st[t][1] + voff, st[t][2] + voff, btri_base + (int)t});
          }
          // within a body, triangles in Morton order of their rest centroids, so that the
          // runs of kTriChunk consecutive triangles whose bounds the search tests are
          // compact (the search breaks ties by the triangle's number, not by this order)
          const double* X = m.rest_pos;
          for (int b = 0; b < ncomp; ++b) {
            auto& tl = per[b];
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            std::vector<std::array<double, 3>> cen(tl.size());
            for (size_t t = 0; t < tl.size(); ++t)
              for (int r = 0; r < 3; ++r) {
                cen[t][r] = (X[3 * (tl[t][0] - voff) + r] + X[3 * (tl[t][1] - voff) + r] +
                             X[3 * (tl[t][2] - voff) + r]) / 3.0;
                lo[r] = std::min(lo[r], cen[t][r]);
                hi[r] = std::max(hi[r], cen[t][r]);
              }
            std::vector<std::pair<uint64_t, int>> key(tl.size());
            for (size_t t = 0; t < tl.size(); ++t) {
              uint64_t code = 0;
              uint32_t qv[3];
              for (int r = 0; r < 3; ++r) {
                const double span = hi[r] - lo[r];
                qv[r] = span > 0 ? (uint32_t)std::min(1023.0, 1023.0 * (cen[t][r] - lo[r]) / span) : 0u;
              }
              for (int bit = 9; bit >= 0; --bit)
                for (int r = 0; r < 3; ++r) code = (code << 1) | ((qv[r] >> bit) & 1u);
              key[t] = {code, tl[t][3]};
            }
            std::vector<int> ord(tl.size());
            std::iota(ord.begin(), ord.end(), 0);
            std::sort(ord.begin(), ord.end(), [&](int a, int c) { return key[a] < key[c]; });
            sd.body_toff.push_back((int)sd.btri.size());
            for (int t : ord) sd.btri.push_back(tl[t]);
          }
          btri_base += (int)st.size();
        }
      }
      const double me = mean_edge(m);
      sd.margin.push_back(margin_override > 0 ? margin_override
                                              : (sc.contact_margin > 0 ? sc.contact_margin : 0.5 * me));
      sd.L_ref.push_back(bbox_diagonal(m));
      for (int r = 0; r < 3; ++r) sd.hvel.push_back(m.handle_vel[r]);
      {
        // FNV-1a over everything that defines the scene (local numbering)
        uint64_t hsh = 1469598103934665603ull;
        auto mix = [&](const void* ptr, size_t bytes) {
          const unsigned char* c = static_cast<const unsigned char*>(ptr);
          for (size_t i = 0; i < bytes; ++i) hsh = (hsh ^ c[i]) * 1099511628211ull;
        };
        mix(&m.n_verts, sizeof(m.n_verts));
        mix(m.rest_pos, sizeof(double) * 3 * (size_t)m.n_verts);
        if (m.n_tets > 0) mix(m.tets, sizeof(int32_t) * 4 * (size_t)m.n_tets);
        if (m.n_tris > 0) mix(m.tris, sizeof(int32_t) * 3 * (size_t)m.n_tris);
        mix(&m.thickness, sizeof(double));
        mix(&m.bending, sizeof(double));
        for (int t = 0; t < m.n_tets; ++t) {
          const int mt = m.tet_material ? m.tet_material[t] : 0;
          if (mt >= 0 && mt < sc.n_materials) {
            const sim_material& ma = sc.materials[mt];
            mix(&ma.model, sizeof(ma.model));
            mix(&ma.E, sizeof(double));
            mix(&ma.nu, sizeof(double));
            mix(&ma.rho, sizeof(double));
          }
        }
        for (int t = 0; t < m.n_tris; ++t) {
          const int mt = m.tri_material ? m.tri_material[t] : 0;
          if (mt >= 0 && mt < sc.n_materials) {
            const sim_material& ma = sc.materials[mt];
            mix(&ma.model, sizeof(ma.model));
            mix(&ma.E, sizeof(double));
            mix(&ma.nu, sizeof(double));
            mix(&ma.rho, sizeof(double));
          }
        }
        if (m.n_pinned > 0) mix(m.pinned, sizeof(int32_t) * m.n_pinned);
        mix(m.handle_vel, sizeof(m.handle_vel));
        for (int q = 0; q < sc.n_obstacles; ++q) {
          const sim_obstacle& ob = sc.obstacles[q];
          mix(&ob.kind, sizeof(ob.kind));
          mix(ob.p, sizeof(ob.p));
          mix(ob.axis, sizeof(ob.axis));
          mix(&ob.radius, sizeof(double));
          mix(&ob.mu, sizeof(double));
          mix(ob.vel, sizeof(ob.vel));
        }
        mix(&sd.margin.back(), sizeof(double));
        mix(&sc.body_contact, sizeof(sc.body_contact));
        if (sc.body_contact) mix(&sc.body_mu, sizeof(double));
        for (int q = 0; q < sc.n_anchors; ++q) {
          const sim_anchor& a = sc.anchors[q];
          mix(&a.vertex, sizeof(a.vertex));
          mix(a.target, sizeof(a.target));
          mix(a.vel, sizeof(a.vel));
          mix(&a.compliance, sizeof(double));
          mix(&a.paired, sizeof(a.paired));
          if (a.paired) mix(&a.partner, sizeof(a.partner));
        }
        s->scene_sig.push_back(hsh);
      }
      voff += m.n_verts;
    }
    if (sd.obstacle_scene.empty()) sd.obstacle_scene.push_back(0);
    sd.scene_bfirst.push_back((int)sd.body_toff.size());
    sd.body_toff.push_back((int)sd.btri.size());
    sim_mesh um{};
    um.n_verts = (int32_t)nv_tot;
    um.n_tets = (int32_t)nt_tot;
    um.rest_pos = X.data();
    um.tets = tets.data();
    um.tet_material = tmat.data();
    um.tris = tris.empty() ? nullptr : tris.data();
    um.tri_material = trmat.empty() ? nullptr : trmat.data();
    um.n_tris = (int32_t)ntr_tot;
    um.pinned = pinned.empty() ? nullptr : pinned.data();
    um.n_pinned = (int32_t)np_tot;
    for (int r = 0; r < 3; ++r) um.handle_vel[r] = scenes[0].mesh.handle_vel[r];
    std::string err;
    int r = silg::build_plan(&um, mats.data(), (int)mats.size(), h, o->n_host_threads, &s->plan,
                             &err, vscene.data(), n_scenes, trthick.data(), vbend.data(),
                             o->s_build == 0);
    if (r != SIM_OK) return r;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return SIM_ECUDA;
    if (o->device < 0 || o->device >= ndev) return SIM_EINVAL;
    s->device = o->device;
    if (cudaSetDevice(s->device) != cudaSuccess) return SIM_ECUDA;
    if (cudaStreamCreateWithFlags(&s->work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->body, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->body_aux, cudaStreamNonBlocking) != cudaSuccess)
      return SIM_ECUDA;
    if (cudaMallocHost(&s->pinned, sizeof(double) * 6 * (size_t)std::max<long long>(1, nv_tot)) !=
        cudaSuccess)
      return SIM_ENOMEM;
    s->fj.resize(2 * silg::kMaxIters + 4);
    for (auto& e : s->fj)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SIM_ECUDA;
    s->launch = o->cuda_stream ? static_cast<cudaStream_t>(o->cuda_stream) : s->work;
    s->n_iters_default = o->n_iters > 0 ? o->n_iters : 5;
    return create_device(s, sd, o);
  });
  if (st != SIM_OK) {
    delete s;
    return st;
  }
  *out = s;
  return SIM_OK;
}

}  // namespace

int sim_create(const sim_mesh* mesh, const sim_material* mats, int32_t n_mat,
               const sim_obstacle* obstacles, int32_t n_obs, double h,
               const sim_options* opts, sim_t** out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (!mesh || n_obs < 0 || (n_obs > 0 && !obstacles)) return SIM_EINVAL;
  sim_options def;
  sim_default_options(&def);
  const sim_options* o = opts ? opts : &def;
  sim_scene sc{};
  sc.mesh = *mesh;
  sc.materials = mats;
  sc.n_materials = n_mat;
  sc.obstacles = obstacles;
  sc.n_obstacles = n_obs;
  sc.contact_margin = o->contact_margin;
  return create_common(&sc, 1, h, o, o->contact_margin, out);
}

int sim_create_batch(const sim_scene* scenes, int32_t n_scenes, double h,
                     const sim_options* opts, sim_t** out) {
  return create_common(scenes, n_scenes, h, opts, 0.0, out);
}

const silg::MlpDev* silg_mlp_dev(const sim_mlp_t* net, int* device);

int sim_set_warmstart(sim_t* s, const sim_mlp_t* net, int32_t mode) {
  if (!s || mode < 0 || mode > 2 || (mode == 1 && !net)) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  cudaError_t e = cudaStreamSynchronize(s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  if (mode == 1) {
    int dev = -1;
    const silg::MlpDev* m = silg_mlp_dev(net, &dev);
    if (!m || dev != s->device) return SIM_EINVAL;
    // on the frame's stream, finished before returning: the next frame reads the copy and
    // the caller may destroy the network right away
    e = cudaMemcpyAsync(s->d.ws_net.theta, m->theta, sizeof(float) * silg::kMlpParams,
                        cudaMemcpyDeviceToDevice, s->launch);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d.ws_net.w_t, m->w_t, sizeof(__nv_bfloat16) * silg::kWTElems,
                          cudaMemcpyDeviceToDevice, s->launch);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->launch);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->d.ws_net.tc != m->tc) {
      // the network's choice of tensor-core instructions is part of the captured frames
      s->d.ws_net.tc = m->tc;
      for (auto& kv : s->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.g) cudaGraphDestroy(kv.second.g);
      }
      s->graphs.clear();
    }
  }
  s->d.ws_mode = mode;   // graphs are cached per mode; the network's weights are read at launch
  delassus_forget(s, s->launch);
  return SIM_OK;
}

int sim_set_warmstart_gains(sim_t* s, float persist, float fresh, float move, float accept) {
  if (!s || !std::isfinite(persist) || !std::isfinite(fresh) || !std::isfinite(move) ||
      persist < 0.f || fresh < 0.f || move < 0.f || !(accept > 0.f && accept <= 1.f))
    return SIM_EINVAL;
  s->d.ws_gain[0] = persist;   // read at graph capture: the cached graphs are dropped
  s->d.ws_gain[1] = fresh;
  s->d.ws_gain[2] = move;
  s->d.ws_gain[3] = accept;
  silg::DeviceGuard dg(s->device);
  cudaStreamSynchronize(s->launch);
  for (auto& kv : s->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  s->graphs.clear();
  return SIM_OK;
}

int sim_set_phase_marks(sim_t* s, int32_t on) {
  if (!s || (on != 0 && on != 1)) return SIM_EINVAL;
  s->phase_marks = on != 0;   // graphs are cached per setting
  return SIM_OK;
}

int sim_set_portfolio(sim_t* s, int32_t copies) {
  if (!s || copies < 1) return SIM_EINVAL;
  const Plan& p = s->plan;
  if (p.n_scenes % copies) return SIM_EINVAL;
  if (copies > 1) {
    // the copies of a group must be the same scene: same vertex count, rest positions and
    // pins, and the same internal numbering relative to the scene's first free vertex
    std::vector<int> voff(p.n_scenes + 1, p.n_verts);
    for (int v = p.n_verts - 1; v >= 0; --v) voff[p.vertex_scene[v]] = v;
    for (int sc = p.n_scenes - 1; sc >= 0; --sc) voff[sc] = std::min(voff[sc], voff[sc + 1]);
    for (int a = 0; a < p.n_scenes; a += copies)
      for (int b = a + 1; b < a + copies; ++b) {
        if (s->scene_sig[a] != s->scene_sig[b]) return SIM_EINVAL;
        const int nv = voff[a + 1] - voff[a];
        if (voff[b + 1] - voff[b] != nv) return SIM_EINVAL;
        for (int i = 0; i < nv; ++i) {
          const int va = voff[a] + i, vb = voff[b] + i;
          if (p.pinned[va] != p.pinned[vb]) return SIM_EINVAL;
          for (int r = 0; r < 3; ++r)
            if (p.X[3 * (size_t)va + r] != p.X[3 * (size_t)vb + r]) return SIM_EINVAL;
          if (!p.pinned[va] &&
              p.internal[vb] - p.scene_vfirst[b] != p.internal[va] - p.scene_vfirst[a])
            return SIM_EINVAL;
        }
      }
  }
  silg::DeviceGuard dg(s->device);
  cudaError_t e = cudaStreamSynchronize(s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  if (s->d.pf_copies != copies) {
    // kernels capture the device view by value: rebuild the frame graphs
    for (auto& kv : s->graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    s->graphs.clear();
    s->d.pf_copies = copies;
    delassus_forget(s, s->launch);
  }
  return SIM_OK;
}

int sim_get_warmstart_samples(sim_t* s, int32_t capacity, float* X, float* T, int32_t* n_out) {
  if (!s || !n_out || capacity < 0) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  int c = 0;
  if (s->has_obstacles && s->frame > 0)
    cudaMemcpy(&c, s->d.counters + silg::kCntContacts, sizeof(int), cudaMemcpyDeviceToHost);
  c = std::min(c, s->d.cap);
  // anchors are not samples (the warm start does not guess them)
  std::vector<int> obst(std::max(1, c));
  if (c > 0) cudaMemcpy(obst.data(), s->d.ct_obst, sizeof(int) * c, cudaMemcpyDeviceToHost);
  int ns = 0;
  for (int j = 0; j < c; ++j) ns += obst[j] >= 0 && obst[j] < s->d.n_obs;
  *n_out = ns;
  if (ns == 0 || capacity < ns) return st;
  std::vector<float> f((size_t)c * silg::kMlpIn), t(4 * (size_t)c);
  cudaMemcpy(f.data(), s->d.ws_feat, f.size() * sizeof(float), cudaMemcpyDeviceToHost);
  cudaError_t e = cudaMemcpy(t.data(), s->d.ws_target, t.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  int row = 0;
  for (int j = 0; j < c; ++j) {
    if (obst[j] < 0 || obst[j] >= s->d.n_obs) continue;
    if (X)
      for (int q = 0; q < silg::kMlpNF; ++q) X[(size_t)row * silg::kMlpNF + q] = f[(size_t)j * silg::kMlpIn + q];
    if (T)
      for (int q = 0; q < 4; ++q) T[4 * (size_t)row + q] = t[4 * (size_t)j + q];
    ++row;
  }
  return st;
}

int sim_get_tuning(const sim_t* s, sim_tuning* out) {
  if (!s || !out) return SIM_EINVAL;
  *out = s->tuning;
  if (!out->tuned) {
    out->pass1_ctas = s->d.s1_grid;
    out->pass2_ctas = s->d.s2_grid;
    out->pass1_unroll = s->d.s1_unroll;
    out->pass2_unroll = s->d.s2_unroll;
    out->pass1_balance = out->pass2_balance = kDefaultBalance;
  }
  return SIM_OK;
}

int sim_get_scene_residuals(sim_t* s, int32_t capacity, double* out) {
  if (!s || !out || capacity < 0) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  const int K = frame_iters(s), S = s->plan.n_scenes;
  if (K < 0) return SIM_ECUDA;
  std::vector<double> r((size_t)S * (silg::kMaxIters + 1));
  cudaError_t e = cudaMemcpy(r.data(), s->d.resid_scene, r.size() * sizeof(double),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  for (int sc = 0; sc < S; ++sc)
    for (int k = 0; k <= K; ++k) {
      const long long idx = (long long)sc * (K + 1) + k;
      if (idx < capacity) out[idx] = s->has_obstacles ? r[(size_t)sc * (silg::kMaxIters + 1) + k] : 0.0;
    }
  return st;
}

void sim_destroy(sim_t* s) {
  if (!s) return;
  silg::DeviceGuard dg(s->device);
  if (s->launch) cudaStreamSynchronize(s->launch);
  delete s;
}

int sim_step(sim_t* s, int32_t n_iters) {
  if (!s) return SIM_EINVAL;
  // n_iters <= 0 with a residual tolerance: iterate to it (K = 0 selects that graph)
  const bool to_tol = n_iters <= 0 && s->d.res_tol > 0.0;
  int K = to_tol ? 0 : (n_iters > 0 ? n_iters : s->n_iters_default);
  if (K > silg::kMaxIters) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  cudaGraphExec_t exec = nullptr;
  int st = get_graph(s, K, &exec);
  if (st != SIM_OK) return st;
  cudaError_t e = cudaGraphLaunch(exec, s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  s->frame += 1;
  s->last_iters = to_tol ? -1 : K;
  s->last_to_tol = to_tol;
  s->last_marks = s->phase_marks;
  return SIM_OK;
}

int sim_synchronize(sim_t* s) {
  if (!s) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  return sync_and_check(s);
}

int sim_get_state(sim_t* s, double* q, double* v, int32_t capacity, double* lambda,
                  int32_t* n_contacts, sim_stats* stats) {
  if (!s || capacity < 0 || (lambda && capacity == 0)) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  const Plan& p = s->plan;
  const size_t m = 3 * (size_t)p.n_verts;
  // both copies on the frame's stream into page-locked staging, then one wait
  if (q) cudaMemcpyAsync(s->pinned, s->d.q_t, m * sizeof(double), cudaMemcpyDeviceToHost, s->launch);
  if (v) cudaMemcpyAsync(s->pinned + m, s->d.v_t, m * sizeof(double), cudaMemcpyDeviceToHost, s->launch);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  const double* srcs[2] = {s->pinned, s->pinned + m};
  double* dsts[2] = {q, v};
  for (int k = 0; k < 2; ++k) {
    if (!dsts[k]) continue;
    for (int vv = 0; vv < p.n_verts; ++vv) {
      const size_t iv = 3 * (size_t)p.internal[vv];
      for (int r = 0; r < 3; ++r) dsts[k][3 * (size_t)vv + r] = srcs[k][iv + r];
    }
  }
  if (lambda || n_contacts) {
    int32_t c = 0;
    const int sc = sim_get_contacts(s, lambda ? capacity : 0, nullptr, nullptr, lambda, nullptr, &c);
    if (sc == SIM_ECUDA) return sc;
    if (n_contacts) *n_contacts = c;
  }
  if (stats) {
    const int ss = sim_get_stats(s, stats);
    if (ss == SIM_ECUDA) return ss;
  }
  return st;
}

int sim_set_state(sim_t* s, const double* q, const double* v) {
  if (!s || !q || !v) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  // the staging may still feed an earlier copy: wait for the frame's stream first
  cudaError_t e = cudaStreamSynchronize(s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  const Plan& p = s->plan;
  const size_t m = 3 * (size_t)p.n_verts;
  double* bq = s->pinned;
  double* bv = s->pinned + m;
  for (int vv = 0; vv < p.n_verts; ++vv) {
    const size_t iv = 3 * (size_t)p.internal[vv];
    for (int r = 0; r < 3; ++r) {
      const double a = q[3 * (size_t)vv + r], b = v[3 * (size_t)vv + r];
      if (!std::isfinite(a) || !std::isfinite(b)) return SIM_EINVAL;
      bq[iv + r] = a;
      bv[iv + r] = b;
    }
  }
  // in stream order before the next frame; the copies read the staging asynchronously
  cudaMemsetAsync(s->d.prev_valid, 0, sizeof(int) * s->d.n, s->launch);
  delassus_forget(s, s->launch);   // a replayed frame is never served from the previous one
  if (s->d.n_anc > 0)   // time restarts at 0: so do the anchors' targets
    cudaMemcpyAsync(s->d.anc_pos, s->d.anc_pos0, 3 * sizeof(double) * s->d.n_anc,
                    cudaMemcpyDeviceToDevice, s->launch);
  cudaMemcpyAsync(s->d.q_t, bq, m * sizeof(double), cudaMemcpyHostToDevice, s->launch);
  cudaMemcpyAsync(s->d.v_t, bv, m * sizeof(double), cudaMemcpyHostToDevice, s->launch);
  cudaMemsetAsync(s->d.err, 0, sizeof(int), s->launch);
  e = cudaGetLastError();
  s->frame = 0;
  return cuda_status(e);
}

namespace {
// A checkpoint: this header, then q_t and v_t (3 n_all doubles each, internal order), the
// anchors' current targets (3 n_anc doubles), and the previous-frame contact record the warm
// starts read (per free vertex: contact flag and obstacle as int32, the impulse D^T lambda in
// world coordinates as 3 doubles, the move along the normal as a double).
struct CheckpointHeader {
  uint64_t magic;        // "SILGCKP1"
  uint64_t signature;    // hash of every scene's inputs: a checkpoint fits its simulator only
  int64_t frame;
  int32_t n_all, n, n_anc, version;
};
constexpr uint64_t kCkptMagic = 0x31504b43474c4953ull;

uint64_t checkpoint_signature(const sim_s* s) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)s->scene_sig.size();
  for (uint64_t x : s->scene_sig) h = (h ^ x) * 1099511628211ull;
  return h;
}

size_t checkpoint_bytes(const sim_s* s) {
  const size_t na = (size_t)s->d.n_all, n = (size_t)s->d.n, nanc = (size_t)s->d.n_anc;
  return sizeof(CheckpointHeader) + sizeof(double) * (6 * na + 3 * nanc + 4 * n) +
         sizeof(int32_t) * 2 * n;
}

// the device arrays of a checkpoint in their order: pointer and bytes
std::vector<std::pair<void*, size_t>> checkpoint_parts(sim_s* s) {
  const size_t na = (size_t)s->d.n_all, n = (size_t)s->d.n, nanc = (size_t)s->d.n_anc;
  return {{s->d.q_t, sizeof(double) * 3 * na},
          {s->d.v_t, sizeof(double) * 3 * na},
          {s->d.anc_pos, sizeof(double) * 3 * nanc},
          {s->d.prev_valid, sizeof(int32_t) * n},
          {s->d.prev_obst, sizeof(int32_t) * n},
          {s->d.prev_force, sizeof(double) * 3 * n},
          {s->d.prev_move, sizeof(double) * n}};
}
}  // namespace

int sim_get_checkpoint(sim_t* s, void* buf, size_t capacity, size_t* bytes) {
  if (!s || (!buf && !bytes)) return SIM_EINVAL;
  const size_t need = checkpoint_bytes(s);
  if (bytes) *bytes = need;
  if (!buf) return SIM_OK;
  if (capacity < need) return SIM_ECAPACITY;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  CheckpointHeader hd{kCkptMagic, checkpoint_signature(s), s->frame, s->d.n_all, s->d.n,
                      s->d.n_anc, 1};
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  cudaError_t e = cudaSuccess;
  for (auto& part : checkpoint_parts(s)) {
    if (part.second && e == cudaSuccess)
      e = cudaMemcpyAsync(out + off, part.first, part.second, cudaMemcpyDeviceToHost, s->launch);
    off += part.second;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->launch);
  return e != cudaSuccess ? cuda_status(e) : st;
}

int sim_set_checkpoint(sim_t* s, const void* buf, size_t bytes) {
  if (!s || !buf) return SIM_EINVAL;
  CheckpointHeader hd;
  if (bytes != checkpoint_bytes(s)) return SIM_EINVAL;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kCkptMagic || hd.version != 1 || hd.signature != checkpoint_signature(s) ||
      hd.n_all != s->d.n_all || hd.n != s->d.n || hd.n_anc != s->d.n_anc || hd.frame < 0)
    return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  cudaError_t e = cudaStreamSynchronize(s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(hd);
  for (auto& part : checkpoint_parts(s)) {
    if (part.second && e == cudaSuccess)
      e = cudaMemcpyAsync(part.first, in + off, part.second, cudaMemcpyHostToDevice, s->launch);
    off += part.second;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.err, 0, sizeof(int), s->launch);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d.dl_state + 1, 0xff, sizeof(int), s->launch);
  // the caller's buffer is read before returning
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->launch);
  if (e != cudaSuccess) return cuda_status(e);
  s->frame = hd.frame;
  return SIM_OK;
}

int sim_load_warmstart(sim_t* s, const void* weights, size_t bytes) {
  if (!s || !weights || bytes != sizeof(float) * SIM_MLP_PARAMS) return SIM_EINVAL;
  std::vector<float> theta(SIM_MLP_PARAMS);
  std::memcpy(theta.data(), weights, bytes);
  for (float x : theta)
    if (!std::isfinite(x)) return SIM_EINVAL;
  sim_mlp_t* net = nullptr;
  int st = sim_mlp_create(s->device, 1, &net);
  if (st != SIM_OK) return st;
  st = sim_mlp_set_params(net, theta.data());
  if (st == SIM_OK) st = sim_set_warmstart(s, net, 1);
  sim_mlp_destroy(net);
  return st;
}

int sim_get_stats(sim_t* s, sim_stats* out) {
  if (!s || !out) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  if (frame_iters(s) < 0) return SIM_ECUDA;
  std::memset(out, 0, sizeof(*out));
  int cnt[silg::kNumCounters];
  double res[silg::kMaxIters + 1];
  cudaMemcpy(cnt, s->d.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  cudaMemcpy(res, s->d.resid, sizeof(res), cudaMemcpyDeviceToHost);
  cudaMemcpy(&out->max_penetration, s->d.max_pen, sizeof(double), cudaMemcpyDeviceToHost);
  out->frame = s->frame;
  out->n_contacts = s->has_obstacles ? cnt[silg::kCntContacts] : 0;
  out->n_contact_verts = s->has_obstacles ? cnt[silg::kCntCv] : 0;
  out->n_iters = s->last_iters;
  out->n_residuals = s->has_obstacles && s->frame > 0 ? s->last_iters + 1 : 0;
  for (int k = 0; k < out->n_residuals; ++k) out->residual[k] = res[k];
  if (s->has_obstacles && s->frame > 0) {
    int dl[3] = {0, 0, 0};
    cudaMemcpy(dl, s->d.dl_state, sizeof(dl), cudaMemcpyDeviceToHost);
    out->delassus_reused = dl[0];
    out->delassus_reuse_frames = dl[2];
  }
  out->kernels_per_frame = s->last_to_tol ? kernels_per_frame_to_tolerance(s, s->last_iters)
                                          : kernels_per_frame(s, s->last_iters > 0 ? s->last_iters
                                                                                   : s->n_iters_default);
  return st;
}

int sim_get_phase_times(sim_t* s, double* ms) {
  if (!s || !ms) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  for (int k = 0; k < SIM_NUM_PHASES; ++k) ms[k] = 0.0;
  if (s->frame == 0 || s->last_iters == 0) return SIM_OK;
  auto el = [&](int a, int b) {
    float t = 0.f;
    cudaEventElapsedTime(&t, s->ev[a], s->ev[b]);
    return (double)t;
  };
  if (s->last_to_tol || !s->last_marks) {
    cudaError_t e = cudaEventSynchronize(s->ev[5]);
    if (e != cudaSuccess) return cuda_status(e);
    ms[SIM_PHASE_COLLIDE] = el(0, 1);
    ms[SIM_PHASE_DELASSUS] = el(1, 2);
    ms[SIM_PHASE_WARMSTART] = el(2, 3);
    ms[SIM_PHASE_ITERATIONS] = el(3, 4);
    ms[SIM_PHASE_INTEGRATE] = el(4, 5);
    return SIM_OK;
  }
  const int K = s->last_iters;
  cudaError_t e = cudaEventSynchronize(s->ev[4 + kMarksPerIter * K]);
  if (e != cudaSuccess) return cuda_status(e);
  ms[SIM_PHASE_COLLIDE] = el(0, 1);
  ms[SIM_PHASE_DELASSUS] = el(1, 2);
  ms[SIM_PHASE_WARMSTART] = el(2, 3);
  for (int k = 0; k < K; ++k) {
    const int b = 4 + kMarksPerIter * k;
    ms[SIM_PHASE_LOCAL] += el(b - 1, b);
    ms[SIM_PHASE_ASSEMBLE] += el(b, b + 1);
    ms[SIM_PHASE_SPMV1] += el(b + 1, b + 2);
    ms[SIM_PHASE_REDUCE] += el(b + 2, b + 3) + el(b + 5, b + 6);
    ms[SIM_PHASE_SOLVE] += el(b + 3, b + 4);
    ms[SIM_PHASE_SPMV2] += el(b + 4, b + 5);
  }
  ms[SIM_PHASE_INTEGRATE] = el(4 + kMarksPerIter * K - 1, 4 + kMarksPerIter * K);
  return SIM_OK;
}

int sim_get_contacts(sim_t* s, int32_t capacity, int32_t* vertex, int32_t* obstacle,
                     double* lambda, double* frame, int32_t* n_out) {
  if (!s || !n_out || capacity < 0) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  int c = 0;
  if (s->has_obstacles) cudaMemcpy(&c, s->d.counters + silg::kCntContacts, sizeof(int), cudaMemcpyDeviceToHost);
  c = std::min(c, s->d.cap);
  *n_out = c;
  if (capacity == 0 || c == 0) return st;
  std::vector<int> cv(c), co(c);
  std::vector<double> cl(3 * (size_t)c), cD(9 * (size_t)c);
  cudaMemcpy(cv.data(), s->d.ct_vert, sizeof(int) * c, cudaMemcpyDeviceToHost);
  cudaMemcpy(co.data(), s->d.ct_obst, sizeof(int) * c, cudaMemcpyDeviceToHost);
  // a contact with another body: its id follows the obstacles' and the anchors'
  for (int& o : co)
    if (o < 0) o = s->d.n_obs + s->d.n_anc + (-1 - o);
  cudaMemcpy(cl.data(), s->d.ct_lam, sizeof(double) * 3 * c, cudaMemcpyDeviceToHost);
  cudaMemcpy(cD.data(), s->d.ct_D, sizeof(double) * 9 * c, cudaMemcpyDeviceToHost);
  std::vector<int> perm(c);
  std::iota(perm.begin(), perm.end(), 0);
  const Plan& p = s->plan;
  std::sort(perm.begin(), perm.end(), [&](int a, int b) {
    int va = p.order[cv[a]], vb = p.order[cv[b]];
    return va < vb || (va == vb && co[a] < co[b]);
  });
  for (int k = 0; k < std::min(c, (int)capacity); ++k) {
    int j = perm[k];
    if (vertex) vertex[k] = p.order[cv[j]];
    if (obstacle) obstacle[k] = co[j];
    if (lambda)
      for (int r = 0; r < 3; ++r) lambda[3 * k + r] = cl[3 * j + r];
    if (frame)
      for (int r = 0; r < 9; ++r) frame[9 * k + r] = cD[9 * j + r];
  }
  return st;
}

int sim_apply_inverse(sim_t* s, const double* b, double* x) {
  if (!s || !b || !x) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  const Plan& p = s->plan;
  const int n = p.n_free, np = p.n_pad;
  std::vector<float> g(3 * (size_t)np, 0.f);
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < 3; ++r) g[(size_t)r * np + k] = (float)b[3 * (size_t)p.order[k] + r];
  cudaStreamSynchronize(s->launch);
  int bits0 = 0;
  if (cudaMemcpy(&bits0, s->d.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SIM_ECUDA;
  cudaMemcpyAsync(s->d.gvec, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, s->work);
  silg::launch_solve(s->d, s->work, silg::kOutX);
  if (s->d.s_bf16 && s->d.refine > 0) {
    // x += S~^T S~ (b - A~ x), the residual summed in FP64
    cudaMemcpyAsync(s->d.gsave, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, s->work);
    silg::launch_residual(s->d, s->work, silg::kResApply);
    DevSim dr = s->d;
    dr.gvec = s->d.gsave;
    silg::launch_solve(dr, s->work, silg::kOutAddX);
  }
  std::vector<float> xo(3 * (size_t)n);
  cudaMemcpyAsync(xo.data(), s->d.xout, xo.size() * sizeof(float), cudaMemcpyDeviceToHost, s->work);
  cudaError_t e = cudaStreamSynchronize(s->work);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  // a wait of the products that ran out (their bulk-copy form) is this call's error; the
  // bits a frame left for its own report are kept
  int bits = 0;
  if (cudaMemcpy(&bits, s->d.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SIM_ECUDA;
  if ((bits & silg::kErrTimeout) && !(bits0 & silg::kErrTimeout)) {
    const int keep = bits0;
    cudaMemcpy(s->d.err, &keep, sizeof(int), cudaMemcpyHostToDevice);
    return SIM_ETIMEOUT;
  }
  std::memset(x, 0, sizeof(double) * 3 * (size_t)p.n_verts);
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < 3; ++r) x[3 * (size_t)p.order[k] + r] = xo[3 * (size_t)k + r];
  return SIM_OK;
}

int sim_local_project(sim_t* s, const double* q, double* pout) {
  if (!s || !q || !pout) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  const Plan& p = s->plan;
  const int n_all = p.n_verts, T = p.n_tets;
  std::vector<double> qi(3 * (size_t)n_all);
  for (int v = 0; v < n_all; ++v)
    for (int r = 0; r < 3; ++r) qi[3 * (size_t)p.internal[v] + r] = q[3 * (size_t)v + r];
  cudaStreamSynchronize(s->launch);
  cudaMemcpyAsync(s->d.q_ref, qi.data(), qi.size() * sizeof(double), cudaMemcpyHostToDevice, s->work);
  cudaMemsetAsync(s->d.dq, 0, sizeof(float) * 3 * (size_t)n_all, s->work);
  silg::launch_local(s->d, s->work, true);
  std::vector<float> po(9 * (size_t)T);
  cudaMemcpyAsync(po.data(), s->d.p_out, po.size() * sizeof(float), cudaMemcpyDeviceToHost, s->work);
  cudaError_t e = cudaStreamSynchronize(s->work);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  for (size_t k = 0; k < po.size(); ++k) pout[k] = po[k];
  return SIM_OK;
}

int sim_get_delassus(sim_t* s, int32_t capacity, double* Wt, int32_t* cv_vertex, int32_t* n_out) {
  if (!s || !n_out || capacity < 0) return SIM_EINVAL;
  silg::DeviceGuard dg(s->device);
  int st = sync_and_check(s);
  if (st == SIM_ECUDA) return st;
  int m = 0;
  if (s->has_obstacles) cudaMemcpy(&m, s->d.counters + silg::kCntCv, sizeof(int), cudaMemcpyDeviceToHost);
  m = std::min(m, s->d.cap);
  *n_out = m;
  if (capacity < m || m == 0) return st;
  // one block per scene (block-diagonal W~): blocks at sc_wtoff with leading dimension sc_ld
  const int S = s->plan.n_scenes;
  std::vector<int> cvb(S + 1), ldv(S);
  std::vector<long long> off(S + 1);
  cudaMemcpy(cvb.data(), s->d.sc_cvb, sizeof(int) * (S + 1), cudaMemcpyDeviceToHost);
  cudaMemcpy(ldv.data(), s->d.sc_ld, sizeof(int) * S, cudaMemcpyDeviceToHost);
  cudaMemcpy(off.data(), s->d.sc_wtoff, sizeof(long long) * (S + 1), cudaMemcpyDeviceToHost);
  std::vector<float> w((size_t)std::max(0LL, off[S]));
  std::vector<int> cv(m), scene_of(m, 0);
  if (!w.empty()) cudaMemcpy(w.data(), s->d.wt, w.size() * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(cv.data(), s->d.cv_vert, sizeof(int) * m, cudaMemcpyDeviceToHost);
  for (int sc = 0; sc < S; ++sc)
    for (int a = cvb[sc]; a < std::min(cvb[sc + 1], m); ++a) scene_of[a] = sc;
  auto entry = [&](int a, int b) -> double {
    const int sa = scene_of[a];
    if (scene_of[b] != sa) return 0.0;
    return w[off[sa] + (size_t)(a - cvb[sa]) * ldv[sa] + (b - cvb[sa])];
  };
  const Plan& p = s->plan;
  std::vector<int> perm(m);
  std::iota(perm.begin(), perm.end(), 0);
  std::sort(perm.begin(), perm.end(), [&](int a, int b) { return p.order[cv[a]] < p.order[cv[b]]; });
  for (int a = 0; a < m; ++a) {
    if (cv_vertex) cv_vertex[a] = p.order[cv[perm[a]]];
    if (Wt)
      for (int b = 0; b < m; ++b) Wt[(size_t)a * m + b] = entry(perm[a], perm[b]);
  }
  return st;
}

}  // extern "C"

// Launch-boundary measurement (a diagnostic of the frame's structure, not part of the method):
// the device time per phase boundary of a chain of phases run (a) as one kernel per phase in a
// CUDA graph with programmatic dependent launch, the form of the frame graph, and (b) as one
// cooperative kernel that separates the phases with a software grid barrier, the form a
// persistent kernel per iteration would take. Every phase does the same small amount of work
// per CTA (a read-modify-write of one value per thread), so the difference per boundary is
// the cost of the boundary itself.
//
// The barrier is a sense-reversing counter in global memory; its wait is bounded (a spin
// limit), after which the kernel records a timeout and returns, so it cannot hang.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "devguard.hpp"
#include "silg.h"

namespace {

constexpr int kDiagThreads = 256;
constexpr unsigned long long kDiagSpin = 1ull << 24;

__device__ __forceinline__ void pdl_wait_diag() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// one phase: every thread updates its own value
__global__ void k_phase(float* buf, int phase) {
  pdl_wait_diag();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  buf[i] = buf[i] * 0.5f + (float)phase;
}

// all phases in one kernel; bar[0]: arrivals, bar[1]: generation, bar[2]: timeout flag
__global__ void k_phases_barrier(float* buf, int n_phases, unsigned* bar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nblocks = gridDim.x;
  for (int phase = 0; phase < n_phases; ++phase) {
    buf[i] = buf[i] * 0.5f + (float)phase;
    if (phase + 1 == n_phases) break;
    __syncthreads();
    if (threadIdx.x == 0) {
      volatile unsigned* gen = bar + 1;
      const unsigned g = *gen;
      __threadfence();
      if (atomicAdd(bar, 1u) == nblocks - 1) {
        bar[0] = 0;
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        unsigned long long spins = 0;
        while (*gen == g) {
          if (++spins > kDiagSpin) {
            atomicExch(bar + 2, 1u);
            break;
          }
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (*(volatile unsigned*)(bar + 2)) return;
  }
}

}  // namespace

extern "C" int sim_measure_phase_boundaries(int32_t device, int32_t n_phases,
                                            int32_t ctas_per_sm, double* graph_us,
                                            double* barrier_us) {
  if (n_phases < 2 || n_phases > 4096 || ctas_per_sm < 1 || ctas_per_sm > 8 || !graph_us ||
      !barrier_us)
    return SIM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SIM_EINVAL;
  silg::DeviceGuard dg(device);
  int n_sm = 0, coop = 0, occ = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (!coop) return SIM_ENOTSUP;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_phases_barrier, kDiagThreads, 0) !=
          cudaSuccess ||
      occ < ctas_per_sm)
    return SIM_ENOTSUP;
  const int grid = n_sm * ctas_per_sm;
  float* buf = nullptr;
  unsigned* bar = nullptr;
  cudaStream_t s = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = SIM_ECUDA;
  auto cleanup = [&]() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (buf) cudaFree(buf);
    if (bar) cudaFree(bar);
  };
  if (cudaMalloc(&buf, sizeof(float) * grid * kDiagThreads) != cudaSuccess ||
      cudaMalloc(&bar, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return SIM_ECUDA;
  }
  cudaMemsetAsync(buf, 0, sizeof(float) * grid * kDiagThreads, s);
  cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s);
  // (a) one kernel per phase, captured into a graph with programmatic dependent launch
  cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  for (int p = 0; p < n_phases; ++p) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kDiagThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = p > 0 ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_phase, buf, p);
  }
  if (cudaStreamEndCapture(s, &g) != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
    cleanup();
    return SIM_ECUDA;
  }
  const int reps = 20;
  float ms = 0.f;
  std::vector<float> t_graph, t_bar;
  for (int r = 0; r < reps + 3; ++r) {
    cudaEventRecord(e0, s);
    cudaGraphLaunch(ge, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cleanup();
      return SIM_ECUDA;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 3) t_graph.push_back(ms);
  }
  // (b) one cooperative kernel, phases separated by the grid barrier
  for (int r = 0; r < reps + 3; ++r) {
    void* args[] = {&buf, &n_phases, &bar};
    cudaEventRecord(e0, s);
    if (cudaLaunchCooperativeKernel((const void*)k_phases_barrier, dim3(grid), dim3(kDiagThreads),
                                    args, 0, s) != cudaSuccess) {
      cleanup();
      return SIM_ECUDA;
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cleanup();
      return SIM_ECUDA;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 3) t_bar.push_back(ms);
  }
  unsigned flags[4] = {0, 0, 0, 0};
  cudaMemcpy(flags, bar, sizeof(flags), cudaMemcpyDeviceToHost);
  std::sort(t_graph.begin(), t_graph.end());
  std::sort(t_bar.begin(), t_bar.end());
  // median per boundary (n_phases - 1 boundaries), microseconds
  *graph_us = 1e3 * t_graph[t_graph.size() / 2] / (n_phases - 1);
  *barrier_us = 1e3 * t_bar[t_bar.size() / 2] / (n_phases - 1);
  status = flags[2] ? SIM_ETIMEOUT : SIM_OK;
  cleanup();
  return status;
}

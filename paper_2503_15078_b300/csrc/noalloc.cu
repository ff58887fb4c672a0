// Global solve x = S~^T (S~ g) that allocates nothing: its scratch lives in a file-scope
// device array instead of memory obtained from the CUDA allocator.
//
// Some callers cannot allocate device memory when they need the solve: real-time loops
// that forbid cudaMalloc because it can synchronise the device and has unbounded latency,
// code that runs while another component is capturing the stream into a CUDA graph, and
// embedders whose device memory is entirely handed out by their own pool. This variant
// runs the same kernels as the simulator's global step, with every intermediate (the
// padded copy of g, the per-item partial sums of both products, z = S~ g) placed in
// g_noalloc_scratch.
#include <cuda_runtime.h>

#include "device.cuh"
#include "silg.h"

const silg::DevSim* silg_sim_devsim(const sim_t* sim, int* device);

namespace {

// 16 MiB of scratch on every device that loads the library, held until the process exits.
constexpr size_t kNoAllocFloats = size_t(4) << 20;
__device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

// Device address of g_noalloc_scratch per device ordinal, looked up on first use. In host
// code the symbol itself names a host-side stand-in, never the device memory.
constexpr int kMaxDevices = 128;
float* g_scratch_addr[kMaxDevices] = {};

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// g (n x 3 row-major) -> SoA of three n_pad vectors, zero padded
__global__ void k_rows_to_soa(const float* g, float* gs, int n, int n_pad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
#pragma unroll
  for (int r = 0; r < 3; ++r) gs[r * n_pad + i] = i < n ? g[3 * i + r] : 0.f;
}

// Runs the solve with `dev` current; the caller restores its own device afterwards.
int solve_on_device(silg::DevSim d, int dev, const float* g, float* x, cudaStream_t s) {
  if (cudaSetDevice(dev) != cudaSuccess) return SIM_ECUDA;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SIM_ECUDA;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  const size_t n_vec = align_up(3 * (size_t)d.n_pad, 64);
  const size_t n_p1 = align_up((size_t)d.n_seg1 * 3 * silg::kRowGroup, 64);
  float* base = g_scratch_addr[dev];
  d.gvec = base;
  d.zvec = base + n_vec;
  d.p1_part = base + 2 * n_vec;
  d.p2_part = base + 2 * n_vec + n_p1;
  d.xout = x;
  // an error left pending by an earlier launch of this library on this thread is not this
  // call's: clear it so that the checks below see only the launches made here (a sticky
  // device error persists and fails them)
  (void)cudaGetLastError();
  k_rows_to_soa<<<(d.n_pad + 255) / 256, 256, 0, s>>>(g, d.gvec, d.n, d.n_pad);
  if (cudaGetLastError() != cudaSuccess) return SIM_ECUDA;
  silg::launch_solve(d, s, silg::kOutX);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

}  // namespace

extern "C" int sim_apply_inverse_noalloc(const sim_t* sim, const float* g, float* x, void* stream) {
  if (!sim || !g || !x) return SIM_EINVAL;
  int dev = 0;
  const silg::DevSim* src = silg_sim_devsim(sim, &dev);
  if (!src || dev < 0 || dev >= kMaxDevices) return SIM_EINVAL;
  silg::DevSim d = *src;
  d.s_bf16 = 0;  // always the FP32 profile (kept on the device in either precision mode)
  const size_t n_vec = align_up(3 * (size_t)d.n_pad, 64);
  const size_t n_p1 = align_up((size_t)d.n_seg1 * 3 * silg::kRowGroup, 64);
  const size_t n_p2 = align_up((size_t)d.n_seg2 * 3 * silg::kTileW, 64);
  if (2 * n_vec + n_p1 + n_p2 > kNoAllocFloats) return SIM_ECAPACITY;
  int caller_dev = -1;
  if (cudaGetDevice(&caller_dev) != cudaSuccess) return SIM_ECUDA;
  const int status = solve_on_device(d, dev, g, x, static_cast<cudaStream_t>(stream));
  // the caller's current device is left as it was
  if (caller_dev != dev && cudaSetDevice(caller_dev) != cudaSuccess && status == SIM_OK)
    return SIM_ECUDA;
  return status;
}

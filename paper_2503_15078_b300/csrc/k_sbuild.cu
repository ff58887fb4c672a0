// The sparse inverse S~ = L~^-1 P built on the device in FP64 (Sec. 4.2, Theorem 1; the
// one-time first line of Alg. 4), from the host's Cholesky factor L~.
//
// Column j of L~^-1 solves L~ x = e_j. By Theorem 1 it is non-zero only on j and its
// elimination-tree ancestors, and column a of L~ is non-zero only on a's ancestors, so the
// forward substitution walks the path j = a_0, a_1 = parent(a_0), ... to the root: at step
// p, x(a_p) /= L(a_p, a_p), then x(k) -= L(k, a_p) x(a_p) for the entries k of column a_p.
// An ancestor k of a_p sits at path position p + depth(a_p) - depth(k), so the path vector
// is a dense array of depth(j) values.
//
// One warp per column, columns taken from a global counter; the warp's path vector lives in
// shared memory; at step p the lanes share the entries of column a_p (one update each, to
// distinct positions), and lane 0 stores x(a_p), final at that step, into row a_p of the
// profile (FP32, rounded to nearest; BF16 rounded to nearest even from that FP32 value).
// The products and differences are rounded separately (no fused multiply-add), in the
// order of the host's loop, so the FP64 values equal the host build bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device.cuh"

namespace silg {
namespace {

constexpr int kSbWarps = 16;

__global__ void __launch_bounds__(32 * kSbWarps) k_sinv_build(
    int nf, const long long* Lp, const int* Ldd, const double* Lx, const int* parent,
    const int* depth, const long long* rowbase, const int* lo, int max_depth, int* next_col,
    float* S, unsigned short* Sb) {
  extern __shared__ double xs[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* x = xs + (size_t)w * max_depth;
  for (;;) {
    int j = 0;
    if (lane == 0) j = atomicAdd(next_col, 1);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= nf) return;
    const int len = depth[j];          // the path j .. root (the root has depth 1)
    for (int p = lane; p < len; p += 32) x[p] = p == 0 ? 1.0 : 0.0;
    __syncwarp();
    int a = j;
    for (int p = 0; p < len; ++p) {
      const long long c0 = Lp[a], c1 = Lp[a + 1];
      const double xa = x[p] / Lx[c0];   // every lane: x[p] is final at this step
      for (long long q = c0 + 1 + lane; q < c1; q += 32) {
        const int pos = p + Ldd[q];
        x[pos] = __dsub_rn(x[pos], __dmul_rn(Lx[q], xa));
      }
      if (lane == 0) {
        const long long at = rowbase[a] + (j - lo[a]);
        const float f = __double2float_rn(xa);
        S[at] = f;
        if (Sb) {
          unsigned u = __float_as_uint(f);
          u += 0x7fffu + ((u >> 16) & 1u);
          Sb[at] = (unsigned short)(u >> 16);
        }
      }
      a = parent[a];
      __syncwarp();
    }
  }
}

}  // namespace

size_t sinv_build_smem(int max_depth) { return sizeof(double) * (size_t)kSbWarps * max_depth; }

bool sinv_build_fits(int max_depth) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return max_depth > 0 && sinv_build_smem(max_depth) <= (size_t)optin;
}

int launch_sinv_build(const SinvBuildArgs& a, cudaStream_t s) {
  const size_t smem = sinv_build_smem(a.max_depth);
  if (cudaFuncSetAttribute(k_sinv_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return SIM_ECUDA;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemsetAsync(a.next_col, 0, sizeof(int), s) != cudaSuccess) return SIM_ECUDA;
  k_sinv_build<<<n_sm, 32 * kSbWarps, smem, s>>>(a.nf, a.Lp, a.Ldd, a.Lx, a.parent, a.depth,
                                                  a.rowbase, a.lo, a.max_depth, a.next_col,
                                                  a.S, a.Sb);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

// depth(a) - depth(row) of every below-diagonal entry of column a of L~ (0 on the diagonal)
void sinv_build_depth_steps(const Plan& p, std::vector<int>* ldd) {
  ldd->assign(p.Li.size(), 0);
  for (int a = 0; a < p.n_free; ++a)
    for (int64_t q = p.Lp[a] + 1; q < p.Lp[a + 1]; ++q)
      (*ldd)[q] = p.depth[a] - p.depth[p.Li[q]];
}

}  // namespace silg

// Inference of the warm-start network on the 5th-generation tensor cores (tcgen05): BF16
// operands in shared memory, FP32 accumulators in tensor memory (TMEM), one CTA of 128
// threads per 128 rows (samples).
//
// Each layer is D (128 x N, FP32, TMEM) = A (128 x K, BF16) B^T with B (N x K, BF16) the
// layer's transposed weights, issued by one thread as K / 16 tcgen05.mma instructions
// (kind::f16, M = 128, N = 128 or 16) and committed to an mbarrier; the four warps then read
// their 32 rows of D (tcgen05.ld, 32 lanes x 32 columns per instruction), add the bias,
// apply GELU, and write the BF16 activations as the next layer's A operand.
//
// Operand layout (K-major, no swizzle): the tensor core reads 8 x 8 BF16 "core matrices",
// each 8 rows of 16 contiguous bytes; element (r, k) of an R x K tile sits at element
// (r % 8) * 8 + (r / 8) * 8K + (k / 8) * 64 + k % 8, so the core matrices adjacent in K are
// 128 bytes apart (the descriptor's leading byte offset) and the 8-row groups 16K bytes apart
// (its stride byte offset). An MMA over columns 16s .. 16s + 15 starts 256 s bytes in.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp.cuh"

namespace silg {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcRows = 128;
constexpr unsigned long long kTcSpin = 1ull << 22;

// element offsets of the operand tiles in shared memory (canonical layout)
constexpr int kW1 = 0;                       // 128 x 16
constexpr int kW2 = kW1 + kMlpH * kMlpIn;    // 128 x 128
constexpr int kW3 = kW2 + kMlpH * kMlpH;     // 128 x 128
constexpr int kW4 = kW3 + kMlpH * kMlpH;     // 16 x 128 (rows 8..15 zero)
constexpr int kXa = kW4 + 16 * kMlpH;        // 128 x 16
constexpr int kH0 = kXa + kTcRows * kMlpIn;  // 128 x 128
constexpr int kH1 = kH0 + kTcRows * kMlpH;   // 128 x 128
constexpr int kTcElems = kH1 + kTcRows * kMlpH;
constexpr int kTcBias = 3 * kMlpH + kMlpOut;
constexpr size_t kTcSmem = sizeof(bf16) * kTcElems + sizeof(float) * kTcBias;

__device__ __forceinline__ int canon(int r, int k, int K) {
  return (r & 7) * 8 + (r >> 3) * (K * 8) + (k >> 3) * 64 + (k & 7);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle, canonical core-matrix layout of a
// tile with K columns starting at p
__device__ __forceinline__ uint64_t smem_desc(const bf16* p, int K) {
  const uint64_t a = smem_addr(p);
  uint64_t d = (a >> 4) & 0x3FFFull;                              // start address / 16
  d |= ((uint64_t)(128 >> 4) & 0x3FFFull) << 16;                  // leading byte offset / 16
  d |= ((uint64_t)((K / 8) * 128 >> 4) & 0x3FFFull) << 32;        // stride byte offset / 16
  d |= 1ull << 46;                                                // descriptor version
  return d;                                                       // base offset 0, no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_issue(unsigned tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          int accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool wait_phase(unsigned bar, unsigned parity) {
  for (unsigned long long i = 0; i < kTcSpin; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu_tc(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// a transposed weight matrix w_t (rows n of ld elements, K used) -> canonical tile of N rows
__device__ __forceinline__ void load_weights(bf16* dst, const bf16* src, int N, int n_src, int K,
                                             int ld) {
  for (int e = threadIdx.x; e < N * (K / 8); e += blockDim.x) {
    const int n = e / (K / 8), k8 = e % (K / 8);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < n_src) v = *reinterpret_cast<const uint4*>(src + (size_t)n * ld + 8 * k8);
    *reinterpret_cast<uint4*>(dst + canon(n, 8 * k8, K)) = v;
  }
}

// n_dev (optional): the row count on the device, at most n; m.err (optional) gets
// kMlpErrTimeout if a wait for the tensor cores gave up (the rows are then not written)
__global__ void __launch_bounds__(128) k_mlp_infer_tc(MlpDev m, const float* X, int n,
                                                      const int* n_dev, float* Y) {
  if (n_dev) n = min(n, *n_dev);
  if (blockIdx.x * kTcRows >= n) return;   // the whole CTA leaves together
  extern __shared__ __align__(128) unsigned char smem[];
  bf16* s = reinterpret_cast<bf16*>(smem);
  float* bias = reinterpret_cast<float*>(s + kTcElems);
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     smem_addr(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operands: weights and this CTA's rows of X in the canonical layout, biases
  // the transposed copies w_t hold W1^T (rows of kLdIn), W2^T, W3^T and W4^T (rows of kLdH)
  const bf16* t1 = m.w_t;
  const bf16* t2 = t1 + kMlpH * kLdIn;
  const bf16* t3 = t2 + kMlpH * kLdH;
  const bf16* t4 = t3 + kMlpH * kLdH;
  load_weights(s + kW1, t1, kMlpH, kMlpH, kMlpIn, kLdIn);
  load_weights(s + kW2, t2, kMlpH, kMlpH, kMlpH, kLdH);
  load_weights(s + kW3, t3, kMlpH, kMlpH, kMlpH, kLdH);
  load_weights(s + kW4, t4, 16, kMlpOut, kMlpH, kLdH);
  for (int e = threadIdx.x; e < kTcBias; e += blockDim.x) {
    const int l = e / kMlpH, c = e % kMlpH;
    const int off = l == 0 ? kOffB1 : l == 1 ? kOffB2 : l == 2 ? kOffB3 : kOffB4;
    bias[e] = m.theta[off + c];
  }
  const int row = threadIdx.x, grow = blockIdx.x * kTcRows + row;
  {
    float x[kMlpIn];
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) x[c] = grow < n ? X[(size_t)grow * kMlpIn + c] : 0.f;
#pragma unroll
    for (int k8 = 0; k8 < kMlpIn / 8; ++k8) {
      uint4 v;
      v.x = pack_bf16(x[8 * k8], x[8 * k8 + 1]);
      v.y = pack_bf16(x[8 * k8 + 2], x[8 * k8 + 3]);
      v.z = pack_bf16(x[8 * k8 + 4], x[8 * k8 + 5]);
      v.w = pack_bf16(x[8 * k8 + 6], x[8 * k8 + 7]);
      *reinterpret_cast<uint4*>(s + kXa + canon(row, 8 * k8, kMlpIn)) = v;
    }
  }
  // the operands written by the threads become visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  const unsigned tl = tmem + ((unsigned)(32 * warp) << 16);   // this warp's lane quarter
  bool ok = true;
  const int a_off[4] = {kXa, kH0, kH1, kH0};
  const int b_off[4] = {kW1, kW2, kW3, kW4};
  const int out_off[3] = {kH0, kH1, kH0};
  for (int layer = 0; layer < 4; ++layer) {
    const int K = layer == 0 ? kMlpIn : kMlpH, N = layer == 3 ? 16 : kMlpH;
    if (threadIdx.x == 0 && ok) {
      const uint32_t idesc = instr_desc(kTcRows, N);
      for (int ks = 0; ks < K / 16; ++ks)
        mma_issue(tmem, smem_desc(s + a_off[layer] + 128 * ks, K),
                  smem_desc(s + b_off[layer] + 128 * ks, K), idesc, ks > 0);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar))
          : "memory");
    }
    // every thread waits; the CTA continues only if all of them saw the phase complete (the
    // TMEM loads below are warp-collective)
    const bool got = ok && wait_phase(smem_addr(&mbar), (unsigned)(layer & 1));
    const bool issued = ok;
    ok = __syncthreads_and(got) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok && issued) {
      // the tensor cores may still be writing TMEM: one more bounded wait before it is freed
      wait_phase(smem_addr(&mbar), (unsigned)(layer & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok && layer < 3) {
      bf16* out = s + out_off[layer];
      const float* b = bias + layer * kMlpH;
#pragma unroll 1
      for (int c = 0; c < kMlpH / 32; ++c) {
        float v[32];
        tmem_ld32(tl + 32 * c, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int k = 32 * c + 8 * g;
          float h[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) h[i] = gelu_tc(v[8 * g + i] + b[k + i]);
          uint4 w;
          w.x = pack_bf16(h[0], h[1]);
          w.y = pack_bf16(h[2], h[3]);
          w.z = pack_bf16(h[4], h[5]);
          w.w = pack_bf16(h[6], h[7]);
          *reinterpret_cast<uint4*>(out + canon(row, k, kMlpH)) = w;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    } else if (ok) {
      float v[32];
      tmem_ld32(tl, v);   // columns 0..31; the layer's 16 are 0..15
      if (grow < n) {
        float4* y = reinterpret_cast<float4*>(Y + (size_t)grow * kMlpOut);
        const float* b = bias + 3 * kMlpH;
        y[0] = make_float4(v[0] + b[0], v[1] + b[1], v[2] + b[2], v[3] + b[3]);
        y[1] = make_float4(v[4] + b[4], v[5] + b[5], v[6] + b[6], v[7] + b[7]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && threadIdx.x == 0 && m.err) atomicOr(m.err, kMlpErrTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

}  // namespace

int mlp_tc_setup() {
  return cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kTcSmem) == cudaSuccess
             ? 0
             : -1;
}

void mlp_launch_infer_tc(const MlpDev& m, const float* X, int n, const int* n_dev, float* Y,
                         cudaStream_t s) {
  if (n <= 0) return;
  k_mlp_infer_tc<<<(n + kTcRows - 1) / kTcRows, 128, kTcSmem, s>>>(m, X, n, n_dev, Y);
}

}  // namespace silg

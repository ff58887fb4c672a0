// The warm-start network on tensor cores: BF16 operands, FP32 accumulation, with
// mma.sync.m16n8k16 (a 16 x 16 by 16 x 8 product per warp instruction). The network is
// tiny (128 units) and the batches are a few hundred to a few thousand contacts, so one
// CTA keeps a whole copy of the weights in shared memory and each warp carries 16 rows
// (samples) through every layer on its own.
//
// Fragment layout of m16n8k16 (per lane: g = lane / 4, t = lane % 4): A (16 x 16,
// row-major) registers hold the pairs (g, 2t..2t+1), (g+8, 2t..), (g, 8+2t..), (g+8, 8+2t..);
// B (16 x 8, k x n) holds (k = 2t..2t+1, n = g) and (k = 8+2t.., n = g); C holds (g, 2t..2t+1)
// and (g+8, 2t..2t+1). Two BF16 values share a 32-bit register, the lower address in the
// low half.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mlp.cuh"

namespace silg {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void st32(bf16* p, float lo, float hi) {
  *reinterpret_cast<uint32_t*>(p) = pack2(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));
}

// A fragment of a row-major matrix M: rows r0.., columns k0..
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const bf16* M, int ld, int r0, int k0, int g, int t) {
  a[0] = ld32(M + (r0 + g) * ld + k0 + 2 * t);
  a[1] = ld32(M + (r0 + g + 8) * ld + k0 + 2 * t);
  a[2] = ld32(M + (r0 + g) * ld + k0 + 8 + 2 * t);
  a[3] = ld32(M + (r0 + g + 8) * ld + k0 + 8 + 2 * t);
}
// A fragment of the transpose of a row-major matrix M: element (m, k) = M[k][m]
__device__ __forceinline__ void frag_a_t(uint32_t (&a)[4], const bf16* M, int ld, int m0, int k0, int g, int t) {
  auto e = [&](int m, int k) { return M[k * ld + m]; };
  a[0] = pack2(e(m0 + g, k0 + 2 * t), e(m0 + g, k0 + 2 * t + 1));
  a[1] = pack2(e(m0 + g + 8, k0 + 2 * t), e(m0 + g + 8, k0 + 2 * t + 1));
  a[2] = pack2(e(m0 + g, k0 + 8 + 2 * t), e(m0 + g, k0 + 8 + 2 * t + 1));
  a[3] = pack2(e(m0 + g + 8, k0 + 8 + 2 * t), e(m0 + g + 8, k0 + 8 + 2 * t + 1));
}
// B fragment (k x n) from an n-major matrix Bt[n][k]
__device__ __forceinline__ void frag_b_nk(uint32_t (&b)[2], const bf16* Bt, int ld, int k0, int n0, int g, int t) {
  b[0] = ld32(Bt + (n0 + g) * ld + k0 + 2 * t);
  b[1] = ld32(Bt + (n0 + g) * ld + k0 + 8 + 2 * t);
}
// B fragment (k x n) from a k-major matrix B[k][n]
__device__ __forceinline__ void frag_b_kn(uint32_t (&b)[2], const bf16* B, int ld, int k0, int n0, int g, int t) {
  b[0] = pack2(B[(k0 + 2 * t) * ld + n0 + g], B[(k0 + 2 * t + 1) * ld + n0 + g]);
  b[1] = pack2(B[(k0 + 8 + 2 * t) * ld + n0 + g], B[(k0 + 8 + 2 * t + 1) * ld + n0 + g]);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// element offsets of the layers in the padded BF16 copies
constexpr int kR1 = 0, kR2 = kR1 + kMlpIn * kLdH, kR3 = kR2 + kMlpH * kLdH, kR4 = kR3 + kMlpH * kLdH;
constexpr int kT1 = 0, kT2 = kT1 + kMlpH * kLdIn, kT3 = kT2 + kMlpH * kLdH, kT4 = kT3 + kMlpH * kLdH;
constexpr int kNBias = 3 * kMlpH + kMlpOut;

__global__ void k_mlp_convert(MlpDev m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const float* th = m.theta;
  if (e < kWRowElems) {
    float v = 0.f;
    if (e < kR2) {
      const int i = e / kLdH, o = e % kLdH;
      if (o < kMlpH) v = th[kOffW1 + i * kMlpH + o];
    } else if (e < kR3) {
      const int i = (e - kR2) / kLdH, o = (e - kR2) % kLdH;
      if (o < kMlpH) v = th[kOffW2 + i * kMlpH + o];
    } else if (e < kR4) {
      const int i = (e - kR3) / kLdH, o = (e - kR3) % kLdH;
      if (o < kMlpH) v = th[kOffW3 + i * kMlpH + o];
    } else {
      const int i = (e - kR4) / kLdOut, o = (e - kR4) % kLdOut;
      if (o < kMlpOut) v = th[kOffW4 + i * kMlpOut + o];
    }
    m.w_row[e] = __float2bfloat16_rn(v);
  }
  if (e < kWTElems) {
    float v = 0.f;
    if (e < kT2) {
      const int o = e / kLdIn, i = e % kLdIn;
      if (i < kMlpIn) v = th[kOffW1 + i * kMlpH + o];
    } else if (e < kT3) {
      const int o = (e - kT2) / kLdH, i = (e - kT2) % kLdH;
      if (i < kMlpH) v = th[kOffW2 + i * kMlpH + o];
    } else if (e < kT4) {
      const int o = (e - kT3) / kLdH, i = (e - kT3) % kLdH;
      if (i < kMlpH) v = th[kOffW3 + i * kMlpH + o];
    } else {
      const int o = (e - kT4) / kLdH, i = (e - kT4) % kLdH;
      if (i < kMlpH) v = th[kOffW4 + i * kMlpOut + o];
    }
    m.w_t[e] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ float bias_of(const float* bias, int layer, int col) {
  return bias[layer * kMlpH + col];
}

// biases b1, b2, b3, b4 gathered from the master vector into shared memory
__device__ __forceinline__ void load_bias(const float* th, float* bias) {
  for (int e = threadIdx.x; e < kNBias; e += blockDim.x) {
    const int l = e / kMlpH, c = e % kMlpH;
    const int off = l == 0 ? kOffB1 : l == 1 ? kOffB2 : l == 2 ? kOffB3 : kOffB4;
    bias[e] = th[off + c];
  }
}

// global -> shared, 16-byte aligned, bytes a multiple of 16: asynchronous copies, all in
// flight at once, then one wait (the callers synchronise the CTA before reading)
__device__ __forceinline__ void copy16(void* dst, const void* src, int bytes) {
  const char* s = static_cast<const char*>(src);
  const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst);
  for (int e = threadIdx.x; e < bytes / 16; e += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16u * (unsigned)e),
                 "l"(s + 16 * (size_t)e) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// One hidden layer for the warp's 16 rows: out = GELU(in W + b), in[16][ld_in] with K
// columns, W given as B fragments by `bfrag(k0, n0, b)`; writes the BF16 activations to
// act_out (and the BF16 pre-activations to z_out when given).
template <int K, class BF>
__device__ __forceinline__ void hidden_layer(const bf16* in, int ld_in, BF bfrag, const float* bias,
                                             int layer, bf16* act_out, bf16* z_out, int g, int t) {
  float acc[kMlpH / 8][4];
#pragma unroll
  for (int j = 0; j < kMlpH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    frag_a(a, in, ld_in, 0, k0, g, t);
#pragma unroll
    for (int j = 0; j < kMlpH / 8; ++j) {
      uint32_t b[2];
      bfrag(k0, 8 * j, b);
      mma_bf16(acc[j], a, b);
    }
  }
#pragma unroll
  for (int j = 0; j < kMlpH / 8; ++j) {
    const int c = 8 * j + 2 * t;
    const float b0 = bias_of(bias, layer, c), b1 = bias_of(bias, layer, c + 1);
    const float z0 = acc[j][0] + b0, z1 = acc[j][1] + b1, z2 = acc[j][2] + b0, z3 = acc[j][3] + b1;
    st32(act_out + g * kLdH + c, gelu(z0), gelu(z1));
    st32(act_out + (g + 8) * kLdH + c, gelu(z2), gelu(z3));
    if (z_out) {
      st32(z_out + g * kLdH + c, z0, z1);
      st32(z_out + (g + 8) * kLdH + c, z2, z3);
    }
  }
}

// ---- inference ---------------------------------------------------------------------
constexpr size_t kInferSmem = sizeof(bf16) * (kWTElems + 4 * (16 * kLdIn + 2 * 16 * kLdH)) +
                              sizeof(float) * kNBias;

// n_dev (optional): the row count on the device, at most n (a launch sized for a capacity)
__global__ void __launch_bounds__(128) k_mlp_infer(MlpDev m, const float* X, int n, const int* n_dev,
                                                   float* Y) {
  if (n_dev) n = min(n, *n_dev);
  if (blockIdx.x * kMlpRows >= n) return;   // the whole CTA leaves together
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* wt = reinterpret_cast<bf16*>(smem);
  bf16* act = wt + kWTElems;                         // per warp: x [16][kLdIn], h0, h1 [16][kLdH]
  float* bias = reinterpret_cast<float*>(act + 4 * (16 * kLdIn + 2 * 16 * kLdH));
  copy16(wt, m.w_t, kWTElems * (int)sizeof(bf16));
  load_bias(m.theta, bias);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  bf16* xs = act + warp * (16 * kLdIn + 2 * 16 * kLdH);
  bf16* h0 = xs + 16 * kLdIn;
  bf16* h1 = h0 + 16 * kLdH;
  const int r0 = blockIdx.x * kMlpRows + warp * 16;
  for (int e = lane; e < 16 * kMlpIn; e += 32) {
    const int r = e / kMlpIn, c = e % kMlpIn;
    xs[r * kLdIn + c] = __float2bfloat16_rn(r0 + r < n ? X[(size_t)(r0 + r) * kMlpIn + c] : 0.f);
  }
  __syncthreads();
  auto b1 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_nk(b, wt + kT1, kLdIn, k0, n0, g, t); };
  auto b2 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_nk(b, wt + kT2, kLdH, k0, n0, g, t); };
  auto b3 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_nk(b, wt + kT3, kLdH, k0, n0, g, t); };
  hidden_layer<kMlpIn>(xs, kLdIn, b1, bias, 0, h0, nullptr, g, t);
  __syncwarp();
  hidden_layer<kMlpH>(h0, kLdH, b2, bias, 1, h1, nullptr, g, t);
  __syncwarp();
  hidden_layer<kMlpH>(h1, kLdH, b3, bias, 2, h0, nullptr, g, t);
  __syncwarp();
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k0 = 0; k0 < kMlpH; k0 += 16) {
    uint32_t a[4], b[2];
    frag_a(a, h0, kLdH, 0, k0, g, t);
    frag_b_nk(b, wt + kT4, kLdH, k0, 0, g, t);
    mma_bf16(acc, a, b);
  }
  const int c = 2 * t;
  const float bb0 = bias_of(bias, 3, c), bb1 = bias_of(bias, 3, c + 1);
  if (r0 + g < n) {
    Y[(size_t)(r0 + g) * kMlpOut + c] = acc[0] + bb0;
    Y[(size_t)(r0 + g) * kMlpOut + c + 1] = acc[1] + bb1;
  }
  if (r0 + g + 8 < n) {
    Y[(size_t)(r0 + g + 8) * kMlpOut + c] = acc[2] + bb0;
    Y[(size_t)(r0 + g + 8) * kMlpOut + c + 1] = acc[3] + bb1;
  }
}

// ---- training: forward and backward of one batch slice per CTA -----------------------
constexpr int kLdY = 24;  // dY rows (8 outputs padded to a 16-wide k block)
constexpr size_t kTrainSmem =
    sizeof(bf16) * (kWRowElems + kMlpRows * kLdIn + 6 * kMlpRows * kLdH + kMlpRows * kLdY) +
    sizeof(float) * (kNBias + 4);

// partial gradient of W = A^T D over this CTA's rows into part (row-major in x out), for
// in = M rows of A^T (M a multiple of 16, split over the warps) and out = N columns
template <int M, int N>
__device__ __forceinline__ void weight_grad(const bf16* A, int lda, const bf16* D, int ldd, float* part,
                                            int warp, int g, int t) {
  constexpr int MT = M / 16, NT = N / 8;
  for (int mt = warp; mt < MT; mt += 4) {
    for (int nh = 0; nh < NT; nh += 8) {
      float acc[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
      for (int k0 = 0; k0 < kMlpRows; k0 += 16) {
        uint32_t a[4];
        frag_a_t(a, A, lda, 16 * mt, k0, g, t);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (nh + j < NT) {
            uint32_t b[2];
            frag_b_kn(b, D, ldd, k0, 8 * (nh + j), g, t);
            mma_bf16(acc[j], a, b);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (nh + j >= NT) continue;
        const int c = 8 * (nh + j) + 2 * t, r = 16 * mt + g;
        part[r * N + c] = acc[j][0];
        part[r * N + c + 1] = acc[j][1];
        part[(r + 8) * N + c] = acc[j][2];
        part[(r + 8) * N + c + 1] = acc[j][3];
      }
    }
  }
}

// dZ_prev = (D W^T) * GELU'(Z_prev) for the warp's 16 rows, written over Z_prev (BF16).
// D: [rows][ldd] with KD columns; W row-major [in][out] (out = KD), in = kMlpH.
template <int KD>
__device__ __forceinline__ void back_layer(const bf16* D, int ldd, const bf16* W, int ldw, bf16* Z,
                                          int g, int t) {
  float acc[kMlpH / 8][4];
#pragma unroll
  for (int j = 0; j < kMlpH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < KD; k0 += 16) {
    uint32_t a[4];
    frag_a(a, D, ldd, 0, k0, g, t);
#pragma unroll
    for (int j = 0; j < kMlpH / 8; ++j) {
      uint32_t b[2];
      frag_b_nk(b, W, ldw, k0, 8 * j, g, t);   // B(k = out, n = in) = W[in][out]
      mma_bf16(acc[j], a, b);
    }
  }
#pragma unroll
  for (int j = 0; j < kMlpH / 8; ++j) {
    const int c = 8 * j + 2 * t;
    bf16* z0 = Z + g * kLdH + c;
    bf16* z1 = Z + (g + 8) * kLdH + c;
    const float d0 = acc[j][0] * gelu_grad(__bfloat162float(z0[0]));
    const float d1 = acc[j][1] * gelu_grad(__bfloat162float(z0[1]));
    const float d2 = acc[j][2] * gelu_grad(__bfloat162float(z1[0]));
    const float d3 = acc[j][3] * gelu_grad(__bfloat162float(z1[1]));
    st32(z0, d0, d1);
    st32(z1, d2, d3);
  }
}

// column sums of a [kMlpRows][ld] BF16 matrix into part[0..N)
template <int N>
__device__ __forceinline__ void bias_grad(const bf16* D, int ld, float* part) {
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < kMlpRows; ++r) s += __bfloat162float(D[r * ld + c]);
    part[c] = s;
  }
}

__global__ void __launch_bounds__(128) k_mlp_train(MlpDev m, const float* X, const float* T,
                                                   const int* idx, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* w = reinterpret_cast<bf16*>(smem);
  bf16* A0 = w + kWRowElems;                       // [64][kLdIn]
  bf16* A1 = A0 + kMlpRows * kLdIn;                // [64][kLdH] each: A1 A2 A3 Z1 Z2 Z3
  bf16* A2 = A1 + kMlpRows * kLdH;
  bf16* A3 = A2 + kMlpRows * kLdH;
  bf16* Z1 = A3 + kMlpRows * kLdH;
  bf16* Z2 = Z1 + kMlpRows * kLdH;
  bf16* Z3 = Z2 + kMlpRows * kLdH;
  bf16* DY = Z3 + kMlpRows * kLdH;                 // [64][kLdY]
  float* bias = reinterpret_cast<float*>(DY + kMlpRows * kLdY);
  float* lsum = bias + kNBias;                     // 4 warps
  copy16(w, m.w_row, kWRowElems * (int)sizeof(bf16));
  load_bias(m.theta, bias);
  const int row0 = blockIdx.x * kMlpRows;
  for (int e = threadIdx.x; e < kMlpRows * kMlpIn; e += blockDim.x) {
    const int r = e / kMlpIn, c = e % kMlpIn, gr = row0 + r;
    float v = 0.f;
    if (gr < n) v = X[(size_t)(idx ? idx[gr] : gr) * kMlpIn + c];
    A0[r * kLdIn + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wr = 16 * warp;  // the warp's rows
  // forward (B fragments of the row-major weights: k = input, n = output)
  auto b1 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_kn(b, w + kR1, kLdH, k0, n0, g, t); };
  auto b2 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_kn(b, w + kR2, kLdH, k0, n0, g, t); };
  auto b3 = [&](int k0, int n0, uint32_t (&b)[2]) { frag_b_kn(b, w + kR3, kLdH, k0, n0, g, t); };
  hidden_layer<kMlpIn>(A0 + wr * kLdIn, kLdIn, b1, bias, 0, A1 + wr * kLdH, Z1 + wr * kLdH, g, t);
  __syncwarp();
  hidden_layer<kMlpH>(A1 + wr * kLdH, kLdH, b2, bias, 1, A2 + wr * kLdH, Z2 + wr * kLdH, g, t);
  __syncwarp();
  hidden_layer<kMlpH>(A2 + wr * kLdH, kLdH, b3, bias, 2, A3 + wr * kLdH, Z3 + wr * kLdH, g, t);
  __syncwarp();
  float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k0 = 0; k0 < kMlpH; k0 += 16) {
    uint32_t a[4], b[2];
    frag_a(a, A3 + wr * kLdH, kLdH, 0, k0, g, t);
    frag_b_kn(b, w + kR4, kLdOut, k0, 0, g, t);
    mma_bf16(y, a, b);
  }
  // dY = (Y - T) / n on the used outputs of valid rows; loss partial sum
  {
    const int c = 2 * t;
    float l2 = 0.f;
    for (int h = 0; h < 2; ++h) {
      const int r = wr + g + 8 * h, gr = row0 + r;
      float d[2] = {0.f, 0.f};
      for (int q = 0; q < 2; ++q) {
        const int col = c + q;
        const float yv = y[2 * h + q] + bias_of(bias, 3, col);
        if (gr < n && col < kMlpNY) {
          const float diff = yv - T[(size_t)(idx ? idx[gr] : gr) * kMlpNY + col];
          d[q] = diff / (float)n;
          l2 += diff * diff;
        }
      }
      st32(DY + r * kLdY + c, d[0], d[1]);
      st32(DY + r * kLdY + 8 + c, 0.f, 0.f);   // the k block's upper half
    }
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    if (lane == 0) lsum[warp] = l2;
  }
  __syncthreads();
  float* part = m.part + (size_t)blockIdx.x * kMlpParams;
  if (threadIdx.x == 0) m.part_loss[blockIdx.x] = 0.5f * (lsum[0] + lsum[1] + lsum[2] + lsum[3]) / (float)n;
  // layer 4: gW4 = A3^T dY, gb4; dZ3 = (dY W4^T) * GELU'(Z3)
  weight_grad<kMlpH, kMlpOut>(A3, kLdH, DY, kLdY, part + kOffW4, warp, g, t);
  bias_grad<kMlpOut>(DY, kLdY, part + kOffB4);
  back_layer<16>(DY + wr * kLdY, kLdY, w + kR4, kLdOut, Z3 + wr * kLdH, g, t);
  __syncthreads();
  // layer 3
  weight_grad<kMlpH, kMlpH>(A2, kLdH, Z3, kLdH, part + kOffW3, warp, g, t);
  bias_grad<kMlpH>(Z3, kLdH, part + kOffB3);
  back_layer<kMlpH>(Z3 + wr * kLdH, kLdH, w + kR3, kLdH, Z2 + wr * kLdH, g, t);
  __syncthreads();
  // layer 2
  weight_grad<kMlpH, kMlpH>(A1, kLdH, Z2, kLdH, part + kOffW2, warp, g, t);
  bias_grad<kMlpH>(Z2, kLdH, part + kOffB2);
  back_layer<kMlpH>(Z2 + wr * kLdH, kLdH, w + kR2, kLdH, Z1 + wr * kLdH, g, t);
  __syncthreads();
  // layer 1
  weight_grad<kMlpIn, kMlpH>(A0, kLdIn, Z1, kLdH, part + kOffW1, warp, g, t);
  bias_grad<kMlpH>(Z1, kLdH, part + kOffB1);
}

// grad = sum of the CTAs' partial gradients in CTA order; loss likewise
__global__ void k_mlp_reduce(MlpDev m, int nctas) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) {
    float s = 0.f;
    for (int c = 0; c < nctas; ++c) s += m.part[(size_t)c * kMlpParams + p];
    m.grad[p] = s;
  }
  if (p == 0) {
    float l = 0.f;
    for (int c = 0; c < nctas; ++c) l += m.part_loss[c];
    *m.loss = l;
  }
}

__global__ void k_mlp_adam(MlpDev m, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float gr = m.grad[p];
  const float mm = 0.9f * m.adam_m[p] + 0.1f * gr;
  const float vv = 0.999f * m.adam_v[p] + 0.001f * gr * gr;
  m.adam_m[p] = mm;
  m.adam_v[p] = vv;
  m.theta[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

}  // namespace

void mlp_launch_convert(const MlpDev& m, cudaStream_t s) {
  const int n = kWRowElems > kWTElems ? kWRowElems : kWTElems;
  k_mlp_convert<<<(n + 255) / 256, 256, 0, s>>>(m);
}

int mlp_setup() {
  if (mlp_tc_setup() != 0 ||
      cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kInferSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTrainSmem) != cudaSuccess)
    return -1;
  return 0;
}

void mlp_launch_infer(const MlpDev& m, const float* X, int n, float* Y, cudaStream_t s) {
  if (n <= 0) return;
  if (m.tc) {
    mlp_launch_infer_tc(m, X, n, nullptr, Y, s);
    return;
  }
  k_mlp_infer<<<(n + kMlpRows - 1) / kMlpRows, 128, kInferSmem, s>>>(m, X, n, nullptr, Y);
}

void mlp_launch_infer_dev(const MlpDev& m, const float* X, const int* n_dev, int n_max, float* Y,
                          cudaStream_t s) {
  if (n_max <= 0) return;
  if (m.tc) {
    mlp_launch_infer_tc(m, X, n_max, n_dev, Y, s);
    return;
  }
  k_mlp_infer<<<(n_max + kMlpRows - 1) / kMlpRows, 128, kInferSmem, s>>>(m, X, n_max, n_dev, Y);
}

void mlp_launch_gradient(const MlpDev& m, const float* X, const float* T, const int* idx, int n,
                         cudaStream_t s) {
  const int nctas = (n + kMlpRows - 1) / kMlpRows;
  if (nctas <= 0 || nctas > m.max_ctas) return;
  k_mlp_train<<<nctas, 128, kTrainSmem, s>>>(m, X, T, idx, n);
  k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, s>>>(m, nctas);
}

void mlp_launch_adam(const MlpDev& m, int t, float lr, cudaStream_t s) {
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(m, lr, c1, c2);
  mlp_launch_convert(m, s);
}

}  // namespace silg

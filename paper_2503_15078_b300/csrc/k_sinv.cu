// The global step as two products with the sparse inverse S~ = L~^-1 P (Eq. 8, Alg. 2):
//   pass 1  z = S~ g      (rows of the profile, dot products)
//   pass 2  x = S~^T y    (columns of the profile, scaled row sums)
// on the per-vertex factor (A = A~ (x) I3, so each S~ value multiplies an x, y, z triple).
//
// Storage: row i holds columns [lo_i, hi_i), a superset of its elimination subtree
// [fd(i), i] aligned to 8 values; rows are concatenated. The work is cut into tiles of
// kRowGroup rows x kTileW columns; a tile's part of a row is one contiguous, 32-byte
// aligned run of at most 1 KB. Each warp owns kRowsPerWarp rows of a tile and each lane
// two fixed 4-column chunks, read with 16-byte loads.
//
// The products are HBM-bound: every S~ value is read once per product. Throughput comes
// from memory-level parallelism, so the inner loops issue all loads of two tiles
// (16 x 16 bytes per lane) before any arithmetic, without branches: a lane whose chunk lies
// outside its row's stored range loads from a small zero buffer instead, which also makes
// masking unnecessary.
//
// Pass-1 work items walk one row group across up to kMaxTilesP1 column tiles (the item's
// slice of g is staged in shared memory); pass-2 items walk one column tile down a list
// of row groups (their row metadata and y values are staged in shared memory). Both
// write per-item partial sums that a second kernel adds in a fixed order, so results are
// deterministic. Items are launched largest first.
#include <cuda_runtime.h>

#include "device.cuh"

namespace silg {
namespace {

constexpr int RG = kRowGroup;
constexpr int TW = kTileW;
constexpr int kChunks = TW / 128;  // float4 chunks per lane per row

// Value formats of the profile. A lane's 4-column chunk is one 16-byte load in FP32 and
// one 8-byte load in BF16; the raw registers are widened to FP32 at the arithmetic.
// BF16 keeps twice as many tiles in flight, so the bytes in flight per warp (and the
// registers holding them) match the FP32 loop.
template <class T> struct Fmt;
template <> struct Fmt<float> {
  using Raw = float4;
  static constexpr int kUnroll = 2;  // tiles in flight per warp
  static __device__ __forceinline__ const float* vals(const DevSim& d) { return d.S; }
  static __device__ __forceinline__ Raw load(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  static __device__ __forceinline__ float4 widen(const Raw& r) { return r; }
};
template <> struct Fmt<unsigned short> {
  using Raw = uint2;
  static constexpr int kUnroll = 4;
  static __device__ __forceinline__ const unsigned short* vals(const DevSim& d) { return d.Sb; }
  static __device__ __forceinline__ Raw load(const unsigned short* p) {
    return __ldg(reinterpret_cast<const uint2*>(p));
  }
  // a BF16 value is the upper half of the FP32 with the same bits
  static __device__ __forceinline__ float4 widen(const Raw& r) {
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u),
                       __uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
  }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}


// z partials: item (rg, [ct0, ct1)) -> p1_part[item][comp][row in group]
template <class T>
__global__ void __launch_bounds__(256, 2) k_pass1(DevSim d) {
  using F = Fmt<T>;
  constexpr int kUnroll = F::kUnroll;
  const T* S = F::vals(d);
  const T* zero = reinterpret_cast<const T*>(d.zero);
  extern __shared__ __align__(16) float4 gsm[];  // [3][q4]
  const int item = d.p1_order[blockIdx.x];
  const int4 it = d.p1_items[item];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c_begin = it.y * TW;
  const int q4 = (it.z - it.y) * (TW / 4);
  for (int e = threadIdx.x; e < 3 * q4; e += blockDim.x) {
    const int comp = e / q4, q = e % q4;
    gsm[e] = *reinterpret_cast<const float4*>(d.gvec + comp * d.n_pad + c_begin + 4 * q);
  }
  const int r_first = it.x * RG + warp * kRowsPerWarp;
  const T* base[kRowsPerWarp];
  int lo[kRowsPerWarp], hi[kRowsPerWarp];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) {
    const int r = r_first + k;
    if (r < d.n) {
      lo[k] = d.lo[r];
      hi[k] = d.hi[r];
      base[k] = S + (d.rowbase[r] - lo[k]);
    } else {
      lo[k] = hi[k] = 0;
      base[k] = S;
    }
  }
  __syncthreads();
  float acc[kRowsPerWarp][3];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
  for (int ct = it.y; ct < it.z; ct += kUnroll) {
    typename F::Raw v[kUnroll][kRowsPerWarp][kChunks];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int m = 0; m < kChunks; ++m) {
        const int c = (ct + u) * TW + 4 * lane + 128 * m;
        const bool tile_ok = ct + u < it.z;
#pragma unroll
        for (int k = 0; k < kRowsPerWarp; ++k) {
          const bool ok = tile_ok && c >= lo[k] && c < hi[k];
          v[u][k][m] = F::load(ok ? base[k] + c : zero + 4 * lane);
        }
      }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (ct + u >= it.z) break;
#pragma unroll
      for (int m = 0; m < kChunks; ++m) {
        const int q = (ct + u - it.y) * (TW / 4) + lane + 32 * m;
        const float4 g0 = gsm[q], g1 = gsm[q4 + q], g2 = gsm[2 * q4 + q];
#pragma unroll
        for (int k = 0; k < kRowsPerWarp; ++k) {
          const float4 sv = F::widen(v[u][k][m]);
          acc[k][0] += dot4(sv, g0);
          acc[k][1] += dot4(sv, g1);
          acc[k][2] += dot4(sv, g2);
        }
      }
    }
  }
  float* out = d.p1_part + (size_t)item * 3 * RG;
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float s = warp_sum(acc[k][comp]);
      if (lane == 0) out[comp * RG + warp * kRowsPerWarp + k] = s;
    }
}

// z_r = sum of its row group's partials, in item order; zero padding beyond n.
__global__ void k_reduce1(DevSim d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.n_pad) return;
  if (r >= d.n) {
    d.zvec[r] = d.zvec[d.n_pad + r] = d.zvec[2 * d.n_pad + r] = 0.f;
    return;
  }
  const int rg = r / RG, lr = r % RG;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = d.p1_first[rg]; i < d.p1_first[rg + 1]; ++i) {
    const float* p = d.p1_part + (size_t)i * 3 * RG;
    s0 += p[lr];
    s1 += p[RG + lr];
    s2 += p[2 * RG + lr];
  }
  d.zvec[r] = s0;
  d.zvec[d.n_pad + r] = s1;
  d.zvec[2 * d.n_pad + r] = s2;
}

struct RowMeta {
  long long base;   // offset of column 0 of the row in S~ (may precede the row)
  int lo, hi;
  float y0, y1, y2, pad;
};

constexpr size_t kP2Meta = sizeof(RowMeta) * kMaxGroupsP2 * RG;
constexpr size_t kP2Smem = kP2Meta + sizeof(float) * kWarps * 3 * TW;

// x partials: item (ct, row-group list) -> p2_part[item][comp][column in tile]
template <class T>
__global__ void __launch_bounds__(256, 2) k_pass2(DevSim d) {
  using F = Fmt<T>;
  constexpr int kUnroll = F::kUnroll;
  const T* S = F::vals(d);
  const T* zero = reinterpret_cast<const T*>(d.zero);
  extern __shared__ __align__(16) unsigned char smem2[];
  RowMeta* meta = reinterpret_cast<RowMeta*>(smem2);
  float* red = reinterpret_cast<float*>(smem2 + kP2Meta);
  const int item = d.p2_order[blockIdx.x];
  const int4 it = d.p2_items[item];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = it.x * TW;
  const int nrg = it.z;
  for (int e = threadIdx.x; e < nrg * RG; e += blockDim.x) {
    const int r = d.p2_list[it.y + e / RG] * RG + e % RG;
    RowMeta m;
    if (r < d.n) {
      m.lo = d.lo[r];
      m.hi = d.hi[r];
      m.base = d.rowbase[r] - m.lo;
      m.y0 = d.zvec[r];
      m.y1 = d.zvec[d.n_pad + r];
      m.y2 = d.zvec[2 * d.n_pad + r];
    } else {
      m.lo = m.hi = 0;
      m.base = 0;
      m.y0 = m.y1 = m.y2 = 0.f;
    }
    m.pad = 0.f;
    meta[e] = m;
  }
  __syncthreads();
  float acc[kChunks][3][4];
#pragma unroll
  for (int m = 0; m < kChunks; ++m)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][comp][e] = 0.f;
  for (int li = 0; li < nrg; li += kUnroll) {
    typename F::Raw v[kUnroll][kRowsPerWarp][kChunks];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool grp_ok = li + u < nrg;
      const RowMeta* rm = meta + (grp_ok ? li + u : li) * RG + warp * kRowsPerWarp;
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const int lo = rm[k].lo, hi = rm[k].hi;
        const T* base = S + rm[k].base;
#pragma unroll
        for (int m = 0; m < kChunks; ++m) {
          const int c = c0 + 4 * lane + 128 * m;
          const bool ok = grp_ok && c >= lo && c < hi;
          v[u][k][m] = F::load(ok ? base + c : zero + 4 * lane);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (li + u >= nrg) break;
      const RowMeta* rm = meta + (li + u) * RG + warp * kRowsPerWarp;
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const float y0 = rm[k].y0, y1 = rm[k].y1, y2 = rm[k].y2;
#pragma unroll
        for (int m = 0; m < kChunks; ++m) {
          const float4 s = F::widen(v[u][k][m]);
          acc[m][0][0] += s.x * y0; acc[m][0][1] += s.y * y0;
          acc[m][0][2] += s.z * y0; acc[m][0][3] += s.w * y0;
          acc[m][1][0] += s.x * y1; acc[m][1][1] += s.y * y1;
          acc[m][1][2] += s.z * y1; acc[m][1][3] += s.w * y1;
          acc[m][2][0] += s.x * y2; acc[m][2][1] += s.y * y2;
          acc[m][2][2] += s.z * y2; acc[m][2][3] += s.w * y2;
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kChunks; ++m)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
      *reinterpret_cast<float4*>(&red[(warp * 3 + comp) * TW + 4 * lane + 128 * m]) =
          make_float4(acc[m][comp][0], acc[m][comp][1], acc[m][comp][2], acc[m][comp][3]);
  __syncthreads();
  float* out = d.p2_part + (size_t)item * 3 * TW;
  for (int idx = threadIdx.x; idx < 3 * TW; idx += blockDim.x) {
    const int comp = idx / TW, c = idx % TW;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[(w * 3 + comp) * TW + c];
    out[comp * TW + c] = s;
  }
}

// x_c = sum of its column tile's partials, in item order, written to the iterate's
// displacement dq (AoS, FP32), to xout (AoS), or added into dq.
template <int kMode>
__global__ void k_reduce2(DevSim d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n) return;
  const int ct = c / TW, lc = c % TW;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = d.p2_first[ct]; i < d.p2_first[ct + 1]; ++i) {
    const float* p = d.p2_part + (size_t)i * 3 * TW;
    s0 += p[lc];
    s1 += p[TW + lc];
    s2 += p[2 * TW + lc];
  }
  float* out = (kMode == kOutDq || kMode == kOutAddDq) ? d.dq : d.xout;
  if (kMode == kOutAddDq || kMode == kOutAddX) {
    out[3 * c] += s0;
    out[3 * c + 1] += s1;
    out[3 * c + 2] += s2;
  } else {
    out[3 * c] = s0;
    out[3 * c + 1] = s1;
    out[3 * c + 2] = s2;
  }
}

// Residual of a global solve, rho = rhs - A~ x per component, into gsave (SoA).
//   kResApply:        rhs = gsave (the saved right-hand side), x = xout
//   kResFrame:        rhs = g (gvec), x = dq
//   kResFrameContact: rhs = g + h^2 J^T dlambda (per contact vertex in uvec), x = dq
// The sum runs in FP64 on the FP32 operands (exact products): the residual of an accurate
// solve is a small difference of large terms, and with FP32 sums its rounding error,
// about 2^-24 |A~| |x|, amplified by cond(A~) in the correction, would exceed the BF16
// error the correction removes on stiff meshes.
template <int kMode>
__global__ void k_residual(DevSim d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_pad) return;
  if (i >= d.n) {
    d.gsave[i] = d.gsave[d.n_pad + i] = d.gsave[2 * d.n_pad + i] = 0.f;
    return;
  }
  const float* x = kMode == kResApply ? d.xout : d.dq;
  const float* rhs = kMode == kResApply ? d.gsave : d.gvec;
  double r0 = rhs[i], r1 = rhs[d.n_pad + i], r2 = rhs[2 * d.n_pad + i];
  if (kMode == kResFrameContact && d.cv_flag[i]) {
    const int c = d.cv_off[i];
    if (c < d.cap) {
      const double h2 = d.h * d.h;
      r0 += h2 * d.uvec[3 * c];
      r1 += h2 * d.uvec[3 * c + 1];
      r2 += h2 * d.uvec[3 * c + 2];
    }
  }
  for (int e = d.A_ptr[i]; e < d.A_ptr[i + 1]; ++e) {
    const int j = d.A_idx[e];
    const double a = d.A_val[e];
    r0 -= a * x[3 * j];
    r1 -= a * x[3 * j + 1];
    r2 -= a * x[3 * j + 2];
  }
  d.gsave[i] = (float)r0;
  d.gsave[d.n_pad + i] = (float)r1;
  d.gsave[2 * d.n_pad + i] = (float)r2;
}

}  // namespace

constexpr size_t kP1Smem = 3 * kMaxTilesP1 * TW * sizeof(float);

int sinv_setup() {
  if (cudaFuncSetAttribute(k_pass2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2Smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_pass1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP1Smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_pass2<unsigned short>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kP2Smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_pass1<unsigned short>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kP1Smem) != cudaSuccess)
    return SIM_ECUDA;
  return SIM_OK;
}

void launch_pass1(const DevSim& d, cudaStream_t s) {
  if (d.s_bf16)
    k_pass1<unsigned short><<<d.n_p1, 256, kP1Smem, s>>>(d);
  else
    k_pass1<float><<<d.n_p1, 256, kP1Smem, s>>>(d);
  k_reduce1<<<(d.n_pad + 255) / 256, 256, 0, s>>>(d);
}

void launch_pass2(const DevSim& d, cudaStream_t s, int out_mode) {
  if (d.s_bf16)
    k_pass2<unsigned short><<<d.n_p2, 256, kP2Smem, s>>>(d);
  else
    k_pass2<float><<<d.n_p2, 256, kP2Smem, s>>>(d);
  const int g = (d.n + 255) / 256;
  switch (out_mode) {
    case kOutDq: k_reduce2<kOutDq><<<g, 256, 0, s>>>(d); break;
    case kOutX: k_reduce2<kOutX><<<g, 256, 0, s>>>(d); break;
    case kOutAddDq: k_reduce2<kOutAddDq><<<g, 256, 0, s>>>(d); break;
    default: k_reduce2<kOutAddX><<<g, 256, 0, s>>>(d); break;
  }
}

void launch_residual(const DevSim& d, cudaStream_t s, int mode) {
  const int g = (d.n_pad + 255) / 256;
  switch (mode) {
    case kResApply: k_residual<kResApply><<<g, 256, 0, s>>>(d); break;
    case kResFrame: k_residual<kResFrame><<<g, 256, 0, s>>>(d); break;
    default: k_residual<kResFrameContact><<<g, 256, 0, s>>>(d); break;
  }
}

}  // namespace silg

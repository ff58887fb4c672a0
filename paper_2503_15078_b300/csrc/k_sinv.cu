// The global step as two products with the sparse inverse S~ = L~^-1 P (Eq. 8, Alg. 2):
//   pass 1  z = S~ g      (rows of the profile, dot products)
//   pass 2  x = S~^T y    (columns of the profile, scaled row sums)
// on the per-vertex factor (A = A~ (x) I3, so each S~ value multiplies an x, y, z triple).
//
// Storage: row i holds columns [lo_i, hi_i), a superset of its elimination subtree
// [fd(i), i] aligned to 8 values; rows are concatenated. Work is tiled into
// kRowGroup x kTileW tiles; each lane owns fixed 4-column chunks of a tile and reads them
// with aligned 16-byte loads. Pass-1 work items walk a row group across column tiles,
// pass-2 items walk a column tile down a list of row groups; both emit partial sums that
// a second kernel adds in a fixed order, so the result is deterministic.
#include <cuda_runtime.h>

#include "device.cuh"

namespace silg {
namespace {

constexpr int RG = kRowGroup;
constexpr int TW = kTileW;
constexpr int kChunks = TW / 128;  // float4 chunks per lane per row

__device__ __forceinline__ float4 ld_stream(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct RowRef {
  const float* base;  // address of column 0 of the row (may point before the row)
  int lo, hi;
};

__device__ __forceinline__ RowRef row_ref(const DevSim& d, int r) {
  RowRef rr;
  if (r < d.n) {
    rr.lo = d.lo[r];
    rr.hi = d.hi[r];
    rr.base = d.S + (d.rowbase[r] - rr.lo);
  } else {
    rr.lo = rr.hi = 0;
    rr.base = d.S;
  }
  return rr;
}

// z partials: item (rg, [ct0, ct1)) -> p1_part[item][comp][row in group]
__global__ void __launch_bounds__(256) k_pass1(DevSim d) {
  __shared__ float4 gs[3][TW / 4];
  const int4 it = d.p1_items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r_first = it.x * RG + warp * kRowsPerWarp;
  RowRef rows[kRowsPerWarp];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) rows[k] = row_ref(d, r_first + k);
  float acc[kRowsPerWarp][3];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
  for (int ct = it.y; ct < it.z; ++ct) {
    const int c0 = ct * TW;
    __syncthreads();
    if (threadIdx.x < 3 * (TW / 4)) {
      int comp = threadIdx.x / (TW / 4), q = threadIdx.x % (TW / 4);
      gs[comp][q] = *reinterpret_cast<const float4*>(d.gvec + comp * d.n_pad + c0 + 4 * q);
    }
    __syncthreads();
    float4 g[3][kChunks];
#pragma unroll
    for (int m = 0; m < kChunks; ++m)
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) g[comp][m] = gs[comp][lane + 32 * m];
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
#pragma unroll
      for (int m = 0; m < kChunks; ++m) {
        const int c = c0 + 4 * lane + 128 * m;
        if (c >= rows[k].lo && c < rows[k].hi) {
          float4 s = ld_stream(rows[k].base + c);
#pragma unroll
          for (int comp = 0; comp < 3; ++comp)
            acc[k][comp] += s.x * g[comp][m].x + s.y * g[comp][m].y + s.z * g[comp][m].z +
                            s.w * g[comp][m].w;
        }
      }
    }
  }
  float* out = d.p1_part + (size_t)blockIdx.x * 3 * RG;
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      float v = warp_sum(acc[k][comp]);
      if (lane == 0) out[comp * RG + warp * kRowsPerWarp + k] = v;
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

// x partials: item (ct, row-group list) -> p2_part[item][comp][column in tile]
__global__ void __launch_bounds__(256) k_pass2(DevSim d) {
  __shared__ float red[kWarps][3][TW];
  const int4 it = d.p2_items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = it.x * TW;
  float acc[kChunks][3][4];
#pragma unroll
  for (int m = 0; m < kChunks; ++m)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][comp][e] = 0.f;
  for (int li = 0; li < it.z; ++li) {
    const int rg = d.p2_list[it.y + li];
    const int r_first = rg * RG + warp * kRowsPerWarp;
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
      const int r = r_first + k;
      RowRef rr = row_ref(d, r);
      if (r >= d.n) continue;
      float y0 = d.zvec[r], y1 = d.zvec[d.n_pad + r], y2 = d.zvec[2 * d.n_pad + r];
#pragma unroll
      for (int m = 0; m < kChunks; ++m) {
        const int c = c0 + 4 * lane + 128 * m;
        if (c >= rr.lo && c < rr.hi) {
          float4 s = ld_stream(rr.base + c);
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
      *reinterpret_cast<float4*>(&red[warp][comp][4 * lane + 128 * m]) =
          make_float4(acc[m][comp][0], acc[m][comp][1], acc[m][comp][2], acc[m][comp][3]);
  __syncthreads();
  float* out = d.p2_part + (size_t)blockIdx.x * 3 * TW;
  for (int idx = threadIdx.x; idx < 3 * TW; idx += blockDim.x) {
    const int comp = idx / TW, c = idx % TW;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w][comp][c];
    out[comp * TW + c] = s;
  }
}

// x_c = sum of its column tile's partials, in item order. to_dq: write the iterate's
// displacement dq (AoS, FP32); otherwise write xout (AoS).
template <bool kToDq>
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
  float* out = kToDq ? d.dq : d.xout;
  out[3 * c] = s0;
  out[3 * c + 1] = s1;
  out[3 * c + 2] = s2;
}

}  // namespace

void launch_pass1(const DevSim& d, cudaStream_t s) {
  k_pass1<<<d.n_p1, 256, 0, s>>>(d);
  k_reduce1<<<(d.n_pad + 255) / 256, 256, 0, s>>>(d);
}

void launch_pass2(const DevSim& d, cudaStream_t s, bool to_dq) {
  k_pass2<<<d.n_p2, 256, 0, s>>>(d);
  if (to_dq)
    k_reduce2<true><<<(d.n + 255) / 256, 256, 0, s>>>(d);
  else
    k_reduce2<false><<<(d.n + 255) / 256, 256, 0, s>>>(d);
}

}  // namespace silg

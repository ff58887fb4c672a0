// The global step as two products with the sparse inverse S~ = L~^-1 P (Eq. 8, Alg. 2):
//   pass 1  z = S~ g      (rows of the profile, dot products)
//   pass 2  x = S~^T y    (columns of the profile, scaled row sums)
// on the per-vertex factor (A = A~ (x) I3, so each S~ value multiplies an x, y, z triple).
//
// Storage: row i holds columns [lo_i, hi_i), a superset of its elimination subtree
// [fd(i), i] aligned to 8 values; rows are concatenated. The work is cut into tiles of
// kRowGroup rows x kTileW columns; a tile's part of a row is one contiguous, aligned run
// of at most 1 KB (FP32). Each warp owns kRowsPerWarp rows of a tile and each lane two
// fixed 4-column chunks, read with one 16-byte (FP32) or 8-byte (BF16) load each.
//
// The products are HBM-bound: every S~ value is read once per product. Each CTA streams
// a contiguous range of the pass's tile order, the ranges cut so that every CTA has about
// the same number of bytes to read (one wave, no tail of large items). Throughput comes
// from memory-level parallelism: a warp issues the loads of kUnroll tiles before any
// arithmetic, without branches (a lane whose chunk lies outside its row's range loads
// from a small zero buffer instead), and the row metadata of the next tiles is fetched
// by the lanes while those loads are in flight. A run of tiles with the same row group
// (pass 1) or column tile (pass 2) accumulates in registers and ends in one partial-sum
// slot; a second kernel adds each row's (column's) slots in a fixed order, so results are
// deterministic. The accumulations use packed FP32 FMAs (fma.rn.f32x2, two columns per
// instruction).
//
// A second form of both products (k_pass1_bulk, k_pass2_bulk, below) moves each tile's row
// runs into shared memory with bulk copies instead of register loads; the autotuner times
// it beside the register form.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "device.cuh"

namespace silg {
namespace {

constexpr int RG = kRowGroup;
constexpr int TW = kTileW;
// Value formats of the profile. A lane's chunk of a row is kVec = 4 values, one 16-byte load
// in FP32 and one 8-byte load in BF16; a row of a tile is kChunks = kTileW / (32 kVec)
// chunks per lane.
// The raw registers are widened to packed FP32 pairs at the arithmetic. BF16 keeps twice
// as many tiles in flight, so the bytes in flight per warp (and the registers holding them)
// match the FP32 loop.
template <class T> struct Fmt;
template <> struct Fmt<float> {
  using Raw = float4;
  static constexpr int kVec = 4;
  static constexpr int kUnroll = 2;  // tiles in flight per warp
  static __device__ __forceinline__ const float* vals(const DevSim& d) { return d.S; }
  // streamed once: first in line for eviction from L1, so the vector slices read by
  // every warp stay cached
  static __device__ __forceinline__ Raw load(const float* p) {
    Raw r;
    asm volatile("ld.global.nc.L1::evict_first.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
  }
  // the chunk's values as the packed pairs (0, 1), (2, 3)
  static __device__ __forceinline__ void pairs(const Raw& r, unsigned long long (&p)[2]) {
    p[0] = f2pack(r.x, r.y);
    p[1] = f2pack(r.z, r.w);
  }
};
// BF16: a chunk of 4 values in one 8-byte load (measured faster on the 64-scene batch than
// 8 values in one 16-byte load, and equal on the star)
template <> struct Fmt<unsigned short> {
  using Raw = uint2;
  static constexpr int kVec = 4;
  static constexpr int kUnroll = 4;
  static __device__ __forceinline__ const unsigned short* vals(const DevSim& d) { return d.Sb; }
  static __device__ __forceinline__ Raw load(const unsigned short* p) {
    Raw r;
    asm volatile("ld.global.nc.L1::evict_first.v2.u32 {%0, %1}, [%2];"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p));
    return r;
  }
  // a BF16 value is the upper half of the FP32 with the same bits; the pairs (0, 1), (2, 3)
  static __device__ __forceinline__ void pairs(const Raw& r, unsigned long long (&p)[2]) {
    p[0] = f2pack(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u));
    p[1] = f2pack(__uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
  }
};
template <class T> struct FmtShape {
  static constexpr int kVec = Fmt<T>::kVec;
  static constexpr int kPairs = kVec / 2;
  static constexpr int kChunks = TW / (32 * kVec);
};

// CTAs per SM the products are built for: two with the format's tiles in flight (or half),
// one with twice as many (their registers hold twice the loads in flight)
template <class T, int U> struct PassOcc {
  static constexpr int kMinBlocks = U > Fmt<T>::kUnroll ? 1 : 2;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Row metadata of the tiles of one batch, held one entry per lane: lane u * 4 + k has
// row k (of the warp's kRowsPerWarp) of tile t + u. base is the offset of column 0 of the
// row (so that S + base + c addresses column c).
struct LaneMeta {
  int key, other;  // the tile's coordinates in the pass's order
  int lo, hi;
  long long base;
  float y0, y1, y2;  // pass 2: the row's values of y
};

template <bool kWithY>
__device__ __forceinline__ LaneMeta fetch_meta(const DevSim& d, const int2* tiles, int t_end,
                                               int t, int lane, int warp, bool pass2) {
  LaneMeta m;
  m.key = m.other = -1;
  m.lo = m.hi = 0;
  m.base = 0;
  m.y0 = m.y1 = m.y2 = 0.f;
  const int u = lane >> 2, k = lane & 3;
  if (t + u < t_end) {
    const int2 tl = tiles[t + u];
    m.key = tl.x;
    m.other = tl.y;
    const int rg = pass2 ? tl.y : tl.x;
    const int r = rg * RG + warp * kRowsPerWarp + k;
    if (r < d.n) {
      m.lo = d.lo[r];
      m.hi = d.hi[r];
      m.base = d.rowbase[r] - m.lo;
      if (kWithY) {
        m.y0 = d.zvec[r];
        m.y1 = d.zvec[d.n_pad + r];
        m.y2 = d.zvec[2 * d.n_pad + r];
      }
    }
  }
  return m;
}

// z partials: one slot per run of tiles of one row group -> p1_part[slot][comp][row].
// U: tiles in flight per warp (the format's default, or half of it).
template <class T, int U>
__global__ void __launch_bounds__(256, PassOcc<T, U>::kMinBlocks) k_pass1(DevSim d) {
  pdl_wait();
  using F = Fmt<T>;
  static_assert(U * kRowsPerWarp <= 32, "one metadata entry per lane");
  const T* S = F::vals(d);
  const T* zero = reinterpret_cast<const T*>(d.zero);
  extern __shared__ __align__(16) float4 gsm[];  // [column slot][comp][kTileW / 4]
  const int t0 = d.s1_cta[blockIdx.x], t1 = d.s1_cta[blockIdx.x + 1];
  if (t0 >= t1) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int slot = d.s1_seg_base[blockIdx.x];
  LaneMeta mt = fetch_meta<false>(d, d.s1_tiles, t1, t0, lane, warp, false);
  {
    // the g slices of the CTA's column tiles, copied asynchronously while the first
    // tiles' loads are issued below
    const int c0 = d.s1_col_first[blockIdx.x], nc = d.s1_col_first[blockIdx.x + 1] - c0;
    for (int e = threadIdx.x; e < nc * 3 * (TW / 4); e += blockDim.x) {
      const int k = e / (3 * (TW / 4)), rem = e % (3 * (TW / 4));
      const int comp = rem / (TW / 4), q = rem % (TW / 4);
      const float* src = d.gvec + comp * d.n_pad + d.s1_cols[c0 + k] * TW + 4 * q;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(gsm + e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  bool g_ready = false;
  int cur = __shfl_sync(0xffffffffu, mt.key, 0);
  // per row and component, two running sums (even and odd columns) in one register pair,
  // advanced by packed FMAs
  unsigned long long acc[kRowsPerWarp][3];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0ull;
  auto flush = [&]() {
    float* out = d.p1_part + (size_t)slot * 3 * RG;
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const float v = warp_sum(f2lo(acc[k][comp]) + f2hi(acc[k][comp]));
        if (lane == 0) out[comp * RG + warp * kRowsPerWarp + k] = v;
        acc[k][comp] = 0ull;
      }
    ++slot;
  };
  using SH = FmtShape<T>;
  constexpr int V = SH::kVec, NC = SH::kChunks;
  for (int t = t0; t < t1; t += U) {
    typename F::Raw v[U][kRowsPerWarp][NC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int ct = __shfl_sync(0xffffffffu, mt.other, u * 4);
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const int src = u * 4 + k;
        const int lo = __shfl_sync(0xffffffffu, mt.lo, src);
        const int hi = __shfl_sync(0xffffffffu, mt.hi, src);
        const long long base = __shfl_sync(0xffffffffu, mt.base, src);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          // runs start and end on multiples of 8 values: a chunk is inside or outside
          const int c = ct * TW + V * lane + 32 * V * m;
          const bool ok = c >= lo && c < hi;   // empty for tiles past the range (lo = hi)
          v[u][k][m] = F::load(ok ? S + base + c : zero + V * lane);
        }
      }
    }
    const int lkey = mt.key;  // this batch's tiles (lanes 4u)
    const int lslot = (lane & 3) == 0 && t + (lane >> 2) < t1 ? d.s1_col_slot[t + (lane >> 2)] : 0;
    mt = fetch_meta<false>(d, d.s1_tiles, t1, t + U, lane, warp, false);
    if (!g_ready) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      g_ready = true;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u >= t1) break;
      const int rg = __shfl_sync(0xffffffffu, lkey, u * 4);
      const int gs = __shfl_sync(0xffffffffu, lslot, u * 4);
      if (rg != cur) {
        flush();
        cur = rg;
      }
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        // g's columns of the chunk as packed pairs, per component
        const unsigned long long* gp = reinterpret_cast<const unsigned long long*>(
            gsm + gs * 3 * (TW / 4) + (V * lane + 32 * V * m) / 4);
        unsigned long long g[3][SH::kPairs];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
#pragma unroll
          for (int i = 0; i < SH::kPairs; ++i) g[comp][i] = gp[comp * (TW / 2) + i];
#pragma unroll
        for (int k = 0; k < kRowsPerWarp; ++k) {
          unsigned long long sp[SH::kPairs];
          F::pairs(v[u][k][m], sp);
#pragma unroll
          for (int i = 0; i < SH::kPairs; ++i) {
            acc[k][0] = ffma2(sp[i], g[0][i], acc[k][0]);
            acc[k][1] = ffma2(sp[i], g[1][i], acc[k][1]);
            acc[k][2] = ffma2(sp[i], g[2][i], acc[k][2]);
          }
        }
      }
    }
  }
  flush();
}

// z_r = sum of its row group's slots, in slot order; zero padding beyond n.
__global__ void k_reduce1(DevSim d) {
  pdl_wait();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.n_pad) return;
  if (r >= d.n) {
    d.zvec[r] = d.zvec[d.n_pad + r] = d.zvec[2 * d.n_pad + r] = 0.f;
    return;
  }
  const int rg = r / RG, lr = r % RG;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = d.s1_seg_first[rg]; i < d.s1_seg_first[rg + 1]; ++i) {
    const float* p = d.p1_part + (size_t)i * 3 * RG;
    s0 += p[lr];
    s1 += p[RG + lr];
    s2 += p[2 * RG + lr];
  }
  d.zvec[r] = s0;
  d.zvec[d.n_pad + r] = s1;
  d.zvec[2 * d.n_pad + r] = s2;
}


constexpr size_t kP2Smem = sizeof(float) * kWarps * 3 * TW;

// x partials: one slot per run of tiles of one column tile -> p2_part[slot][comp][column]
template <class T, int U>
__global__ void __launch_bounds__(256, PassOcc<T, U>::kMinBlocks) k_pass2(DevSim d) {
  pdl_wait();
  using F = Fmt<T>;
  static_assert(U * kRowsPerWarp <= 32, "one metadata entry per lane");
  const T* S = F::vals(d);
  const T* zero = reinterpret_cast<const T*>(d.zero);
  extern __shared__ __align__(16) float red[];  // [warp][comp][column]
  const int t0 = d.s2_cta[blockIdx.x], t1 = d.s2_cta[blockIdx.x + 1];
  if (t0 >= t1) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int slot = d.s2_seg_base[blockIdx.x];
  LaneMeta mt = fetch_meta<true>(d, d.s2_tiles, t1, t0, lane, warp, true);
  int cur = __shfl_sync(0xffffffffu, mt.key, 0);
  // per chunk and component, the chunk's columns' sums as packed pairs
  using SH = FmtShape<T>;
  constexpr int V = SH::kVec, NC = SH::kChunks, NP = SH::kPairs;
  unsigned long long acc[NC][3][NP];
#pragma unroll
  for (int m = 0; m < NC; ++m)
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
      for (int i = 0; i < NP; ++i) acc[m][comp][i] = 0ull;
  // every warp reaches a flush at the same tile, so the barriers are uniform
  auto flush = [&]() {
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        ulonglong2* dst =
            reinterpret_cast<ulonglong2*>(&red[(warp * 3 + comp) * TW + V * lane + 32 * V * m]);
#pragma unroll
        for (int i = 0; i < NP / 2; ++i) {
          dst[i] = make_ulonglong2(acc[m][comp][2 * i], acc[m][comp][2 * i + 1]);
          acc[m][comp][2 * i] = acc[m][comp][2 * i + 1] = 0ull;
        }
      }
    __syncthreads();
    float* out = d.p2_part + (size_t)slot * 3 * TW;
    for (int idx = threadIdx.x; idx < 3 * TW; idx += blockDim.x) {
      const int comp = idx / TW, c = idx % TW;
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += red[(w * 3 + comp) * TW + c];
      out[comp * TW + c] = s;
    }
    __syncthreads();
    ++slot;
  };
  for (int t = t0; t < t1; t += U) {
    typename F::Raw v[U][kRowsPerWarp][NC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int ctu = __shfl_sync(0xffffffffu, mt.key, u * 4);
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const int src = u * 4 + k;
        const int lo = __shfl_sync(0xffffffffu, mt.lo, src);
        const int hi = __shfl_sync(0xffffffffu, mt.hi, src);
        const long long base = __shfl_sync(0xffffffffu, mt.base, src);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          const int c = ctu * TW + V * lane + 32 * V * m;
          const bool ok = c >= lo && c < hi;
          v[u][k][m] = F::load(ok ? S + base + c : zero + V * lane);
        }
      }
    }
    const float ly0 = mt.y0, ly1 = mt.y1, ly2 = mt.y2;  // this batch's y, one row per lane
    const int lkey = mt.key;
    mt = fetch_meta<true>(d, d.s2_tiles, t1, t + U, lane, warp, true);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t + u >= t1) break;
      const int ct = __shfl_sync(0xffffffffu, lkey, u * 4);
      if (ct != cur) {
        flush();
        cur = ct;
      }
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const float y0 = __shfl_sync(0xffffffffu, ly0, u * 4 + k);
        const float y1 = __shfl_sync(0xffffffffu, ly1, u * 4 + k);
        const float y2 = __shfl_sync(0xffffffffu, ly2, u * 4 + k);
        const unsigned long long y00 = f2pack(y0, y0), y11 = f2pack(y1, y1),
                                 y22 = f2pack(y2, y2);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          unsigned long long sp[NP];
          F::pairs(v[u][k][m], sp);
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            acc[m][0][i] = ffma2(sp[i], y00, acc[m][0][i]);
            acc[m][1][i] = ffma2(sp[i], y11, acc[m][1][i]);
            acc[m][2][i] = ffma2(sp[i], y22, acc[m][2][i]);
          }
        }
      }
    }
  }
  flush();
}

// x_c = sum of its column tile's slots, in slot order, written to the iterate's
// displacement dq (AoS, FP32), to xout (AoS), or added into one of them.
template <int kMode>
__global__ void k_reduce2(DevSim d) {
  pdl_wait();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n) return;
  const int ct = c / TW, lc = c % TW;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = d.s2_seg_first[ct]; i < d.s2_seg_first[ct + 1]; ++i) {
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


// ---- the products through bulk copies ----------------------------------------------------
// The same tile streams, partial-sum slots and reductions as k_pass1 / k_pass2, with the
// S~ values moved into shared memory by bulk copies (cp.async.bulk, one per row run of a
// tile) instead of register loads. A producer warp walks the CTA's tiles and fills a ring
// of stages: per tile the row runs, in pass 1 the g slice of its column tile, in pass 2
// the y of its rows; each stage completes on an mbarrier when its bytes have arrived.
// Eight consumer warps (kRowsPerWarp rows of every tile each) multiply and release the
// stage on a second mbarrier. A lane reads eight consecutive values of a row: runs start
// and end on 8-value boundaries (16 bytes in BF16), so the lane's values lie either inside
// the row's run in that tile or outside it (zeros). Every wait is bounded: on a timeout the
// kernel records kErrTimeout and the waits that follow are skipped (the frame reports
// SIM_ETIMEOUT); before it exits, the producer waits (bounded) for the copies it issued.
constexpr int kBulkConsumers = kWarps;
constexpr int kBulkThreads = 32 * (kBulkConsumers + 1);
constexpr int kBulkMaxStages = 8;
constexpr int kSmemPerSm = 228 * 1024;
int g_bulk_smem_max = 0;   // dynamic shared memory a bulk-copy CTA may take (sinv_setup)

template <class T, bool kPass2> struct BulkLayout {
  static constexpr int kVals = RG * TW * (int)sizeof(T);          // the tile's values
  static constexpr int kSide = kPass2 ? RG * 16 : 3 * TW * 4;      // y (float4 per row) | g
  static constexpr int kRuns = RG * 8;                             // int2 [a, b) per row
  static constexpr int kStage = (kVals + kSide + kRuns + 127) / 128 * 128;
  static constexpr int kRed = kPass2 ? kBulkConsumers * 3 * TW * 4 : 0;   // pass 2 flush
};

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// wait for the phase of the given parity to complete, at most `limit` polls (0: 2^22, the
// default of sim_options.spin_limit)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity,
                                                  unsigned long long limit) {
  if (limit == 0) limit = 1ull << 22;
  for (unsigned long long i = 0; i < limit; ++i) {
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
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// the eight values of a lane's part of a row, as four packed pairs (zeros outside the run)
template <class T> struct BulkRow;
template <> struct BulkRow<unsigned short> {
  static __device__ __forceinline__ void get(const char* row, int lane, bool ok,
                                             unsigned long long (&p)[4]) {
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (ok) r = *reinterpret_cast<const uint4*>(row + 16 * lane);
    p[0] = f2pack(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u));
    p[1] = f2pack(__uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
    p[2] = f2pack(__uint_as_float(r.z << 16), __uint_as_float(r.z & 0xffff0000u));
    p[3] = f2pack(__uint_as_float(r.w << 16), __uint_as_float(r.w & 0xffff0000u));
  }
};
template <> struct BulkRow<float> {
  static __device__ __forceinline__ void get(const char* row, int lane, bool ok,
                                             unsigned long long (&p)[4]) {
    ulonglong2 a = make_ulonglong2(0ull, 0ull), b = make_ulonglong2(0ull, 0ull);
    if (ok) {
      a = *reinterpret_cast<const ulonglong2*>(row + 32 * lane);
      b = *reinterpret_cast<const ulonglong2*>(row + 32 * lane + 16);
    }
    p[0] = a.x;
    p[1] = a.y;
    p[2] = b.x;
    p[3] = b.y;
  }
};

// The producer lane's row of one tile: its run [a, b) in the tile's columns, the offset of
// the row's column 0, and (pass 2) its y.
struct BulkRowMeta {
  int a, b, ct;
  long long base;
  float4 y;
};

template <bool kPass2>
__device__ __forceinline__ BulkRowMeta bulk_row_meta(const DevSim& d, int2 tl, int lane) {
  BulkRowMeta m;
  const int rg = kPass2 ? tl.y : tl.x;
  m.ct = kPass2 ? tl.x : tl.y;
  const int r = rg * RG + lane;
  m.a = m.b = 0;
  m.base = 0;
  m.y = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r < d.n) {
    const int lo = d.lo[r], hi = d.hi[r];
    m.a = max(lo, m.ct * TW);
    m.b = max(m.a, min(hi, m.ct * TW + TW));
    m.base = d.rowbase[r] - lo;
    if (kPass2) m.y = make_float4(d.zvec[r], d.zvec[d.n_pad + r], d.zvec[2 * d.n_pad + r], 0.f);
  }
  return m;
}

// The producer warp: fills stage i % S with tile t0 + i once the consumers have released
// its previous use. The loads are software-pipelined: while tile t is issued, the rows of
// tile t + 1 and the entry of tile t + 2 are already on their way. Returns the number of
// tiles issued.
template <class T, bool kPass2>
__device__ int bulk_produce(const DevSim& d, const int2* tiles, int t0, int t1, char* stages,
                            int S, unsigned full0, unsigned empty0, int lane, bool& dead) {
  using L = BulkLayout<T, kPass2>;
  const T* vals = Fmt<T>::vals(d);
  const int2 none = make_int2(0, 0);
  BulkRowMeta cur = bulk_row_meta<kPass2>(d, tiles[t0], lane);
  int2 tl_next = t0 + 1 < t1 ? tiles[t0 + 1] : none;
  int i = 0;
  for (int t = t0; t < t1; ++t, ++i) {
    const BulkRowMeta nxt = t + 1 < t1 ? bulk_row_meta<kPass2>(d, tl_next, lane) : cur;
    const int2 tl_next2 = t + 2 < t1 ? tiles[t + 2] : none;
    const int s = i % S;
    const unsigned full = full0 + 8u * s, empty = empty0 + 8u * s;
    if (i >= S && !dead && !mbar_wait_bounded(empty, (unsigned)((i / S) - 1) & 1u, d.spin_limit)) {
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      dead = true;
    }
    if (dead) break;
    char* st = stages + (size_t)s * L::kStage;
    const int c0 = cur.ct * TW;
    reinterpret_cast<int2*>(st + L::kVals + L::kSide)[lane] = make_int2(cur.a - c0, cur.b - c0);
    if (kPass2) reinterpret_cast<float4*>(st + L::kVals)[lane] = cur.y;
    const unsigned bytes = (unsigned)(cur.b - cur.a) * (unsigned)sizeof(T);
    unsigned total = bytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (!kPass2) total += 3u * TW * 4u;
    // lane 0 announces the bytes the copies will deliver before any copy is issued; every
    // lane's writes of the stage's metadata are released by its own arrival
    __syncwarp();
    if (lane == 0) mbar_arrive_tx(full, total);
    __syncwarp();
    if (lane != 0) mbar_arrive(full);
    if (bytes)
      bulk_g2s((unsigned)__cvta_generic_to_shared(st + (size_t)(cur.a - c0) * sizeof(T) +
                                                   (size_t)lane * TW * sizeof(T)),
               vals + cur.base + cur.a, bytes, full);
    if (!kPass2 && lane < 3)
      bulk_g2s((unsigned)__cvta_generic_to_shared(st + L::kVals + lane * TW * 4),
               d.gvec + (size_t)lane * d.n_pad + (size_t)c0, TW * 4u, full);
    cur = nxt;
    tl_next = tl_next2;
  }
  return i;
}

// the producer's last act: wait (bounded) until the copies of the last use of every stage
// have landed, so that no copy is in flight into the CTA's shared memory when it exits
template <class T, bool kPass2>
__device__ void bulk_drain(const DevSim& d, int issued, int S, unsigned full0) {
  for (int i = max(0, issued - S); i < issued; ++i)
    mbar_wait_bounded(full0 + 8u * (i % S), (unsigned)(i / S) & 1u, d.spin_limit);
}

// z partials, as k_pass1
template <class T>
__global__ void __launch_bounds__(kBulkThreads, 2) k_pass1_bulk(DevSim d, int S) {
  pdl_wait();
  using L = BulkLayout<T, false>;
  extern __shared__ __align__(128) char bsm[];
  __shared__ __align__(8) unsigned long long bar_full[kBulkMaxStages], bar_empty[kBulkMaxStages];
  const int t0 = d.s1_cta[blockIdx.x], t1 = d.s1_cta[blockIdx.x + 1];
  if (t0 >= t1) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full0 = (unsigned)__cvta_generic_to_shared(bar_full);
  const unsigned empty0 = (unsigned)__cvta_generic_to_shared(bar_empty);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8u * s, 32);
      mbar_init(empty0 + 8u * s, kBulkConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  bool dead = false;
  if (warp == kBulkConsumers) {
    const int issued = bulk_produce<T, false>(d, d.s1_tiles, t0, t1, bsm, S, full0, empty0, lane,
                                              dead);
    if (lane == 0) bulk_drain<T, false>(d, issued, S, full0);
    return;
  }
  int slot = d.s1_seg_base[blockIdx.x];
  int cur = d.s1_tiles[t0].x;
  unsigned long long acc[kRowsPerWarp][3];
#pragma unroll
  for (int k = 0; k < kRowsPerWarp; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0ull;
  auto flush = [&]() {
    float* out = d.p1_part + (size_t)slot * 3 * RG;
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const float v = warp_sum(f2lo(acc[k][comp]) + f2hi(acc[k][comp]));
        if (lane == 0) out[comp * RG + warp * kRowsPerWarp + k] = v;
        acc[k][comp] = 0ull;
      }
    ++slot;
  };
  int i = 0;
  int key_next = cur;
  for (int t = t0; t < t1; ++t, ++i) {
    // the next tile's key is loaded one tile ahead
    const int key = key_next;
    if (t + 1 < t1) key_next = d.s1_tiles[t + 1].x;
    const int s = i % S;
    if (!dead && !mbar_wait_bounded(full0 + 8u * s, (unsigned)(i / S) & 1u, d.spin_limit)) {
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      dead = true;
    }
    const char* st = bsm + (size_t)s * L::kStage;
    if (key != cur) {
      flush();
      cur = key;
    }
    // g of the lane's eight columns, as packed pairs per component
    const ulonglong2* gp = reinterpret_cast<const ulonglong2*>(st + L::kVals) + 2 * lane;
    const ulonglong2 g0a = gp[0], g0b = gp[1], g1a = gp[64], g1b = gp[65], g2a = gp[128],
                     g2b = gp[129];
    const int2* runs = reinterpret_cast<const int2*>(st + L::kVals + L::kSide);
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
      const int row = warp * kRowsPerWarp + k;
      const int2 run = runs[row];
      const bool ok = 8 * lane >= run.x && 8 * lane < run.y;
      unsigned long long p[4];
      BulkRow<T>::get(st + (size_t)row * TW * sizeof(T), lane, ok, p);
      acc[k][0] = ffma2(p[3], g0b.y, ffma2(p[2], g0b.x, ffma2(p[1], g0a.y, ffma2(p[0], g0a.x, acc[k][0]))));
      acc[k][1] = ffma2(p[3], g1b.y, ffma2(p[2], g1b.x, ffma2(p[1], g1a.y, ffma2(p[0], g1a.x, acc[k][1]))));
      acc[k][2] = ffma2(p[3], g2b.y, ffma2(p[2], g2b.x, ffma2(p[1], g2a.y, ffma2(p[0], g2a.x, acc[k][2]))));
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8u * s);
  }
  flush();
}

// x partials, as k_pass2
template <class T>
__global__ void __launch_bounds__(kBulkThreads, 2) k_pass2_bulk(DevSim d, int S) {
  pdl_wait();
  using L = BulkLayout<T, true>;
  extern __shared__ __align__(128) char bsm[];
  __shared__ __align__(8) unsigned long long bar_full[kBulkMaxStages], bar_empty[kBulkMaxStages];
  __shared__ __align__(8) unsigned long long bar_red;   // the consumers' flush barrier
  const int t0 = d.s2_cta[blockIdx.x], t1 = d.s2_cta[blockIdx.x + 1];
  if (t0 >= t1) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full0 = (unsigned)__cvta_generic_to_shared(bar_full);
  const unsigned empty0 = (unsigned)__cvta_generic_to_shared(bar_empty);
  const unsigned redb = (unsigned)__cvta_generic_to_shared(&bar_red);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8u * s, 32);
      mbar_init(empty0 + 8u * s, kBulkConsumers);
    }
    mbar_init(redb, kBulkConsumers * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  bool dead = false;
  if (warp == kBulkConsumers) {
    const int issued = bulk_produce<T, true>(d, d.s2_tiles, t0, t1, bsm, S, full0, empty0, lane,
                                             dead);
    if (lane == 0) bulk_drain<T, true>(d, issued, S, full0);
    return;
  }
  float* red = reinterpret_cast<float*>(bsm + (size_t)S * L::kStage);   // [warp][comp][TW]
  int slot = d.s2_seg_base[blockIdx.x];
  int cur = d.s2_tiles[t0].x;
  unsigned red_phase = 0;
  // the consumers' barrier (all 256 consumer threads arrive; bounded wait)
  auto consumers_sync = [&]() {
    mbar_arrive(redb);
    if (!dead && !mbar_wait_bounded(redb, red_phase & 1u, d.spin_limit)) {
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      dead = true;
    }
    ++red_phase;
  };
  // per component, the lane's eight columns as four packed pairs
  unsigned long long acc[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0ull;
  auto flush = [&]() {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(red + (warp * 3 + c) * TW + 8 * lane);
      dst[0] = make_ulonglong2(acc[c][0], acc[c][1]);
      dst[1] = make_ulonglong2(acc[c][2], acc[c][3]);
      acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0ull;
    }
    consumers_sync();
    float* out = d.p2_part + (size_t)slot * 3 * TW;
    for (int idx = threadIdx.x; idx < 3 * TW; idx += kBulkConsumers * 32) {
      const int comp = idx / TW, c = idx % TW;
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < kBulkConsumers; ++w) sum += red[(w * 3 + comp) * TW + c];
      out[comp * TW + c] = sum;
    }
    consumers_sync();
    ++slot;
  };
  int i = 0;
  int key_next = cur;
  for (int t = t0; t < t1; ++t, ++i) {
    // the next tile's key is loaded one tile ahead
    const int key = key_next;
    if (t + 1 < t1) key_next = d.s2_tiles[t + 1].x;
    const int s = i % S;
    if (!dead && !mbar_wait_bounded(full0 + 8u * s, (unsigned)(i / S) & 1u, d.spin_limit)) {
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      dead = true;
    }
    const char* st = bsm + (size_t)s * L::kStage;
    if (key != cur) {
      flush();
      cur = key;
    }
    const int2* runs = reinterpret_cast<const int2*>(st + L::kVals + L::kSide);
    const float4* ys = reinterpret_cast<const float4*>(st + L::kVals);
#pragma unroll
    for (int k = 0; k < kRowsPerWarp; ++k) {
      const int row = warp * kRowsPerWarp + k;
      const int2 run = runs[row];
      const float4 y = ys[row];
      const bool ok = 8 * lane >= run.x && 8 * lane < run.y;
      unsigned long long p[4];
      BulkRow<T>::get(st + (size_t)row * TW * sizeof(T), lane, ok, p);
      const unsigned long long y0 = f2pack(y.x, y.x), y1 = f2pack(y.y, y.y), y2 = f2pack(y.z, y.z);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[0][q] = ffma2(p[q], y0, acc[0][q]);
        acc[1][q] = ffma2(p[q], y1, acc[1][q]);
        acc[2][q] = ffma2(p[q], y2, acc[2][q]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8u * s);
  }
  flush();
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

// One Jacobi sweep of A~ dq = g (the incomplete global step of the comparison in Sec. 8):
// dst_i = src_i + (g_i - (A~ src)_i) / A~_ii for the free vertices, sums in FP64.
__global__ void k_jacobi(DevSim d, const float* src, float* dst) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double r0 = d.gvec[i], r1 = d.gvec[d.n_pad + i], r2 = d.gvec[2 * d.n_pad + i], dia = 1.0;
  for (int e = d.A_ptr[i]; e < d.A_ptr[i + 1]; ++e) {
    const int j = d.A_idx[e];
    const double a = d.A_val[e];
    if (j == i) dia = a;
    r0 -= a * src[3 * j];
    r1 -= a * src[3 * j + 1];
    r2 -= a * src[3 * j + 2];
  }
  dst[3 * i] = (float)(src[3 * i] + r0 / dia);
  dst[3 * i + 1] = (float)(src[3 * i + 1] + r1 / dia);
  dst[3 * i + 2] = (float)(src[3 * i + 2] + r2 / dia);
}

}  // namespace

void launch_jacobi(const DevSim& d, cudaStream_t s) {
  float* a = d.dq;
  float* b = d.dq_alt;
  for (int k = 0; k < d.jacobi_sweeps; ++k) {
    launch_k(d.pdl, k_jacobi, (d.n + 255) / 256, 256, 0, s, d, (const float*)a, b);
    std::swap(a, b);
  }
  if (a != d.dq) cudaMemcpyAsync(d.dq, a, 3 * sizeof(float) * (size_t)d.n, cudaMemcpyDeviceToDevice, s);
}

int sinv_setup() {
  // pass 1 stages the g slices of a CTA's column tiles: up to 3 KB per tile of its range
  const int most = kMaxStagedCols * 3 * TW * (int)sizeof(float);
  const void* fns[] = {(const void*)k_pass1<float, 2>, (const void*)k_pass1<float, 1>,
                       (const void*)k_pass1<float, 4>, (const void*)k_pass1<unsigned short, 4>,
                       (const void*)k_pass1<unsigned short, 2>,
                       (const void*)k_pass1<unsigned short, 8>};
  for (const void* f : fns)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most) != cudaSuccess)
      return SIM_ECUDA;
  // the bulk-copy forms may take all of a block's shared memory beside their static part
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void* bulk[] = {(const void*)k_pass1_bulk<float>, (const void*)k_pass1_bulk<unsigned short>,
                        (const void*)k_pass2_bulk<float>, (const void*)k_pass2_bulk<unsigned short>};
  int dyn_max = optin;
  for (const void* f : bulk) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return SIM_ECUDA;
    dyn_max = std::min(dyn_max, optin - (int)fa.sharedSizeBytes);
  }
  for (const void* f : bulk)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) !=
        cudaSuccess)
      return SIM_ECUDA;
  g_bulk_smem_max = dyn_max;
  return SIM_OK;
}

// stages of a bulk-copy product with `grid` CTAs over the device's SMs (the CTAs of one
// wave share an SM's shared memory); 0 if fewer than two fit
template <class T, bool kPass2>
int bulk_stages(const DevSim& d, int grid) {
  using L = BulkLayout<T, kPass2>;
  const int per_sm = std::max(1, (grid + d.n_sm - 1) / d.n_sm);
  const int budget = std::min(g_bulk_smem_max, kSmemPerSm / per_sm - 1024 - 256) - L::kRed;
  const int S = std::min(kBulkMaxStages, budget / L::kStage);
  return S >= 2 ? S : 0;
}

template <class T>
bool launch_pass1_bulk(const DevSim& d, cudaStream_t s) {
  const int S = bulk_stages<T, false>(d, d.s1_grid);
  if (!S) return false;
  launch_k(d.pdl, k_pass1_bulk<T>, d.s1_grid, kBulkThreads,
           (size_t)S * BulkLayout<T, false>::kStage, s, d, S);
  return true;
}

template <class T>
bool launch_pass2_bulk(const DevSim& d, cudaStream_t s) {
  const int S = bulk_stages<T, true>(d, d.s2_grid);
  if (!S) return false;
  launch_k(d.pdl, k_pass2_bulk<T>, d.s2_grid, kBulkThreads,
           (size_t)S * BulkLayout<T, true>::kStage + BulkLayout<T, true>::kRed, s, d, S);
  return true;
}

// unroll: 1 = the format's default tiles in flight, 0 = half of it, 2 = twice; kUnrollBulk:
// the bulk-copy form (the register form where its stages do not fit)
void launch_pass1(const DevSim& d, cudaStream_t s) {
  const size_t smem = (size_t)d.s1_max_cols * 3 * TW * sizeof(float);
  const int g = d.s1_grid;
  if (d.s1_unroll == kUnrollBulk &&
      (d.s_bf16 ? launch_pass1_bulk<unsigned short>(d, s) : launch_pass1_bulk<float>(d, s)))
    return;
  if (d.s_bf16) {
    if (d.s1_unroll == 2) launch_k(d.pdl, k_pass1<unsigned short, 8>, g, 256, smem, s, d);
    else if (d.s1_unroll == 1) launch_k(d.pdl, k_pass1<unsigned short, 4>, g, 256, smem, s, d);
    else launch_k(d.pdl, k_pass1<unsigned short, 2>, g, 256, smem, s, d);
  } else {
    if (d.s1_unroll == 2) launch_k(d.pdl, k_pass1<float, 4>, g, 256, smem, s, d);
    else if (d.s1_unroll == 1) launch_k(d.pdl, k_pass1<float, 2>, g, 256, smem, s, d);
    else launch_k(d.pdl, k_pass1<float, 1>, g, 256, smem, s, d);
  }
}

void launch_reduce1(const DevSim& d, cudaStream_t s) {
  launch_k(d.pdl, k_reduce1, (d.n_pad + 255) / 256, 256, 0, s, d);
}

void launch_pass2(const DevSim& d, cudaStream_t s) {
  const int g = d.s2_grid;
  if (d.s2_unroll == kUnrollBulk &&
      (d.s_bf16 ? launch_pass2_bulk<unsigned short>(d, s) : launch_pass2_bulk<float>(d, s)))
    return;
  if (d.s_bf16) {
    if (d.s2_unroll == 2) launch_k(d.pdl, k_pass2<unsigned short, 8>, g, 256, kP2Smem, s, d);
    else if (d.s2_unroll == 1) launch_k(d.pdl, k_pass2<unsigned short, 4>, g, 256, kP2Smem, s, d);
    else launch_k(d.pdl, k_pass2<unsigned short, 2>, g, 256, kP2Smem, s, d);
  } else {
    if (d.s2_unroll == 2) launch_k(d.pdl, k_pass2<float, 4>, g, 256, kP2Smem, s, d);
    else if (d.s2_unroll == 1) launch_k(d.pdl, k_pass2<float, 2>, g, 256, kP2Smem, s, d);
    else launch_k(d.pdl, k_pass2<float, 1>, g, 256, kP2Smem, s, d);
  }
}

void launch_reduce2(const DevSim& d, cudaStream_t s, int out_mode) {
  const int g = (d.n + 255) / 256;
  switch (out_mode) {
    case kOutDq: launch_k(d.pdl, k_reduce2<kOutDq>, g, 256, 0, s, d); break;
    case kOutX: launch_k(d.pdl, k_reduce2<kOutX>, g, 256, 0, s, d); break;
    case kOutAddDq: launch_k(d.pdl, k_reduce2<kOutAddDq>, g, 256, 0, s, d); break;
    default: launch_k(d.pdl, k_reduce2<kOutAddX>, g, 256, 0, s, d); break;
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

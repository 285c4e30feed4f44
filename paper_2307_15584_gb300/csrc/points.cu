// points.cu -- materialised low-discrepancy points (HBM-write bound).
//
//   sobol_points_*    Alg. 3 / Eq. (ts): y_j(i) = XOR of the generator columns
//                     selected by the bits of i, randomised in integers
//                     (Sec. 2.3), mapped to [0,1) (Sec. 2.1).
//   lattice_points_*  Eq. (R1LS) / Alg. 4: x_j(k) = phi_2(k) g_j + shift_j mod 2^32.
//
// Fast path layout.  Output rows are [count][s] u32/f32.  A warp writes a
// "group" of Q = 128 / gcd(s,128) consecutive points per step: Q*s = 128*K
// elements, i.e. K 16-byte chunks per lane, so every store is a coalesced
// 128-bit store.  Lane l owns chunks l, l+32, .. of the group; element e of
// a group is point p_e = e / s, dimension j_e = e % s, the same in every group.
//
// Linearity over GF(2) makes the per-element cost O(1): for a group starting
// at enumeration index G*Q (index_begin is a multiple of Q), the bits of the
// enumeration index J split into three disjoint fields,
//   J = (G_hi << (u + q)) | (G_in << q) | p_e,   G_in < 2^u, p_e < Q,
// and y_j(i) = Hout_j(G_hi) ^ Hin_j[G_in] ^ lo_e for i = (J << col0) | pconst.
// lo_e (which also carries the fixed low part pconst) is fixed per lane, Hin
// is a shared-memory table of 2^u rows, and Hout changes once every 2^u groups,
// by the columns of the G_hi bits that flip.  G_hi takes up to 64 bits (Alg. 3's
// wide indices).  For the lattice, phi_2 of disjoint bit fields adds without
// carries, so x = phi_2(G*Q) g_j + lo_e with one bit reversal per group.
#include <cstdint>
#include <mutex>
#include <vector>

#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void store4(uint32_t* out_u32, float* out_f32, uint64_t off,
                                       const uint32_t (&v)[4]) {
  if (out_u32) __stcs(reinterpret_cast<uint4*>(out_u32 + off), make_uint4(v[0], v[1], v[2], v[3]));
  if (out_f32)
    __stcs(reinterpret_cast<float4*>(out_f32 + off),
           make_float4(map_u32_to_unifloat(v[0]), map_u32_to_unifloat(v[1]),
                       map_u32_to_unifloat(v[2]), map_u32_to_unifloat(v[3])));
}

__device__ __forceinline__ void store1(uint32_t* out_u32, float* out_f32, uint64_t off,
                                       uint32_t v) {
  if (out_u32) out_u32[off] = v;
  if (out_f32) out_f32[off] = map_u32_to_unifloat(v);
}

// --- TMA bulk stores (cp.async.bulk): shared memory -> global, asynchronous ---
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one bulk group may still be reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every bulk group of this thread has completed its global writes
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Build-time choices of the Sobol' store path: TMA bulk stores from staged
// shared-memory tiles (1) or direct 128-bit stores (0), and the groups per
// staged tile (per warp, double-buffered).  Measured on GB300 at s = 32, 2^24
// points, u32 + f32: direct stores 0.714 ms; TMA with 1 / 2 / 4 / 8 groups per
// tile 0.726 / 0.728 / 0.653 / 0.866 ms (4 groups: 2 KiB bulk stores, 2 CTAs per
// SM; 8 groups: 1 CTA per SM).
#ifndef QMC_POINTS_TMA
#define QMC_POINTS_TMA 1
#endif
#ifndef QMC_POINTS_STAGE_GROUPS
#define QMC_POINTS_STAGE_GROUPS 4
#endif
constexpr bool kPointsTma = QMC_POINTS_TMA != 0;
constexpr uint32_t kStageGroups = QMC_POINTS_STAGE_GROUPS;

// This warp's contiguous share [g0, g1) of n_groups groups.
__device__ __forceinline__ void warp_range(uint64_t n_groups, uint64_t& g0, uint64_t& g1) {
  const uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t W = (uint64_t)gridDim.x * (blockDim.x >> 5);
  g0 = n_groups * w / W;
  g1 = n_groups * (w + 1) / W;
}

// Per-warp staging of full groups for TMA bulk stores: two tiles of
// kStageGroups groups (u32 and f32 halves) in shared memory; lane 0 sends a
// full tile with one bulk store per output, and the warp refills a tile once
// the copy engine has read it.  Calls are warp-uniform.
template <int K>
struct WarpStager {
  static constexpr uint32_t kTileWords = kStageGroups * 128u * K;  // one output of one tile
  static constexpr uint32_t kWarpWords = 4 * kTileWords;           // [2 tiles][2 outputs]
  uint32_t* base;
  uint32_t tile, staged;
  uint64_t tile_off;  // global element offset of the tile's first group

  __device__ explicit WarpStager(uint32_t* warp_base) : base(warp_base), tile(0), staged(0), tile_off(0) {}

  // chunk c (elements 4 (lane + 32 c) .. +3) of the group being staged
  __device__ __forceinline__ void put(uint32_t lane, int c, const uint32_t (&v)[4]) {
    uint32_t* t = base + tile * 2 * kTileWords + staged * 128u * K + 4u * (lane + 32u * c);
    *reinterpret_cast<uint4*>(t) = make_uint4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(t + kTileWords) =
        make_float4(map_u32_to_unifloat(v[0]), map_u32_to_unifloat(v[1]), map_u32_to_unifloat(v[2]),
                    map_u32_to_unifloat(v[3]));
  }

  // the group at element offset off (this lane's first element) is complete;
  // `last`: no further full group of this warp follows
  __device__ __forceinline__ void group_done(uint32_t lane, uint64_t off, bool last, uint32_t* out_u32,
                                             float* out_f32) {
    if (staged == 0) tile_off = off - 4u * lane;
    if (++staged == kStageGroups || last) flush(lane, out_u32, out_f32);
  }

  __device__ __forceinline__ void flush(uint32_t lane, uint32_t* out_u32, float* out_f32) {
    fence_smem_to_async();
    __syncwarp();
    if (lane == 0) {
      const uint32_t bytes = staged * 128u * K * 4u;
      const uint32_t* t = base + tile * 2 * kTileWords;
      if (out_u32) bulk_store(out_u32 + tile_off, t, bytes);
      if (out_f32) bulk_store(out_f32 + tile_off, t + kTileWords, bytes);
      bulk_commit();
      bulk_wait_read_1();  // the other tile's previous copy has read its source
    }
    __syncwarp();
    tile ^= 1u;
    staged = 0;
  }

  // every bulk store of this warp has completed before the kernel ends
  __device__ __forceinline__ void finish(uint32_t lane) {
    if (lane == 0) bulk_wait_all();
  }
};

// ---------------------------------------------------------------------------
// K1 fast path.  MODE: 0 none, 1 XOR, 2 nested.  K: 16-byte chunks per lane.
// Shared memory: cols[s][m] (mirrored for nested), hin[2^u][s], pc[s].  Table
// entries for index bits at or above m stay zero: no enumerated index sets them.
// ---------------------------------------------------------------------------
// TMA: full groups go through a WarpStager (bulk stores from shared memory).
template <int K, int MODE, bool V4, bool TMA>  // V4: s % 4 == 0, chunks hold 4 consecutive dimensions
__global__ void __launch_bounds__(kThreads) sobol_points_fast(PointsArgs a) {
  extern __shared__ __align__(128) uint32_t smem[];
  const uint32_t s = a.s;
  const uint32_t nin = 1u << a.u_log2;
  // [warps][WarpStager words], then the tables
  uint32_t* cols = smem + (TMA ? (kThreads / 32) * WarpStager<K>::kWarpWords : 0);
  const uint32_t m = a.m;
  uint32_t* hin = cols + s * m;
  uint32_t* pc = hin + nin * s;

  for (uint32_t idx = threadIdx.x; idx < s * m; idx += blockDim.x) {
    const uint32_t c = __ldg(a.matrices + idx);
    cols[idx] = (MODE == 2) ? __brev(c) : c;
  }
  __syncthreads();
  const uint32_t cin = a.col0 + a.q_log2;  // column of the lowest G_in bit
  for (uint32_t idx = threadIdx.x; idx < nin * s; idx += blockDim.x) {
    const uint32_t g = idx / s, j = idx - g * s;
    uint32_t y = 0;
    for (uint32_t k = 0; (g >> k) != 0 && cin + k < m; ++k)
      if ((g >> k) & 1u) y ^= cols[j * m + cin + k];
    hin[idx] = y;
  }
  for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) {
    uint32_t y = 0;
    for (uint32_t k = 0; k < a.col0; ++k)
      if ((a.pconst >> k) & 1u) y ^= cols[j * m + k];
    pc[j] = y;
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t Q = 1u << a.q_log2;
  uint32_t jd[4 * K], lo[4 * K], hout[4 * K];
  NestedKey key[4 * K];
#pragma unroll
  for (int c = 0; c < K; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t e = 4u * (lane + 32u * c) + t;
      const uint32_t p = e / s, j = e - p * s;
      uint32_t y = pc[j];
      for (uint32_t k = 0; k < a.q_log2 && a.col0 + k < m; ++k)
        if ((p >> k) & 1u) y ^= cols[j * m + a.col0 + k];
      if (MODE == 1) y ^= __ldg(a.seeds + j);
      jd[4 * c + t] = j;
      lo[4 * c + t] = y;
      key[4 * c + t] = nested_key(MODE == 2 ? __ldg(a.seeds + j) : 0u);
    }

  const uint64_t n_groups = (a.count + Q - 1) >> a.q_log2;
  const uint64_t full_groups = a.count >> a.q_log2;  // groups whose Q rows all exist
  uint64_t g0, g1;
  warp_range(n_groups, g0, g1);
  const uint64_t G_first = a.index_begin >> a.q_log2;
  const uint32_t hi_col = a.col0 + a.q_log2 + a.u_log2;  // column of the lowest G_hi bit
  const uint64_t step = (uint64_t)Q * s;  // elements per group
  uint64_t off = g0 * step + 4u * lane;   // this lane's first element in group g0

  WarpStager<K> stager(smem + (threadIdx.x >> 5) * WarpStager<K>::kWarpWords);

  for (uint64_t g = g0; g < g1; ++g, off += step) {
    const uint64_t G = G_first + g;
    const uint32_t G_in = (uint32_t)G & (nin - 1u);
    if (g == g0) {
      const uint64_t G_hi = G >> a.u_log2;  // below 2^(m - hi_col) for every enumerated group
#pragma unroll
      for (int e = 0; e < 4 * K; ++e) {
        uint32_t y = 0;
        for (uint32_t k = 0; (G_hi >> k) != 0; ++k)
          if ((G_hi >> k) & 1u) y ^= cols[jd[e] * m + hi_col + k];
        hout[e] = y;
      }
    } else if (G_in == 0) {
      // G_hi advanced by one: exactly the bits of G_hi ^ (G_hi - 1) flipped
      // (the trailing ones and the bit above them), two on average.
      const uint64_t G_hi = G >> a.u_log2;
      const uint32_t nflip = (uint32_t)__ffsll((long long)G_hi);  // G_hi > 0 here
#pragma unroll
      for (int e = 0; e < 4 * K; ++e) {
        uint32_t y = hout[e];
        for (uint32_t k = 0; k < nflip; ++k) y ^= cols[jd[e] * m + hi_col + k];
        hout[e] = y;
      }
    }
    const uint32_t* hrow = hin + G_in * s;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      uint32_t h[4];
      if (V4) {  // four consecutive dimensions: one 128-bit shared-memory load
        const uint4 q = *reinterpret_cast<const uint4*>(hrow + jd[4 * c]);
        h[0] = q.x, h[1] = q.y, h[2] = q.z, h[3] = q.w;
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) h[t] = hrow[jd[4 * c + t]];
      }
      uint32_t v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        uint32_t y = h[t] ^ hout[4 * c + t] ^ lo[4 * c + t];
        if (MODE == 2) y = __brev(nested_mix(y, key[4 * c + t]));
        v[t] = y;
      }
      const uint64_t o = off + 128u * c;
      if (g < full_groups) {
        if (TMA)
          stager.put(lane, c, v);
        else
          store4(a.out_u32, a.out_f32, o, v);
      } else {  // ragged last group: per-element row test
        const uint64_t rows_left = a.count - (g << a.q_log2);
        const uint32_t e0 = 4u * (lane + 32u * c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if ((uint64_t)((e0 + t) / s) < rows_left) store1(a.out_u32, a.out_f32, o + t, v[t]);
      }
    }
    if (TMA && g < full_groups)
      stager.group_done(lane, off, g + 1 == g1 || g + 1 == full_groups, a.out_u32, a.out_f32);
  }
  if (TMA) stager.finish(lane);
}

// K1 generic path: one element per thread, columns read through the cache.
template <int MODE>
__global__ void __launch_bounds__(kThreads) sobol_points_generic(PointsArgs a) {
  const uint64_t total = a.count * a.s;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
    const uint64_t r = f / a.s;
    const uint32_t j = (uint32_t)(f - r * a.s);
    uint64_t i = ((a.index_begin + r) << a.col0) | a.pconst;  // below 2^m (checked by the caller)
    const uint32_t* Cj = a.matrices + (uint64_t)j * a.m;
    uint32_t y = 0;
    for (; i != 0; i &= i - 1u) y ^= __ldg(Cj + (__ffsll((long long)i) - 1));
    if (MODE == 1) y ^= __ldg(a.seeds + j);
    if (MODE == 2) y = __brev(nested_mix(__brev(y), nested_key(__ldg(a.seeds + j))));
    store1(a.out_u32, a.out_f32, f, y);
  }
}

// ---------------------------------------------------------------------------
// K2: rank-1 lattice.  BACKWARD follows Alg. 4: phi_2(~k) = ~phi_2(k), so
// x = shift - g - phi_2(k) g (mod 2^32).
// ---------------------------------------------------------------------------
template <int K, bool BACKWARD, bool TMA>
__global__ void __launch_bounds__(kThreads) lattice_points_fast(PointsArgs a) {
  extern __shared__ __align__(128) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  WarpStager<K> stager(smem + (threadIdx.x >> 5) * WarpStager<K>::kWarpWords);
  const uint32_t s = a.s;
  const uint32_t Q = 1u << a.q_log2;
  uint32_t gj[4 * K], lo[4 * K];
#pragma unroll
  for (int c = 0; c < K; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t e = 4u * (lane + 32u * c) + t;
      const uint32_t p = e / s, j = e - p * s;
      const uint32_t g = __ldg(a.matrices + j) | 1u;  // generator words
      const uint32_t sh = a.seeds ? __ldg(a.seeds + j) : 0u;
      const uint32_t phi_p = __brev(p);
      gj[4 * c + t] = g;
      lo[4 * c + t] = BACKWARD ? sh - g - phi_p * g : phi_p * g + sh;
    }
  const uint64_t n_groups = (a.count + Q - 1) >> a.q_log2;
  const uint64_t full_groups = a.count >> a.q_log2;
  uint64_t g0, g1;
  warp_range(n_groups, g0, g1);
  const uint32_t G_first = (uint32_t)(a.index_begin >> a.q_log2);
  const uint64_t step = (uint64_t)Q * s;
  uint64_t off = g0 * step + 4u * lane;
  for (uint64_t g = g0; g < g1; ++g, off += step) {
    const uint32_t phib = __brev((G_first + (uint32_t)g) << a.q_log2);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      uint32_t v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        v[t] = BACKWARD ? lo[4 * c + t] - phib * gj[4 * c + t] : phib * gj[4 * c + t] + lo[4 * c + t];
      const uint64_t o = off + 128u * c;
      if (g < full_groups) {
        if (TMA)
          stager.put(lane, c, v);
        else
          store4(a.out_u32, a.out_f32, o, v);
      } else {  // ragged last group: per-element row test
        const uint64_t rows_left = a.count - (g << a.q_log2);
        const uint32_t e0 = 4u * (lane + 32u * c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if ((uint64_t)((e0 + t) / s) < rows_left) store1(a.out_u32, a.out_f32, o + t, v[t]);
      }
    }
    if (TMA && g < full_groups)
      stager.group_done(lane, off, g + 1 == g1 || g + 1 == full_groups, a.out_u32, a.out_f32);
  }
  if (TMA) stager.finish(lane);
}

template <bool BACKWARD>
__global__ void __launch_bounds__(kThreads) lattice_points_generic(PointsArgs a) {
  const uint64_t total = a.count * a.s;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
    const uint64_t r = f / a.s;
    const uint32_t j = (uint32_t)(f - r * a.s);
    const uint32_t k = (uint32_t)a.index_begin + (uint32_t)r;
    const uint32_t phi = __brev(BACKWARD ? ~k : k);
    const uint32_t g = __ldg(a.matrices + j) | 1u;
    const uint32_t sh = a.seeds ? __ldg(a.seeds + j) : 0u;
    store1(a.out_u32, a.out_f32, f, phi * g + sh);
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// Pixel-shifted lattice, coalesced path (s % 4 == 0, 16-byte aligned outputs,
// 32 spp s <= 2^31).  A warp takes batches of 32 consecutive pixels: lane l
// computes the shift of pixel l of the batch once (Hilbert position, then
// phi_3), and the batch's 32 spp rows are written as consecutive 16-byte chunks,
// each chunk's pixel shift fetched from its lane with a shuffle.
__global__ void __launch_bounds__(kThreads) pixel_lattice_points_fast(PixelPointsArgs a) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t n_batches = (a.n_pixels + 31) >> 5;
  uint64_t b0, b1;
  warp_range(n_batches, b0, b1);
  // x / d = umulhi(x, floor(2^64 / d) + 1) exactly for x < 2^32 and d > 1
  const uint64_t mag_s = ~0ull / a.s + 1;  // s >= 4
  const uint64_t mag_spp = a.spp > 1 ? ~0ull / a.spp + 1 : 0;
  const uint32_t chunks_per_pixel = a.spp * (a.s >> 2);
  for (uint64_t b = b0; b < b1; ++b) {
    const uint64_t first = b << 5;  // batch's first pixel, relative to pixel_begin
    const uint64_t left = a.n_pixels - first;
    const uint32_t npx = left < 32 ? (uint32_t)left : 32u;
    uint32_t sh = 0;
    if (lane < npx) {
      const uint64_t p = a.pixel_begin + first + lane;
      sh = pixel_shift((uint32_t)(p % a.width), (uint32_t)(p / a.width), a.grid_log2);
    }
    const uint32_t chunks = npx * chunks_per_pixel;
    const uint64_t off0 = first * a.spp * a.s;  // element offset of the batch
    for (uint32_t c0 = 0; c0 < chunks; c0 += 32) {  // same trip count in every lane
      const uint32_t c = c0 + lane;
      const uint32_t e = 4u * c;  // element within the batch, < 2^32
      const uint32_t row = (uint32_t)__umul64hi(e, mag_s);
      const uint32_t j = e - row * a.s;
      const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
      const uint32_t smp = row - pl * a.spp;
      const uint32_t shift = __shfl_sync(0xffffffffu, sh, pl & 31u);
      if (c < chunks) {
        const uint32_t base = __brev(smp) + shift;
        const uint32_t v[4] = {base * (__ldg(a.g + j) | 1u), base * (__ldg(a.g + j + 1) | 1u),
                               base * (__ldg(a.g + j + 2) | 1u), base * (__ldg(a.g + j + 3) | 1u)};
        store4(a.out_u32, a.out_f32, off0 + e, v);
      }
    }
  }
}


// Pixel-shifted rank-1 lattice (Sec. 3): one thread per (pixel, sample) row;
// row r holds sample r % spp of pixel pixel_begin + r / spp.
__global__ void __launch_bounds__(kThreads) pixel_lattice_points_kernel(PixelPointsArgs a) {
  const uint64_t rows = a.n_pixels * a.spp;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    const uint64_t p = a.pixel_begin + r / a.spp;
    const uint32_t i = (uint32_t)(r % a.spp);
    const uint32_t shift = pixel_shift((uint32_t)(p % a.width), (uint32_t)(p / a.width), a.grid_log2);
    const uint32_t base = __brev(i) + shift;
    for (uint32_t j = 0; j < a.s; ++j) store1(a.out_u32, a.out_f32, r * a.s + j, base * (__ldg(a.g + j) | 1u));
  }
}

// Halton points: element (r, j) = phi_b(i') of index
// i = ((index_begin + r) << q) | pconst (q > 0: one element of a sequence
// partitioned by its base-2 dimension, Sec. 2.5.1) with b the (dim0 + j)-th
// prime; digits permuted (Faure table or linear multiplier), i' = i mod 2^32
// for b = 2 (the bit reversal of the low 32 bits), otherwise i mod b^K with b^K
// the largest power below 2^32 (Alg. 1's domain limit).
//
// Multi-digit tables (Sec. 2.2): the K digits of i' are taken in G groups of L
// digits (the most significant group holding the remaining L' digits), and a
// table per output dimension maps a group to its permuted, mirrored L-digit
// numerator, so the K-digit numerator N = sum_k sigma(d_k) b^(K-1-k) is a
// G-step Horner sum of table entries.  The tables depend on the call's
// permutation; each block builds them in shared memory.  Divisions by b^L and
// by b^K use multiply-high reciprocals (exact for 32-bit operands), and the
// result floor(N 2^32 / b^K) one multiply-high plus a remainder correction.
constexpr uint32_t kHaltonPermWords = 8896;  // sum of the first 64 primes (8893), rounded up
constexpr uint32_t kHaltonGroupCap = 1024;   // largest table (b^L) for bases that allow L >= 2
struct HaltonTables {
  uint32_t base[kHaltonMaxDims];
  uint32_t max_power[kHaltonMaxDims];  // b^K: the largest power of the base below 2^32
  uint32_t perm_off[kHaltonMaxDims];   // Faure table of dimension j at perm[perm_off[j]]
  uint32_t digits[kHaltonMaxDims];     // L, digits per full group
  uint32_t groups[kHaltonMaxDims];     // G
  uint32_t top_digits[kHaltonMaxDims]; // L', digits of the most significant group (1 <= L' <= L)
  uint32_t group_pow[kHaltonMaxDims];  // b^L
  uint32_t top_pow[kHaltonMaxDims];    // b^L'
  uint64_t magic_group[kHaltonMaxDims];  // floor(2^64 / b^L) + 1: x / b^L = umulhi(x, .) for x < 2^32
  uint64_t magic_max[kHaltonMaxDims];    // floor(2^64 / b^K) + 1: the same for b^K
  uint64_t scale[kHaltonMaxDims];        // floor(2^64 / b^K): floor(N 2^32 / b^K) up to one correction
  uint16_t perm[kHaltonPermWords];
};
__device__ HaltonTables g_halton;

// Work layout.  A block takes tiles of R rows (R a multiple of 128).  A warp
// takes one output dimension for 128 rows of the tile at a time, so its lanes
// share the dimension's constants and group count, and each lane carries four
// independent rows (lane, lane+32, ..) through the group loop.  Results go to a
// shared-memory tile [R][s] (odd row stride: no bank conflicts), which the block
// then writes out with coalesced stores.
constexpr uint32_t kHaltonRowsPerUnit = 128;

// floor(N 2^32 / b^K) for N < b^K <= 2^32: one multiply-high by floor(2^64 / b^K)
// is at most one below; the remainder decides.
__device__ __forceinline__ uint32_t halton_scale(uint32_t N, uint32_t mp, uint64_t scale) {
  const uint64_t num = (uint64_t)N << 32;
  uint64_t w = __umul64hi(num, scale);
  if (num - w * mp >= mp) ++w;
  return (uint32_t)w;
}

__global__ void __launch_bounds__(kThreads) halton_points_kernel(HaltonArgs p) {
  extern __shared__ __align__(16) uint32_t hsmem[];
  uint32_t* stage = hsmem;                                            // [R][stride]
  uint16_t* htab = reinterpret_cast<uint16_t*>(hsmem + p.stage_words);  // digit-group tables
  for (uint32_t jo = 0; jo < p.s; ++jo) {
    const uint32_t j = p.dim0 + jo;
    const uint32_t b = g_halton.base[j];
    if (b == 2) continue;
    const uint32_t bL = g_halton.group_pow[j], bLp = g_halton.top_pow[j];
    const uint32_t poff = g_halton.perm_off[j];
    uint16_t* t = htab + p.table_off[jo];
    for (uint32_t e = threadIdx.x; e < bL + bLp; e += blockDim.x) {
      const bool top = e >= bL;
      uint32_t x = top ? e - bL : e;
      const uint32_t nd = top ? g_halton.top_digits[j] : g_halton.digits[j];
      uint32_t num = 0;
      for (uint32_t k = 0; k < nd; ++k) {  // lowest digit first: it becomes the most significant
        uint32_t d = x % b;
        x /= b;
        if (p.mode == 1) d = g_halton.perm[poff + d];
        else if (p.mode == 2) d = (p.mult[jo] * d) % b;
        num = num * b + d;
      }
      t[e] = (uint16_t)num;
    }
  }

  const uint32_t s = p.s, R = p.tile_rows, stride = p.stage_stride;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const uint32_t units = s * (R / kHaltonRowsPerUnit);
  const uint64_t mag_s = s > 1 ? ~0ull / s + 1 : 0;  // e / s for e < 2^32
  const uint64_t n_tiles = (p.count + R - 1) / R;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t row0 = tile * R;
    const uint64_t left = p.count - row0;
    const uint32_t rows = left < R ? (uint32_t)left : R;
    __syncthreads();  // tables built / the previous tile written out
    for (uint32_t u = warp; u < units; u += warps) {
      const uint32_t jo = u / (R / kHaltonRowsPerUnit);
      const uint32_t r0 = (u - jo * (R / kHaltonRowsPerUnit)) * kHaltonRowsPerUnit + lane;
      const uint32_t j = p.dim0 + jo;
      const uint32_t b = g_halton.base[j];
      uint32_t v[4];
      if (b == 2) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = __brev((uint32_t)(((p.index_begin + row0 + r0 + 32u * c) << p.q) | p.pconst));
      } else {
        const uint32_t mp = g_halton.max_power[j], bL = g_halton.group_pow[j], G = g_halton.groups[j];
        const uint64_t mg = g_halton.magic_group[j], mm = g_halton.magic_max[j];
        const uint16_t* t = htab + p.table_off[jo];
        uint32_t x[4], N[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint64_t i = ((p.index_begin + row0 + r0 + 32u * c) << p.q) | p.pconst;
          x[c] = (i >> 32) ? (uint32_t)(i % mp) : (uint32_t)i - mp * (uint32_t)__umul64hi((uint32_t)i, mm);
          N[c] = 0;
        }
        for (uint32_t m = 1; m < G; ++m) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t q = (uint32_t)__umul64hi(x[c], mg);
            N[c] = N[c] * bL + t[x[c] - q * bL];
            x[c] = q;
          }
        }
        const uint32_t bLp = g_halton.top_pow[j];
        const uint64_t sc = g_halton.scale[j];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = halton_scale(N[c] * bLp + t[bL + x[c]], mp, sc);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) stage[(r0 + 32u * c) * stride + jo] = v[c];
    }
    __syncthreads();
    const uint32_t elems = rows * s;
    for (uint32_t e = threadIdx.x; e < elems; e += blockDim.x) {
      const uint32_t r = s > 1 ? (uint32_t)__umul64hi(e, mag_s) : e;
      store1(p.out_u32, p.out_f32, row0 * s + e, stage[r * stride + (e - r * s)]);
    }
  }
}

// Chunks per lane of the fast path, or 0 when the generic path must run.
uint32_t fast_k(uint32_t s) {
  uint32_t g = 128;
  while (s % g) g >>= 1;  // gcd(s, 128): the largest power of two dividing both
  const uint32_t K = s / g;
  return K <= 4 ? K : 0;
}

uint32_t log2_exact(uint32_t v) {
  uint32_t l = 0;
  while ((1u << l) < v) ++l;
  return l;
}

template <typename KernelT>
cudaError_t launch_persistent(KernelT kernel, uint64_t warps_needed, size_t smem,
                              cudaStream_t stream, const PointsArgs& a) {
  const DeviceInfo& dev = device_info();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t blocks = (uint64_t)dev.sm_count * per_sm;
  const uint64_t need = (warps_needed + kThreads / 32 - 1) / (kThreads / 32);
  if (need < blocks) blocks = need;
  if (blocks < 1) blocks = 1;
  kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

// True for device (or managed) memory and for null; false for host memory the
// GPU reaches through the interconnect (pinned or registered host buffers).
bool device_resident(const void* p) {
  if (!p) return true;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

template <typename KernelT>
cudaError_t launch_grid_stride(KernelT kernel, uint64_t elements, cudaStream_t stream,
                               const PointsArgs& a) {
  const DeviceInfo& dev = device_info();
  uint64_t blocks = (elements + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)dev.sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sobol_points(PointsArgs a, cudaStream_t stream) {
  const uint32_t K = fast_k(a.s);
  a.q_log2 = log2_exact(K ? 128u * K / a.s : 1u);
  bool fast = K != 0 && a.s <= 256 && (a.index_begin & ((1ull << a.q_log2) - 1u)) == 0 &&
              aligned16(a.out_u32) && aligned16(a.out_f32);
  // inner table of at most 16 KiB and 256 rows
  uint32_t u = 0;
  while (u < 8 && (2u << u) * a.s * 4u <= 16384u) ++u;
  a.u_log2 = u;
  // TMA bulk stores target device memory; outputs in host memory that the GPU
  // writes directly (pinned, mapped) take the 128-bit store path.
  bool tma = kPointsTma && device_resident(a.out_u32) && device_resident(a.out_f32);
  const size_t table_words = (size_t)a.s * a.m + ((size_t)1 << u) * a.s + a.s;
  const size_t stage_words = (size_t)(kThreads / 32) * 4 * kStageGroups * 128u * K;
  const size_t optin = device_info().smem_per_block_optin;
  if (tma && (stage_words + table_words) * sizeof(uint32_t) > optin) tma = false;
  if (table_words * sizeof(uint32_t) > optin) fast = false;
  if (!fast) {
    switch (a.scramble) {
      case 0: return launch_grid_stride(sobol_points_generic<0>, a.count * a.s, stream, a);
      case 1: return launch_grid_stride(sobol_points_generic<1>, a.count * a.s, stream, a);
      default: return launch_grid_stride(sobol_points_generic<2>, a.count * a.s, stream, a);
    }
  }
  const size_t smem = ((tma ? stage_words : 0) + table_words) * sizeof(uint32_t);
  const uint64_t groups = (a.count + (1u << a.q_log2) - 1) >> a.q_log2;
  const bool v4 = (a.s & 3u) == 0;
#define QMC_SOBOL_MODES(KK, V, T)                                                                       \
  if (a.scramble == 0) return launch_persistent(sobol_points_fast<KK, 0, V, T>, groups, smem, stream, a); \
  if (a.scramble == 1) return launch_persistent(sobol_points_fast<KK, 1, V, T>, groups, smem, stream, a); \
  return launch_persistent(sobol_points_fast<KK, 2, V, T>, groups, smem, stream, a);
#define QMC_SOBOL_CASE(KK)                \
  case KK:                                \
    if (v4 && tma) {                      \
      QMC_SOBOL_MODES(KK, true, kPointsTma)  \
    } else if (v4) {                      \
      QMC_SOBOL_MODES(KK, true, false)    \
    } else if (tma) {                     \
      QMC_SOBOL_MODES(KK, false, kPointsTma) \
    } else {                              \
      QMC_SOBOL_MODES(KK, false, false)   \
    }
  switch (K) {
    QMC_SOBOL_CASE(1)
    QMC_SOBOL_CASE(2)
    QMC_SOBOL_CASE(3)
    QMC_SOBOL_CASE(4)
    default: return cudaErrorInvalidValue;
  }
#undef QMC_SOBOL_CASE
#undef QMC_SOBOL_MODES
}

// Faure permutations sigma_k for k = 0 .. max_k, built bottom-up from Sec. 2.2's
// rule (even k: twice sigma_{k/2}, then twice plus one; odd k: sigma_{k-1} with
// the middle value (k-1)/2 inserted and the values above it moved up).
static std::vector<std::vector<uint16_t>> faure_tables(uint32_t max_k) {
  std::vector<std::vector<uint16_t>> t(max_k + 1);
  for (uint32_t k = 0; k <= max_k; ++k) {
    if (k <= 2) {
      for (uint32_t d = 0; d < k; ++d) t[k].push_back((uint16_t)d);
    } else if (k % 2 == 0) {
      for (uint16_t v : t[k / 2]) t[k].push_back((uint16_t)(2 * v));
      for (uint16_t v : t[k / 2]) t[k].push_back((uint16_t)(2 * v + 1));
    } else {
      const uint32_t mid = (k - 1) / 2;
      for (uint32_t d = 0; d < k - 1; ++d) {
        if (d == mid) t[k].push_back((uint16_t)mid);
        const uint16_t v = t[k - 1][d];
        t[k].push_back((uint16_t)(v >= mid ? v + 1 : v));
      }
    }
  }
  return t;
}

static const std::vector<uint32_t>& first_primes() {
  static const std::vector<uint32_t> primes = [] {
    std::vector<uint32_t> v;
    for (uint32_t c = 2; v.size() < kHaltonMaxDims; ++c) {
      bool prime = true;
      for (uint32_t q : v)
        if (c % q == 0) {
          prime = false;
          break;
        }
      if (prime) v.push_back(c);
    }
    return v;
  }();
  return primes;
}

// Per-base constants of the Halton engine (host copy; g_halton holds the same),
// or null if the Faure tables would not fit their array.
static const HaltonTables* halton_host_tables() {
  static const HaltonTables* tables = [] {
    static HaltonTables h;  // ~20 KB: static storage, not the stack
    h = HaltonTables{};
    const std::vector<uint32_t>& primes = first_primes();
    const std::vector<std::vector<uint16_t>> faure = faure_tables(primes.back());
    uint32_t off = 0;
    for (uint32_t j = 0; j < kHaltonMaxDims; ++j) {
      const uint32_t b = primes[j];
      uint64_t mp = 1;
      uint32_t K = 0;
      while (mp * b <= 0xFFFFFFFFull) mp *= b, ++K;
      uint32_t L = 1;
      uint64_t bL = b;
      while (bL * b <= kHaltonGroupCap) bL *= b, ++L;
      const uint32_t G = (K + L - 1) / L, Lp = K - (G - 1) * L;
      uint64_t bLp = 1;
      for (uint32_t t = 0; t < Lp; ++t) bLp *= b;
      h.base[j] = b;
      h.max_power[j] = (uint32_t)mp;
      h.digits[j] = L;
      h.groups[j] = G;
      h.top_digits[j] = Lp;
      h.group_pow[j] = (uint32_t)bL;
      h.top_pow[j] = (uint32_t)bLp;
      h.magic_group[j] = UINT64_MAX / bL + 1;
      h.magic_max[j] = UINT64_MAX / mp + 1;
      h.scale[j] = UINT64_MAX / mp;  // mp is odd for b > 2: floor(2^64 / mp) = floor((2^64 - 1) / mp)
      h.perm_off[j] = off;
      if (off + b <= kHaltonPermWords)
        for (uint32_t d = 0; d < b; ++d) h.perm[off + d] = faure[b][d];
      off += b;
    }
    return off <= kHaltonPermWords ? &h : nullptr;  // table sized for the first 64 primes
  }();
  return tables;
}

// Writes g_halton on the current device once (synchronous copy, under a mutex).
static cudaError_t ensure_halton_tables() {
  static std::mutex mu;
  static uint64_t ready_mask = 0;  // bit d: device d holds the table
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (ready_mask & (1ull << dev)) return cudaSuccess;
  const HaltonTables* h = halton_host_tables();
  if (!h) return cudaErrorInvalidValue;
  e = cudaMemcpyToSymbol(g_halton, h, sizeof(HaltonTables));
  if (e == cudaSuccess) ready_mask |= 1ull << dev;
  return e;
}

uint32_t halton_base(uint32_t j) { return first_primes()[j]; }

cudaError_t launch_halton_points(const HaltonArgs& args, cudaStream_t stream) {
  const cudaError_t e = ensure_halton_tables();
  if (e != cudaSuccess) return e;
  const HaltonTables& h = *halton_host_tables();  // non-null: ensure_halton_tables succeeded
  HaltonArgs p = args;
  // tile rows: a multiple of 128, at least 32 units of (dimension, 128 rows) per tile
  p.tile_rows = kHaltonRowsPerUnit * ((32 + p.s - 1) / p.s > 2 ? (32 + p.s - 1) / p.s : 2);
  p.stage_stride = p.s | 1u;  // odd: the lanes of a warp hit distinct banks
  p.stage_words = p.tile_rows * p.stage_stride;
  uint32_t table_words = 0;  // uint16 entries
  for (uint32_t jo = 0; jo < p.s; ++jo) {
    const uint32_t j = p.dim0 + jo;
    p.table_off[jo] = table_words;
    if (h.base[j] != 2) table_words += h.group_pow[j] + h.top_pow[j];
  }
  const size_t smem = (size_t)p.stage_words * sizeof(uint32_t) + (size_t)table_words * sizeof(uint16_t);
  const DeviceInfo& dev = device_info();
  if (smem > dev.smem_per_block_optin) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    const cudaError_t ea =
        cudaFuncSetAttribute(halton_points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
  }
  int per_sm = 0;
  cudaError_t eo = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, halton_points_kernel, kThreads, smem);
  if (eo != cudaSuccess) return eo;
  uint64_t blocks = (uint64_t)dev.sm_count * (per_sm < 1 ? 1 : per_sm);
  const uint64_t tiles = (p.count + p.tile_rows - 1) / p.tile_rows;
  if (tiles < blocks) blocks = tiles;
  if (blocks < 1) blocks = 1;
  halton_points_kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

namespace {

// LFSR jump tables of the materialising kernels: level b advances a state by
// 32 * 2^b steps (b < kJumpLevels), each level the square of the one below, so a
// chunk reaches dimension j0 in popcount(j0) jumps.
constexpr uint32_t kJumpLevels = 5;

template <int KIND>
__device__ __forceinline__ void rlat_jump_tables_fill(uint32_t* jump) {
  if (KIND != QMC_RLAT_LFSR) return;
  lfsr_jump_table_fill(jump);
  __syncthreads();
  for (uint32_t b = 1; b < kJumpLevels; ++b) {
    const uint32_t* lower = jump + (b - 1) * kLfsrJumpWords;
    for (uint32_t e = threadIdx.x; e < kLfsrJumpWords; e += blockDim.x) {
      const uint32_t v = (e & 255u) << (8u * (e >> 8));
      jump[b * kLfsrJumpWords + e] = lfsr_jump32(lower, lfsr_jump32(lower, v));
    }
    __syncthreads();
  }
}

// Generator component j of instance k of pixel (px, py), for one chunk of
// consecutive dimensions j0 .. j0+N-1 (LFSR: 32 register steps per dimension
// from the pixel's seed state, taken through the jump tables).
template <int KIND, int N>
__device__ __forceinline__ void rlat_generators(uint32_t seed, uint32_t k, uint32_t j0, uint32_t px,
                                                uint32_t py, const uint32_t* jump, uint32_t (&g)[N]) {
  if (KIND == QMC_RLAT_HASH) {
#pragma unroll
    for (int q = 0; q < N; ++q) g[q] = rlat_hash(seed, k, j0 + q, px, py) | 1u;
  } else {
    uint32_t xi = rlat_lfsr_seed(seed, k, px, py);
#pragma unroll
    for (uint32_t b = 0; b + 1 < kJumpLevels; ++b)
      if ((j0 >> b) & 1u) xi = lfsr_jump32(jump + b * kLfsrJumpWords, xi);
    for (uint32_t u = 0; u < (j0 >> (kJumpLevels - 1)); ++u)
      xi = lfsr_jump32(jump + (kJumpLevels - 1) * kLfsrJumpWords, xi);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      g[q] = 2u * xi + 1u;
      xi = lfsr_jump32(jump, xi);
    }
  }
}

// Coalesced path (s % 4 == 0, 16-byte aligned outputs, batch_pixels spp s <= 2^31).
// A block takes batches of batch_pixels consecutive pixels: it first derives the
// generator words of every (pixel, instance, dimension) of the batch into
// shared memory ([pixel][R][s]; spp / R samples share each word), then writes
// the batch's rows as consecutive 16-byte chunks, each chunk one sample and
// four consecutive dimensions: one 128-bit shared load, four multiplies.
template <int KIND>
__global__ void __launch_bounds__(kThreads) random_lattice_points_fast(RandomPointsArgs a) {
  extern __shared__ __align__(16) uint32_t rsm[];
  uint32_t* jump = rsm;  // LFSR jump tables
  uint32_t* pxy = rsm + (KIND == QMC_RLAT_LFSR ? kJumpLevels * kLfsrJumpWords : 0);  // [batch][2]
  uint32_t* gvec = pxy + ((2 * a.batch_pixels + 3u) & ~3u);  // [batch][R][s], 16-byte aligned
  rlat_jump_tables_fill<KIND>(jump);
  const uint32_t s = a.s, R = 1u << a.r_log2, Rs = R * s;
  const uint64_t mag_s = ~0ull / s + 1;  // s >= 4
  const uint64_t mag_spp = a.spp > 1 ? ~0ull / a.spp + 1 : 0;
  const uint64_t n_batches = (a.n_pixels + a.batch_pixels - 1) / a.batch_pixels;
  for (uint64_t b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const uint64_t first = b * a.batch_pixels;
    const uint64_t left = a.n_pixels - first;
    const uint32_t npx = left < a.batch_pixels ? (uint32_t)left : a.batch_pixels;
    __syncthreads();  // the previous batch's words are no longer read
    for (uint32_t q = threadIdx.x; q < npx; q += blockDim.x) {
      const uint64_t p = a.pixel_begin + first + q;
      pxy[2 * q] = (uint32_t)(p % a.width);
      pxy[2 * q + 1] = (uint32_t)(p / a.width);
    }
    __syncthreads();
    if (KIND == QMC_RLAT_HASH) {  // every component independently
      for (uint32_t idx = threadIdx.x; idx < npx * Rs; idx += blockDim.x) {
        const uint32_t row = (uint32_t)__umul64hi(idx, mag_s);  // (pixel, instance)
        const uint32_t j = idx - row * s, q = row >> a.r_log2;
        gvec[idx] = rlat_hash(a.seed, row & (R - 1u), j, pxy[2 * q], pxy[2 * q + 1]) | 1u;
      }
    } else {  // one thread per (pixel, instance) walks the register through the dimensions
      for (uint32_t w = threadIdx.x; w < npx * R; w += blockDim.x) {
        const uint32_t q = w >> a.r_log2;
        uint32_t xi = rlat_lfsr_seed(a.seed, w & (R - 1u), pxy[2 * q], pxy[2 * q + 1]);
        for (uint32_t j = 0; j < s; ++j) {
          gvec[w * s + j] = 2u * xi + 1u;
          xi = lfsr_jump32(jump, xi);
        }
      }
    }
    __syncthreads();
    const uint32_t chunks = npx * a.spp * (s >> 2);
    const uint64_t off0 = first * a.spp * s;
    for (uint32_t c = threadIdx.x; c < chunks; c += blockDim.x) {
      const uint32_t e = 4u * c;  // element within the batch, < 2^31
      const uint32_t row = (uint32_t)__umul64hi(e, mag_s);
      const uint32_t j = e - row * s;
      const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
      const uint32_t t = row - pl * a.spp;
      const uint4 g = *reinterpret_cast<const uint4*>(gvec + (pl * R + (t & (R - 1u))) * s + j);
      const uint32_t phi = __brev(~(t >> a.r_log2));  // phi_2(2^32 - 1 - i), Alg. 4
      const uint32_t v[4] = {phi * g.x, phi * g.y, phi * g.z, phi * g.w};
      store4(a.out_u32, a.out_f32, off0 + e, v);
    }
  }
}

// Generic path: one element per thread.
template <int KIND>
__global__ void __launch_bounds__(kThreads) random_lattice_points_generic(RandomPointsArgs a) {
  __shared__ uint32_t jump[KIND == QMC_RLAT_LFSR ? kJumpLevels * kLfsrJumpWords : 1];
  rlat_jump_tables_fill<KIND>(jump);
  const uint64_t total = a.n_pixels * a.spp * a.s;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
    const uint64_t row = f / a.s;
    const uint32_t j = (uint32_t)(f - row * a.s);
    const uint64_t q = row / a.spp;
    const uint32_t t = (uint32_t)(row - q * a.spp);
    const uint64_t p = a.pixel_begin + q;
    uint32_t g[1];
    rlat_generators<KIND, 1>(a.seed, t & ((1u << a.r_log2) - 1u), j, (uint32_t)(p % a.width),
                             (uint32_t)(p / a.width), jump, g);
    store1(a.out_u32, a.out_f32, f, __brev(~(t >> a.r_log2)) * g[0]);
  }
}

}  // namespace

cudaError_t launch_random_lattice_points(const RandomPointsArgs& args, cudaStream_t stream) {
  const DeviceInfo& dev = device_info();
  RandomPointsArgs a = args;
  const bool hash = a.kind == QMC_RLAT_HASH;
  const uint64_t Rs = (uint64_t)a.s << a.r_log2;
  // batch: up to 48 KiB of generator words (at least one pixel), at most 256 pixels
  uint64_t pixels = (48u * 1024u / 4u) / Rs;
  if (pixels > 256) pixels = 256;
  if (pixels < 1) pixels = 1;
  a.batch_pixels = (uint32_t)pixels;
  const size_t smem =
      ((hash ? 0 : (size_t)kJumpLevels * kLfsrJumpWords) + ((2 * pixels + 3) & ~3ull) + pixels * Rs) * sizeof(uint32_t);
  if ((a.s & 3u) == 0 && pixels * a.spp * a.s <= (1ull << 31) && aligned16(a.out_u32) && aligned16(a.out_f32) &&
      smem <= dev.smem_per_block_optin) {
    const auto kernel = hash ? random_lattice_points_fast<QMC_RLAT_HASH> : random_lattice_points_fast<QMC_RLAT_LFSR>;
    if (smem > 48 * 1024) {
      const cudaError_t ea = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ea != cudaSuccess) return ea;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (uint64_t)dev.sm_count * (per_sm < 1 ? 1 : per_sm);
    const uint64_t batches = (a.n_pixels + pixels - 1) / pixels;
    if (batches < blocks) blocks = batches;
    if (blocks < 1) blocks = 1;
    kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
  }
  uint64_t blocks = (a.n_pixels * a.spp * a.s + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)dev.sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (hash)
    random_lattice_points_generic<QMC_RLAT_HASH><<<(unsigned)blocks, kThreads, 0, stream>>>(a);
  else
    random_lattice_points_generic<QMC_RLAT_LFSR><<<(unsigned)blocks, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pixel_lattice_points(const PixelPointsArgs& a, cudaStream_t stream) {
  const DeviceInfo& dev = device_info();
  if ((a.s & 3u) == 0 && (uint64_t)32 * a.spp * a.s <= (1ull << 31) && aligned16(a.out_u32) &&
      aligned16(a.out_f32)) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pixel_lattice_points_fast, kThreads, 0);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (uint64_t)dev.sm_count * (per_sm < 1 ? 1 : per_sm);
    const uint64_t need = (((a.n_pixels + 31) >> 5) + kThreads / 32 - 1) / (kThreads / 32);
    if (need < blocks) blocks = need;
    if (blocks < 1) blocks = 1;
    pixel_lattice_points_fast<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
  }
  uint64_t blocks = (a.n_pixels * a.spp + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)dev.sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  pixel_lattice_points_kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_lattice_points(PointsArgs a, cudaStream_t stream) {
  const bool backward = (a.scramble & 1u) != 0;
  const uint32_t K = fast_k(a.s);
  a.q_log2 = log2_exact(K ? 128u * K / a.s : 1u);
  const bool fast = K != 0 && (a.index_begin & ((1ull << a.q_log2) - 1u)) == 0 && aligned16(a.out_u32) &&
                    aligned16(a.out_f32);
  if (!fast) {
    return backward ? launch_grid_stride(lattice_points_generic<true>, a.count * a.s, stream, a)
                    : launch_grid_stride(lattice_points_generic<false>, a.count * a.s, stream, a);
  }
  const uint64_t groups = (a.count + (1u << a.q_log2) - 1) >> a.q_log2;
  // TMA bulk stores for device-memory outputs whose staging tiles fit (K <= 3)
  const size_t stage = (size_t)(kThreads / 32) * 4 * kStageGroups * 128u * K * sizeof(uint32_t);
  const bool tma = kPointsTma && device_resident(a.out_u32) && device_resident(a.out_f32) &&
                   stage <= device_info().smem_per_block_optin;
  const size_t smem = tma ? stage : 0;
#define QMC_LATTICE_CASE(KK)                                                                                 \
  case KK:                                                                                                   \
    if (tma)                                                                                                 \
      return backward ? launch_persistent(lattice_points_fast<KK, true, kPointsTma>, groups, smem, stream, a)  \
                      : launch_persistent(lattice_points_fast<KK, false, kPointsTma>, groups, smem, stream, a); \
    return backward ? launch_persistent(lattice_points_fast<KK, true, false>, groups, 0, stream, a)          \
                    : launch_persistent(lattice_points_fast<KK, false, false>, groups, 0, stream, a);
  switch (K) {
    QMC_LATTICE_CASE(1)
    QMC_LATTICE_CASE(2)
    QMC_LATTICE_CASE(3)
    QMC_LATTICE_CASE(4)
    default: return cudaErrorInvalidValue;
  }
#undef QMC_LATTICE_CASE
}

}  // namespace qmc

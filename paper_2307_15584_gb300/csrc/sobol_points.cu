// sobol_points.cu -- materialised Sobol' points (HBM-write bound): Alg. 3 /
// Eq. (ts), y_j(i) = XOR of the generator columns selected by the bits of i,
// randomised in integers (Sec. 2.3), mapped to [0,1) (Sec. 2.1); 32-bit, 64-bit
// (Alg. 3's wide indices) and partitioned (Sec. 2.5.1) enumeration.
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
// wide indices).
#include <cstdint>

#include "points_common.cuh"

namespace qmc {

namespace {
using namespace pts;

// ---------------------------------------------------------------------------
// K1 fast path.  MODE: 0 none, 1 XOR, 2 nested (a.scramble = NESTED_XOR adds the
// digital shift before the nested scramble, folded into the fixed per-lane terms).
// K: 16-byte chunks per lane.
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
      if (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR) y ^= __brev(__ldg(a.seeds + j));  // mirrored shift
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
          store4(a.out_u32, a.out_f32, o, v, a.chk);
      } else {  // ragged last group: per-element row test
        const uint64_t rows_left = a.count - (g << a.q_log2);
        const uint32_t e0 = 4u * (lane + 32u * c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if ((uint64_t)((e0 + t) / s) < rows_left) store1(a.out_u32, a.out_f32, o + t, v[t], a.chk);
      }
    }
    if (TMA && g < full_groups)
      stager.group_done(lane, off, g + 1 == g1 || g + 1 == full_groups, a.out_u32, a.out_f32);
  }
  if (TMA) stager.finish(lane);
}

// K1 walking path, for what the fast path's 16-byte groups do not fit (s / gcd(s, 128) > 4, or
// an index_begin off the group grid).  Lanes own dimensions: a warp takes a chunk of up to 32
// consecutive output dimensions (w of them) and k = floor(32 / w) consecutive rows per step, lane l
// holding dimension l mod w of row l / w, so each step writes k whole rows of the chunk with
// coalesced 4-byte stores.  Each lane walks its dimension down kWalkSteps steps: with the
// enumeration index J = (J_hi << u) | J_lo, y_j = pc_j ^ Hlo_j[J_lo] ^ Hhi_j(J_hi), Hlo a
// shared-memory table of 2^u rows (u >= 5, so one step of k <= 32 wraps J_lo at most once) and Hhi
// changed, when J_lo wraps, by the columns of the J_hi bits that flip.
constexpr uint32_t kWalkSteps = 256;

template <int MODE>
__global__ void __launch_bounds__(kThreads) sobol_points_walk(PointsArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t s = a.s, m = a.m, u = a.u_log2, nlo = 1u << u;
  uint32_t* cols = smem;          // [s][m], mirrored for nested
  uint32_t* hlo = cols + s * m;   // [2^u][s]
  uint32_t* pc = hlo + nlo * s;   // [s]: the fixed low index part
  for (uint32_t idx = threadIdx.x; idx < s * m; idx += blockDim.x) {
    const uint32_t c = __ldg(a.matrices + idx);
    cols[idx] = (MODE == 2) ? __brev(c) : c;
  }
  __syncthreads();
  for (uint32_t idx = threadIdx.x; idx < nlo * s; idx += blockDim.x) {
    const uint32_t g = idx / s, j = idx - g * s;
    uint32_t y = 0;
    for (uint32_t b = 0; (g >> b) != 0 && a.col0 + b < m; ++b)
      if ((g >> b) & 1u) y ^= cols[j * m + a.col0 + b];
    hlo[idx] = y;
  }
  for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) {
    uint32_t y = 0;
    for (uint32_t b = 0; b < a.col0; ++b)
      if ((a.pconst >> b) & 1u) y ^= cols[j * m + b];
    pc[j] = y;
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nch = (s + 31u) >> 5, wl = s - 32u * (nch - 1u), kl = 32u / wl;  // the last chunk: wl wide
  const uint64_t Uf = kWalkSteps, Ul = (uint64_t)kWalkSteps * kl;  // rows per unit: full chunks, the last
  const uint64_t nf = (a.count + Uf - 1) / Uf, nl = (a.count + Ul - 1) / Ul;
  const uint64_t n_units = (uint64_t)(nch - 1u) * nf + nl;
  const uint32_t hi_col = a.col0 + u;  // column of the lowest J_hi bit
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t un = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); un < n_units; un += nw) {
    const bool last = un >= (uint64_t)(nch - 1u) * nf;
    const uint32_t c = last ? nch - 1u : (uint32_t)(un / nf);
    const uint32_t w = last ? wl : 32u, k = last ? kl : 1u;
    const uint64_t U = last ? Ul : Uf;
    const uint64_t r0 = (last ? un - (uint64_t)(nch - 1u) * nf : un - (uint64_t)c * nf) * U;
    if (lane >= k * w) continue;  // w does not divide 32: the remaining lanes idle
    const uint32_t jo = 32u * c + lane % w;
    const uint64_t row = r0 + lane / w;
    const uint64_t r_end = r0 + U < a.count ? r0 + U : a.count;
    if (row >= r_end) continue;
    const uint32_t steps = ((uint32_t)(r_end - row) + k - 1) / k;  // r_end - row <= U <= kWalkSteps k
    const uint64_t J = a.index_begin + row;
    uint32_t jlo = (uint32_t)J & (nlo - 1u);
    uint64_t jhi = J >> u;
    const uint32_t* cj = cols + jo * m;
    uint32_t base = pc[jo];
    for (uint32_t b = 0; (jhi >> b) != 0 && hi_col + b < m; ++b)
      if ((jhi >> b) & 1u) base ^= cj[hi_col + b];
    const uint32_t seed = MODE != 0 ? __ldg(a.seeds + jo) : 0u;
    if (MODE == 1) base ^= seed;
    if (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR) base ^= __brev(seed);  // the shift, mirrored
    const NestedKey key = nested_key(seed);
    // the unit's outputs from its first row on: at most kWalkSteps k s <= 2^23 elements (s <= 1024)
    const uint64_t off0 = row * s + jo;
    uint32_t* const ou = a.out_u32 ? a.out_u32 + off0 : nullptr;
    float* const of = a.out_f32 ? a.out_f32 + off0 : nullptr;
    const uint32_t dofs = k * s;
    uint32_t ofs = 0;
    for (uint32_t t = 0; t < steps; ++t) {
      uint32_t y = hlo[jlo * s + jo] ^ base;
      if (MODE == 2) y = __brev(nested_mix(y, key));
      if (a.out_u32) ou[ofs] = y;
      if (a.out_f32) of[ofs] = map_u32_to_unifloat(y);
      ofs += dofs;
      jlo += k;
      if (jlo >= nlo) {  // J_hi advances by one: the bits of jhi ^ (jhi + 1) flip
        jlo -= nlo;
        ++jhi;
        const uint32_t nflip = (uint32_t)__ffsll((long long)jhi);  // jhi > 0
        for (uint32_t b = 0; b < nflip && hi_col + b < m; ++b) base ^= cj[hi_col + b];
      }
    }
  }
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
    if (MODE == 1 || (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR)) y ^= __ldg(a.seeds + j);
    if (MODE == 2) y = __brev(nested_mix(__brev(y), nested_key(__ldg(a.seeds + j))));
    store1(a.out_u32, a.out_f32, f, y, a.chk);
  }
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
    // the walking path: the columns and a low table of 2^w rows, 5 <= w <= 8, in shared memory
    uint32_t w = 8;
    while (w > 5 && ((size_t)a.s * a.m + ((size_t)1 << w) * a.s + a.s) * sizeof(uint32_t) > optin) --w;
    const size_t walk_smem = ((size_t)a.s * a.m + ((size_t)1 << w) * a.s + a.s) * sizeof(uint32_t);
    if (walk_smem <= optin && a.s <= 1024) {
      a.u_log2 = w;
      const uint32_t nch = (a.s + 31u) >> 5, wl = a.s - 32u * (nch - 1u);
      const uint64_t Ul = (uint64_t)kWalkSteps * (32u / wl);
      const uint64_t units = (uint64_t)(nch - 1u) * ((a.count + kWalkSteps - 1) / kWalkSteps) + (a.count + Ul - 1) / Ul;
      switch (a.scramble) {
        case 0: return launch_persistent(sobol_points_walk<0>, units, walk_smem, stream, a);
        case 1: return launch_persistent(sobol_points_walk<1>, units, walk_smem, stream, a);
        default: return launch_persistent(sobol_points_walk<2>, units, walk_smem, stream, a);
      }
    }
    switch (a.scramble) {  // tables beyond shared memory: one element per thread
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

}  // namespace qmc

// halton_points.cu -- materialised Halton points (Sec. 2.2, Alg. 1, Alg. 2):
// radical inverses in the first 64 prime bases, plain, Faure-permuted or with a
// linear digit scramble, 64-bit indices, partitioned by the base-2 dimension
// (Sec. 2.5.1).
#include <cstdint>
#include <mutex>
#include <vector>

#include "points_common.cuh"

namespace qmc {

namespace {
using namespace pts;

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

}  // namespace

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

}  // namespace qmc

// halton_points.cu -- materialised Halton points (Sec. 2.2, Alg. 1, Alg. 2):
// radical inverses in the first 64 prime bases, plain, Faure-permuted or with a
// linear digit scramble, 64-bit indices, partitioned by the base-2 dimension
// (Sec. 2.5.1).
#include <cstdint>
#include <mutex>
#include <vector>

#include "halton_points.h"
#include "points_common.cuh"

namespace qmc {

namespace {
using namespace pts;

// Halton points: element (r, j) = phi_b(i') of index
// i = ((index_begin + r) << q) | pconst (q > 0: one element of a sequence
// partitioned by its base-2 dimension, Sec. 2.5.1) with b the (dim0 + j)-th
// prime; digits permuted (Faure table or linear multiplier), i' = i mod 2^32
// for b = 2 (the bit reversal of the low 32 bits), otherwise i mod b^K with b^K
// the largest power below 2^32 (Alg. 1's domain limit).  Base 2 runs the same
// tables with b^K = 2^32 (K = 32 digits; the scale 2^32 / b^K is then 1), so no
// lane of a warp takes a path of its own.
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
  uint32_t max_power[kHaltonMaxDims];  // b^K: the largest power of the base below 2^32; 0 for base 2 (2^32)
  uint32_t perm_off[kHaltonMaxDims];   // Faure table of dimension j at perm[perm_off[j]]
  uint32_t digits[kHaltonMaxDims];     // L, digits per full group
  uint32_t groups[kHaltonMaxDims];     // G
  uint32_t top_digits[kHaltonMaxDims]; // L', digits of the most significant group (1 <= L' <= L)
  uint32_t group_pow[kHaltonMaxDims];  // b^L
  uint32_t top_pow[kHaltonMaxDims];    // b^L'
  uint64_t magic_group[kHaltonMaxDims];  // floor(2^64 / b^L) + 1: x / b^L = umulhi(x, .) for x < 2^32
  uint64_t magic_max[kHaltonMaxDims];    // floor(2^64 / b^K) + 1: the same for b^K
  uint32_t recip96[kHaltonMaxDims][3];   // ceil(2^96 / b^K) = [2] 2^64 + [1] 2^32 + [0]: floor(N 2^32 / b^K)
  uint64_t magic_base[kHaltonMaxDims];   // floor(2^64 / b) + 1: x / b = umulhi(x, .) for x < 2^32
  uint16_t perm[kHaltonPermWords];
};
__device__ HaltonTables g_halton;

// Work layout.  The output is [count][s] row-major.  Lanes own dimensions: a
// warp takes a chunk of up to 32 consecutive output dimensions (w of them) and
// k = floor(32 / w) consecutive rows per step, lane l holding dimension l mod w
// of row l / w, so each step writes k whole rows of the chunk, coalesced.  A
// unit is NSTEPS steps of one chunk; each lane walks its dimension down
// the rows, advancing the digit groups of i mod b^K by the index step k 2^q
// instead of recomputing them: one table lookup and one multiply-add per row,
// the higher groups touched only on a carry (or every row when the step has
// higher digits, as in a partitioned sequence).  A 32-wide chunk with 16-byte
// aligned rows passes each group of four rows through a per-warp 4 x 32
// shared-memory tile, so each lane stores four consecutive dimensions of one
// row as one 16-byte chunk.
// Steps per unit: shorter units keep the resident warps' stores closer together, longer ones
// pay each unit's set-up (the digit groups of its first index) over more rows; measured at
// s = 32: 128 steps for a plain sequence (4 % faster than 256), 256 for a partition element
// (whose set-up is costlier: 128 steps ran 5 % slower).
constexpr uint32_t kHaltonStepsPlain = 128, kHaltonStepsPartitioned = 256;
constexpr uint32_t kHaltonStageWords = 128;  // per warp: 4 rows x 32 dimensions
constexpr int kHaltonMaxGroups = 6;  // G <= 6 for every base up to the 64th prime (base 37: L = 1, K = 6)

// floor(N 2^32 / b^K) for N < b^K < 2^32, exactly: with M = ceil(2^96 / b^K) = M2 2^64 + M1 2^32 + M0,
// N M / 2^64 exceeds N 2^32 / b^K by less than N / 2^64 < 1 / b^K (as N b^K < 2^64), which never
// reaches the next integer, so the result is floor(N M / 2^64) = N M2 + hi32(N M1 + umulhi(N, M0)).
__device__ __forceinline__ uint32_t halton_scale(uint32_t N, uint32_t m0, uint32_t m1, uint32_t m2) {
  const uint64_t a = (uint64_t)N * m1 + __umulhi(N, m0);
  return N * m2 + (uint32_t)(a >> 32);
}

// The digit groups of x < b^K, least significant first: g < G-1 hold L digits
// (x mod b^L by the magic reciprocal), the top group the remaining L' digits.
__device__ __forceinline__ void halton_groups(uint32_t x, uint32_t G, uint32_t bL, uint64_t mg,
                                              uint32_t (&out)[kHaltonMaxGroups]) {
#pragma unroll
  for (int g = 0; g < kHaltonMaxGroups; ++g) {
    if ((uint32_t)g + 1 < G) {
      const uint32_t q = (uint32_t)__umul64hi(x, mg);
      out[g] = x - q * bL;
      x = q;
    } else if ((uint32_t)g + 1 == G) {
      out[g] = x;
    } else {
      out[g] = 0;
    }
  }
}

template <uint32_t NSTEPS>  // steps per unit
__global__ void __launch_bounds__(kThreads, 2) halton_points_kernel(HaltonArgs p) {
  extern __shared__ __align__(16) uint32_t hsmem[];
  uint16_t* htab = reinterpret_cast<uint16_t*>(hsmem);  // digit-group tables
  // this warp's 4 x 32 tile for the transposed stores, after the tables (16-byte aligned)
  uint32_t* stage = hsmem + p.stage_word + (threadIdx.x >> 5) * kHaltonStageWords;
  for (uint32_t jo = 0; jo < p.s; ++jo) {
    const uint32_t j = p.dim0 + jo;
    const uint32_t b = g_halton.base[j];
    const uint32_t bL = g_halton.group_pow[j], bLp = g_halton.top_pow[j];
    const uint32_t poff = g_halton.perm_off[j];
    uint16_t* t = htab + p.table_off[jo];
    for (uint32_t e = threadIdx.x; e < bL + bLp; e += blockDim.x) {
      const bool top = e >= bL;
      uint32_t x = top ? e - bL : e;
      const uint32_t nd = top ? g_halton.top_digits[j] : g_halton.digits[j];
      const uint64_t mb = g_halton.magic_base[j];
      uint32_t num = 0;
      for (uint32_t k = 0; k < nd; ++k) {  // lowest digit first: it becomes the most significant
        const uint32_t q = (uint32_t)__umul64hi(x, mb);
        uint32_t d = x - q * b;
        x = q;
        if (p.mode == 1) {
          d = g_halton.perm[poff + d];
        } else if (p.mode == 2) {
          const uint32_t md = p.mult[jo] * d;  // < b^2
          d = md - (uint32_t)__umul64hi(md, mb) * b;
        }
        num = num * b + d;
      }
      t[e] = (uint16_t)num;
    }
  }
  __syncthreads();

  const uint32_t s = p.s, lane = threadIdx.x & 31u;
  const uint32_t w0 = s < 32u ? s : 32u, k0 = 32u / w0;
  const uint32_t w1 = s > 32u ? s - 32u : 0u, k1 = w1 ? 32u / w1 : 1u;
  constexpr uint32_t nsteps = NSTEPS;
  const uint64_t U0 = (uint64_t)nsteps * k0, U1 = (uint64_t)nsteps * k1;
  // Two chunks (s > 32, so k0 = 1): units go by row blocks of U1 rows, k1 units of the first
  // chunk then one of the second, so the two chunks of the same rows -- which share cache lines
  // when a row is not a whole number of lines -- are written at about the same time.
  const uint32_t per_block = w1 ? k1 + 1u : 1u;
  const uint64_t n_units = w1 ? (p.count + U1 - 1) / U1 * per_block : (p.count + U0 - 1) / U0;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  // this lane's place in a unit of either chunk: (row offset, output dimension)
  const uint32_t ro0 = lane / w0, jo0 = lane % w0;
  const uint32_t ro1 = w1 ? lane / w1 : 0u, jo1 = w1 ? 32u + lane % w1 : 0u;
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units; u += nw) {
    const uint64_t rb = u / per_block;
    const uint32_t within = (uint32_t)(u - rb * per_block);
    const bool c1 = w1 && within == k1;
    const uint32_t w = c1 ? w1 : w0, k = c1 ? k1 : k0;
    const uint64_t U = c1 ? U1 : U0;
    const uint64_t r0 = w1 ? rb * U1 + (c1 ? 0u : (uint64_t)within * nsteps) : u * U0;
    if (r0 >= p.count) continue;  // the last row block is cut by the range
    if (lane >= k * w) continue;  // w does not divide 32: the remaining lanes idle
    const uint32_t jo = c1 ? jo1 : jo0;
    const uint64_t row = r0 + (c1 ? ro1 : ro0);
    const uint64_t r_end = r0 + U < p.count ? r0 + U : p.count;
    if (row >= r_end) continue;
    const uint32_t steps = ((uint32_t)(r_end - row) + k - 1) / k;  // r_end - row <= U = nsteps k
    // the unit's outputs from its first row on; a unit spans at most 256 k s <= 2^19 elements,
    // so the step offset stays 32-bit (the null tests are on the kernel parameters: uniform)
    const uint64_t off0 = row * s + jo;
    uint32_t* const ou = p.out_u32 ? p.out_u32 + off0 : nullptr;
    float* const of = p.out_f32 ? p.out_f32 + off0 : nullptr;
    const uint32_t dofs = k * s;
    uint32_t ofs = 0;
    const uint32_t j = p.dim0 + jo;
    const uint64_t i = ((p.index_begin + row) << p.q) | p.pconst;
    const uint32_t mp = g_halton.max_power[j];  // 0: base 2, whose b^K is 2^32
    const uint32_t m0 = g_halton.recip96[j][0], m1 = g_halton.recip96[j][1], m2 = g_halton.recip96[j][2];
    const uint32_t bL = g_halton.group_pow[j], bLp = g_halton.top_pow[j];
    const uint32_t G = g_halton.groups[j];
    const uint64_t mg = g_halton.magic_group[j];
    const uint16_t* tab = htab + p.table_off[jo];
    const uint32_t x = mp == 0 ? (uint32_t)i
                       : (i >> 32) ? (uint32_t)(i % mp)
                                   : (uint32_t)i - mp * (uint32_t)__umul64hi((uint32_t)i, g_halton.magic_max[j]);
    uint32_t xg[kHaltonMaxGroups], dg[kHaltonMaxGroups], wg[kHaltonMaxGroups];
    halton_groups(x, G, bL, mg, xg);
    const uint32_t D = p.delta[jo];  // (k 2^q) mod b^K
    halton_groups(D, G, bL, mg, dg);
    const bool d_hi = D >= bL;  // the step reaches beyond the lowest group
    // weights of the mirrored groups: N = sum_g T_g[x_g] wg[g], the lowest group the most significant
    uint32_t wacc = 1;
#pragma unroll
    for (int g = kHaltonMaxGroups - 1; g >= 0; --g) {
      wg[g] = wacc;
      if ((uint32_t)g + 1 == G) wacc = bLp;
      else if ((uint32_t)g + 1 < G) wacc *= bL;
    }
    auto entry = [&](int g) -> uint32_t {  // T_g[x_g]: the top group has its own table after the full one
      return (uint32_t)tab[(uint32_t)g + 1 == G ? bL + xg[g] : xg[g]];
    };
    auto rest = [&]() {  // the groups above the lowest
      uint32_t r = 0;
#pragma unroll
      for (int g = 1; g < kHaltonMaxGroups; ++g)
        if ((uint32_t)g < G) r += entry(g) * wg[g];
      return r;
    };
    // add the step's higher digits (when d_hi) and a carry to groups 1.., wrapping mod b^K
    auto add_high = [&](uint32_t carry) {
#pragma unroll
      for (int g = 1; g < kHaltonMaxGroups; ++g) {
        if ((uint32_t)g < G) {
          const uint32_t lim = (uint32_t)g + 1 == G ? bLp : bL;
          const uint32_t v = xg[g] + (d_hi ? dg[g] : 0u) + carry;
          carry = v >= lim ? 1u : 0u;
          xg[g] = carry ? v - lim : v;
        }
      }
    };
    uint32_t nrest = rest();
    uint32_t t1 = entry(1);  // group 1's current entry
    const uint32_t lim1 = G == 2 ? bLp : bL, w1g = wg[1];
    uint32_t x0 = xg[0];
    const uint32_t d0 = dg[0], w0g = wg[0];
    auto put = [&](uint32_t o, uint32_t v) {  // one coordinate, element o of the unit's outputs
      if (in_bounds(p.chk, off0 + o, 1, kCheckPoints)) {
        if (p.out_u32) ou[o] = v;
        if (p.out_f32) of[o] = map_u32_to_unifloat(v);
      }
    };
    auto emit = [&]() {  // the current row's coordinate
      put(ofs, halton_scale(nrest + (uint32_t)tab[x0] * w0g, m0, m1, m2));
      ofs += dofs;
      x0 += d0;
      const bool carry0 = x0 >= bL;
      if (carry0) x0 -= bL;
      return carry0;
    };
    auto carry1 = [&]() {  // a carry out of the lowest group
      if (xg[1] + 1 < lim1) {  // the common carry: group 1 moves by one
        ++xg[1];
        const uint32_t t1n = entry(1);
        nrest += (t1n - t1) * w1g;  // exact modulo 2^32, and the result is below b^K
        t1 = t1n;
      } else {
        add_high(1u);
        nrest = rest();
        t1 = entry(1);
      }
    };
    uint32_t t = 0;
    // Four steps at a time while the step lies in the lowest group and four of them wrap it at
    // most once: the four table reads go out together, and the rows past the wrap take the
    // carried higher part.  A 32-wide chunk (all lanes on the same rows, so the choice is made
    // for the whole warp) with 16-byte aligned rows transposes its four rows through the warp's
    // tile and stores 16-byte chunks of four consecutive dimensions.
    bool grouped = !d_hi && 4u * d0 <= bL;
    if (w == 32u) grouped = __all_sync(0xffffffffu, grouped);
    if (grouped) {
      const bool rows16 = w == 32u && (s & 3u) == 0 &&
                          (((uintptr_t)p.out_u32 | (uintptr_t)p.out_f32) & 15u) == 0;
      uint64_t vo = (row + (lane >> 3)) * s + (c1 ? 32u : 0u) + 4u * (lane & 7u);  // after the transpose
      for (; t + 4u <= steps; t += 4u) {
        uint32_t e[4];
        bool wr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t v = x0 + (uint32_t)q * d0;  // below 2 b^L
          wr[q] = v >= bL;
          e[q] = tab[wr[q] ? v - bL : v];
        }
        const uint32_t xn = x0 + 4u * d0, nlow = nrest;
        if (xn >= bL) carry1();  // at one of the four rows or at the next group's first
        x0 = xn >= bL ? xn - bL : xn;
        uint32_t y4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) y4[q] = halton_scale((wr[q] ? nrest : nlow) + e[q] * w0g, m0, m1, m2);
        if (rows16) {
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 4; ++q) stage[q * 32u + lane] = y4[q];
          __syncwarp();
          const uint4 v = *reinterpret_cast<const uint4*>(stage + (lane >> 3) * 32u + 4u * (lane & 7u));
          const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
          store4(p.out_u32, p.out_f32, vo, vv, p.chk);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) put(ofs + (uint32_t)q * dofs, y4[q]);
        }
        ofs += 4u * dofs;
        vo += 4u * s;
      }
    }
    if (!d_hi) {  // the step lies in the lowest group: the higher groups move only on its carry
      for (; t < steps; ++t)
        if (emit()) carry1();
    } else {  // every step moves the higher groups (a partitioned sequence)
      for (; t < steps; ++t) {
        add_high(emit() ? 1u : 0u);
        nrest = rest();
      }
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
      if (b == 2) mp = 1ull << 32, K = 32;  // base 2 keeps all 32 index bits: its b^K is 2^32
      uint32_t L = 1;
      uint64_t bL = b;
      while (bL * b <= kHaltonGroupCap) bL *= b, ++L;
      const uint32_t G = (K + L - 1) / L, Lp = K - (G - 1) * L;
      uint64_t bLp = 1;
      for (uint32_t t = 0; t < Lp; ++t) bLp *= b;
      h.base[j] = b;
      h.max_power[j] = (uint32_t)mp;  // 0 for base 2
      h.digits[j] = L;
      h.groups[j] = G;
      h.top_digits[j] = Lp;
      h.group_pow[j] = (uint32_t)bL;
      h.top_pow[j] = (uint32_t)bLp;
      h.magic_group[j] = UINT64_MAX / bL + 1;
      h.magic_max[j] = b == 2 ? 0 : UINT64_MAX / mp + 1;  // base 2 takes i mod 2^32 directly
      // ceil(2^96 / b^K): for odd b^K the quotient's floor plus one; for 2^32 exactly 2^64
      const unsigned __int128 r96 = ((((unsigned __int128)1) << 96) - 1) / mp + 1;
      h.recip96[j][0] = (uint32_t)r96;
      h.recip96[j][1] = (uint32_t)(r96 >> 32);
      h.recip96[j][2] = (uint32_t)(r96 >> 64);
      h.magic_base[j] = UINT64_MAX / b + 1;
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
  uint32_t table_words = 0;  // uint16 entries
  for (uint32_t jo = 0; jo < p.s; ++jo) {
    const uint32_t j = p.dim0 + jo;
    p.table_off[jo] = table_words;
    if (h.groups[j] < 2) return cudaErrorInvalidValue;  // the lowest group is a full one
    table_words += h.group_pow[j] + h.top_pow[j];
    // the index step of this dimension's lanes: k rows, k = floor(32 / w) for the chunk's width w
    const uint32_t chunk_w = jo < 32 ? (p.s < 32 ? p.s : 32) : p.s - 32;
    const uint64_t k = 32 / chunk_w, mp = h.base[j] == 2 ? 1ull << 32 : h.max_power[j];
    const uint64_t pow2q = (p.q < 64 ? (1ull << p.q) : 0ull) % mp;
    p.delta[jo] = (uint32_t)((k % mp) * pow2q % mp);
  }
  p.stage_word = (uint32_t)((((size_t)table_words * sizeof(uint16_t) + 15) & ~(size_t)15) / sizeof(uint32_t));
  const size_t smem = ((size_t)p.stage_word + (size_t)(kThreads / 32) * kHaltonStageWords) * sizeof(uint32_t);
  const DeviceInfo& dev = device_info();
  if (smem > dev.smem_per_block_optin) return cudaErrorInvalidValue;
  const uint32_t nsteps = p.q == 0 ? kHaltonStepsPlain : kHaltonStepsPartitioned;
  const auto kernel = p.q == 0 ? halton_points_kernel<kHaltonStepsPlain>
                               : halton_points_kernel<kHaltonStepsPartitioned>;
  if (smem > 48 * 1024) {
    const cudaError_t ea = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
  }
  int per_sm = 0;
  cudaError_t eo = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
  if (eo != cudaSuccess) return eo;
  uint64_t blocks = (uint64_t)dev.sm_count * (per_sm < 1 ? 1 : per_sm);
  // units of nsteps steps: one chunk of up to 32 dimensions, k rows per step; with two
  // chunks, row blocks of one second-chunk unit's rows, 32 / w1 + 1 units each
  const uint32_t w0 = p.s < 32 ? p.s : 32, w1 = p.s > 32 ? p.s - 32 : 0;
  const uint64_t U0 = (uint64_t)nsteps * (32 / w0);
  uint64_t units = (p.count + U0 - 1) / U0;
  if (w1) {
    const uint64_t U1 = (uint64_t)nsteps * (32 / w1);
    units = (p.count + U1 - 1) / U1 * (32 / w1 + 1);
  }
  const uint64_t need = (units + kThreads / 32 - 1) / (kThreads / 32);
  if (need < blocks) blocks = need;
  if (blocks < 1) blocks = 1;
  kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace qmc

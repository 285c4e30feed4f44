// integrate.cu -- massively parallel QMC integro-approximation (Sec. 2.5).
//
// Launch sequence of one qmc_integrate* call (all on the caller's stream):
//   1. scan_totals   per block of 1024 integrals: sum of work items
//                    ceil(n_p / C) and of samples n_p (u64)
//   2. scan_carry    one block: exclusive scan of the block totals, resets the
//                    scheduler, checks the item count against the workspace
//   3. scan_write    item_off[p] (u32) and, for the unfused path, row_off[p] (u64)
//   4. integrate_main  persistent: each warp takes a work item (integral p,
//                    chunk k) from an atomic counter, generates the chunk's
//                    points in registers, evaluates f in fp32, accumulates
//                    with Kahan sums, merges the 32 lanes in a fixed
//                    butterfly and writes the compensated partial to slot
//                    `item` -- so the result never depends on scheduling
//   5. reduce_*      per integral, the partials in item order in fp64
//                    (the only fp64 arithmetic of the path), divided by n_p
//   6. loss_reduce   (fused fwd+bwd only) fixed-order fp64 sum of the loss terms
//
// Sample i of integral p lives in chunk k = i >> log2(C), iteration
// r = (i >> 5) mod C/32 and lane i mod 32.  These bit fields are disjoint, so
// the Sobol' digits split as y(i) = Y(kC) ^ T[r] ^ L[lane] (linearity of
// Eq. (ts) over GF(2)): one shared-memory load and two XORs per coordinate.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/qmc.h"
#include "qmc_device.cuh"
#include "qmc_integrate.h"
#include "qmc_internal.h"

namespace qmc {

namespace {

constexpr uint32_t kScanBlock = 1024;  // integrals per scan block
constexpr uint32_t kScanThreads = 256;

// ---------------------------------------------------------------------------
// 1-3: work-item offsets
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v, uint64_t* sh) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  uint64_t t = 0;
  for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}

// Exclusive scan of v over the block; returns the block total in `total`.
__device__ __forceinline__ uint64_t block_exscan_u64(uint64_t v, uint64_t* sh, uint64_t& total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  uint64_t warp_off = 0;
  total = 0;
  for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
    if (w < warp) warp_off += sh[w];
    total += sh[w];
  }
  __syncthreads();
  return warp_off + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_totals(IntegrateArgs a) {
  __shared__ uint64_t sh[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock;
  uint64_t items = 0, rows = 0;
  for (uint32_t t = threadIdx.x; t < kScanBlock; t += blockDim.x) {
    const uint64_t p = base + t;
    if (p < a.n) {
      const uint64_t c = a.counts[p];
      items += (c + (1ull << a.chunk_log2) - 1) >> a.chunk_log2;
      rows += c;
    }
  }
  items = block_sum_u64(items, sh);
  rows = block_sum_u64(rows, sh);
  if (threadIdx.x == 0) {
    a.ws_block_items[blockIdx.x] = items;
    a.ws_block_rows[blockIdx.x] = rows;
  }
}

__global__ void __launch_bounds__(1024) scan_carry(IntegrateArgs a, uint32_t n_blocks) {
  __shared__ uint64_t sh[32];
  uint64_t carry_items = 0, carry_rows = 0;
  for (uint32_t b0 = 0; b0 < n_blocks; b0 += blockDim.x) {
    const uint32_t b = b0 + threadIdx.x;
    const uint64_t vi = b < n_blocks ? a.ws_block_items[b] : 0;
    const uint64_t vr = b < n_blocks ? a.ws_block_rows[b] : 0;
    uint64_t ti, tr;
    const uint64_t ei = block_exscan_u64(vi, sh, ti);
    const uint64_t er = block_exscan_u64(vr, sh, tr);
    if (b < n_blocks) {
      a.ws_block_items[b] = carry_items + ei;
      a.ws_block_rows[b] = carry_rows + er;
    }
    carry_items += ti;
    carry_rows += tr;
  }
  if (threadIdx.x == 0) {
    WsHeader* h = a.hdr;
    h->next_item = 0;
    h->error_bits = 0;
    if (carry_items > a.capacity_items || carry_items >= 0xFFFFFFFFull) {
      h->error_bits = kErrCapacity;
      h->total_items = 0;  // integrate nothing rather than write past the workspace
    } else {
      h->total_items = (uint32_t)carry_items;
    }
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_write(IntegrateArgs a) {
  __shared__ uint64_t sh[32];
  constexpr uint32_t kPer = kScanBlock / kScanThreads;
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kPer;
  uint64_t items[kPer], rows[kPer];
  uint64_t ti = 0, tr = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint64_t p = base + q;
    const uint64_t c = p < a.n ? a.counts[p] : 0;
    items[q] = (c + (1ull << a.chunk_log2) - 1) >> a.chunk_log2;
    rows[q] = c;
    ti += items[q];
    tr += rows[q];
  }
  uint64_t dummy;
  uint64_t oi = block_exscan_u64(ti, sh, dummy) + a.ws_block_items[blockIdx.x];
  uint64_t orow = block_exscan_u64(tr, sh, dummy) + a.ws_block_rows[blockIdx.x];
  const bool ok = a.hdr->error_bits == 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint64_t p = base + q;
    if (p <= a.n) {  // entry n is the total
      if (ok) a.item_off[p] = (uint32_t)oi;
      if (a.row_off) a.row_off[p] = orow;
    }
    oi += items[q];
    orow += rows[q];
  }
}

// ---------------------------------------------------------------------------
// Point sources.  Each produces the S coordinates of local sample il of the
// current item (sample index start + il) in the scaled form X = x * 2^32 of
// unifloat_x2p32 (exact: x = map_u32_to_unifloat(u) = X * 2^-32); the
// integrands fold the 2^-32 into their constants.
// ---------------------------------------------------------------------------
template <int S, int SCR>  // SCR: 0 none, 1 XOR, 2 nested
struct SobolSource {
  static constexpr int kRow = (S + 3) & ~3;  // table row stride: whole 128-bit words
  const uint32_t* cols;  // shared: [s][32], mirrored when nested
  const uint32_t* tab;   // shared: [C/32][kRow], y(32 r)
  uint32_t s;
  uint32_t lane_y[S];    // y(lane)
  uint32_t yl[S];        // y(start) ^ y(lane) (^ seed for XOR)
  NestedKey key[S];

  // the columns first (a multiple of 32 words keeps the table 16-byte aligned)
  static size_t smem_bytes(uint32_t s, uint32_t chunk_log2) {
    return ((size_t)s * 32 + ((size_t)1 << (chunk_log2 - 5)) * kRow) * sizeof(uint32_t);
  }

  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t* smem) {
    s = a.s;
    uint32_t* c = smem;
    uint32_t* t = smem + s * 32;
    for (uint32_t i = threadIdx.x; i < s * 32; i += blockDim.x) {
      const uint32_t v = __ldg(a.matrices + i);
      c[i] = SCR == 2 ? __brev(v) : v;
    }
    __syncthreads();
    const uint32_t rows = 1u << (a.chunk_log2 - 5);
    for (uint32_t i = threadIdx.x; i < rows * kRow; i += blockDim.x) {
      const uint32_t r = i / kRow, j = i - r * kRow;
      uint32_t y = 0;
      if (j < s)
        for (uint32_t b = 0; (r >> b) != 0; ++b)
          if ((r >> b) & 1u) y ^= c[j * 32 + 5 + b];
      t[i] = y;
    }
    __syncthreads();
    cols = c;
    tab = t;
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t y = 0;
      if ((uint32_t)j < s)
        for (uint32_t b = 0; b < 5; ++b)
          if ((lane >> b) & 1u) y ^= c[j * 32 + b];
      lane_y[j] = y;
    }
  }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t start) {
    const uint32_t khi = start >> a.chunk_log2;
    const uint32_t* sd = a.seeds ? a.seeds + (a.seeds_per_integral ? (size_t)p * s : 0) : nullptr;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t y = 0;
      if ((uint32_t)j < s)
        for (uint32_t b = 0; (khi >> b) != 0; ++b)
          if ((khi >> b) & 1u) y ^= cols[j * 32 + a.chunk_log2 + b];
      const uint32_t seed = (sd && (uint32_t)j < s) ? __ldg(sd + j) : 0u;
      yl[j] = y ^ lane_y[j] ^ (SCR == 1 ? seed : 0u);
      key[j] = nested_key(seed);
    }
  }

  __device__ __forceinline__ void point(uint32_t r, uint32_t /*il*/, bool /*valid*/, float* x) const {
    uint32_t row[kRow];
#pragma unroll
    for (int q = 0; q < kRow / 4; ++q) {  // 128-bit shared loads
      const uint4 w = reinterpret_cast<const uint4*>(tab + r * kRow)[q];
      row[4 * q] = w.x, row[4 * q + 1] = w.y, row[4 * q + 2] = w.z, row[4 * q + 3] = w.w;
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t y = row[j] ^ yl[j];
      if (SCR == 2) y = __brev(nested_mix(y, key[j]));
      x[j] = unifloat_x2p32(y);
    }
  }
};

template <int S, bool BACKWARD>
struct LatticeSource {
  uint32_t s;
  uint32_t start;
  uint32_t g[S];
  uint32_t sh[S];

  static size_t smem_bytes(uint32_t, uint32_t) { return 0; }

  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t*) {
    s = a.s;
#pragma unroll
    for (int j = 0; j < S; ++j) g[j] = (uint32_t)j < s ? (__ldg(a.g + j) | 1u) : 1u;
  }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t st) {
    start = st;
    const uint32_t* sd = a.seeds ? a.seeds + (a.seeds_per_integral ? (size_t)p * s : 0) : nullptr;
#pragma unroll
    for (int j = 0; j < S; ++j) sh[j] = (sd && (uint32_t)j < s) ? __ldg(sd + j) : 0u;
  }

  __device__ __forceinline__ void point(uint32_t, uint32_t il, bool, float* x) const {
    const uint32_t k = start + il;
    const uint32_t phi = __brev(BACKWARD ? ~k : k);
#pragma unroll
    for (int j = 0; j < S; ++j) x[j] = unifloat_x2p32(phi * g[j] + sh[j]);
  }
};

// Pixel-shifted rank-1 lattice (Sec. 3, Eq. (PixelShiftedR1LS)): integral p
// is the pixel (p % width, p / width); its samples are
// (phi_2(i) + phi_3(hilbert(x, y))) g mod 1, one shift per pixel.
template <int S>
struct PixelLatticeSource {
  uint32_t start;
  uint32_t shift;
  uint32_t g[S];

  static size_t smem_bytes(uint32_t, uint32_t) { return 0; }

  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t*) {
#pragma unroll
    for (int j = 0; j < S; ++j) g[j] = (uint32_t)j < a.s ? (__ldg(a.g + j) | 1u) : 1u;
  }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t st) {
    start = st;
    shift = pixel_shift(p % a.image_width, p / a.image_width, a.grid_log2);
  }

  __device__ __forceinline__ void point(uint32_t, uint32_t il, bool, float* x) const {
    const uint32_t base = __brev(start + il) + shift;  // mod 2^32
#pragma unroll
    for (int j = 0; j < S; ++j) x[j] = unifloat_x2p32(base * g[j]);
  }
};

// Random rank-1 lattice per pixel (Alg. 4, Sec. 3): integral p is pixel
// (p % width, p / width).  Sample t of an item lives in lane t mod 32 (items
// start at multiples of the chunk, a multiple of 32), so with R | 32 instances
// every lane keeps one instance k = lane mod R for the whole item and derives
// its generator vector once per item; point i = t div R of that instance is
// phi_2(2^32 - 1 - i) g mod 1.
template <int S, int KIND>
struct RandomLatticeSource {
  uint32_t start, seed, r_log2;
  const uint32_t* jump;  // LFSR: the 32-step jump table in shared memory
  uint32_t g[S];

  static size_t smem_bytes(uint32_t, uint32_t) {
    return KIND == QMC_RLAT_LFSR ? kLfsrJumpWords * sizeof(uint32_t) : 0;
  }

  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t* smem) {
    seed = __ldg(a.seeds);
    r_log2 = a.rlat_log2;
    jump = smem;
    if (KIND == QMC_RLAT_LFSR) {
      lfsr_jump_table_fill(smem);
      __syncthreads();
    }
  }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t st) {
    start = st;
    const uint32_t px = p % a.image_width, py = p / a.image_width;
    const uint32_t k = threadIdx.x & ((1u << r_log2) - 1u);
    if (KIND == QMC_RLAT_HASH) {
#pragma unroll
      for (int j = 0; j < S; ++j) g[j] = rlat_hash(seed, k, j, px, py) | 1u;
    } else {
      uint32_t xi = rlat_lfsr_seed(seed, k, px, py);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        g[j] = 2u * xi + 1u;
        xi = lfsr_jump32(jump, xi);
      }
    }
  }

  __device__ __forceinline__ void point(uint32_t, uint32_t il, bool, float* x) const {
    const uint32_t phi = __brev(~((start + il) >> r_log2));
#pragma unroll
    for (int j = 0; j < S; ++j) x[j] = unifloat_x2p32(phi * g[j]);
  }
};

// Unfused comparison path: coordinates read back from HBM.
template <int S>
struct PointsSource {
  const float* rows;
  uint32_t s;

  static size_t smem_bytes(uint32_t, uint32_t) { return 0; }

  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t*) { s = a.s; }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t start) {
    const uint64_t row0 = (a.points_shared ? 0ull : a.row_off[p]) + start;
    rows = a.points + row0 * s;
  }

  __device__ __forceinline__ void point(uint32_t, uint32_t il, bool valid, float* x) const {
    const float* r = rows + (size_t)il * s;
#pragma unroll
    for (int j = 0; j < S; ++j)
      x[j] = (valid && (uint32_t)j < s) ? __fmul_rn(__ldcs(r + j), 0x1p32f) : 0x1p31f;  // exact scale
  }
};

// ---------------------------------------------------------------------------
// Integrands (fp32).  Per-integral constants are built with error-free
// transformations so that no rounding error is shared by all samples.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float t) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}

// log2(e) split into two fp32 words (hi + lo to ~2^-48).
constexpr float kLog2eHi = 1.44269502162933349609375f;
constexpr float kLog2eLo = 1.925963033500011079e-08f;

template <int FN>
struct Integrand;

// Every integrand offers eval<EXACT>(x, err): f(x) in fp32 and, for adaptive
// integrands, err = an estimate of the sample's rounding error scale.  EXACT
// selects the float-float evaluation used when an item's error estimate is
// over budget; non-adaptive integrands ignore it.
template <>
struct Integrand<QMC_F_BILINEAR2D> {
  static constexpr int S = 2;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  __device__ void setup(const float*, uint32_t) {}
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    return __fmaf_rn(0x1p-33f, x[0], 0.75f) * __fmaf_rn(0x1p-33f, x[1], 0.75f);  // 0.75 + x/2
  }
};

template <>
struct Integrand<QMC_F_GENZ_PRODUCT_PEAK> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  uint32_t s;
  float ch[16], cl[16], u[16];  // a^-2 = ch + cl
  __device__ void setup(const float* th, uint32_t s_) {
    s = s_;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float a = (uint32_t)j < s ? __ldg(th + j) : 1.0f;
      u[j] = (uint32_t)j < s ? __ldg(th + s + j) : 0.0f;
      float e;
      const float a2 = two_prod(a, a, e);
      ch[j] = ff_recip(a2, e, cl[j]);
    }
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    float prod = 1.0f;
    if (s == 16) {  // every dimension (a warp-uniform branch: no per-dimension test)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float d = __fmaf_rn(x[j], 0x1p-32f, -u[j]);  // x - u, one rounding
        prod = __fmul_rn(prod, __fadd_rn(__fmaf_rn(d, d, ch[j]), cl[j]));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if ((uint32_t)j < s) {
          const float d = __fmaf_rn(x[j], 0x1p-32f, -u[j]);
          prod = __fmul_rn(prod, __fadd_rn(__fmaf_rn(d, d, ch[j]), cl[j]));
        }
      }
    }
    return __frcp_rn(prod);
  }
};

template <>
struct Integrand<QMC_F_GENZ_OSCILLATORY> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  uint32_t s;
  float a[16];
  float c0, s0;  // cos, sin of 2 pi u_1
  __device__ void setup(const float* th, uint32_t s_) {
    s = s_;
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = (uint32_t)j < s ? __ldg(th + j) * 0x1p-32f : 0.0f;  // a_j x_j = (a_j 2^-32) X_j
    sincospif(2.0f * __ldg(th + s), &s0, &c0);
  }
  // cos(2 pi u_1 + B) = cos(2 pi u_1) cos B - sin(2 pi u_1) sin B, B = sum_j a_j x_j
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    float B = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) B = __fmaf_rn(a[j], x[j], B);  // a_j = 0 beyond s adds exactly 0
    float sb, cb;
    sincosf(B, &sb, &cb);
    return __fmaf_rn(c0, cb, -__fmul_rn(s0, sb));
  }
};

constexpr float kLn2 = 0.693147180559945309f;

// Mixture of four separable Gaussians.  G_c = 2^t with t = -q_c k_c,
// q_c = sum_d (x_d - m_{c,d})^2 and k_c = log2(e)/(2 sigma_c^2) held as a
// float pair.  In fp32, q carries up to ~8 unit roundoffs of relative error,
// so G_c's relative error grows like 8u ln2 |t|; err returns sum_c w_c G_c |t_c|
// for the caller's budget test.  The EXACT path forms |x - m| exactly
// (Fast2Sum on the ordered pair), squares it with an FMA residual, sums the
// squares with TwoSum and applies the low word of t as a first-order factor.
template <>
struct Integrand<QMC_F_GAUSSMIX4_6D> {
  static constexpr int S = 6;
  static constexpr bool kAdaptive = true;
  float wsum;
  float w[4], mu[4], nu[4], kh[4], kl[4];
  float is2[4], is3[4];  // 1/sigma^2, 1/sigma^3 (gradient only)
  __device__ void setup(const float* th, uint32_t) {
    wsum = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(th) + c);
      w[c] = t.x;
      mu[c] = t.y;
      nu[c] = t.z;
      wsum += fabsf(t.x);
      const float sg = t.w;
      float e;
      const float s2 = two_prod(sg, sg, e);  // sigma^2 = s2 + e exactly
      float rl;
      const float rh = ff_recip(2.0f * s2, 2.0f * e, rl);  // 1/(2 sigma^2)
      float pe;
      const float p = two_prod(rh, kLog2eHi, pe);
      kh[c] = p;
      kl[c] = pe + rh * kLog2eLo + rl * kLog2eHi;
      is2[c] = __frcp_rn(s2);
      is3[c] = is2[c] * __frcp_rn(sg);
    }
  }

  // 2^(-q k) for component c of the scaled point X (x = X 2^-32); q_out receives q
  // (its leading word when EXACT); with SUMS, se / so receive the sums of the
  // differences over the even / odd dimensions (gradient).
  template <bool EXACT, bool SUMS>
  __device__ __forceinline__ float gauss(const float* X, int c, float& q_out, float& t_abs, float& se,
                                         float& so) const {
    if constexpr (!EXACT) {
      float q = 0.0f;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const float diff = __fmaf_rn(X[d], 0x1p-32f, (d & 1) ? -nu[c] : -mu[c]);  // x - m, one rounding
        q = __fmaf_rn(diff, diff, q);
        if constexpr (SUMS) {  // the differences themselves: sum x - 3 mu would cancel near the mean
          if (d & 1) so = __fadd_rn(so, diff); else se = __fadd_rn(se, diff);
        }
      }
      const float t = __fmaf_rn(q, kh[c], __fmul_rn(q, kl[c]));
      q_out = q;
      t_abs = t;
      return ex2_approx(-t);
    } else {
      float qh = 0.0f, ql = 0.0f;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const float m = (d & 1) ? nu[c] : mu[c];
        const float xd = __fmul_rn(X[d], 0x1p-32f);  // exact
        if constexpr (SUMS) {
          const float diff = __fsub_rn(xd, m);
          if (d & 1) so = __fadd_rn(so, diff); else se = __fadd_rn(se, diff);
        }
        const float hi = fmaxf(xd, m), lo = fminf(xd, m);
        const float D = __fsub_rn(hi, lo);                        // |x - m| rounded
        const float e = __fsub_rn(-lo, __fsub_rn(D, hi));         // exact remainder (Fast2Sum)
        const float p = __fmul_rn(D, D);
        const float pe = __fmaf_rn(2.0f * D, e, __fmaf_rn(D, D, -p));
        float se;
        qh = two_sum(qh, p, se);
        ql = __fadd_rn(ql, __fadd_rn(se, pe));
      }
      const float th = __fmul_rn(qh, kh[c]);
      const float tl = __fadd_rn(__fmaf_rn(qh, kh[c], -th), __fmaf_rn(qh, kl[c], __fmul_rn(ql, kh[c])));
      q_out = qh;
      t_abs = th;
      return __fmul_rn(ex2_approx(-th), __fmaf_rn(-kLn2, tl, 1.0f));
    }
  }

  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    float f = 0.0f;
    err = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float q, t, se, so;
      const float wG = __fmul_rn(w[c], gauss<EXACT, false>(x, c, q, t, se, so));
      f = __fadd_rn(f, wG);
      err = __fmaf_rn(fabsf(wG), t, err);
    }
    return f;
  }

  // f and the per-sample factors of df/dtheta (theta order w, mu, nu, sigma per
  // component): gq[4c..4c+3] = (G_c, sum_even (x_d - mu_c), sum_odd (x_d - nu_c),
  // q_c), so that df/dw = G, df/dmu = (w / sigma^2) G se, df/dnu = (w / sigma^2)
  // G so, df/dsigma = (w / sigma^3) G q.  The constant factors multiply the
  // item's sums once (grad_scale) instead of every sample.
  template <bool EXACT>
  __device__ __forceinline__ float eval_grad(const float* x, float* gq, float& err) const {
    float f = 0.0f;
    err = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float q, t, se = 0.0f, so = 0.0f;
      const float G = gauss<EXACT, true>(x, c, q, t, se, so);
      const float wG = __fmul_rn(w[c], G);
      f = __fadd_rn(f, wG);
      err = __fmaf_rn(fabsf(wG), t, err);
      gq[4 * c + 0] = G;
      gq[4 * c + 1] = se;
      gq[4 * c + 2] = so;
      gq[4 * c + 3] = q;
    }
    return f;
  }

  // factor of value v (1..16, theta order) that eval_grad's sums leave out
  __device__ __forceinline__ float grad_scale(int v) const {
    const int c = (v - 1) >> 2, k = (v - 1) & 3;
    return k == 0 ? 1.0f : k == 3 ? __fmul_rn(w[c], is3[c]) : __fmul_rn(w[c], is2[c]);
  }
};

// The procedural scene (a Fig. 1 substitute): irradiance from a square light,
// through a spherical occluder, onto a checkerboard plane seen from above.
// theta = (fx, fy, fw, fh, cx, cy, h, side, Le, ox, oy, oz, rho, freq, -, -).
// The checker and occlusion decisions use explicitly rounded fp32 operations
// in a fixed order (no contraction into fused multiply-adds), so any IEEE
// machine that evaluates the same sequence takes the same decisions.
template <>
struct Integrand<QMC_F_SCENE4D> {
  static constexpr int S = 4;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  float fx, fy, fw, fh, cx, cy, h, side, ox, oy, oz, rho2, freq, K;
  __device__ void setup(const float* th, uint32_t) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(th));
    const float4 b = __ldg(reinterpret_cast<const float4*>(th) + 1);
    const float4 c = __ldg(reinterpret_cast<const float4*>(th) + 2);
    const float4 d = __ldg(reinterpret_cast<const float4*>(th) + 3);
    fx = a.x, fy = a.y, fw = a.z, fh = a.w;
    cx = b.x, cy = b.y, h = b.z, side = b.w;
    ox = c.y, oy = c.z, oz = c.w;
    rho2 = __fmul_rn(d.x, d.x);
    freq = d.y;
    K = c.x * side * side * h * h;  // Le side^2 h^2 (shading only)
    wsum = K / (h * h * h * h);     // the largest value of f / albedo: the scale of the estimate
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* X, float& err) const {
    err = 0.0f;
    const float u0 = __fmul_rn(X[0], 0x1p-32f), u1 = __fmul_rn(X[1], 0x1p-32f);  // exact
    const float u2 = __fmul_rn(X[2], 0x1p-32f), u3 = __fmul_rn(X[3], 0x1p-32f);
    const float Px = __fadd_rn(fx, __fmul_rn(fw, u0));
    const float Py = __fadd_rn(fy, __fmul_rn(fh, u1));
    const float Lx = __fadd_rn(cx, __fmul_rn(side, __fsub_rn(u2, 0.5f)));
    const float Ly = __fadd_rn(cy, __fmul_rn(side, __fsub_rn(u3, 0.5f)));
    const float Dx = __fsub_rn(Lx, Px), Dy = __fsub_rn(Ly, Py), Dz = h;
    const float Ex = __fsub_rn(Px, ox), Ey = __fsub_rn(Py, oy), Ez = -oz;
    const float DE = __fadd_rn(__fadd_rn(__fmul_rn(Dx, Ex), __fmul_rn(Dy, Ey)), __fmul_rn(Dz, Ez));
    const float DD = __fadd_rn(__fadd_rn(__fmul_rn(Dx, Dx), __fmul_rn(Dy, Dy)), __fmul_rn(Dz, Dz));
    const float EE = __fadd_rn(__fadd_rn(__fmul_rn(Ex, Ex), __fmul_rn(Ey, Ey)), __fmul_rn(Ez, Ez));
    const float disc = __fsub_rn(__fmul_rn(DE, DE), __fmul_rn(DD, __fsub_rn(EE, rho2)));
    if (!(disc < 0.0f)) return 0.0f;  // the sphere blocks the light
    const int cell = ((int)floorf(__fmul_rn(Px, freq)) + (int)floorf(__fmul_rn(Py, freq))) & 1;
    return __fdividef(cell ? 0.8f * K : 0.2f * K, __fmul_rn(DD, DD));  // DD = |L - P|^2
  }
};

// ---------------------------------------------------------------------------
// Kahan accumulation (true value = s - c) and the per-item store.
// ---------------------------------------------------------------------------
struct Kahan {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ Comp comp() const { return {s, -c}; }
};

// Warp-cooperative search: the integral p with item_off[p] <= item < item_off[p+1]
// (32 probes per round, so about log32(n) dependent loads).
__device__ __forceinline__ uint32_t find_integral(const uint32_t* off, uint32_t n, uint32_t item) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t lo = 0, hi = n;  // off[lo] <= item < off[hi]
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) >> 5;
    const uint64_t pos = (uint64_t)lo + (uint64_t)(lane + 1) * step;
    const bool le = pos < hi && __ldg(off + pos) <= item;
    const uint32_t m = __popc(__ballot_sync(0xffffffffu, le));
    const uint64_t nhi = (uint64_t)lo + (uint64_t)(m + 1) * step;
    lo += m * step;
    if (nhi < hi) hi = (uint32_t)nhi;
  }
  return lo;
}

// Per-sample rounding-error coefficient of the fp32 mixture path: relative
// error of G <= 8 u ln2 |t| (u = 2^-24), see Integrand<GAUSSMIX4_6D>.
constexpr float kKappa = 8.0f * 5.9604645e-8f * kLn2;

// One pass over the samples of the current item.  Returns nothing; adds into
// acc and, on the fp32 pass, the squared per-sample error scales into e2.
// Samples are summed in blocks of kBlock consecutive iterations with plain fp32
// adds, and each block sum enters the lane's Kahan sum (a two-level reduction,
// Sec. 2.5.1): the block adds carry at most (kBlock-1) unit roundoffs of the
// block's absolute sum, the compensated sum carries almost nothing.
constexpr uint32_t kBlock = 4;

template <bool EXACT, bool GRAD, int NV, class Src, class F>
__device__ __forceinline__ void run_item(const Src& src, const F& f, uint32_t len, Kahan (&acc)[NV],
                                         float& e2) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t R = (len + 31u) >> 5;
  for (uint32_t r0 = 0; r0 < R; r0 += kBlock) {
    float blk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) blk[v] = 0.0f;
    const uint32_t r1 = min(R, r0 + kBlock);
    for (uint32_t r = r0; r < r1; ++r) {
      const uint32_t il = (r << 5) + lane;
      const bool valid = il < len;
      float x[F::S];
      src.point(r, il, valid, x);
      float err;
      if constexpr (GRAD) {
        float gq[16];
        const float v = f.template eval_grad<EXACT>(x, gq, err);
        if (valid) {
          blk[0] = __fadd_rn(blk[0], v);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float G = gq[4 * c];
            blk[1 + 4 * c] = __fadd_rn(blk[1 + 4 * c], G);
            blk[2 + 4 * c] = __fmaf_rn(G, gq[4 * c + 1], blk[2 + 4 * c]);
            blk[3 + 4 * c] = __fmaf_rn(G, gq[4 * c + 2], blk[3 + 4 * c]);
            blk[4 + 4 * c] = __fmaf_rn(G, gq[4 * c + 3], blk[4 + 4 * c]);
          }
          if constexpr (F::kAdaptive && !EXACT) e2 = __fmaf_rn(err, err, e2);
        }
      } else {
        const float v = f.template eval<EXACT>(x, err);
        if (valid) {
          blk[0] = __fadd_rn(blk[0], v);
          if constexpr (F::kAdaptive && !EXACT) e2 = __fmaf_rn(err, err, e2);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      // The estimate keeps the compensated sum.  The parameter gradients are
      // held to a tolerance relative to the mean absolute derivative, which a
      // plain sum of the lane's block sums meets with a wide margin (about
      // (kBlock - 1 + blocks) unit roundoffs of the sum of absolute terms).
      if (v == 0) acc[v].add(blk[v]);
      else acc[v].s = __fadd_rn(acc[v].s, blk[v]);
    }
  }
}

template <class Src, int FN, bool GRAD>
__global__ void __launch_bounds__(256) integrate_main(IntegrateArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  using F = Integrand<FN>;
  constexpr int NV = GRAD ? 17 : 1;
  Src src;
  src.kernel_setup(a, smem);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t total = a.hdr->total_items;
  const uint32_t C = 1u << a.chunk_log2;
  const uint32_t pstride = a.theta_stride;

  uint32_t next = 0;
  if (lane == 0) next = atomicAdd(&a.hdr->next_item, 1u);
  next = __shfl_sync(0xffffffffu, next, 0);
  while (next < total) {
    const uint32_t item = next;
    if (lane == 0) next = atomicAdd(&a.hdr->next_item, 1u);  // prefetch the next item
    const uint32_t p = find_integral(a.item_off, a.n, item);
    const uint32_t start = (item - __ldg(a.item_off + p)) << a.chunk_log2;
    const uint32_t n_p = __ldg(a.counts + p);
    const uint32_t len = min(C, n_p - start);
    F f;
    f.setup(a.theta ? a.theta + (size_t)p * pstride : nullptr, a.s);
    src.item_setup(a, p, start);

    Kahan acc[NV];
    float e2 = 0.0f;
    run_item<false, GRAD>(src, f, len, acc, e2);
    if constexpr (F::kAdaptive) {
      // Budget test on the item: the fp32 rounding errors of the samples are
      // treated as independent, so their sum has scale kKappa sqrt(e2); an
      // item whose 3-sigma error exceeds 0.6e-6 of its sum (plus its share of
      // the 1e-12 W absolute floor) is recomputed on the exact path.  The test
      // depends only on the item's data, so results stay reproducible.
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      const Comp tot = warp_comp_sum(acc[0].comp());
      const float budget = 0.6e-6f * fabsf(tot.sum + tot.err) + 0.5e-12f * f.wsum * (float)len;
      if (3.0f * kKappa * sqrtf(e2) > budget) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = Kahan{};
        run_item<true, GRAD>(src, f, len, acc, e2);
      }
    }
    float* out = a.partials + (size_t)item * (2 * NV);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const Comp c = warp_comp_sum(acc[v].comp());
      float k = 1.0f;
      if constexpr (GRAD) {
        if (v > 0) k = f.grad_scale(v);
      }
      if (lane == (uint32_t)(v & 31)) {
        out[2 * v] = __fmul_rn(c.sum, k);
        out[2 * v + 1] = __fmul_rn(c.err, k);
      }
    }
    next = __shfl_sync(0xffffffffu, next, 0);
  }
}

// ---------------------------------------------------------------------------
// 5-6: per-integral reductions.  The compensated partials of an integral are
// merged in item order with error-free fp32 transformations (TwoSum), which
// keep the sum exact to ~2^-48; fp64 -- slow on GB300 -- is used only for the
// final combination of that float pair and the division by n_p.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Comp comp_load(const float* q) { return {q[0], q[1]}; }

__device__ __forceinline__ double comp_to_double(Comp c) { return (double)c.sum + (double)c.err; }

// One warp per integral: lane l merges items l, l+32, ..., then a fixed butterfly.
__global__ void __launch_bounds__(256) reduce_forward(IntegrateArgs a) {
  const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (p >= a.n) return;
  if (a.hdr->error_bits) {  // offsets were not written: report NaN, touch no partial
    if (lane == 0) a.estimate[p] = __longlong_as_double(0x7FF8000000000000ll);
    return;
  }
  const uint32_t b = a.item_off[p], e = a.item_off[p + 1];
  Comp acc{0.0f, 0.0f};
  for (uint32_t it = b + lane; it < e; it += 32) acc = comp_merge(acc, comp_load(a.partials + 2 * (size_t)it));
  acc = warp_comp_sum(acc);
  if (lane == 0) {
    const uint32_t n_p = a.counts[p];
    a.estimate[p] = n_p ? comp_to_double(acc) / (double)n_p : 0.0;
  }
}

// GRAD partials: 17 values per item (f, 16 derivatives).  Lane v < 17 merges
// value v over the integral's items in item order.  The estimate I_p and the
// loss term are fp64; the Jacobian J = sum/n_p and the gradient product are fp32
// (relative error ~2e-7, far inside the gradient tolerance).
__global__ void __launch_bounds__(256) reduce_grad(IntegrateArgs a) {
  const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (p >= a.n) return;
  if (a.hdr->error_bits) {  // offsets were not written: report NaN, touch no partial
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    if (lane == 0 && a.target) {
      a.estimate[p] = nan;
      a.ws_loss_terms[p] = nan;
    }
    if (lane >= 1 && lane < 17) a.grad_theta[p * 16 + (lane - 1)] = __int_as_float(0x7FC00000);
    return;
  }
  const uint32_t b = a.item_off[p], e = a.item_off[p + 1];
  Comp acc{0.0f, 0.0f};
  if (lane < 17)
    for (uint32_t it = b; it < e; ++it) acc = comp_merge(acc, comp_load(a.partials + (size_t)it * 34 + 2 * lane));
  const uint32_t n_p = a.counts[p];
  float scale = 0.0f;
  if (lane == 0) {
    const double I = n_p ? comp_to_double(acc) / (double)n_p : 0.0;
    if (a.target) {  // fused squared-error loss
      const double diff = I - a.target[p];
      a.estimate[p] = I;
      a.ws_loss_terms[p] = diff * diff;
      scale = (float)(2.0 * diff);
    } else {
      scale = (float)a.grad_est[p];
    }
  }
  scale = __shfl_sync(0xffffffffu, scale, 0);
  if (lane >= 1 && lane < 17) {
    const float J = n_p ? __fadd_rn(acc.sum, acc.err) * __frcp_rn((float)n_p) : 0.0f;
    a.grad_theta[p * 16 + (lane - 1)] = scale * J;
  }
}

// Fixed-order sum of the loss terms: kLossBlocks blocks each add a contiguous
// range (thread-strided, then a block tree), one block adds the block sums.
constexpr uint32_t kLossBlocks = 256;

__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += sh[w];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(256) loss_partial(IntegrateArgs a) {
  __shared__ double sh[8];
  const uint64_t per = (a.n + kLossBlocks - 1) / kLossBlocks;
  const uint64_t lo = blockIdx.x * per, hi = min((uint64_t)a.n, lo + per);
  double s = 0.0;
  for (uint64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) s += a.ws_loss_terms[p];
  const double t = block_sum_f64(s, sh);
  if (threadIdx.x == 0) a.ws_loss_terms[a.n + blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) loss_final(IntegrateArgs a) {
  __shared__ double sh[8];
  const double s = threadIdx.x < kLossBlocks ? a.ws_loss_terms[a.n + threadIdx.x] : 0.0;
  const double t = block_sum_f64(s, sh);
  if (threadIdx.x == 0) a.loss[0] = t;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <class Src, int FN, bool GRAD>
cudaError_t launch_main_t(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  auto kernel = integrate_main<Src, FN, GRAD>;
  const size_t smem = Src::smem_bytes(a.s, a.chunk_log2);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)block, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const DeviceInfo& dev = device_info();
  kernel<<<(unsigned)(dev.sm_count * per_sm), block, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int FN, bool GRAD>
cudaError_t launch_main_fn(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  constexpr int S = Integrand<FN>::S;
  if (a.points) return launch_main_t<PointsSource<S>, FN, GRAD>(a, block, stream);
  if (a.source == QMC_SOURCE_PIXEL_LATTICE) return launch_main_t<PixelLatticeSource<S>, FN, GRAD>(a, block, stream);
  if (a.source == QMC_SOURCE_RANDOM_LATTICE)
    return (a.randomize & 0xFFu) == QMC_RLAT_HASH
               ? launch_main_t<RandomLatticeSource<S, QMC_RLAT_HASH>, FN, GRAD>(a, block, stream)
               : launch_main_t<RandomLatticeSource<S, QMC_RLAT_LFSR>, FN, GRAD>(a, block, stream);
  if (a.source == QMC_SOURCE_LATTICE)
    return (a.randomize & QMC_LATTICE_BACKWARD) ? launch_main_t<LatticeSource<S, true>, FN, GRAD>(a, block, stream)
                                                : launch_main_t<LatticeSource<S, false>, FN, GRAD>(a, block, stream);
  const uint32_t scr = a.seeds ? a.randomize : 0u;
  if (scr == QMC_SCRAMBLE_NESTED) return launch_main_t<SobolSource<S, 2>, FN, GRAD>(a, block, stream);
  if (scr == QMC_SCRAMBLE_XOR) return launch_main_t<SobolSource<S, 1>, FN, GRAD>(a, block, stream);
  return launch_main_t<SobolSource<S, 0>, FN, GRAD>(a, block, stream);
}

}  // namespace

cudaError_t launch_integrate(const IntegrateArgs& a, uint32_t block, bool grad, cudaStream_t stream) {
  const uint32_t n_blocks = (uint32_t)(((uint64_t)a.n + kScanBlock) / kScanBlock);  // covers entry n
  scan_totals<<<n_blocks, kScanThreads, 0, stream>>>(a);
  scan_carry<<<1, 1024, 0, stream>>>(a, n_blocks);
  scan_write<<<n_blocks, kScanThreads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (a.integrand) {
    case QMC_F_BILINEAR2D: e = launch_main_fn<QMC_F_BILINEAR2D, false>(a, block, stream); break;
    case QMC_F_GENZ_PRODUCT_PEAK: e = launch_main_fn<QMC_F_GENZ_PRODUCT_PEAK, false>(a, block, stream); break;
    case QMC_F_GENZ_OSCILLATORY: e = launch_main_fn<QMC_F_GENZ_OSCILLATORY, false>(a, block, stream); break;
    case QMC_F_SCENE4D: e = launch_main_fn<QMC_F_SCENE4D, false>(a, block, stream); break;
    default:
      e = grad ? launch_main_fn<QMC_F_GAUSSMIX4_6D, true>(a, block, stream)
               : launch_main_fn<QMC_F_GAUSSMIX4_6D, false>(a, block, stream);
  }
  if (e != cudaSuccess) return e;
  const uint64_t threads = (uint64_t)a.n * 32;
  const unsigned rblocks = (unsigned)((threads + 255) / 256);
  if (grad) {
    reduce_grad<<<rblocks, 256, 0, stream>>>(a);
    if (a.target) {
      loss_partial<<<kLossBlocks, 256, 0, stream>>>(a);
      loss_final<<<1, 256, 0, stream>>>(a);
    }
  } else {
    reduce_forward<<<rblocks, 256, 0, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace qmc

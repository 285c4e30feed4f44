// integrate_kernel.cuh -- the persistent integration kernel of the fused path
// (Sec. 2.5): the point sources, the per-sample accumulation, the work-item loop
// and its launcher, as templates over the source and the integrand.  Each
// integrand family instantiates them in its own translation unit
// (integrate_bilinear.cu, integrate_genz.cu, integrate_gaussmix.cu,
// integrate_scene.cu); integrate.cu holds the scans, the reductions and the
// dispatch.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/qmc.h"
#include "qmc_checked.cuh"
#include "qmc_device.cuh"
#include "qmc_integrate.h"
#include "qmc_internal.h"

namespace qmc {
namespace integ {

// ---------------------------------------------------------------------------
// Point sources.  Each produces the S coordinates of local sample il of the
// current item (sample index start + il) in the scaled form X = x * 2^32 of
// unifloat_x2p32 (exact: x = map_u32_to_unifloat(u) = X * 2^-32); the
// integrands fold the 2^-32 into their constants.
// ---------------------------------------------------------------------------
template <int S, int SCR>  // SCR: 0 none, 1 XOR, 2 nested (or, by a.randomize, XOR then nested)
struct SobolSource {
  static constexpr int kRow = (S + 3) & ~3;  // table row stride: whole 128-bit words
  const uint32_t* cols;  // shared: [s][m], mirrored when nested
  const uint32_t* tab;   // shared: [C/32][kRow], y(32 r)
  uint32_t s;
  uint32_t lane_y[S];    // y(lane)
  uint32_t yl[S];        // y(start) ^ y(lane) (^ seed for XOR) (^ the element's fixed low part)
  NestedKey key[S];

  // offset of the table: the columns, rounded up to whole 16-byte words
  __host__ __device__ static uint32_t table_offset(uint32_t s, uint32_t m) { return (s * m + 3u) & ~3u; }

  static size_t smem_bytes(const IntegrateArgs& a) {
    return ((size_t)table_offset(a.s, a.sobol_m) + ((size_t)1 << (a.chunk_log2 - 5)) * kRow) * sizeof(uint32_t);
  }

  // Sample J of an item (J below 2^32) is index i = (J << q) | c_p of an m-column sequence
  // (m = a.sobol_m, q = a.part_log2, read from the kernel parameters where used); every
  // column touched lies below q + 32 <= m (checked on the host).
  __device__ void kernel_setup(const IntegrateArgs& a, uint32_t* smem) {
    s = a.s;
    const uint32_t m = a.sobol_m, q = a.part_log2;
    uint32_t* c = smem;
    uint32_t* t = smem + table_offset(s, m);
    for (uint32_t i = threadIdx.x; i < s * m; i += blockDim.x) {
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
          if ((r >> b) & 1u) y ^= c[j * m + q + 5 + b];
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
          if ((lane >> b) & 1u) y ^= c[j * m + q + b];
      lane_y[j] = y;
    }
  }

  __device__ void item_setup(const IntegrateArgs& a, uint32_t p, uint32_t start) {
    const uint32_t khi = start >> a.chunk_log2;
    const uint32_t m = a.sobol_m, q = a.part_log2;
    const uint32_t* sd = a.seeds ? a.seeds + (a.seeds_per_integral ? (size_t)p * s : 0) : nullptr;
    // partitioned: integral p enumerates element p mod 2^q, whose indices carry the q-bit
    // reversal of the element number in their low bits
    const uint32_t cp = q ? __brev(p) >> (32u - q) : 0u;  // the low q bits of p, reversed
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t y = 0;
      if ((uint32_t)j < s) {
        for (uint32_t b = 0; (khi >> b) != 0; ++b)
          if ((khi >> b) & 1u) y ^= cols[j * m + q + a.chunk_log2 + b];
        for (uint32_t b = 0; (cp >> b) != 0; ++b)
          if ((cp >> b) & 1u) y ^= cols[j * m + b];
      }
      const uint32_t seed = (sd && (uint32_t)j < s) ? __ldg(sd + j) : 0u;
      // XOR: the digital shift; NESTED_XOR: the same shift before the nested scramble, in the
      // mirrored domain the columns are stored in
      const bool shift_mirrored = SCR == 2 && a.randomize == QMC_SCRAMBLE_NESTED_XOR;
      yl[j] = y ^ lane_y[j] ^ (SCR == 1 ? seed : 0u) ^ (shift_mirrored ? __brev(seed) : 0u);
      key[j] = nested_key(seed);
    }
  }

  __device__ __forceinline__ void point(uint32_t r, uint32_t /*il*/, bool /*valid*/, float* x) const {
    uint32_t row[kRow];
#pragma unroll
    for (int k = 0; k < kRow / 4; ++k) {  // 128-bit shared loads
      const uint4 w = reinterpret_cast<const uint4*>(tab + r * kRow)[k];
      row[4 * k] = w.x, row[4 * k + 1] = w.y, row[4 * k + 2] = w.z, row[4 * k + 3] = w.w;
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

  static size_t smem_bytes(const IntegrateArgs&) { return 0; }

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

  static size_t smem_bytes(const IntegrateArgs&) { return 0; }

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

  static size_t smem_bytes(const IntegrateArgs&) {
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

  static size_t smem_bytes(const IntegrateArgs&) { return 0; }

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
// integrands, err = an estimate of the sample's rounding error scale (kErrUnit
// turns it into an absolute scale).  EXACT selects the float-float evaluation
// used when an item's error estimate is over budget; non-adaptive integrands
// ignore it.  With kExactPair the EXACT evaluation returns f as a float pair
// (the value and, in err, its low word), and both words enter the compensated
// sum sample by sample.  kMinBlocks is the kernel's minimum of resident
// 256-thread blocks per SM (0: the compiler's choice of registers).
constexpr float kLn2 = 0.693147180559945309f;

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

// Unit roundoff of fp32 (2^-24).  Each adaptive integrand states kErrUnit, the
// factor that turns its per-sample err into an absolute error scale.
constexpr float kU32 = 5.9604645e-8f;

// One pass over the samples of the current item.  Returns nothing; adds into
// acc and, on the fp32 pass, the squared per-sample error scales into e2.
// Samples are summed in blocks of kBlock consecutive iterations with plain fp32
// adds, and each block sum enters the lane's Kahan sum of the estimate (a
// two-level reduction, Sec. 2.5.1): the block adds carry at most (kBlock-1)
// unit roundoffs of the block's absolute sum, the compensated sum carries
// almost nothing.  The parameter gradients' block sums enter plain running
// sums: their error against the fp64 oracle is set by the fp32 evaluation of
// each term (about 8u ln2 |t| relative, see the mixture), which a compensated
// sum was measured not to reduce, at 16 more registers and 10 % of the fused
// kernel's rate.  Whole blocks of full rows (all 32 samples of each row in the
// item) run unrolled -- by kBlock, by two with the gradient, whose 17 sums leave
// fewer registers -- with no per-sample test of the sample's existence; the
// remaining rows (fewer than kBlock full ones and the ragged last) run sample by
// sample with it.
constexpr uint32_t kBlock = 4;

template <bool EXACT, bool GRAD, bool FULL, int NV, class Src, class F>
__device__ __forceinline__ void run_sample(const Src& src, const F& f, uint32_t r, uint32_t len, float (&blk)[NV],
                                           Kahan (&acc)[NV], float& e2) {
  const uint32_t il = (r << 5) + (threadIdx.x & 31u);
  const bool valid = FULL || il < len;
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
      if constexpr (EXACT && F::kExactPair) {  // f = v + err: both words, each compensated
        acc[0].add(v);
        acc[0].add(err);
      } else {
        blk[0] = __fadd_rn(blk[0], v);
      }
      if constexpr (F::kAdaptive && !EXACT) e2 = __fmaf_rn(err, err, e2);
    }
  }
}

template <bool EXACT, bool GRAD, int NV, class Src, class F>
__device__ __forceinline__ void run_item(const Src& src, const F& f, uint32_t len, Kahan (&acc)[NV],
                                         float& e2) {
  const uint32_t R = (len + 31u) >> 5;
  auto fold = [&](const float (&blk)[NV]) {
    if constexpr (!(EXACT && F::kExactPair)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (v == 0) acc[v].add(blk[v]);                // the estimate: compensated
        else acc[v].s = __fadd_rn(acc[v].s, blk[v]);   // the gradients: plain
      }
    }
  };
  uint32_t r0 = 0;
  const uint32_t Rfull = len >> 5;  // rows whose 32 samples all exist
  for (; r0 + kBlock <= Rfull; r0 += kBlock) {
    float blk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) blk[v] = 0.0f;
#pragma unroll (GRAD ? 2 : kBlock)
    for (uint32_t k = 0; k < kBlock; ++k) run_sample<EXACT, GRAD, true>(src, f, r0 + k, len, blk, acc, e2);
    fold(blk);
  }
  while (r0 < R) {  // the rest: at most kBlock - 1 full rows and the ragged last row, in blocks
    float blk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) blk[v] = 0.0f;
    const uint32_t r1 = min(R, r0 + kBlock);
    for (uint32_t r = r0; r < r1; ++r) run_sample<EXACT, GRAD, false>(src, f, r, len, blk, acc, e2);
    fold(blk);
    r0 = r1;
  }
}

template <class Src, int FN, bool GRAD>
__global__ void __launch_bounds__(256, Integrand<FN>::kMinBlocks) integrate_main(IntegrateArgs a) {
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
      // treated as independent, so their sum has scale kErrUnit sqrt(e2); an
      // item whose 3-sigma error exceeds 0.6e-6 of its sum (plus its share of
      // the 1e-12 W absolute floor) is recomputed on the exact path.  The test
      // depends only on the item's data, so results stay reproducible.
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      const Comp tot = warp_comp_sum(acc[0].comp());
      const float budget = 0.6e-6f * fabsf(tot.sum + tot.err) + 0.5e-12f * f.wsum * (float)len;
      if (3.0f * F::kErrUnit * sqrtf(e2) > budget) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = Kahan{};
        run_item<true, GRAD>(src, f, len, acc, e2);
      }
    }
    float* out = a.partials + (size_t)item * (2 * NV);
    const bool store_ok = in_bounds(CheckCtx{a.check_word, a.capacity_items}, item, 1, kCheckPartials);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const Comp c = warp_comp_sum(acc[v].comp());
      float k = 1.0f;
      if constexpr (GRAD) {
        if (v > 0) k = f.grad_scale(v);
      }
      if (store_ok && lane == (uint32_t)(v & 31)) {
        out[2 * v] = __fmul_rn(c.sum, k);
        out[2 * v + 1] = __fmul_rn(c.err, k);
      }
    }
    next = __shfl_sync(0xffffffffu, next, 0);
  }
}

// ---------------------------------------------------------------------------
// Host side: launch the persistent kernel for one integrand, every source
// ---------------------------------------------------------------------------
template <class Src, int FN, bool GRAD>
cudaError_t launch_main_t(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  auto kernel = integrate_main<Src, FN, GRAD>;
  const size_t smem = Src::smem_bytes(a);
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
  if (scr >= QMC_SCRAMBLE_NESTED) return launch_main_t<SobolSource<S, 2>, FN, GRAD>(a, block, stream);
  if (scr == QMC_SCRAMBLE_XOR) return launch_main_t<SobolSource<S, 1>, FN, GRAD>(a, block, stream);
  return launch_main_t<SobolSource<S, 0>, FN, GRAD>(a, block, stream);
}

}  // namespace integ
}  // namespace qmc

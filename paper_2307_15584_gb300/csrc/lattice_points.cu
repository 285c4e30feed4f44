// lattice_points.cu -- materialised rank-1 lattice points (HBM-write bound):
//   lattice_points_*          Eq. (R1LS) / Alg. 4: x_j(k) = phi_2(k) g_j + shift_j mod 2^32,
//                             forward or backward;
//   pixel_lattice_points_*    Sec. 3, Eq. (PixelShiftedR1LS): one phi_3 shift per pixel
//                             along the Hilbert curve;
//   random_lattice_points_*   Alg. 4, Sec. 2.4.2, Sec. 3: a random generator vector per
//                             pixel (hashed or LFSR) and superimposed instances.
// Layouts as in sobol_points.cu: rows [count][s] u32/f32, coalesced 16-byte chunks;
// phi_2 of disjoint index bit fields adds without carries, so the rank-1 lattice
// takes x = phi_2(G*Q) g_j + lo_e with one bit reversal per group.
#include <cstdint>

#include "points_common.cuh"

namespace qmc {

namespace {
using namespace pts;

// ---------------------------------------------------------------------------
// K2: rank-1 lattice.  BACKWARD follows Alg. 4: phi_2(~k) = ~phi_2(k), so
// x = shift - g - phi_2(k) g (mod 2^32).  Direct 16-byte stores; each warp takes
// a short range of groups (launch_spread), so the resident warps write
// neighbouring parts of the output.
// ---------------------------------------------------------------------------
template <int K, bool BACKWARD>
__global__ void __launch_bounds__(kThreads) lattice_points_fast(PointsArgs a) {
  const uint32_t lane = threadIdx.x & 31u;
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
        store4(a.out_u32, a.out_f32, o, v, a.chk);
      } else {  // ragged last group: per-element row test
        const uint64_t rows_left = a.count - (g << a.q_log2);
        const uint32_t e0 = 4u * (lane + 32u * c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if ((uint64_t)((e0 + t) / s) < rows_left) store1(a.out_u32, a.out_f32, o + t, v[t], a.chk);
      }
    }
  }
}

// K2 for the shapes the fast path's groups do not fit (s / gcd(s, 128) > 4, or an
// index_begin off the group grid): a warp takes batches of kFlatRows consecutive
// rows and writes them as 16-byte chunks of the flat [row][s] layout, each element
// of a chunk finding its own row and dimension (one exact multiply-high division).
// kFlatRows is a multiple of 4, so every batch starts on a 16-byte boundary.
constexpr uint32_t kFlatRows = 512;

template <bool BACKWARD>
__global__ void __launch_bounds__(kThreads) lattice_points_flat(PointsArgs a) {
  const uint32_t lane = threadIdx.x & 31u, s = a.s;
  const uint64_t mag_s = s > 1 ? ~0ull / s + 1 : 0;  // x / s = umulhi(x, .) for x < 2^32, s > 1
  const uint64_t n_batches = (a.count + kFlatRows - 1) / kFlatRows;
  uint64_t b0, b1;
  warp_range(n_batches, b0, b1);
  for (uint64_t b = b0; b < b1; ++b) {
    const uint64_t row0 = b * kFlatRows;
    const uint64_t left = a.count - row0;
    const uint32_t rows = left < kFlatRows ? (uint32_t)left : kFlatRows;
    const uint32_t total = rows * s;  // <= 2^19 elements (s <= 1024)
    const uint64_t off0 = row0 * s;   // a multiple of 4
    const uint32_t k0 = (uint32_t)a.index_begin + (uint32_t)row0;  // index of the batch's first row, mod 2^32
    for (uint32_t e = 4u * lane; e < total; e += 128u) {
      uint32_t v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t et = e + t < total ? e + t : total - 1u;
        const uint32_t r = s > 1 ? (uint32_t)__umul64hi(et, mag_s) : et;
        const uint32_t j = et - r * s;
        const uint32_t g = __ldg(a.matrices + j) | 1u;
        const uint32_t sh = a.seeds ? __ldg(a.seeds + j) : 0u;
        const uint32_t phi = __brev(k0 + r);
        v[t] = BACKWARD ? sh - g - phi * g : phi * g + sh;  // phi_2(~k) = ~phi_2(k)
      }
      if (e + 4u <= total) {
        store4(a.out_u32, a.out_f32, off0 + e, v, a.chk);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (e + t < total) store1(a.out_u32, a.out_f32, off0 + e + t, v[t], a.chk);
      }
    }
  }
}

// K2 fallback for outputs that are not 16-byte aligned: one element per thread.
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
    store1(a.out_u32, a.out_f32, f, phi * g + sh, a.chk);
  }
}

// Pixel-shifted lattice, coalesced path (16-byte aligned outputs, 32 spp s <= 2^31).
// A warp takes batches of 2^BLOG2 <= 32 consecutive pixels: lane l computes the shift
// of pixel l of the batch once (Hilbert position, then phi_3), and the batch's rows
// are written as consecutive 16-byte chunks, each element's pixel shift fetched from
// its lane with a shuffle.  LAYOUT 1 (s % 4 == 0): a chunk holds four dimensions of
// one row; LAYOUT 2 (s = 1, 2): a chunk holds 4 / s whole rows; LAYOUT 0: each of its
// four elements finds its own row, dimension and pixel.
template <int LAYOUT, int BLOG2, int NB>  // NB: batches whose shifts a warp computes together
__global__ void __launch_bounds__(kThreads, 4) pixel_lattice_points_fast(PixelPointsArgs a) {
  constexpr uint32_t kBatch = 1u << BLOG2;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t n_batches = (a.n_pixels + kBatch - 1) >> BLOG2;
  uint64_t b0, b1;
  warp_range(n_batches, b0, b1);
  // x / d = umulhi(x, floor(2^64 / d) + 1) exactly for x < 2^32 and d > 1
  const uint64_t mag_s = a.s > 1 ? ~0ull / a.s + 1 : 0;
  const uint64_t mag_spp = a.spp > 1 ? ~0ull / a.spp + 1 : 0;
  const uint32_t per_pixel = a.spp * a.s;  // elements
  // the shift of pixel `lane` of batch b (0 past the batch's pixels)
  auto shift_of = [&](uint64_t b) -> uint32_t {
    const uint64_t first = b << BLOG2;
    const uint64_t left = a.n_pixels - first;
    const uint32_t npx = left < kBatch ? (uint32_t)left : kBatch;
    if (lane >= npx) return 0u;
    const uint64_t p = a.pixel_begin + first + lane;
    return pixel_shift((uint32_t)(p % a.width), (uint32_t)(p / a.width), a.grid_log2);
  };
  // the rows of batch b, its pixels' shifts in lanes 0 .. npx - 1 of sh
  auto write_batch = [&](uint64_t b, uint32_t sh) {
    const uint64_t first = b << BLOG2;  // batch's first pixel, relative to pixel_begin
    const uint64_t left = a.n_pixels - first;
    const uint32_t npx = left < kBatch ? (uint32_t)left : kBatch;
    const uint32_t total = npx * per_pixel;  // the batch's elements
    const uint32_t chunks = (total + 3u) >> 2;
    const uint64_t off0 = first * per_pixel;  // element offset of the batch: a multiple of 8
    for (uint32_t c0 = 0; c0 < chunks; c0 += 32) {  // same trip count in every lane
      const uint32_t c = c0 + lane;
      const uint32_t e = 4u * c;  // element within the batch, < 2^32
      uint32_t v[4];
      if (LAYOUT == 2) {
        const uint32_t rpc = 4u / a.s;  // rows per chunk
        const uint32_t g0 = __ldg(a.g) | 1u, g1 = a.s == 2 ? (__ldg(a.g + 1) | 1u) : 0u;
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
          if (q < rpc) {
            const uint32_t row = (a.s == 2 ? e >> 1 : e) + q;
            const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
            const uint32_t smp = row - pl * a.spp;
            const uint32_t base = __brev(smp) + __shfl_sync(0xffffffffu, sh, pl & 31u);
            if (a.s == 2) {
              v[2 * q] = base * g0;
              v[2 * q + 1] = base * g1;
            } else {
              v[q] = base * g0;
            }
          }
        }
      } else if (LAYOUT == 1) {
        const uint32_t row = (uint32_t)__umul64hi(e, mag_s);
        const uint32_t j = e - row * a.s;
        const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
        const uint32_t smp = row - pl * a.spp;
        const uint32_t base = __brev(smp) + __shfl_sync(0xffffffffu, sh, pl & 31u);
        if (c < chunks) {
#pragma unroll
          for (int t = 0; t < 4; ++t) v[t] = base * (__ldg(a.g + j + t) | 1u);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t et = e + t;
          const uint32_t row = a.s > 1 ? (uint32_t)__umul64hi(et, mag_s) : et;
          const uint32_t j = et - row * a.s;
          const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
          const uint32_t smp = row - pl * a.spp;
          const uint32_t base = __brev(smp) + __shfl_sync(0xffffffffu, sh, pl & 31u);
          v[t] = base * (__ldg(a.g + j) | 1u);  // j < s for every element
        }
      }
      if (c < chunks) {
        if (e + 4u <= total) {
          store4(a.out_u32, a.out_f32, off0 + e, v, a.chk);
        } else {  // the batch's ragged end (s % 4 != 0)
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (e + t < total) store1(a.out_u32, a.out_f32, off0 + e + t, v[t], a.chk);
        }
      }
    }
  };
  // NB batches at a time: their shifts are independent dependency chains, computed together
  for (uint64_t b = b0; b < b1; b += NB) {
    uint32_t shv[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) shv[k] = b + k < b1 ? shift_of(b + k) : 0u;
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (b + k < b1) write_batch(b + k, shv[k]);
  }
}


// Pixel-shifted rank-1 lattice (Sec. 3), fallback for outputs that are not 16-byte aligned
// (or 32 spp s beyond 2^31): one thread per (pixel, sample) row; row r holds sample r % spp
// of pixel pixel_begin + r / spp.
__global__ void __launch_bounds__(kThreads) pixel_lattice_points_kernel(PixelPointsArgs a) {
  const uint64_t rows = a.n_pixels * a.spp;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    const uint64_t p = a.pixel_begin + r / a.spp;
    const uint32_t i = (uint32_t)(r % a.spp);
    const uint32_t shift = pixel_shift((uint32_t)(p % a.width), (uint32_t)(p / a.width), a.grid_log2);
    const uint32_t base = __brev(i) + shift;
    for (uint32_t j = 0; j < a.s; ++j) store1(a.out_u32, a.out_f32, r * a.s + j, base * (__ldg(a.g + j) | 1u), a.chk);
  }
}


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
template <int KIND, int LAYOUT>  // LAYOUT as in pixel_lattice_points_fast
__global__ void __launch_bounds__(kThreads) random_lattice_points_fast(RandomPointsArgs a) {
  extern __shared__ __align__(16) uint32_t rsm[];
  uint32_t* jump = rsm;  // LFSR: the 32-step jump table (the walk below needs no other level)
  uint32_t* pxy = rsm + (KIND == QMC_RLAT_LFSR ? kLfsrJumpWords : 0);  // [batch][2]
  // generator words [batch][R][stride]: a row stride of s + 4 keeps rows 16-byte aligned and
  // spreads the LFSR walk's per-thread rows over the banks (4-way instead of 32-way conflicts)
  uint32_t* gvec = pxy + ((2 * a.batch_pixels + 3u) & ~3u);
  if (KIND == QMC_RLAT_LFSR) {
    lfsr_jump_table_fill(jump);
    __syncthreads();
  }
  const uint32_t s = a.s, R = 1u << a.r_log2, Rs = R * s, stride = s + 4u;
  const uint64_t mag_s = s > 1 ? ~0ull / s + 1 : 0;
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
        const uint32_t row = s > 1 ? (uint32_t)__umul64hi(idx, mag_s) : idx;  // (pixel, instance)
        const uint32_t j = idx - row * s, q = row >> a.r_log2;
        gvec[row * stride + j] = rlat_hash(a.seed, row & (R - 1u), j, pxy[2 * q], pxy[2 * q + 1]) | 1u;
      }
    } else {  // one thread per (pixel, instance) walks the register through the dimensions
      for (uint32_t w = threadIdx.x; w < npx * R; w += blockDim.x) {
        const uint32_t q = w >> a.r_log2;
        uint32_t xi = rlat_lfsr_seed(a.seed, w & (R - 1u), pxy[2 * q], pxy[2 * q + 1]);
        for (uint32_t j = 0; j < s; ++j) {
          gvec[w * stride + j] = 2u * xi + 1u;
          xi = lfsr_jump32(jump, xi);
        }
      }
    }
    __syncthreads();
    const uint32_t total = npx * a.spp * s;  // the batch's elements
    const uint32_t chunks = (total + 3u) >> 2;
    const uint64_t off0 = first * a.spp * s;  // a multiple of 4 (16-byte chunks)
    for (uint32_t c = threadIdx.x; c < chunks; c += blockDim.x) {
      const uint32_t e = 4u * c;  // element within the batch, < 2^31
      uint32_t v[4];
      if (LAYOUT == 2) {  // 4 / s whole rows: the index math once per row
        const uint32_t rpc = 4u / s;
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
          if (q < rpc) {
            const uint32_t row0 = s == 2 ? e >> 1 : e;
            const uint32_t row = row0 + q < total / s ? row0 + q : total / s - 1u;  // past the end: any row
            const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
            const uint32_t t = row - pl * a.spp;
            const uint32_t phi = __brev(~(t >> a.r_log2));
            const uint32_t* gw = gvec + (pl * R + (t & (R - 1u))) * stride;
            if (s == 2) {
              v[2 * q] = phi * gw[0];
              v[2 * q + 1] = phi * gw[1];
            } else {
              v[q] = phi * gw[0];
            }
          }
        }
      } else if (LAYOUT == 1) {  // four dimensions of one row: one 128-bit shared load
        const uint32_t row = (uint32_t)__umul64hi(e, mag_s);
        const uint32_t j = e - row * s;
        const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
        const uint32_t t = row - pl * a.spp;
        const uint4 g = *reinterpret_cast<const uint4*>(gvec + (pl * R + (t & (R - 1u))) * stride + j);
        const uint32_t phi = __brev(~(t >> a.r_log2));  // phi_2(2^32 - 1 - i), Alg. 4
        v[0] = phi * g.x, v[1] = phi * g.y, v[2] = phi * g.z, v[3] = phi * g.w;
      } else {  // each element its own row
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t et = e + q < total ? e + q : total - 1u;  // past the end: any valid word
          const uint32_t row = s > 1 ? (uint32_t)__umul64hi(et, mag_s) : et;
          const uint32_t j = et - row * s;
          const uint32_t pl = a.spp > 1 ? (uint32_t)__umul64hi(row, mag_spp) : row;
          const uint32_t t = row - pl * a.spp;
          v[q] = __brev(~(t >> a.r_log2)) * gvec[(pl * R + (t & (R - 1u))) * stride + j];
        }
      }
      if (e + 4u <= total) {
        store4(a.out_u32, a.out_f32, off0 + e, v, a.chk);
      } else {  // the batch's ragged end (s % 4 != 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (e + q < total) store1(a.out_u32, a.out_f32, off0 + e + q, v[q], a.chk);
      }
    }
  }
}

// Fallback for outputs that are not 16-byte aligned or batches beyond shared memory:
// one element per thread.
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
    store1(a.out_u32, a.out_f32, f, __brev(~(t >> a.r_log2)) * g[0], a.chk);
  }
}

}  // namespace

cudaError_t launch_random_lattice_points(const RandomPointsArgs& args, cudaStream_t stream) {
  const DeviceInfo& dev = device_info();
  RandomPointsArgs a = args;
  const bool hash = a.kind == QMC_RLAT_HASH;
  const uint64_t Rrow = (uint64_t)(a.s + 4) << a.r_log2;  // words per pixel (padded rows)
  // batch: up to 48 KiB of generator words (at least one pixel), at most 1024 / s pixels within
  // [32, 256] -- a batch writes about 32-64 KiB per output, so the resident blocks' stores stay
  // close together (measured at s = 32: 32-pixel batches 2 % faster than 256; at s = 2, 256)
  uint64_t pixels = (48u * 1024u / 4u) / Rrow;
  const uint64_t pixel_cap = a.s >= 32 ? 32 : a.s <= 4 ? 256 : 1024 / a.s;
  if (pixels > pixel_cap) pixels = pixel_cap;
  if ((a.s & 3u) != 0) pixels &= ~3ull;  // batches of 4k pixels: every batch's first element offset
                                         // first spp s is a multiple of 4, so 16-byte chunks stay aligned
  const bool batched = pixels >= 1;
  if (pixels < 1) pixels = 1;
  a.batch_pixels = (uint32_t)pixels;
  const size_t smem =
      ((hash ? 0 : (size_t)kLfsrJumpWords) + ((2 * pixels + 3) & ~3ull) + pixels * Rrow) * sizeof(uint32_t);
  if (batched && pixels * a.spp * a.s <= (1ull << 31) && aligned16(a.out_u32) && aligned16(a.out_f32) &&
      smem <= dev.smem_per_block_optin) {
    const int layout = (a.s & 3u) == 0 ? 1 : a.s <= 2 ? 2 : 0;
    const auto kernel = hash ? (layout == 1   ? random_lattice_points_fast<QMC_RLAT_HASH, 1>
                                : layout == 2 ? random_lattice_points_fast<QMC_RLAT_HASH, 2>
                                              : random_lattice_points_fast<QMC_RLAT_HASH, 0>)
                             : (layout == 1   ? random_lattice_points_fast<QMC_RLAT_LFSR, 1>
                                : layout == 2 ? random_lattice_points_fast<QMC_RLAT_LFSR, 2>
                                              : random_lattice_points_fast<QMC_RLAT_LFSR, 0>);
    if (smem > 48 * 1024) {
      const cudaError_t ea = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ea != cudaSuccess) return ea;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (uint64_t)dev.sm_count * (per_sm < 1 ? 1 : per_sm);
    const uint64_t batches = (a.n_pixels + pixels - 1) / pixels;
    // one batch per block on a grid sized by the batches when a batch writes at least 64 KiB of
    // each output (the resident blocks then write one neighbourhood: at s = 32, 2^20 pixels x 16
    // samples, 960 / 953 Gdims/s against 835 / 822 on the persistent grid); smaller batches keep
    // the persistent grid, whose blocks pay the LFSR jump table once (at s = 2 the spread grid
    // measured 4 % / 17 % slower)
    if (pixels * a.spp * a.s * sizeof(uint32_t) >= 64u * 1024u || batches < blocks) blocks = batches;
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
  if ((uint64_t)32 * a.spp * a.s <= (1ull << 31) && aligned16(a.out_u32) && aligned16(a.out_f32)) {
    // one batch per warp: the kernel has no per-block set-up, and a persistent grid's warps would
    // end unevenly when they hold only a few batches each.  Batches of 8 pixels when a pixel has
    // 256 or more elements (short ranges keep the resident warps' stores together: s = 32 at 16
    // spp 920 Gdims/s against 880 with 32-pixel batches), else 32 (at s = 2, 16 spp, a warp
    // computing 8 shifts for 256 elements ran at a third of the speed)
    // With 32-pixel batches a warp takes four of them and computes their shifts together: one
    // shift is a long dependent chain, and a warp with a single batch spent most of its life on it
    // (s = 2, 16 spp: 0.79 of the copy bandwidth at any image size).
    const bool small = a.spp * a.s >= 256u;
    const auto kernel = (a.s & 3u) == 0 ? (small ? pixel_lattice_points_fast<1, 3, 1> : pixel_lattice_points_fast<1, 5, 4>)
                        : a.s <= 2       ? (small ? pixel_lattice_points_fast<2, 3, 1> : pixel_lattice_points_fast<2, 5, 4>)
                                         : (small ? pixel_lattice_points_fast<0, 3, 1> : pixel_lattice_points_fast<0, 5, 4>);
    const uint32_t blog2 = small ? 3u : 5u, per_warp = small ? 1u : 4u;
    uint64_t blocks = (((a.n_pixels + (1u << blog2) - 1) >> blog2) + per_warp * (kThreads / 32) - 1) /
                      (per_warp * (kThreads / 32));
    if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;  // warp_range spreads the batches over the grid
    if (blocks < 1) blocks = 1;
    kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
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
    if (aligned16(a.out_u32) && aligned16(a.out_f32) && a.s <= 1024) {
      const uint64_t batches = (a.count + kFlatRows - 1) / kFlatRows;
      return backward ? launch_spread(lattice_points_flat<true>, batches, 1, 0, stream, a)
                      : launch_spread(lattice_points_flat<false>, batches, 1, 0, stream, a);
    }
    return backward ? launch_grid_stride(lattice_points_generic<true>, a.count * a.s, stream, a)
                    : launch_grid_stride(lattice_points_generic<false>, a.count * a.s, stream, a);
  }
  const uint64_t groups = (a.count + (1u << a.q_log2) - 1) >> a.q_log2;
  // direct 16-byte stores, four groups per warp on a grid sized by the groups: at s = 32 this
  // wrote 2^24 points 21 % faster than TMA bulk stores from a persistent grid of long ranges
#define QMC_LATTICE_CASE(KK)                                                                  \
  case KK:                                                                                    \
    return backward ? launch_spread(lattice_points_fast<KK, true>, groups, 4, 0, stream, a) \
                    : launch_spread(lattice_points_fast<KK, false>, groups, 4, 0, stream, a);
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

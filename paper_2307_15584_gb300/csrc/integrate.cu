// integrate.cu -- massively parallel QMC integro-approximation (Sec. 2.5): the
// scans, the reductions and the dispatch; the persistent kernel of step 4 lives
// in integrate_kernel.cuh, instantiated per integrand in integrate_<name>.cu.
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
  const bool items_ok = in_bounds(CheckCtx{a.check_word, a.capacity_items}, b, e - b, kCheckPartials);
  if (items_ok)
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
  const bool items_ok = in_bounds(CheckCtx{a.check_word, a.capacity_items}, b, e - b, kCheckPartials);
  if (items_ok && lane < 17)
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

}  // namespace

cudaError_t launch_integrate(const IntegrateArgs& a, uint32_t block, bool grad, cudaStream_t stream) {
  const uint32_t n_blocks = (uint32_t)(((uint64_t)a.n + kScanBlock) / kScanBlock);  // covers entry n
  scan_totals<<<n_blocks, kScanThreads, 0, stream>>>(a);
  scan_carry<<<1, 1024, 0, stream>>>(a, n_blocks);
  scan_write<<<n_blocks, kScanThreads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (a.integrand) {
    case QMC_F_BILINEAR2D: e = launch_integrand_bilinear(a, block, stream); break;
    case QMC_F_GENZ_PRODUCT_PEAK:
    case QMC_F_GENZ_OSCILLATORY: e = launch_integrand_genz(a, block, stream); break;
    case QMC_F_SCENE4D: e = launch_integrand_scene(a, block, stream); break;
    default: e = launch_integrand_gaussmix(a, block, grad, stream);
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

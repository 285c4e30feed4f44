// points_common.cuh -- helpers shared by the materialising point kernels
// (sobol_points.cu, lattice_points.cu, halton_points.cu): 16-byte and scalar
// stores, TMA bulk stores from shared memory, warp work ranges, per-warp staging,
// and the host-side launch helpers.
#pragma once

#include <cstdint>

#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmc {
namespace pts {

constexpr int kThreads = 256;

__device__ __forceinline__ void store4(uint32_t* out_u32, float* out_f32, uint64_t off,
                                       const uint32_t (&v)[4], const CheckCtx& chk) {
  if (!in_bounds(chk, off, 4, kCheckPoints)) return;
  if (out_u32) __stcs(reinterpret_cast<uint4*>(out_u32 + off), make_uint4(v[0], v[1], v[2], v[3]));
  if (out_f32)
    __stcs(reinterpret_cast<float4*>(out_f32 + off),
           make_float4(map_u32_to_unifloat(v[0]), map_u32_to_unifloat(v[1]),
                       map_u32_to_unifloat(v[2]), map_u32_to_unifloat(v[3])));
}

__device__ __forceinline__ void store1(uint32_t* out_u32, float* out_f32, uint64_t off,
                                       uint32_t v, const CheckCtx& chk) {
  if (!in_bounds(chk, off, 1, kCheckPoints)) return;
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
// shared-memory tiles on a persistent grid (1) or direct 128-bit stores on a
// grid of short per-warp ranges (0), and the groups per staged tile (per warp,
// double-buffered).  Measured on GB300 at s = 32, 2^24 points, u32 + f32, on a
// persistent grid of long per-warp ranges: direct stores 0.714 ms; TMA with
// 1 / 2 / 4 / 8 groups per tile 0.726 / 0.728 / 0.653 / 0.866 ms.  Direct stores
// with 64 groups per warp on a grid sized by the groups (launch_spread): 0.60 ms;
// TMA on that grid 0.83 ms (each block stages 86 KB).
#ifndef QMC_POINTS_TMA
#define QMC_POINTS_TMA 0
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


inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Chunks per lane of the fast path, or 0 when the generic path must run.
inline uint32_t fast_k(uint32_t s) {
  uint32_t g = 128;
  while (s % g) g >>= 1;  // gcd(s, 128): the largest power of two dividing both
  const uint32_t K = s / g;
  return K <= 4 ? K : 0;
}

inline uint32_t log2_exact(uint32_t v) {
  uint32_t l = 0;
  while ((1u << l) < v) ++l;
  return l;
}

template <typename KernelT>
inline cudaError_t launch_persistent(KernelT kernel, uint64_t warps_needed, size_t smem,
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

// A grid of one range of per_warp units per warp, as many blocks as the units ask, so that the
// warps resident at any time write neighbouring parts of the output (measured on GB300: a
// persistent grid of long per-warp ranges spreads the concurrent stores over the whole output
// and writes 5-20 % slower).  Kernels with a per-block set-up take ranges long enough to pay it.
template <typename KernelT>
inline cudaError_t launch_spread(KernelT kernel, uint64_t units, uint64_t per_warp, size_t smem,
                                 cudaStream_t stream, const PointsArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  uint64_t blocks = (units + per_warp * (kThreads / 32) - 1) / (per_warp * (kThreads / 32));
  if (blocks > 0x7FFFFFFFull) blocks = 0x7FFFFFFFull;  // warp_range spreads any remainder over the grid
  if (blocks < 1) blocks = 1;
  kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

// True for device (or managed) memory and for null; false for host memory the
// GPU reaches through the interconnect (pinned or registered host buffers).
inline bool device_resident(const void* p) {
  if (!p) return true;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

template <typename KernelT>
inline cudaError_t launch_grid_stride(KernelT kernel, uint64_t elements, cudaStream_t stream,
                               const PointsArgs& a) {
  const DeviceInfo& dev = device_info();
  uint64_t blocks = (elements + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)dev.sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace pts
}  // namespace qmc

// qmc_internal.h -- host-side declarations shared by the translation units of
// libqmc_gb300.so (never installed; the public interface is include/qmc.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/qmc.h"

namespace qmc {

struct DeviceInfo {
  int device;
  int sm_count;
  int cc_major, cc_minor;
  size_t smem_per_block_optin;
};

// Properties of the current device (cached per device id).
const DeviceInfo& device_info();

// Arguments of the materialising kernels.
struct PointsArgs {
  const uint32_t* matrices;  // Sobol': [s][32] columns; lattice: [s] generator words
  const uint32_t* seeds;     // Sobol': scramble seeds [s]; lattice: shifts [s] (nullable)
  uint32_t* out_u32;         // [count][s] or null
  float* out_f32;            // [count][s] or null
  uint64_t count;
  uint32_t s;
  uint32_t index_begin;      // index_begin + count <= 2^32 was checked by the caller
  uint32_t scramble;         // Sobol': 0 none, 1 XOR, 2 nested; lattice: bit 0 = backward
  uint32_t q_log2;           // set by the launcher
  uint32_t u_log2;           // set by the launcher
};

// Arguments of the pixel-shifted lattice points (Sec. 3).
struct PixelPointsArgs {
  const uint32_t* g;  // [s] generator words
  uint32_t* out_u32;  // [n_pixels * spp][s] or null
  float* out_f32;     // [n_pixels * spp][s] or null
  uint64_t pixel_begin, n_pixels;
  uint32_t spp, s, width, grid_log2;
};

cudaError_t launch_pixel_lattice_points(const PixelPointsArgs& a, cudaStream_t stream);

// Radical inversion in prime bases (Sec. 2.2).  The per-base constants (the
// first 64 primes, their domain limits, division reciprocals and Faure tables)
// never change; points.cu writes them once per device into a device table.
// The per-call arguments stay small (kernel parameters).
constexpr uint32_t kHaltonMaxDims = 64;
struct HaltonArgs {
  uint32_t* out_u32;
  float* out_f32;
  uint64_t count;
  uint32_t index_begin, s, mode;       // mode: 0 identity, 1 Faure, 2 linear
  uint32_t mult[kHaltonMaxDims];       // linear digit scramble multipliers
};

// Enqueues the Halton kernel; writes the device table first if this device has
// not received it yet (a synchronous copy).
cudaError_t launch_halton_points(const HaltonArgs& p, cudaStream_t stream);
// The j-th prime (j < kHaltonMaxDims).
uint32_t halton_base(uint32_t j);
cudaError_t launch_sobol_points(PointsArgs a, cudaStream_t stream);
cudaError_t launch_lattice_points(PointsArgs a, cudaStream_t stream);

// Work split recorded by qmc_tune_integrate for this problem class, if any.
bool tuned_lookup(const qmc_problem* p, uint32_t n, bool grad, uint32_t* chunk, uint32_t* block);

}  // namespace qmc

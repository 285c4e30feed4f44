// qmc_internal.h -- host-side declarations shared by the translation units of
// libqmc_gb300.so (never installed; the public interface is include/qmc.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/qmc.h"
#include "qmc_checked.cuh"

namespace qmc {

struct DeviceInfo {
  int device;
  int sm_count;
  int cc_major, cc_minor;
  size_t smem_per_block_optin;
};

// Properties of the current device (cached per device id).
const DeviceInfo& device_info();

// Arguments of the materialising kernels.  Sobol' row r is the point of index
// i = ((index_begin + r) << col0) | pconst, evaluated with the m columns per
// dimension of matrices (Alg. 3; m = 32 below 2^32).  col0 > 0 enumerates one
// element of a partitioned sequence (Sec. 2.5.1): pconst < 2^col0 is its fixed
// low index part.
struct PointsArgs {
  const uint32_t* matrices;  // Sobol': [s][m] columns; lattice: [s] generator words
  const uint32_t* seeds;     // Sobol': scramble seeds [s]; lattice: shifts [s] (nullable)
  uint32_t* out_u32;         // [count][s] or null
  float* out_f32;            // [count][s] or null
  uint64_t count;
  uint64_t index_begin;      // the caller checked the whole range (2^32 for the lattice)
  uint64_t pconst;           // Sobol': low index bits below col0
  uint32_t s;
  uint32_t m;                // Sobol': columns per dimension (32 .. 64)
  uint32_t col0;             // Sobol': first column of the enumerated index
  uint32_t scramble;         // Sobol': 0 none, 1 XOR, 2 nested; lattice: bit 0 = backward
  uint32_t q_log2;           // set by the launcher
  uint32_t u_log2;           // set by the launcher
  CheckCtx chk;              // checked build: the output extent count * s and the error word
};

// Arguments of the pixel-shifted lattice points (Sec. 3).
struct PixelPointsArgs {
  const uint32_t* g;  // [s] generator words
  uint32_t* out_u32;  // [n_pixels * spp][s] or null
  float* out_f32;     // [n_pixels * spp][s] or null
  uint64_t pixel_begin, n_pixels;
  uint32_t spp, s, width, grid_log2;
  CheckCtx chk;  // checked build: the output extent n_pixels * spp * s and the error word
};

cudaError_t launch_pixel_lattice_points(const PixelPointsArgs& a, cudaStream_t stream);

// Arguments of the per-pixel random lattice points (Alg. 4, Sec. 3).
struct RandomPointsArgs {
  uint32_t* out_u32;  // [n_pixels * spp][s] or null
  float* out_f32;     // [n_pixels * spp][s] or null
  uint64_t pixel_begin, n_pixels;
  uint32_t spp, s, width;
  uint32_t kind, seed, r_log2;  // qmc_rlat_kind, hash seed, log2 of the instance count
  uint32_t batch_pixels;        // set by the launcher: pixels per shared-memory batch
  CheckCtx chk;                 // checked build: the output extent n_pixels * spp * s and the error word
};

cudaError_t launch_random_lattice_points(const RandomPointsArgs& a, cudaStream_t stream);

cudaError_t launch_sobol_points(PointsArgs a, cudaStream_t stream);
cudaError_t launch_lattice_points(PointsArgs a, cudaStream_t stream);

// The checked build's error word of the current device and the extent `limit`
// (less QMC_CHECK_SLACK elements, a test hook that makes the last stores of a
// launch report themselves); {nullptr, limit} in the normal build.
CheckCtx check_ctx(uint64_t limit);

// Work split recorded by qmc_tune_integrate for this problem class, if any.
bool tuned_lookup(const qmc_problem* p, uint32_t n, bool grad, uint32_t* chunk, uint32_t* block);

}  // namespace qmc

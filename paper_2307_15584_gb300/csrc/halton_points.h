// halton_points.h -- host-side declarations of the Halton engine (radical
// inversion in prime bases, Sec. 2.2), shared by halton_points.cu and api.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qmc_checked.cuh"

namespace qmc {

// Radical inversion in prime bases (Sec. 2.2).  The per-base constants (the
// first 64 primes, their domain limits, division reciprocals and Faure tables)
// never change; halton_points.cu writes them once per device into a device table.
// The per-call arguments stay small (kernel parameters).
constexpr uint32_t kHaltonMaxDims = 64;
struct HaltonArgs {
  uint32_t* out_u32;
  float* out_f32;
  uint64_t count;
  uint64_t index_begin;                // row r: index ((index_begin + r) << q) | pconst
  uint64_t pconst;
  uint32_t q, dim0;                    // output dimension j is Halton dimension dim0 + j
  uint32_t s, mode;                    // mode: 0 identity, 1 Faure, 2 linear
  uint32_t mult[kHaltonMaxDims];       // linear digit scramble multipliers per output dimension
  // set by the launcher
  uint32_t table_off[kHaltonMaxDims];  // output dimension jo's digit-group tables in shared memory
  uint32_t delta[kHaltonMaxDims];      // (k 2^q) mod b^K: the index step of the lanes of dimension jo
  uint32_t stage_word;                 // first 32-bit word of the warps' store tiles, after the tables
  CheckCtx chk;                        // checked build: the output extent count * s and the error word
};

// Enqueues the Halton kernel; writes the device table first if this device has
// not received it yet (a synchronous copy).
cudaError_t launch_halton_points(const HaltonArgs& p, cudaStream_t stream);
// The j-th prime (j < kHaltonMaxDims).
uint32_t halton_base(uint32_t j);

}  // namespace qmc

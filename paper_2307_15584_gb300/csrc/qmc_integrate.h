// qmc_integrate.h -- host/device declarations of the integration launcher.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace qmc {

constexpr uint32_t kErrCapacity = 1u;  // more work items than the workspace holds

struct WsHeader {
  uint32_t next_item;    // dynamic scheduler counter
  uint32_t total_items;  // work items of this call (0 after a capacity error)
  uint32_t error_bits;
  uint32_t reserved;
};

struct IntegrateArgs {
  // problem
  uint32_t source, integrand, s, randomize;
  const uint32_t* matrices;
  const uint32_t* g;
  const uint32_t* seeds;
  uint32_t seeds_per_integral;
  uint32_t chunk_log2;
  uint32_t image_width;  // pixel-shifted lattice: integral p is pixel (p % width, p / width)
  uint32_t grid_log2;    // ... on the 2^grid_log2 square grid of the Hilbert curve
  uint32_t rlat_log2;    // random lattice: log2 of the superimposed instances (kind in randomize)
  uint32_t n;
  const uint32_t* counts;
  const float* theta;
  uint32_t theta_stride;
  // unfused path (null for the fused kernels)
  const float* points;
  uint32_t points_shared;
  // workspace views
  WsHeader* hdr;
  uint32_t* item_off;       // [n+1]
  uint64_t* row_off;        // [n+1] or null
  uint64_t* ws_block_items; // [ceil((n+1)/1024)]
  uint64_t* ws_block_rows;
  double* ws_loss_terms;    // [n]
  float* partials;          // [capacity][2 * values]
  uint64_t capacity_items;
  // outputs / upstream
  double* estimate;
  const double* grad_est;
  float* grad_theta;
  const double* target;
  double* loss;
  // Sobol' (kept last: the fused kernels' code is sensitive to the parameter layout, and
  // placing these before the hot fields measured 1.5 % slower)
  uint32_t sobol_m;      // columns per dimension of matrices (32 .. 64)
  uint32_t part_log2;    // integral p enumerates element p mod 2^part_log2 (0: the sequence)
  uint32_t* check_word;  // checked build: where out-of-range stores report themselves
};

// Offsets of the workspace regions (bytes from the 256-byte aligned base).
struct WsLayout {
  size_t header, item_off, row_off, block_items, block_rows, loss_terms, partials, total;
};

WsLayout workspace_layout(uint32_t n, uint64_t capacity_items, uint32_t values_per_item);

cudaError_t launch_integrate(const IntegrateArgs& a, uint32_t block, bool grad, cudaStream_t stream);

// Persistent integration kernel of one integrand family (integrate_<name>.cu).
cudaError_t launch_integrand_bilinear(const IntegrateArgs& a, uint32_t block, cudaStream_t stream);
cudaError_t launch_integrand_genz(const IntegrateArgs& a, uint32_t block, cudaStream_t stream);
cudaError_t launch_integrand_gaussmix(const IntegrateArgs& a, uint32_t block, bool grad, cudaStream_t stream);
cudaError_t launch_integrand_scene(const IntegrateArgs& a, uint32_t block, cudaStream_t stream);

}  // namespace qmc

// qmc_checked.cuh -- the checked build of the library (compiled with
// -DQMC_CHECKED=1 into libqmc_gb300_checked.so).  Every store of a materialising
// kernel and every per-item and per-integral store of the integration kernels
// tests its element offset against the extent the host validated; an offset
// outside it sets a bit of a device error word (qmc_checked_error) and the store
// is skipped -- no trap and no fault, so a broken index shows up as a status on
// the host.  The normal build compiles the tests out.
#pragma once

#include <cstdint>

#ifndef QMC_CHECKED
#define QMC_CHECKED 0
#endif

namespace qmc {

constexpr bool kChecked = QMC_CHECKED != 0;

// Bits of the checked build's error word.
constexpr uint32_t kCheckPoints = 1u;    // a point kernel stored beyond count x s elements
constexpr uint32_t kCheckPartials = 2u;  // an integration work item beyond the workspace's capacity
constexpr uint32_t kCheckIntegral = 4u;  // a per-integral store beyond the n integrals

// The extent a kernel may write and where to report a store outside it (null in
// the normal build).
struct CheckCtx {
  uint32_t* word;
  uint64_t limit;
};

// True when elements [off, off + n) lie inside [0, c.limit); otherwise records
// `bit` and returns false (always true in the normal build).
__device__ __forceinline__ bool in_bounds(const CheckCtx& c, uint64_t off, uint64_t n, uint32_t bit) {
#if QMC_CHECKED
  if (off + n <= c.limit) return true;
  if (c.word) atomicOr(c.word, bit);
  return false;
#else
  (void)c;
  (void)off;
  (void)n;
  (void)bit;
  return true;
#endif
}

}  // namespace qmc

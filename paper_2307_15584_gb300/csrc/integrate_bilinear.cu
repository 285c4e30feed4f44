// integrate_bilinear.cu -- the 2-D bilinear test integrand of the fused integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

template <>
struct Integrand<QMC_F_BILINEAR2D> {
  static constexpr int S = 2;
  static constexpr bool kAdaptive = false;
  static constexpr bool kExactPair = false;
  static constexpr int kMinBlocks = 0;  // resident 256-thread blocks per SM to fit (0: the compiler's choice)
  float wsum = 1.0f;
  __device__ void setup(const float*, uint32_t) {}
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    return __fmaf_rn(0x1p-33f, x[0], 0.75f) * __fmaf_rn(0x1p-33f, x[1], 0.75f);  // 0.75 + x/2
  }
};

}  // namespace integ

cudaError_t launch_integrand_bilinear(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  return integ::launch_main_fn<QMC_F_BILINEAR2D, false>(a, block, stream);
}
}  // namespace qmc

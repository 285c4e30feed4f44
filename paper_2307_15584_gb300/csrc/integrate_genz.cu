// integrate_genz.cu -- the Genz product-peak and oscillatory test integrands (s <= 16) of the
// fused integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

template <>
struct Integrand<QMC_F_GENZ_PRODUCT_PEAK> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  uint32_t s;
  float ch[16], cl[16], u[16];  // a^-2 = ch + cl
  __device__ void setup(const float* th, uint32_t s_) {
    s = s_;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float a = (uint32_t)j < s ? __ldg(th + j) : 1.0f;
      u[j] = (uint32_t)j < s ? __ldg(th + s + j) : 0.0f;
      float e;
      const float a2 = two_prod(a, a, e);
      ch[j] = ff_recip(a2, e, cl[j]);
    }
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    float prod = 1.0f;
    if (s == 16) {  // every dimension (a warp-uniform branch: no per-dimension test)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float d = __fmaf_rn(x[j], 0x1p-32f, -u[j]);  // x - u, one rounding
        prod = __fmul_rn(prod, __fadd_rn(__fmaf_rn(d, d, ch[j]), cl[j]));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if ((uint32_t)j < s) {
          const float d = __fmaf_rn(x[j], 0x1p-32f, -u[j]);
          prod = __fmul_rn(prod, __fadd_rn(__fmaf_rn(d, d, ch[j]), cl[j]));
        }
      }
    }
    return __frcp_rn(prod);
  }
};

template <>
struct Integrand<QMC_F_GENZ_OSCILLATORY> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = false;
  float wsum = 1.0f;
  uint32_t s;
  float a[16];
  float c0, s0;  // cos, sin of 2 pi u_1
  __device__ void setup(const float* th, uint32_t s_) {
    s = s_;
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = (uint32_t)j < s ? __ldg(th + j) * 0x1p-32f : 0.0f;  // a_j x_j = (a_j 2^-32) X_j
    sincospif(2.0f * __ldg(th + s), &s0, &c0);
  }
  // cos(2 pi u_1 + B) = cos(2 pi u_1) cos B - sin(2 pi u_1) sin B, B = sum_j a_j x_j
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    err = 0.0f;
    float B = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) B = __fmaf_rn(a[j], x[j], B);  // a_j = 0 beyond s adds exactly 0
    float sb, cb;
    sincosf(B, &sb, &cb);
    return __fmaf_rn(c0, cb, -__fmul_rn(s0, sb));
  }
};

}  // namespace integ

cudaError_t launch_integrand_genz(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  return a.integrand == QMC_F_GENZ_PRODUCT_PEAK ? integ::launch_main_fn<QMC_F_GENZ_PRODUCT_PEAK, false>(a, block, stream)
                                                : integ::launch_main_fn<QMC_F_GENZ_OSCILLATORY, false>(a, block, stream);
}
}  // namespace qmc

// integrate_genz.cu -- the Genz product-peak and oscillatory test integrands (s <= 16) of the
// fused integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

template <>
struct Integrand<QMC_F_GENZ_PRODUCT_PEAK> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = false;
  static constexpr int kMinBlocks = 1;  // resident 256-thread blocks per SM the registers must allow
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

// Oscillatory: f = cos(2 pi u_1 + B), B = sum_j a_j x_j.  The fp32 path sums B
// with one FMA per dimension and applies the angle-addition formula to
// cos/sin(2 pi u_1) from setup; its error is dominated by B's roundings, at
// most u |B_k| <= u sum_j |a_j| each (uniform, so rms over s of them
// u sqrt(s/3) sum_j |a_j|) and |sin| <= 1, so err returns the per-integral
// constant sqrt(s/3) sum_j |a_j| + 3 in units of u (3 for the sine/cosine and
// product roundings).  An item whose sum is small next to that error (few
// samples, or samples that cancel) is recomputed on the EXACT path: the
// phase phi = 2 pi u_1 + B as a float pair (exact products,
// TwoSum accumulation, 2 pi u_1 from a two-word 2 pi), then
// cos(phi) = cos(phi_h) - sin(phi_h) phi_l, whose error is that of one fp32
// cosine relative to its own value.
template <>
struct Integrand<QMC_F_GENZ_OSCILLATORY> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = true;
  static constexpr int kMinBlocks = 3;  // the fp32 loop fits 80 registers; the exact path must too
  static constexpr float kErrUnit = kU32;
  float wsum = 1.0f;
  uint32_t s;
  float a[16];
  float c0, s0;    // cos, sin of 2 pi u_1
  float wh, wl;    // 2 pi u_1 as a float pair
  float errc;      // sqrt(s/3) sum_j |a_j| + 3
  __device__ void setup(const float* th, uint32_t s_) {
    s = s_;
    float asum = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float aj = (uint32_t)j < s ? __ldg(th + j) : 0.0f;
      a[j] = aj * 0x1p-32f;  // a_j x_j = (a_j 2^-32) X_j
      asum += fabsf(aj);
    }
    const float u1 = __ldg(th + s);
    sincospif(2.0f * u1, &s0, &c0);
    // 2 pi = 6.28318548202514648 - 1.74845553e-7 (the nearest float and its remainder)
    float e;
    wh = two_prod(6.28318548202514648f, u1, e);
    wl = __fmaf_rn(-1.74845553e-7f, u1, e);
    errc = __fmaf_rn(sqrtf((float)s * (1.0f / 3.0f)), asum, 3.0f);
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    if constexpr (!EXACT) {
      float B = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) B = __fmaf_rn(a[j], x[j], B);  // a_j = 0 beyond s adds exactly 0
      float sb, cb;
      sincosf(B, &sb, &cb);
      err = errc;
      return __fmaf_rn(c0, cb, -__fmul_rn(s0, sb));
    } else {
      err = 0.0f;
      float bh = 0.0f, bl = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float pe, se;
        const float p = two_prod(a[j], x[j], pe);
        bh = two_sum(bh, p, se);
        bl = __fadd_rn(bl, __fadd_rn(se, pe));
      }
      float he;
      const float h = two_sum(wh, bh, he);
      const float l = __fadd_rn(he, __fadd_rn(wl, bl));
      const float ph = __fadd_rn(h, l);
      const float pl = __fsub_rn(l, __fsub_rn(ph, h));  // Fast2Sum: |h| >= |l|
      float sp, cp;
      sincosf(ph, &sp, &cp);
      return __fmaf_rn(-sp, pl, cp);
    }
  }
};

}  // namespace integ

cudaError_t launch_integrand_genz(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  return a.integrand == QMC_F_GENZ_PRODUCT_PEAK ? integ::launch_main_fn<QMC_F_GENZ_PRODUCT_PEAK, false>(a, block, stream)
                                                : integ::launch_main_fn<QMC_F_GENZ_OSCILLATORY, false>(a, block, stream);
}
}  // namespace qmc

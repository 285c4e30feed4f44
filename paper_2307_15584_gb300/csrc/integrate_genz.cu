// integrate_genz.cu -- the Genz product-peak and oscillatory test integrands (s <= 16) of the
// fused integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

// Product peak: f = prod_j 1 / (a_j^-2 + (x_j - u_j)^2), a_j^-2 held as a float
// pair.  Each fp32 factor carries four roundings (x - u, whose relative error
// doubles in the square, the FMA, the low word's add and the product), rms
// sqrt(7/3) u together, and the reciprocal one more, so err returns
// sqrt((7s + 1)/3) f.  An item over the error budget (in practice one of a
// few samples) is recomputed on the EXACT path: x - u exactly (TwoSum),
// its square with an FMA residual, each factor and the running product as
// float pairs, and a float-pair reciprocal.
template <>
struct Integrand<QMC_F_GENZ_PRODUCT_PEAK> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = true;
  static constexpr bool kExactPair = false;
  static constexpr int kMinBlocks = 2;  // 128 registers: the exact path must not cost the fp32 loop occupancy
  static constexpr float kErrUnit = kU32;
  float wsum = 1.0f;
  uint32_t s;
  float errc;                   // sqrt((7s + 1)/3)
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
    errc = sqrtf((7.0f * (float)s + 1.0f) * (1.0f / 3.0f));
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    if constexpr (!EXACT) {
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
      const float f = __frcp_rn(prod);
      err = __fmul_rn(errc, f);
      return f;
    } else {
      err = 0.0f;
      float ph = 1.0f, pl = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if ((uint32_t)j < s) {
          float dl, sqe, te, ne;
          const float dh = two_sum(__fmul_rn(x[j], 0x1p-32f), -u[j], dl);  // x - u = dh + dl
          const float sqh = two_prod(dh, dh, sqe);
          const float sql = __fmaf_rn(2.0f * dh, dl, sqe);
          const float th = two_sum(sqh, ch[j], te);
          const float tl = __fadd_rn(te, __fadd_rn(sql, cl[j]));
          const float nh = two_prod(ph, th, ne);
          const float nl = __fmaf_rn(ph, tl, __fmaf_rn(pl, th, ne));
          ph = __fadd_rn(nh, nl);
          pl = __fsub_rn(nl, __fsub_rn(ph, nh));  // Fast2Sum: |nh| >= |nl|
        }
      }
      float fl;
      const float fh = ff_recip(ph, pl, fl);
      return __fadd_rn(fh, fl);
    }
  }
};

// Float pairs (h + l, |l| <= ulp(h)/2) for the oscillatory integrand's exact path.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_fast(float h, float l) {  // Fast2Sum, |h| >= |l|
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float e;
  const float s = two_sum(a.h, b.h, e);
  return ff_fast(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float e;
  const float p = two_prod(a.h, b.h, e);
  return ff_fast(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}

// cos(ph + pl) as a float pair, for |ph| < 2^12.  Cody-Waite reduction
// phi = k pi/2 + r (|r| <= pi/4 up to the rounding of k) with pi/2 in three
// words: k times each of the first two is an exact TwoProd pair, ph minus the
// leading head is exact (Sterbenz), and the heads of the rest combine by
// TwoSum, so r carries only the rounding of terms below 2^-40 |phi|.  Then the
// quadrant's Taylor series, cos r = sum (-z)^k/(2k)! or
// sin r = r sum (-z)^k/(2k+1)! with z = r^2: the terms from z^5 on (below
// 3e-8 of the result) in fp32, the rest by float-pair Horner steps with
// two-word coefficients 1/n!.  Absolute error below 1e-14 (measured in an
// fp32 emulation against a 200-bit cosine).
__device__ __forceinline__ FF ff_cos(float ph, float pl) {
  const float k = rintf(__fmul_rn(ph, 0x1.45f306p-1f));  // 2/pi
  float e1, e2;
  const float a1 = two_prod(k, 0x1.921fb6p+0f, e1);
  const float a2 = two_prod(k, -0x1.777a5cp-25f, e2);
  const float rh = __fsub_rn(ph, a1);  // exact
  float e, ul;
  const float t = two_sum(rh, -a2, e);
  const float uh = two_sum(pl, -e1, ul);
  const FF r = ff_add(FF{t, e}, FF{uh, __fsub_rn(__fsub_rn(ul, e2), __fmul_rn(k, -0x1.ee59dap-50f))});
  const FF z = ff_mul(r, r);
  const int q = (int)k & 3;
  FF p;
  if (q & 1) {  // sin r: coefficients (-1)^k / (2k+1)!
    const float t5 = __fmaf_rn(__fmaf_rn(-0x1.ae7f3ep-41f, z.h, 0x1.612462p-33f), z.h, -0x1.ae6456p-26f);
    p = {t5, 0.0f};
    p = ff_add(ff_mul(p, z), FF{0x1.71de3ap-19f, 0x1.55b1ccp-45f});
    p = ff_add(ff_mul(p, z), FF{-0x1.a01a02p-13f, 0x1.7f97fap-39f});
    p = ff_add(ff_mul(p, z), FF{0x1.111112p-7f, -0x1.dddddep-32f});
    p = ff_add(ff_mul(p, z), FF{-0x1.555556p-3f, 0x1.555556p-28f});
    p = ff_add(ff_mul(p, z), FF{1.0f, 0.0f});
    p = ff_mul(p, r);
  } else {  // cos r: coefficients (-1)^k / (2k)!
    const float t5 =
        __fmaf_rn(__fmaf_rn(__fmaf_rn(0x1.ae7f3ep-45f, z.h, -0x1.93974ap-37f), z.h, 0x1.1eed8ep-29f), z.h,
                  -0x1.27e4fcp-22f);
    p = {t5, 0.0f};
    p = ff_add(ff_mul(p, z), FF{0x1.a01a02p-16f, -0x1.7f97fap-42f});
    p = ff_add(ff_mul(p, z), FF{-0x1.6c16c2p-10f, 0x1.27d27ep-35f});
    p = ff_add(ff_mul(p, z), FF{0x1.555556p-5f, -0x1.555556p-30f});
    p = ff_add(ff_mul(p, z), FF{-0.5f, 0.0f});
    p = ff_add(ff_mul(p, z), FF{1.0f, 0.0f});
  }
  // cos(r + q pi/2) = cos r, -sin r, -cos r, sin r
  return (q == 1 || q == 2) ? FF{-p.h, -p.l} : p;
}

// Oscillatory: f = cos(2 pi u_1 + B), B = sum_j a_j x_j.  The fp32 path sums B
// with one FMA per dimension and applies the angle-addition formula to
// cos/sin(2 pi u_1) from setup; its error is dominated by B's roundings, at
// most u |B_k| <= u sum_j |a_j| each (uniform, so rms over s of them
// u sqrt(s/3) sum_j |a_j|) and |sin| <= 1, so err returns the per-integral
// constant sqrt(s/3) sum_j |a_j| + 3 in units of u (3 for the sine/cosine and
// product roundings).  An item whose sum is small next to that error (few
// samples, or samples that cancel) is recomputed on the EXACT path: the
// phase phi = 2 pi u_1 + B as a float pair (exact products, TwoSum
// accumulation, 2 pi u_1 from a two-word 2 pi) and f = cos(phi) as a float pair
// (ff_cos), both of whose words enter the compensated sum (kExactPair), so
// that samples of both signs cancel without fp32 rounding of f.
template <>
struct Integrand<QMC_F_GENZ_OSCILLATORY> {
  static constexpr int S = 16;
  static constexpr bool kAdaptive = true;
  static constexpr bool kExactPair = true;
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
    // 2 pi as the nearest float and its remainder
    float e;
    wh = two_prod(0x1.921fb6p+2f, u1, e);
    wl = __fmaf_rn(-0x1.777a5cp-23f, u1, e);
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
    } else {  // err: the low word of f
      err = 0.0f;
      float bh = 0.0f, bl = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float pe, se;
        const float p = two_prod(a[j], x[j], pe);
        bh = two_sum(bh, p, se);
        bl = __fadd_rn(bl, __fadd_rn(se, pe));
      }
      const FF phi = ff_add(FF{wh, wl}, ff_fast(bh, bl));
      if (fabsf(phi.h) < 4096.0f) {
        const FF c = ff_cos(phi.h, phi.l);
        err = c.l;  // the low word, which the caller adds as well
        return c.h;
      }
      float sp, cp;  // beyond the reduction's range: one fp32 cosine and the first-order term
      sincosf(phi.h, &sp, &cp);
      return __fmaf_rn(-sp, phi.l, cp);
    }
  }
};

}  // namespace integ

cudaError_t launch_integrand_genz(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  return a.integrand == QMC_F_GENZ_PRODUCT_PEAK ? integ::launch_main_fn<QMC_F_GENZ_PRODUCT_PEAK, false>(a, block, stream)
                                                : integ::launch_main_fn<QMC_F_GENZ_OSCILLATORY, false>(a, block, stream);
}
}  // namespace qmc

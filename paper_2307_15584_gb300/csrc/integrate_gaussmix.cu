// integrate_gaussmix.cu -- the 6-D mixture of four Gaussians (forward and, with its parameter
// gradient, the fused forward+backward) of the fused integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

// Mixture of four separable Gaussians.  G_c = 2^t with t = -q_c k_c,
// q_c = sum_d (x_d - m_{c,d})^2 and k_c = log2(e)/(2 sigma_c^2) held as a
// float pair.  In fp32, q carries up to ~8 unit roundoffs of relative error,
// so G_c's relative error grows like 8u ln2 |t|; err returns sum_c w_c G_c |t_c|
// for the caller's budget test.  The EXACT path forms |x - m| exactly
// (Fast2Sum on the ordered pair), squares it with an FMA residual, sums the
// squares with TwoSum and applies the low word of t as a first-order factor.
template <>
struct Integrand<QMC_F_GAUSSMIX4_6D> {
  static constexpr int S = 6;
  static constexpr bool kAdaptive = true;
  static constexpr bool kExactPair = false;
  static constexpr int kMinBlocks = 0;  // resident 256-thread blocks per SM to fit (0: the compiler's choice)
  static constexpr float kErrUnit = 8.0f * kU32 * kLn2;  // relative error of G per unit |t|
  float wsum;
  float w[4], mu[4], nu[4], kh[4], kl[4];
  float is2[4], is3[4];  // 1/sigma^2, 1/sigma^3 (gradient only)
  __device__ void setup(const float* th, uint32_t) {
    wsum = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(th) + c);
      w[c] = t.x;
      mu[c] = t.y;
      nu[c] = t.z;
      wsum += fabsf(t.x);
      const float sg = t.w;
      float e;
      const float s2 = two_prod(sg, sg, e);  // sigma^2 = s2 + e exactly
      float rl;
      const float rh = ff_recip(2.0f * s2, 2.0f * e, rl);  // 1/(2 sigma^2)
      float pe;
      const float p = two_prod(rh, kLog2eHi, pe);
      kh[c] = p;
      kl[c] = pe + rh * kLog2eLo + rl * kLog2eHi;
      is2[c] = __frcp_rn(s2);
      is3[c] = is2[c] * __frcp_rn(sg);
    }
  }

  // 2^(-q k) for component c of the scaled point X (x = X 2^-32); q_out receives q
  // (its leading word when EXACT); with SUMS, se / so are set to the sums of the
  // differences over the even / odd dimensions (gradient).
  template <bool EXACT, bool SUMS>
  __device__ __forceinline__ float gauss(const float* X, int c, float& q_out, float& t_abs, float& se,
                                         float& so) const {
    if constexpr (!EXACT) {
      float q = 0.0f;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const float diff = __fmaf_rn(X[d], 0x1p-32f, (d & 1) ? -nu[c] : -mu[c]);  // x - m, one rounding
        q = __fmaf_rn(diff, diff, q);
        if constexpr (SUMS) {  // the differences themselves: sum x - 3 mu would cancel near the mean
          if (d < 2) (d & 1 ? so : se) = diff;
          else if (d & 1) so = __fadd_rn(so, diff);
          else se = __fadd_rn(se, diff);
        }
      }
      const float t = __fmaf_rn(q, kh[c], __fmul_rn(q, kl[c]));
      q_out = q;
      t_abs = t;
      return ex2_approx(-t);
    } else {
      float qh = 0.0f, ql = 0.0f;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const float m = (d & 1) ? nu[c] : mu[c];
        const float xd = __fmul_rn(X[d], 0x1p-32f);  // exact
        if constexpr (SUMS) {
          const float diff = __fsub_rn(xd, m);
          if (d < 2) (d & 1 ? so : se) = diff;
          else if (d & 1) so = __fadd_rn(so, diff);
          else se = __fadd_rn(se, diff);
        }
        const float hi = fmaxf(xd, m), lo = fminf(xd, m);
        const float D = __fsub_rn(hi, lo);                        // |x - m| rounded
        const float e = __fsub_rn(-lo, __fsub_rn(D, hi));         // exact remainder (Fast2Sum)
        const float p = __fmul_rn(D, D);
        const float pe = __fmaf_rn(2.0f * D, e, __fmaf_rn(D, D, -p));
        float se;
        qh = two_sum(qh, p, se);
        ql = __fadd_rn(ql, __fadd_rn(se, pe));
      }
      const float th = __fmul_rn(qh, kh[c]);
      const float tl = __fadd_rn(__fmaf_rn(qh, kh[c], -th), __fmaf_rn(qh, kl[c], __fmul_rn(ql, kh[c])));
      q_out = qh;
      t_abs = th;
      return __fmul_rn(ex2_approx(-th), __fmaf_rn(-kLn2, tl, 1.0f));
    }
  }

  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* x, float& err) const {
    float f = 0.0f;
    err = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float q, t, se, so;
      const float wG = __fmul_rn(w[c], gauss<EXACT, false>(x, c, q, t, se, so));
      f = __fadd_rn(f, wG);
      err = __fmaf_rn(fabsf(wG), t, err);
    }
    return f;
  }

  // f and the per-sample factors of df/dtheta (theta order w, mu, nu, sigma per
  // component): gq[4c..4c+3] = (G_c, sum_even (x_d - mu_c), sum_odd (x_d - nu_c),
  // q_c), so that df/dw = G, df/dmu = (w / sigma^2) G se, df/dnu = (w / sigma^2)
  // G so, df/dsigma = (w / sigma^3) G q.  The constant factors multiply the
  // item's sums once (grad_scale) instead of every sample.
  template <bool EXACT>
  __device__ __forceinline__ float eval_grad(const float* x, float* gq, float& err) const {
    float f = 0.0f;
    err = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float q, t, se, so;
      const float G = gauss<EXACT, true>(x, c, q, t, se, so);
      const float wG = __fmul_rn(w[c], G);
      f = __fadd_rn(f, wG);
      err = __fmaf_rn(fabsf(wG), t, err);
      gq[4 * c + 0] = G;
      gq[4 * c + 1] = se;
      gq[4 * c + 2] = so;
      gq[4 * c + 3] = q;
    }
    return f;
  }

  // factor of value v (1..16, theta order) that eval_grad's sums leave out
  __device__ __forceinline__ float grad_scale(int v) const {
    const int c = (v - 1) >> 2, k = (v - 1) & 3;
    return k == 0 ? 1.0f : k == 3 ? __fmul_rn(w[c], is3[c]) : __fmul_rn(w[c], is2[c]);
  }
};

}  // namespace integ

cudaError_t launch_integrand_gaussmix(const IntegrateArgs& a, uint32_t block, bool grad, cudaStream_t stream) {
  return grad ? integ::launch_main_fn<QMC_F_GAUSSMIX4_6D, true>(a, block, stream)
              : integ::launch_main_fn<QMC_F_GAUSSMIX4_6D, false>(a, block, stream);
}
}  // namespace qmc

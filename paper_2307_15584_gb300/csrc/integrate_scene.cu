// integrate_scene.cu -- the procedural scene integrand (a Fig. 1 substitute) of the fused
// integration kernel.
#include "integrate_kernel.cuh"

namespace qmc {
namespace integ {

// The procedural scene (a Fig. 1 substitute): irradiance from a square light,
// through a spherical occluder, onto a checkerboard plane seen from above.
// theta = (fx, fy, fw, fh, cx, cy, h, side, Le, ox, oy, oz, rho, freq, -, -).
// The checker and occlusion decisions use explicitly rounded fp32 operations
// in a fixed order (no contraction into fused multiply-adds), so any IEEE
// machine that evaluates the same sequence takes the same decisions.
template <>
struct Integrand<QMC_F_SCENE4D> {
  static constexpr int S = 4;
  static constexpr bool kAdaptive = false;
  static constexpr bool kExactPair = false;
  static constexpr int kMinBlocks = 0;  // resident 256-thread blocks per SM to fit (0: the compiler's choice)
  float wsum = 1.0f;
  float fx, fy, fw, fh, cx, cy, h, side, ox, oy, oz, rho2, freq, K;
  __device__ void setup(const float* th, uint32_t) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(th));
    const float4 b = __ldg(reinterpret_cast<const float4*>(th) + 1);
    const float4 c = __ldg(reinterpret_cast<const float4*>(th) + 2);
    const float4 d = __ldg(reinterpret_cast<const float4*>(th) + 3);
    fx = a.x, fy = a.y, fw = a.z, fh = a.w;
    cx = b.x, cy = b.y, h = b.z, side = b.w;
    ox = c.y, oy = c.z, oz = c.w;
    rho2 = __fmul_rn(d.x, d.x);
    freq = d.y;
    K = c.x * side * side * h * h;  // Le side^2 h^2 (shading only)
    wsum = K / (h * h * h * h);     // the largest value of f / albedo: the scale of the estimate
  }
  template <bool EXACT>
  __device__ __forceinline__ float eval(const float* X, float& err) const {
    err = 0.0f;
    const float u0 = __fmul_rn(X[0], 0x1p-32f), u1 = __fmul_rn(X[1], 0x1p-32f);  // exact
    const float u2 = __fmul_rn(X[2], 0x1p-32f), u3 = __fmul_rn(X[3], 0x1p-32f);
    const float Px = __fadd_rn(fx, __fmul_rn(fw, u0));
    const float Py = __fadd_rn(fy, __fmul_rn(fh, u1));
    const float Lx = __fadd_rn(cx, __fmul_rn(side, __fsub_rn(u2, 0.5f)));
    const float Ly = __fadd_rn(cy, __fmul_rn(side, __fsub_rn(u3, 0.5f)));
    const float Dx = __fsub_rn(Lx, Px), Dy = __fsub_rn(Ly, Py), Dz = h;
    const float Ex = __fsub_rn(Px, ox), Ey = __fsub_rn(Py, oy), Ez = -oz;
    const float DE = __fadd_rn(__fadd_rn(__fmul_rn(Dx, Ex), __fmul_rn(Dy, Ey)), __fmul_rn(Dz, Ez));
    const float DD = __fadd_rn(__fadd_rn(__fmul_rn(Dx, Dx), __fmul_rn(Dy, Dy)), __fmul_rn(Dz, Dz));
    const float EE = __fadd_rn(__fadd_rn(__fmul_rn(Ex, Ex), __fmul_rn(Ey, Ey)), __fmul_rn(Ez, Ez));
    const float disc = __fsub_rn(__fmul_rn(DE, DE), __fmul_rn(DD, __fsub_rn(EE, rho2)));
    if (!(disc < 0.0f)) return 0.0f;  // the sphere blocks the light
    const int cell = ((int)floorf(__fmul_rn(Px, freq)) + (int)floorf(__fmul_rn(Py, freq))) & 1;
    return __fdividef(cell ? 0.8f * K : 0.2f * K, __fmul_rn(DD, DD));  // DD = |L - P|^2
  }
};

}  // namespace integ

cudaError_t launch_integrand_scene(const IntegrateArgs& a, uint32_t block, cudaStream_t stream) {
  return integ::launch_main_fn<QMC_F_SCENE4D, false>(a, block, stream);
}
}  // namespace qmc

// qmc_device.cuh -- device building blocks of the QMC hot path (sm_103a).
//
// Everything here is integer or fp32 register arithmetic; none of it touches
// memory.  The definitions follow Keller, Waechter, Binder, "Quasi-Monte Carlo
// Algorithms (not only) for Graphics Software": Sec. 2.1 (float conversion),
// Sec. 2.3 (digital sequences, randomisation in integers), Sec. 2.4 (rank-1
// lattices) and Sec. 2.5 (compensated, order-controlled reduction).
#pragma once

#include <cstdint>

namespace qmc {

// Sec. 2.1: the largest fp32 value not above u * 2^-32, so every component
// stays in [0,1).  A uint->float conversion rounding toward zero keeps the 24
// leading significant bits of u (all of them below 2^24, where the result is
// exact and collision free); the scale by 2^-32 is exact because every
// non-zero result is a normal number >= 2^-32.
__device__ __forceinline__ float map_u32_to_unifloat(uint32_t u) {
  return __uint2float_rz(u) * 0x1p-32f;
}

// The same value before the exact scale: map_u32_to_unifloat(u) == unifloat_x2p32(u) * 2^-32
// bit for bit.  Fused integrands take this form and fold the power of two into
// their own constants (x - m == fma(X, 2^-32, -m) with the same single rounding).
__device__ __forceinline__ float unifloat_x2p32(uint32_t u) { return __uint2float_rz(u); }

// Hash-based nested (Owen-type) scramble, applied in the mirrored digit domain
// where the first digit 2^-1 sits in bit 0.  Each step changes bit b only as a
// function of bits below b -- an add, a multiply by an odd number, an XOR
// with a multiple by an even number -- so digit d of the scrambled value is
// digit d of the input flipped by a function of the digits before it, and
// the map is a bijection.  The seed enters as the addend and, rotated by 16
// and made odd, as the multiplier.
struct NestedKey {
  uint32_t add;
  uint32_t mul;
};

__device__ __forceinline__ NestedKey nested_key(uint32_t seed) {
  return {seed, __funnelshift_l(seed, seed, 16) | 1u};
}

__device__ __forceinline__ uint32_t nested_mix(uint32_t v, NestedKey k) {
  v += k.add;
  v ^= v * 0xD37A65C4u;
  v *= k.mul;
  v ^= v * 0x2AAE6212u;
  v ^= v * 0x2BB2601Eu;
  return v;
}

// ---------------------------------------------------------------------------
// Sec. 3, Eq. (PixelShiftedR1LS): one shift per pixel, phi_3 of the pixel's
// position along the Hilbert curve, added to phi_2(i) before the generator
// multiplication.
// ---------------------------------------------------------------------------

// Position of (x, y) along the Hilbert curve of the 2^k x 2^k grid (curve from
// the origin through quadrants (0,0), (0,1), (1,1), (1,0) of (x-bit, y-bit)):
// per level, the quadrant code, then the point is carried into the frame of
// the quadrant's sub-curve (reflected through the centre for the lower-right
// quadrant, transposed for both lower quadrants).
__device__ __forceinline__ uint32_t hilbert_position(uint32_t x, uint32_t y, uint32_t k) {
  const uint32_t n = 1u << k;
  uint32_t d = 0;
  for (uint32_t half = n >> 1; half > 0; half >>= 1) {
    const uint32_t rx = (x & half) ? 1u : 0u, ry = (y & half) ? 1u : 0u;
    d += half * half * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = n - 1u - x;
        y = n - 1u - y;
      }
      const uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

// floor(phi_3(h) * 2^32): two base-3 digits per step through the base-9 digit
// reversal of Alg. 2 ({0,3,6,1,4,7,2,5,8}, packed as nibbles), exact division.
__device__ __forceinline__ uint32_t radinv3_u32(uint32_t h) {
  constexpr uint64_t kPerm9 = 0x852741630ull;  // nibble d holds the reversal of digit pair d
  uint64_t num = 0, den = 1;
  while (h) {
    num = num * 9u + ((kPerm9 >> (4u * (h % 9u))) & 15u);
    den *= 9u;
    h /= 9u;
  }
  // num < den <= 9^11 < 2^35, so num * 2^32 < 2^67 would overflow 64 bits:
  // divide in two 16-bit steps (exact long division).
  const uint64_t q1 = (num << 16) / den, r1 = (num << 16) % den;
  const uint64_t q2 = (r1 << 16) / den;
  return (uint32_t)((q1 << 16) | q2);
}

__device__ __forceinline__ uint32_t pixel_shift(uint32_t px, uint32_t py, uint32_t k) {
  return radinv3_u32(hilbert_position(px, py, k));
}

// --- Random rank-1 lattices per pixel (Alg. 4, Sec. 2.4.2) -------------------
// Alg. 4 names a hash_value of (dimension, pixel) without defining it.  Here it
// is the high word of SplitMix64 (Steele, Lea, Flood 2014) output number
// c = py*2^44 + px*2^24 + k*2^20 + j of the stream seeded with `seed`, i.e.
// the finaliser applied to seed + (c+1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ uint32_t rlat_hash(uint32_t seed, uint32_t k, uint32_t j, uint32_t px,
                                              uint32_t py) {
  const uint64_t c = ((uint64_t)py << 44) | ((uint64_t)px << 24) | ((uint64_t)k << 20) | j;
  uint64_t z = (uint64_t)seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (uint32_t)(z >> 32);
}

// Galois LFSR of Sec. 2.4.2: the state times x modulo x^32 + x^22 + x^2 + x + 1.
__device__ __forceinline__ uint32_t lfsr_step(uint32_t st) {
  return (st << 1) ^ (0x00400007u & (0u - (st >> 31)));
}

// The LFSR yields one 32-bit number per 32 register steps.  Advancing a state by
// 32 steps multiplies it by x^32 modulo the polynomial, a linear map over GF(2),
// so it is the XOR of four byte-indexed tables (the multi-digit table idea of
// Sec. 2.2 carried over to GF(2)): T[b][v] = (v << 8b) advanced 32 steps.
constexpr uint32_t kLfsrJumpWords = 1024;  // [4][256]

// Block-cooperative fill of T; the caller synchronises the block afterwards.
__device__ __forceinline__ void lfsr_jump_table_fill(uint32_t* T) {
  for (uint32_t e = threadIdx.x; e < kLfsrJumpWords; e += blockDim.x) {
    uint32_t v = (e & 255u) << (8u * (e >> 8));
    for (int t = 0; t < 32; ++t) v = lfsr_step(v);
    T[e] = v;
  }
}

__device__ __forceinline__ uint32_t lfsr_jump32(const uint32_t* T, uint32_t xi) {
  return T[xi & 255u] ^ T[256u + ((xi >> 8) & 255u)] ^ T[512u + ((xi >> 16) & 255u)] ^ T[768u + (xi >> 24)];
}

// Seed state of the LFSR generator of instance k of a pixel: the hash at the
// reserved dimension 2^20 - 1 (never zero: 0 maps to 1).
__device__ __forceinline__ uint32_t rlat_lfsr_seed(uint32_t seed, uint32_t k, uint32_t px, uint32_t py) {
  const uint32_t x0 = rlat_hash(seed, k, (1u << 20) - 1u, px, py);
  return x0 ? x0 : 1u;
}

// ---------------------------------------------------------------------------
// Compensated fp32 summation (Sec. 2.5.1 names Kahan's algorithm; this is
// the Neumaier variant, whose error term is exact for either operand order).
// ---------------------------------------------------------------------------
struct Comp {
  float sum;
  float err;
};

// Knuth's TwoSum: t + e = a + b exactly (round-to-nearest, no branch).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float t = __fadd_rn(a, b);
  const float bv = __fsub_rn(t, a);
  const float av = __fsub_rn(t, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return t;
}

__device__ __forceinline__ void comp_add(Comp& c, float v) {
  float e;
  c.sum = two_sum(c.sum, v, e);
  c.err = __fadd_rn(c.err, e);
}

// Merge two compensated states without losing the rounding error of the sums.
__device__ __forceinline__ Comp comp_merge(Comp a, Comp b) {
  float e;
  Comp r;
  r.sum = two_sum(a.sum, b.sum, e);
  r.err = __fadd_rn(__fadd_rn(a.err, b.err), e);
  return r;
}

// Fixed butterfly over the warp: every lane ends with the same merged state,
// and the order of merges depends only on lane numbers (reproducible).
__device__ __forceinline__ Comp warp_comp_sum(Comp c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Comp o;
    o.sum = __shfl_xor_sync(0xffffffffu, c.sum, off);
    o.err = __shfl_xor_sync(0xffffffffu, c.err, off);
    // merge in lane order so both partners compute bit-identical results
    c = ((threadIdx.x & off) == 0) ? comp_merge(c, o) : comp_merge(o, c);
  }
  return c;
}

// ---------------------------------------------------------------------------
// Error-free fp32 products and a float-float reciprocal, used to keep
// per-integral constants exact to ~2^-48 so that no systematic rounding error
// is shared by all samples of an integral.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

// 1 / (a_hi + a_lo) as hi + lo (one Newton correction of the rounded reciprocal).
__device__ __forceinline__ float ff_recip(float a_hi, float a_lo, float& lo) {
  const float r = __frcp_rn(a_hi);
  // residual 1 - r (a_hi + a_lo), exact in its leading part thanks to the FMA
  const float res = __fmaf_rn(-r, a_hi, 1.0f) - r * a_lo;
  lo = r * res;
  return r;
}

}  // namespace qmc

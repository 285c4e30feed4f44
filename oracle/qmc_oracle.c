/*
 * qmc_oracle.c -- plain, slow CPU oracle for the QMC hot path of
 * Keller, Waechter, Binder, "Quasi-Monte Carlo Algorithms (not only) for
 * Graphics Software" (arXiv 2307.15584).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The CUDA
 * product path never calls it, and the two share no code, header, table or
 * constant generator: each writes its arithmetic from the paper (and from the
 * readings the library documents where the paper is silent).
 *
 * Every routine computes its result the literal way -- one index bit, one
 * digit, one sample at a time, in the order the paper states -- and all
 * integrand arithmetic is fp64.  Nothing is blocked, fused or reordered.
 *
 * Pins (tests/test_oracle_*.py check these against things other than this
 * file): the float mapping against an integer-truncation closed form and the
 * paper's special cases; dimension 0 against the radical inverse in exact
 * rational arithmetic; dimensions 0-1 against the (0,m,2)-net property by
 * brute-force counting; the polynomial enumeration against the counts
 * phi(2^d-1)/d; dimension 1 against the Pascal matrix mod 2; the lattice
 * against its closed form; integrands against closed-form integrals and
 * numerical quadrature; gradients against finite differences; the wide
 * (up to 64-column) matrices against the Pascal closed form and Niederreiter's
 * rank criterion for the t-value of the first 2^m points, m up to 64; the
 * partitioning of Sec. 2.5.1 against brute-force selection by the extra
 * coordinate and the (t, s-1)-sequence property of each element's points;
 * SplitMix64 against its published outputs, the LFSR against polynomial
 * arithmetic and a primitivity test, the per-pixel random lattice against
 * exact rational arithmetic and the Latin hypercube property of odd
 * generators.  The procedural scene: its light-square integral against a closed form
 * (itself checked by quadrature), its fp32 visibility and checker decisions
 * against fp64 geometry.
 *
 * Parity unpinned beyond those properties: the particular values of
 * qo_rlat_hash (Alg. 4's hash_value is not defined by the paper; this
 * library defines it from SplitMix64, whose outputs are pinned).
 *
 * Parity unpinned: the exact output bits of qo_nested_scramble.  The paper
 * names Owen scrambling but prints no algorithm; the hash below is this
 * library's own definition.  Its structure (nestedness, bijectivity, exact
 * per-point uniformity over seeds, preservation of the net property) is
 * pinned; its particular constants are not pinned to anything in the paper.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define QO_EXPORT __attribute__((visibility("default")))

enum { QO_SOURCE_SOBOL = 0, QO_SOURCE_LATTICE = 1, QO_SOURCE_PIXEL_LATTICE = 2,
       QO_SOURCE_RANDOM_LATTICE = 3 };
enum { QO_RLAT_HASH = 0, QO_RLAT_LFSR = 1 };
enum { QO_SCRAMBLE_NONE = 0, QO_SCRAMBLE_XOR = 1, QO_SCRAMBLE_NESTED = 2, QO_SCRAMBLE_NESTED_XOR = 3 };
enum {
    QO_F_BILINEAR2D = 0,
    QO_F_GENZ_PRODUCT_PEAK = 1,
    QO_F_GENZ_OSCILLATORY = 2,
    QO_F_GAUSSMIX4_6D = 3,
    QO_F_SCENE4D = 4
};

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: floating point conversion.                                      */
/* ------------------------------------------------------------------------ */

/* The best fp32 representation of u / 2^32 inside [0,1): the largest float
 * that is not above the exact value (0 for u = 0).  Sec. 2.1 asks for a value
 * in the right-open unit interval, so rounding may never go up. */
QO_EXPORT float qo_map_u32_to_unifloat(uint32_t u)
{
    if (u == 0) return 0.0f;
    double exact = (double)u / 4294967296.0; /* exact: u has <= 32 significant bits */
    float f = (float)exact;                  /* nearest float, may lie above */
    if ((double)f > exact) f = nextafterf(f, 0.0f);
    return f;
}

QO_EXPORT void qo_map_array(const uint32_t* u, uint64_t n, float* out)
{
    for (uint64_t k = 0; k < n; ++k) out[k] = qo_map_u32_to_unifloat(u[k]);
}

/* Mirror the 32 bits of v: bit b moves to bit 31-b. */
QO_EXPORT uint32_t qo_bit_reverse(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 32; ++b)
        if ((v >> b) & 1u) r |= 1u << (31 - b);
    return r;
}

/* Sec. 2.2: radical inverse phi_b(i) = sum_k a_k(i) b^(-k-1), returned as the
 * integer floor(phi_b(i) * 2^32).  Digits are peeled off one at a time. */
QO_EXPORT uint32_t qo_radical_inverse_u32(uint32_t b, uint64_t i)
{
    /* numerator / denominator of phi_b(i) as exact integers */
    unsigned __int128 num = 0, den = 1;
    while (i > 0) {
        num = num * b + (i % b);
        den *= b;
        i /= b;
    }
    return (uint32_t)((num << 32) / den);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: radical inversion in prime bases, digit permutations, Halton.   */
/* ------------------------------------------------------------------------ */

/* The j-th prime (j = 0 gives 2), by trial division. */
QO_EXPORT uint32_t qo_prime(uint32_t j)
{
    uint32_t count = 0;
    for (uint32_t p = 2;; ++p) {
        int is_prime = 1;
        for (uint32_t q = 2; q * q <= p; ++q)
            if (p % q == 0) { is_prime = 0; break; }
        if (is_prime && count++ == j) return p;
    }
}

/* Faure's permutation sigma_b(d), by its recursive definition (Sec. 2.2):
 * sigma_2 = (0, 1); for even b, sigma_b = 2 sigma_{b/2} followed by
 * 2 sigma_{b/2} + 1; for odd b, sigma_b is sigma_{b-1} with every value
 * >= (b-1)/2 raised by one and (b-1)/2 inserted in the middle. */
QO_EXPORT uint32_t qo_faure(uint32_t b, uint32_t d)
{
    if (b <= 2) return d;
    if (b % 2 == 0) {
        uint32_t h = b / 2;
        return d < h ? 2 * qo_faure(h, d) : 2 * qo_faure(h, d - h) + 1;
    }
    uint32_t c = (b - 1) / 2;
    if (d == c) return c;
    uint32_t v = qo_faure(b - 1, d < c ? d : d - 1);
    return v >= c ? v + 1 : v;
}

/* Component j of Halton point i (base b = the j-th prime), as
 * floor(phi(i') 2^32) where the digits of i' are permuted digit by digit:
 *   mode 0: identity; mode 1: Faure sigma_b; mode 2: linear d -> (m d) mod b
 *   (Alg. 2, radinv_linscramble, multiplier m).
 * i' = i mod b^K with b^K the largest power of b that the 32-bit result
 * resolves: 2^32 for base 2 (the bit reversal of the low 32 index bits),
 * otherwise the largest power of b below 2^32 (Alg. 1's domain limit).  Digits
 * are peeled off one at a time.  Indices take 64 bits (Sec. 2.5.1). */
QO_EXPORT uint32_t qo_halton_u64(uint64_t i, uint32_t j, uint32_t mode, uint32_t m)
{
    uint32_t b = qo_prime(j);
    uint64_t maxp = 1;
    if (b == 2) {
        maxp = 1ull << 32;
    } else {
        while (maxp * b <= 0xFFFFFFFFull) maxp *= b;
    }
    uint64_t ii = i % maxp;
    unsigned __int128 num = 0, den = 1;
    while (ii > 0) {
        uint32_t dgt = (uint32_t)(ii % b);
        if (mode == 1) dgt = qo_faure(b, dgt);
        else if (mode == 2) dgt = (uint32_t)(((uint64_t)m * dgt) % b);
        num = num * b + dgt;
        den *= b;
        ii /= b;
    }
    return (uint32_t)((num << 32) / den);
}

QO_EXPORT uint32_t qo_halton_u32(uint32_t i, uint32_t j, uint32_t mode, uint32_t m)
{
    return qo_halton_u64(i, j, mode, m);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3, Eq. (ts): Sobol' generator matrices over GF(2).                 */
/* ------------------------------------------------------------------------ */

/* Multiplicative order of x modulo the GF(2) polynomial p of degree d with
 * p(0) = 1 (bit k of p is the coefficient of x^k), found by multiplying by x
 * until the residue returns to 1; 0 when it does not within 2^d steps. */
static uint32_t order_of_x(uint32_t p, uint32_t d)
{
    uint32_t r = 1;
    for (uint32_t k = 1; k <= (1u << d); ++k) {
        r <<= 1;                    /* multiply by x */
        if ((r >> d) & 1u) r ^= p;  /* reduce modulo p */
        if (r == 1u) return k;
    }
    return 0;
}

/* All primitive polynomials of degree 1..max_degree, by increasing degree and
 * then increasing integer encoding.  A polynomial of degree d with p(0) = 1
 * is primitive exactly when x has order 2^d - 1 modulo p.  Writes at most cap
 * encodings and returns how many exist. */
QO_EXPORT uint32_t qo_primitive_polynomials(uint32_t max_degree, uint32_t* out, uint32_t cap)
{
    uint32_t n = 0;
    for (uint32_t d = 1; d <= max_degree; ++d)
        for (uint32_t p = (1u << d) | 1u; p < (2u << d); p += 2)
            if (order_of_x(p, d) == (1u << d) - 1u) {
                if (n < cap) out[n] = p;
                ++n;
            }
    return n;
}

static uint32_t degree_of(uint32_t p)
{
    uint32_t d = 0;
    while (p >> (d + 1)) ++d;
    return d;
}

/* Generator matrices of the s-dimensional Sobol' sequence for indices of up
 * to m bits (32 <= m <= 64; Alg. 3 stores 52), as m columns per dimension:
 * C[m*j + k] is the image of index bit k, truncated to the first 32 digits of
 * Eq. (ts), bit 31 being the first digit b^-1.
 *   dimension 0: the identity (van der Corput, phi_2); its columns beyond the
 *   32nd are zero (2^-k has no digit among the first 32 when k > 32);
 *   dimension j >= 1: the j-th primitive polynomial of the enumeration above,
 *   initial direction numbers m_k = (raw[7*j + k - 1] mod 2^k) | 1 for k <= deg,
 *   then m_k = m_{k-d} ^ (m_{k-d} << d) ^ XOR_{l=1}^{d-1} a_l (m_{k-l} << l)
 *   for k = d+1..m (a_l the coefficient of x^(d-l)).  Column k-1 holds the
 *   first 32 digits of v_k = m_k / 2^k: m_k << (32-k) for k <= 32 and
 *   m_k >> (k-32) beyond.  m_k < 2^k is carried exactly in 128 bits.
 * Returns 0, or -1 when s exceeds 1 + the number of polynomials of degree <= 7
 * or m lies outside [32, 64]. */
QO_EXPORT int qo_sobol_matrices_wide(uint32_t s, uint32_t m, const uint32_t* raw, uint32_t* C)
{
    uint32_t polys[64];
    uint32_t npoly = qo_primitive_polynomials(7, polys, 64);
    if (s > npoly + 1 || m < 32 || m > 64) return -1;
    for (uint32_t j = 0; j < s; ++j) {
        uint32_t* Cj = C + (uint64_t)m * j;
        if (j == 0) {
            for (uint32_t k = 0; k < m; ++k) Cj[k] = k < 32 ? 1u << (31 - k) : 0u;
            continue;
        }
        uint32_t p = polys[j - 1];
        uint32_t d = degree_of(p);
        unsigned __int128 mk[65];
        for (uint32_t k = 1; k <= d; ++k)
            mk[k] = (raw[7 * j + (k - 1)] % (1ull << k)) | 1ull;
        for (uint32_t k = d + 1; k <= m; ++k) {
            unsigned __int128 v = mk[k - d] ^ (mk[k - d] << d);
            for (uint32_t l = 1; l < d; ++l)
                if ((p >> (d - l)) & 1u) v ^= mk[k - l] << l;
            mk[k] = v;
        }
        for (uint32_t k = 1; k <= m; ++k)
            Cj[k - 1] = k <= 32 ? (uint32_t)(mk[k] << (32 - k)) : (uint32_t)(mk[k] >> (k - 32));
    }
    return 0;
}

/* The 32-column matrices (indices below 2^32): the first 32 columns of the
 * wide construction. */
QO_EXPORT int qo_sobol_matrices(uint32_t s, const uint32_t* raw, uint32_t* C)
{
    return qo_sobol_matrices_wide(s, 32, raw, C);
}

/* Eq. (ts) over F_2 and Alg. 3 with a zero scramble: the XOR of the columns
 * selected by the set bits of the index. */
QO_EXPORT uint32_t qo_sobol_u32(const uint32_t* Cj, uint32_t i)
{
    uint32_t y = 0;
    for (uint32_t k = 0; k < 32; ++k)
        if ((i >> k) & 1u) y ^= Cj[k];
    return y;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1 / 2.3 / 2.5.2: randomisation kept in integers.                   */
/* ------------------------------------------------------------------------ */

/* Hash-based nested (Owen-type) scramble of the 32 digits of y.  The digits
 * are mirrored so that the first digit b^-1 sits in bit 0; each step below
 * changes bit b only as a function of bits below b (an add, a multiply by an
 * odd number, or an XOR with a multiple by an even number), so digit d of the
 * result is digit d of the input flipped by a function of the digits before
 * it.  Arithmetic is mod 2^32, carried in 64 bits and masked. */
QO_EXPORT uint32_t qo_nested_scramble(uint32_t y, uint32_t seed)
{
    const uint64_t M = 0xFFFFFFFFull;
    uint64_t v = qo_bit_reverse(y);
    uint64_t odd = ((((uint64_t)seed << 16) | ((uint64_t)seed >> 16)) & M) | 1ull;
    v = (v + seed) & M;
    v = (v ^ (v * 0xD37A65C4ull)) & M;
    v = (v * odd) & M;
    v = (v ^ (v * 0x2AAE6212ull)) & M;
    v = (v ^ (v * 0x2BB2601Eull)) & M;
    return qo_bit_reverse((uint32_t)v);
}

/* The randomisations of a Sobol' coordinate: the random digital shift of
 * Sec. 2.3, the nested scramble above, or the shift followed by the nested
 * scramble, both selected by the dimension's one seed word. */
static uint32_t randomise_sobol(uint32_t y, uint32_t mode, uint32_t seed)
{
    if (mode == QO_SCRAMBLE_XOR) return y ^ seed;  /* Sec. 2.3: random digital shift */
    if (mode == QO_SCRAMBLE_NESTED) return qo_nested_scramble(y, seed);
    if (mode == QO_SCRAMBLE_NESTED_XOR) return qo_nested_scramble(y ^ seed, seed);
    return y;
}

/* Materialised Sobol' points: row r holds point begin + r, dimension j at
 * column j; both outputs optional. */
QO_EXPORT void qo_sobol_points(const uint32_t* C, uint32_t s, uint64_t begin, uint64_t count,
                               uint32_t mode, const uint32_t* seeds, uint32_t* out_u32,
                               float* out_f32)
{
    for (uint64_t r = 0; r < count; ++r) {
        uint32_t i = (uint32_t)(begin + r);
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t y = qo_sobol_u32(C + 32 * j, i);
            y = randomise_sobol(y, mode, seeds ? seeds[j] : 0u);
            if (out_u32) out_u32[r * s + j] = y;
            if (out_f32) out_f32[r * s + j] = qo_map_u32_to_unifloat(y);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 with wide indices, and Sec. 2.5.1: partitioning one sequence.      */
/* ------------------------------------------------------------------------ */

/* Eq. (ts) for an index of up to m bits: the XOR of the columns of Cj (m of
 * them) selected by the set bits of i.  Bits of i at or above m must be 0. */
QO_EXPORT uint32_t qo_sobol_u64(const uint32_t* Cj, uint32_t m, uint64_t i)
{
    uint32_t y = 0;
    for (uint32_t k = 0; k < m; ++k)
        if ((i >> k) & 1u) y ^= Cj[k];
    return y;
}

/* Materialised Sobol' points with 64-bit indices: row r holds point begin + r
 * of the matrices C ([s][m]); randomisation and outputs as qo_sobol_points. */
QO_EXPORT void qo_sobol_points_wide(const uint32_t* C, uint32_t m, uint32_t s, uint64_t begin,
                                    uint64_t count, uint32_t mode, const uint32_t* seeds,
                                    uint32_t* out_u32, float* out_f32)
{
    for (uint64_t r = 0; r < count; ++r) {
        uint64_t i = begin + r;
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t y = qo_sobol_u64(C + (uint64_t)m * j, m, i);
            y = randomise_sobol(y, mode, seeds ? seeds[j] : 0u);
            if (out_u32) out_u32[r * s + j] = y;
            if (out_f32) out_f32[r * s + j] = qo_map_u32_to_unifloat(y);
        }
    }
}

/* Sec. 2.5.1: the sequence is extended by one radical-inversion dimension in
 * base b, whose unit interval is cut into P = b^q intervals; processing element
 * p (0 <= p < P) owns the points whose extra coordinate phi_b(i) lies in
 * [p/P, (p+1)/P).  The first q digits of phi_b(i) are the q lowest base-b digits
 * of i in reverse order, so those points are exactly i = J P + c_p, J = 0, 1,
 * .., where c_p is p with its q base-b digits reversed.  Returns the global
 * index of the J-th point of element p (the caller keeps it below 2^64). */
QO_EXPORT uint64_t qo_partition_index(uint32_t b, uint32_t q, uint64_t p, uint64_t J)
{
    uint64_t P = 1, c = 0, rest = p;
    for (uint32_t k = 0; k < q; ++k) {
        c = c * b + rest % b;  /* digit k of p becomes digit q-1-k of c */
        rest /= b;
        P *= b;
    }
    return J * P + c;
}

/* Points J = j_begin .. j_begin+count-1 of element p of P = 2^q, partitioned by
 * dimension 0 of the Sobol' matrices C ([s+1][m], dimension 0 the identity =
 * phi_2): row r holds dimensions 1..s of point qo_partition_index(2, q, p,
 * j_begin + r); seeds[s] randomise those s dimensions. */
QO_EXPORT void qo_sobol_points_partitioned(const uint32_t* C, uint32_t m, uint32_t s,
                                           uint32_t q, uint64_t p, uint64_t j_begin,
                                           uint64_t count, uint32_t mode,
                                           const uint32_t* seeds, uint32_t* out_u32,
                                           float* out_f32)
{
    for (uint64_t r = 0; r < count; ++r) {
        uint64_t i = qo_partition_index(2, q, p, j_begin + r);
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t y = qo_sobol_u64(C + (uint64_t)m * (j + 1), m, i);
            y = randomise_sobol(y, mode, seeds ? seeds[j] : 0u);
            if (out_u32) out_u32[r * s + j] = y;
            if (out_f32) out_f32[r * s + j] = qo_map_u32_to_unifloat(y);
        }
    }
}

/* Halton points partitioned by dimension 0 (base 2, P = 2^q elements): row r
 * holds dimensions 1..s (bases 3, 5, ..) of point qo_partition_index(2, q, p,
 * j_begin + r); mult[j] is the linear multiplier of output dimension j. */
QO_EXPORT void qo_halton_points_partitioned(uint32_t s, uint32_t mode, const uint32_t* mult,
                                            uint32_t q, uint64_t p, uint64_t j_begin,
                                            uint64_t count, uint32_t* out_u32)
{
    for (uint64_t r = 0; r < count; ++r) {
        uint64_t i = qo_partition_index(2, q, p, j_begin + r);
        for (uint32_t j = 0; j < s; ++j)
            out_u32[r * s + j] = qo_halton_u64(i, j + 1, mode, mult ? mult[j] : 0u);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4, Eq. (R1LS) and Alg. 4: rank-1 lattice sequence in base 2.       */
/* ------------------------------------------------------------------------ */

/* Component j of point k, as an integer in units of 2^-32:
 * (phi_2(k) * g_j + shift_j) mod 1, with g_j forced odd (Alg. 4 sets its
 * least significant bit) and the Cranley-Patterson shift added mod 2^32.
 * Backward enumeration uses phi_2(2^32 - 1 - k) as Alg. 4 does. */
QO_EXPORT uint32_t qo_lattice_u32(uint32_t k, uint32_t g, uint32_t shift, uint32_t backward)
{
    uint32_t phi = qo_bit_reverse(backward ? 0xFFFFFFFFu - k : k);
    uint64_t prod = (uint64_t)phi * (uint64_t)(g | 1u);
    return (uint32_t)((prod + shift) & 0xFFFFFFFFull);
}

QO_EXPORT void qo_lattice_points(const uint32_t* g, const uint32_t* shift, uint32_t s,
                                 uint64_t begin, uint64_t count, uint32_t backward,
                                 uint32_t* out_u32, float* out_f32)
{
    for (uint64_t r = 0; r < count; ++r) {
        uint32_t k = (uint32_t)(begin + r);
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t x = qo_lattice_u32(k, g[j], shift ? shift[j] : 0u, backward);
            if (out_u32) out_u32[r * s + j] = x;
            if (out_f32) out_f32[r * s + j] = qo_map_u32_to_unifloat(x);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3, Eq. (PixelShiftedR1LS): the pixel-shifted rank-1 lattice.         */
/* ------------------------------------------------------------------------ */

/* Position of pixel (x, y) along the Hilbert curve filling the 2^k x 2^k grid
 * (the inverse of the curve's index -> position map).  The curve starts at the
 * origin, visits the quadrants in the order (0,0), (0,1), (1,1), (1,0) of
 * (x-bit, y-bit), and each quadrant holds a copy of the curve turned so that
 * consecutive positions stay neighbours: the lower-left copy is mirrored in
 * the diagonal, the lower-right one in the anti-diagonal. */
QO_EXPORT uint32_t qo_hilbert_index(uint32_t x, uint32_t y, uint32_t k)
{
    uint32_t d = 0;
    for (int level = (int)k - 1; level >= 0; --level) {
        uint32_t rx = (x >> level) & 1u, ry = (y >> level) & 1u;
        uint32_t quad = rx ? (ry ? 2u : 3u) : (ry ? 1u : 0u);
        d = d * 4u + quad;
        uint32_t mask = (1u << level) - 1u;  /* the coordinates inside the quadrant */
        uint32_t lx = x & mask, ly = y & mask;
        if (!ry) {
            if (rx) { lx = mask - lx; ly = mask - ly; }  /* anti-diagonal mirror */
            uint32_t t = lx; lx = ly; ly = t;          /* diagonal mirror */
        }
        x = lx;
        y = ly;
    }
    return d;
}

/* One shift per pixel: floor(phi_3(h) 2^32) of its Hilbert index h. */
QO_EXPORT uint32_t qo_pixel_shift(uint32_t px, uint32_t py, uint32_t k)
{
    return qo_radical_inverse_u32(3, qo_hilbert_index(px, py, k));
}

/* Component j of sample i of the pixel with shift `shift` (units of 2^-32):
 * (phi_2(i) + phi_3(h)) g_j mod 1, with g_j forced odd. */
QO_EXPORT uint32_t qo_pixel_lattice_u32(uint32_t i, uint32_t g, uint32_t shift)
{
    uint64_t base = ((uint64_t)qo_bit_reverse(i) + shift) & 0xFFFFFFFFull;
    return (uint32_t)((base * (uint64_t)(g | 1u)) & 0xFFFFFFFFull);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4.2 and Alg. 4: a random rank-1 lattice sequence per pixel; Sec. 3: */
/* superimposed instances.                                                   */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", 2014): output n (n = 0, 1, ..) of the generator whose state
 * starts at z0 is mix(z0 + (n + 1) gamma), gamma = 0x9E3779B97F4A7C15, where
 * mix applies z ^= z >> 30, z *= 0xBF58476D1CE4E5B9, z ^= z >> 27,
 * z *= 0x94D049BB133111EB, z ^= z >> 31 (arithmetic mod 2^64). */
QO_EXPORT uint64_t qo_splitmix64(uint64_t z0, uint64_t n)
{
    uint64_t z = z0 + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Alg. 4's hash_value, which the paper leaves open, defined here as the high
 * 32 bits of SplitMix64 output number
 *   (py << 44) | (px << 24) | (k << 20) | j
 * of the stream seeded with `seed`: one counter per pixel (px, py < 2^20),
 * superimposed instance k < 16 and dimension j < 2^20. */
QO_EXPORT uint32_t qo_rlat_hash(uint32_t seed, uint32_t k, uint32_t j, uint32_t px, uint32_t py)
{
    uint64_t counter = ((uint64_t)py << 44) | ((uint64_t)px << 24) | ((uint64_t)k << 20) | j;
    return (uint32_t)(qo_splitmix64(seed, counter) >> 32);
}

/* One step of the linear feedback shift register of Sec. 2.4.2: the state is
 * a polynomial of degree < 32 over GF(2) (bit k = coefficient of x^k),
 * multiplied by x modulo the primitive polynomial x^32 + x^22 + x^2 + x + 1.
 * A nonzero state runs through all 2^32 - 1 nonzero states. */
QO_EXPORT uint32_t qo_lfsr_step(uint32_t state)
{
    uint64_t v = (uint64_t)state << 1;           /* multiply by x */
    if ((v >> 32) & 1u) v ^= 0x100400007ull;     /* reduce: subtract (xor) the polynomial */
    return (uint32_t)v;
}

/* Component j of the generator vector of instance k of pixel (px, py):
 *   HASH (Alg. 4): hash_value | 1;
 *   LFSR (Sec. 2.4.2): g_j = 2 xi_j + 1 mod 2^32, where the LFSR serves as the
 *   pseudo-random number generator of 32-bit numbers xi: xi_0 is the instance's
 *   seed state (the hash at the reserved dimension 2^20 - 1, replaced by 1 if 0)
 *   and xi_{j+1} the state 32 steps after xi_j, so that every number holds 32
 *   fresh register bits (one step alone only shifts the state, which would make
 *   g_{j+1} nearly 2 g_j).  One seed defines the whole vector. */
QO_EXPORT uint32_t qo_rlat_generator(uint32_t kind, uint32_t seed, uint32_t k, uint32_t j,
                                     uint32_t px, uint32_t py)
{
    if (kind == QO_RLAT_HASH) return qo_rlat_hash(seed, k, j, px, py) | 1u;
    uint32_t xi = qo_rlat_hash(seed, k, (1u << 20) - 1u, px, py);
    if (xi == 0) xi = 1;
    for (uint64_t t = 0; t < 32ull * j; ++t) xi = qo_lfsr_step(xi);
    return (uint32_t)(((uint64_t)xi * 2u + 1u) & 0xFFFFFFFFull);
}

/* Sample t of pixel (px, py), dimension j, with R superimposed instances
 * (Sec. 3): instance k = t mod R takes its samples i = t div R = 0, 1, ..,
 * enumerated backwards as Alg. 4 does, x = phi_2(2^32 - 1 - i) g_j mod 1, in
 * units of 2^-32. */
QO_EXPORT uint32_t qo_random_lattice_u32(uint32_t kind, uint32_t seed, uint32_t R, uint32_t t,
                                         uint32_t j, uint32_t px, uint32_t py)
{
    uint32_t k = t % R, i = t / R;
    uint64_t prod = (uint64_t)qo_bit_reverse(0xFFFFFFFFu - i) *
                    qo_rlat_generator(kind, seed, k, j, px, py);
    return (uint32_t)(prod & 0xFFFFFFFFull);
}

/* Materialised samples: row q*spp + t holds sample t of pixel pixel_begin + q
 * of a row-major image `width` pixels wide, s dimensions. */
QO_EXPORT void qo_random_lattice_points(uint32_t kind, uint32_t seed, uint32_t R, uint32_t s,
                                        uint32_t width, uint64_t pixel_begin, uint64_t n_pixels,
                                        uint32_t spp, uint32_t* out_u32)
{
    for (uint64_t q = 0; q < n_pixels; ++q) {
        uint64_t p = pixel_begin + q;
        uint32_t px = (uint32_t)(p % width), py = (uint32_t)(p / width);
        for (uint32_t t = 0; t < spp; ++t)
            for (uint32_t j = 0; j < s; ++j)
                out_u32[(q * spp + t) * s + j] = qo_random_lattice_u32(kind, seed, R, t, j, px, py);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.6: test integrands with analytic integrals, in fp64.               */
/* Parameters are fp32 values promoted exactly to double.                    */
/* ------------------------------------------------------------------------ */

/* f(x, y) = (1 + (x - 1/2)/2) (1 + (y - 1/2)/2); its integral over [0,1)^2 is 1. */
static double f_bilinear(const double* x)
{
    return (1.0 + 0.5 * (x[0] - 0.5)) * (1.0 + 0.5 * (x[1] - 0.5));
}

/* Genz product peak: prod_j 1 / (a_j^-2 + (x_j - u_j)^2); theta = a[s], u[s]. */
static double f_genz_product_peak(const double* x, uint32_t s, const float* theta)
{
    double f = 1.0;
    for (uint32_t j = 0; j < s; ++j) {
        double a = theta[j], u = theta[s + j];
        double d = x[j] - u;
        f *= 1.0 / (1.0 / (a * a) + d * d);
    }
    return f;
}

/* Genz oscillatory: cos(2 pi u_1 + sum_j a_j x_j); theta = a[s], u[s]. */
static double f_genz_oscillatory(const double* x, uint32_t s, const float* theta)
{
    const double two_pi = 6.283185307179586476925286766559;
    double arg = two_pi * (double)theta[s];
    for (uint32_t j = 0; j < s; ++j) arg += (double)theta[j] * x[j];
    return cos(arg);
}

/* Mixture of four separable Gaussians in six dimensions.  Component c uses
 * theta[4c..4c+3] = (w_c, mu_c, nu_c, sigma_c): mean mu_c in dimensions
 * 0, 2, 4, mean nu_c in dimensions 1, 3, 5, width sigma_c in all six:
 *   f = sum_c w_c exp(-sum_d (x_d - m_{c,d})^2 / (2 sigma_c^2)).
 * When grad is given, it receives df/dtheta (16 values). */
/* The mixture and, when grad is given, its 16 partial derivatives; with
 * grad_abs, also the sum of the absolute values of the terms each derivative
 * is a sum of (|w| G sum_d |x_d - m| / sigma^2 for a mean, whose differences
 * may cancel; |df/dtheta| for w and sigma, whose terms all have one sign). */
static double f_gaussmix_terms(const double* x, const float* theta, double* grad, double* grad_abs)
{
    double f = 0.0;
    for (uint32_t c = 0; c < 4; ++c) {
        double w = theta[4 * c + 0], mu = theta[4 * c + 1];
        double nu = theta[4 * c + 2], sg = theta[4 * c + 3];
        double q = 0.0, se = 0.0, so = 0.0, ae = 0.0, ao = 0.0;
        for (uint32_t d = 0; d < 6; ++d) {
            double m = (d % 2 == 0) ? mu : nu;
            double diff = x[d] - m;
            q += diff * diff;
            if (d % 2 == 0) se += diff, ae += fabs(diff);
            else so += diff, ao += fabs(diff);
        }
        double G = exp(-q / (2.0 * sg * sg));
        f += w * G;
        if (grad) {
            grad[4 * c + 0] = G;
            grad[4 * c + 1] = w * G * se / (sg * sg);
            grad[4 * c + 2] = w * G * so / (sg * sg);
            grad[4 * c + 3] = w * G * q / (sg * sg * sg);
        }
        if (grad_abs) {
            grad_abs[4 * c + 0] = G;
            grad_abs[4 * c + 1] = fabs(w) * G * ae / (sg * sg);
            grad_abs[4 * c + 2] = fabs(w) * G * ao / (sg * sg);
            grad_abs[4 * c + 3] = fabs(w * G * q / (sg * sg * sg));
        }
    }
    return f;
}

static double f_gaussmix(const double* x, const float* theta, double* grad)
{
    return f_gaussmix_terms(x, theta, grad, NULL);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.5: one integral, samples reduced in index order.                   */
/* ------------------------------------------------------------------------ */

typedef struct { double s, c; } neumaier;

/* Neumaier's compensated addition (the paper names Kahan's algorithm). */
static void neu_add(neumaier* a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/* ------------------------------------------------------------------------ */
/* A procedural scene standing in for Fig. 1's rendering: the irradiance that */
/* a square area light delivers through a spherical occluder onto a          */
/* checkerboard ground plane, seen orthographically from above.              */
/* ------------------------------------------------------------------------ */

/* The scene function of a 4-D sample (x0, x1: position in the pixel's footprint
 * on the plane z = 0; x2, x3: position on the light), theta[16] =
 *   (fx, fy, fw, fh,  cx, cy, h, side,  Le,  ox, oy, oz, rho,  freq, 0, 0):
 * P = (fx + fw x0, fy + fh x1, 0); L = (cx + side (x2 - 1/2), cy + side (x3 - 1/2), h),
 * a light facing down; occluder = sphere (ox, oy, oz) of radius rho inside the
 * slab 0 < z < h.  f = albedo(P) V(P, L) Le side^2 h^2 / |L - P|^4 (the geometry
 * term cos cos / d^2 of two facing horizontal surfaces times the light's area),
 * albedo 0.8 or 0.2 by the parity of floor(freq P_x) + floor(freq P_y).
 * The two decisions -- the checker cell and whether the segment P-L meets the
 * sphere (the discriminant of |P + t (L - P) - O|^2 = rho^2 is >= 0; with the
 * sphere inside the slab every meeting lies inside the segment) -- are taken in
 * fp32 with each operation rounded separately in the order written here, the
 * precision the GPU takes them in; the shading value is fp64. */
static double f_scene(const double* x, const float* th)
{
    float u0 = (float)x[0], u1 = (float)x[1], u2 = (float)x[2], u3 = (float)x[3];  /* exact */
    float Px = th[0] + th[2] * u0;
    float Py = th[1] + th[3] * u1;
    float Lx = th[4] + th[7] * (u2 - 0.5f);
    float Ly = th[5] + th[7] * (u3 - 0.5f);
    float Dx = Lx - Px, Dy = Ly - Py, Dz = th[6];
    float Ex = Px - th[9], Ey = Py - th[10], Ez = -th[11];
    float DE = (Dx * Ex + Dy * Ey) + Dz * Ez;
    float DD = (Dx * Dx + Dy * Dy) + Dz * Dz;
    float EE = (Ex * Ex + Ey * Ey) + Ez * Ez;
    float disc = DE * DE - DD * (EE - th[12] * th[12]);
    if (!(disc < 0.0f)) return 0.0;  /* the sphere blocks the light */
    int cell = ((int)floorf(Px * th[13]) + (int)floorf(Py * th[13])) & 1;
    double albedo = cell ? 0.8 : 0.2;
    double px = (double)th[0] + (double)th[2] * x[0], py = (double)th[1] + (double)th[3] * x[1];
    double lx = (double)th[4] + (double)th[7] * (x[2] - 0.5), ly = (double)th[5] + (double)th[7] * (x[3] - 0.5);
    double h = th[6];
    double d2 = (lx - px) * (lx - px) + (ly - py) * (ly - py) + h * h;
    return albedo * (double)th[8] * (double)th[7] * (double)th[7] * h * h / (d2 * d2);
}

/* QMC estimate (1/n) sum_{i<n} f(x_i; theta) of one integral.
 *   source 0 (Sobol'): x_i = Sobol' point i of C[s][32] randomised by
 *     `scramble` with seeds[s];
 *   source 1 (lattice): x_i = lattice point i of g[s] shifted by seeds[s]
 *     (the Cranley-Patterson rotation), backward when scramble & 1;
 *   source 2 (pixel-shifted lattice, Eq. (PixelShiftedR1LS)): seeds[0] holds
 *     the pixel's shift floor(phi_3(h) 2^32) from qo_pixel_shift;
 *   source 3 (random lattice per pixel, Alg. 4 / Sec. 3): seeds[0..2] hold
 *     (seed, px, py), scramble = kind + 256 R (R superimposed instances).
 * Coordinates are the fp32 values of the float mapping, promoted to fp64.
 * Outputs (each may be NULL except est): est = estimate; mass = (1/n) sum |f|;
 * grad[16] = (1/n) sum df/dtheta, grad_mass[16] = (1/n) sum |df/dtheta| and
 * grad_scale[16] = (1/n) sum of the absolute values of the terms of each
 * df/dtheta (>= grad_mass: the mean's own differences may cancel inside one
 * sample) (Gaussian mixture only; grad_scale needs grad).  n = 0 gives zeros.
 * Returns 0, or -1 on bad arguments. */
QO_EXPORT int qo_integrate_one(uint32_t source, uint32_t integrand, uint32_t s,
                               uint32_t scramble, const uint32_t* C, const uint32_t* g,
                               const uint32_t* seeds, uint32_t n, const float* theta,
                               double* est, double* mass, double* grad, double* grad_mass,
                               double* grad_scale)
{
    if (s == 0 || s > 32) return -1;
    if (integrand == QO_F_BILINEAR2D && s != 2) return -1;
    if (integrand == QO_F_GAUSSMIX4_6D && s != 6) return -1;
    if (integrand == QO_F_SCENE4D && s != 4) return -1;
    if (integrand > QO_F_SCENE4D || source > QO_SOURCE_RANDOM_LATTICE) return -1;
    if (source == QO_SOURCE_RANDOM_LATTICE && (!seeds || (scramble >> 8) == 0)) return -1;

    neumaier sum = {0, 0}, abs_sum = {0, 0};
    neumaier gsum[16], gabs[16], gterm[16];
    for (int k = 0; k < 16; ++k) gsum[k] = gabs[k] = gterm[k] = (neumaier){0, 0};

    double x[32], df[16], dfa[16];
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t v;
            if (source == QO_SOURCE_SOBOL)
                v = randomise_sobol(qo_sobol_u32(C + 32 * j, i), scramble, seeds ? seeds[j] : 0u);
            else if (source == QO_SOURCE_LATTICE)
                v = qo_lattice_u32(i, g[j], seeds ? seeds[j] : 0u, scramble & 1u);
            else if (source == QO_SOURCE_PIXEL_LATTICE)  /* seeds[0]: the pixel's shift */
                v = qo_pixel_lattice_u32(i, g[j], seeds ? seeds[0] : 0u);
            else
                v = qo_random_lattice_u32(scramble & 0xFFu, seeds[0], scramble >> 8, i, j,
                                          seeds[1], seeds[2]);
            x[j] = (double)qo_map_u32_to_unifloat(v);
        }
        double f;
        switch (integrand) {
        case QO_F_BILINEAR2D: f = f_bilinear(x); break;
        case QO_F_GENZ_PRODUCT_PEAK: f = f_genz_product_peak(x, s, theta); break;
        case QO_F_GENZ_OSCILLATORY: f = f_genz_oscillatory(x, s, theta); break;
        case QO_F_SCENE4D: f = f_scene(x, theta); break;
        default: f = f_gaussmix_terms(x, theta, grad ? df : NULL, grad ? dfa : NULL); break;
        }
        neu_add(&sum, f);
        neu_add(&abs_sum, fabs(f));
        if (grad && integrand == QO_F_GAUSSMIX4_6D)
            for (int k = 0; k < 16; ++k) {
                neu_add(&gsum[k], df[k]);
                neu_add(&gabs[k], fabs(df[k]));
                neu_add(&gterm[k], dfa[k]);
            }
    }
    double inv = n ? 1.0 / (double)n : 0.0;
    *est = n ? (sum.s + sum.c) / (double)n : 0.0;
    if (mass) *mass = (abs_sum.s + abs_sum.c) * inv;
    if (grad)
        for (int k = 0; k < 16; ++k) {
            grad[k] = n ? (gsum[k].s + gsum[k].c) / (double)n : 0.0;
            if (grad_mass) grad_mass[k] = (gabs[k].s + gabs[k].c) * inv;
            if (grad_scale) grad_scale[k] = (gterm[k].s + gterm[k].c) * inv;
        }
    return 0;
}

/* qo_integrate_one for integrals p0 .. p1-1 of a batch, one after another:
 * integral p reads seeds + p * seed_stride (NULL: none), counts[p] and
 * theta + p * theta_stride, and writes est[p], mass[p], grad[16 p ..] and
 * grad_mass[16 p ..] and grad_scale[16 p ..] (the last four optional).  Returns 0, or the first
 * non-zero return of qo_integrate_one. */
QO_EXPORT int qo_integrate_range(uint32_t source, uint32_t integrand, uint32_t s, uint32_t scramble,
                                 const uint32_t* C, const uint32_t* g, const uint32_t* seeds,
                                 uint64_t seed_stride, const uint32_t* counts, const float* theta,
                                 uint64_t theta_stride, uint64_t p0, uint64_t p1, double* est,
                                 double* mass, double* grad, double* grad_mass, double* grad_scale)
{
    for (uint64_t p = p0; p < p1; ++p) {
        int rc = qo_integrate_one(source, integrand, s, scramble, C, g,
                                  seeds ? seeds + p * seed_stride : NULL, counts[p],
                                  theta + p * theta_stride, est + p, mass ? mass + p : NULL,
                                  grad ? grad + 16 * p : NULL, grad_mass ? grad_mass + 16 * p : NULL,
                                  grad_scale ? grad_scale + 16 * p : NULL);
        if (rc != 0) return rc;
    }
    return 0;
}

/* Sec. 2.5.1 for integration: the QMC estimate over element p of a Sobol'
 * sequence partitioned across 2^q processing elements by its dimension 0 --
 * samples x_J = dimensions 1..s of point qo_partition_index(2, q, p, J),
 * J = 0 .. n-1, of the m-column matrices C ([s+1][m]) randomised by `scramble`
 * with seeds[s].  The 2^q elements' points together are the sequence's first
 * 2^q n points, so with equal counts the mean of their estimates is the
 * estimate over those points -- an integral of up to 2^(32+q) samples from
 * 32-bit counts.  Outputs as qo_integrate_one. */
QO_EXPORT int qo_integrate_partitioned(uint32_t integrand, uint32_t s, uint32_t scramble,
                                       const uint32_t* C, uint32_t m, uint32_t q, uint64_t p,
                                       const uint32_t* seeds, uint32_t n, const float* theta,
                                       double* est, double* mass, double* grad, double* grad_mass,
                                       double* grad_scale)
{
    if (s == 0 || s > 32 || m < 32 || m > 64 || q > 32 || m < 32 + q) return -1;
    if (integrand == QO_F_BILINEAR2D && s != 2) return -1;
    if (integrand == QO_F_GAUSSMIX4_6D && s != 6) return -1;
    if (integrand == QO_F_SCENE4D && s != 4) return -1;
    if (integrand > QO_F_SCENE4D) return -1;

    neumaier sum = {0, 0}, abs_sum = {0, 0};
    neumaier gsum[16], gabs[16], gterm[16];
    for (int k = 0; k < 16; ++k) gsum[k] = gabs[k] = gterm[k] = (neumaier){0, 0};

    double x[32], df[16], dfa[16];
    for (uint32_t J = 0; J < n; ++J) {
        uint64_t i = qo_partition_index(2, q, p, J);
        for (uint32_t j = 0; j < s; ++j) {
            uint32_t v = randomise_sobol(qo_sobol_u64(C + (uint64_t)m * (j + 1), m, i), scramble,
                                         seeds ? seeds[j] : 0u);
            x[j] = (double)qo_map_u32_to_unifloat(v);
        }
        double f;
        switch (integrand) {
        case QO_F_BILINEAR2D: f = f_bilinear(x); break;
        case QO_F_GENZ_PRODUCT_PEAK: f = f_genz_product_peak(x, s, theta); break;
        case QO_F_GENZ_OSCILLATORY: f = f_genz_oscillatory(x, s, theta); break;
        case QO_F_SCENE4D: f = f_scene(x, theta); break;
        default: f = f_gaussmix_terms(x, theta, grad ? df : NULL, grad ? dfa : NULL); break;
        }
        neu_add(&sum, f);
        neu_add(&abs_sum, fabs(f));
        if (grad && integrand == QO_F_GAUSSMIX4_6D)
            for (int k = 0; k < 16; ++k) {
                neu_add(&gsum[k], df[k]);
                neu_add(&gabs[k], fabs(df[k]));
                neu_add(&gterm[k], dfa[k]);
            }
    }
    double inv = n ? 1.0 / (double)n : 0.0;
    *est = n ? (sum.s + sum.c) / (double)n : 0.0;
    if (mass) *mass = (abs_sum.s + abs_sum.c) * inv;
    if (grad)
        for (int k = 0; k < 16; ++k) {
            grad[k] = n ? (gsum[k].s + gsum[k].c) / (double)n : 0.0;
            if (grad_mass) grad_mass[k] = (gabs[k].s + gabs[k].c) * inv;
            if (grad_scale) grad_scale[k] = (gterm[k].s + gterm[k].c) * inv;
        }
    return 0;
}

/* Integrand value (and Gaussian-mixture gradient) at one fp64 point; used by
 * the finite-difference pins. */
QO_EXPORT double qo_integrand(uint32_t integrand, uint32_t s, const double* x,
                              const float* theta, double* grad)
{
    switch (integrand) {
    case QO_F_BILINEAR2D: return f_bilinear(x);
    case QO_F_GENZ_PRODUCT_PEAK: return f_genz_product_peak(x, s, theta);
    case QO_F_GENZ_OSCILLATORY: return f_genz_oscillatory(x, s, theta);
    case QO_F_SCENE4D: return f_scene(x, theta);
    default: return f_gaussmix(x, theta, grad);
    }
}

/* Gaussian-mixture integrand with fp64 parameters (for central differences in
 * theta, whose perturbed values are not fp32). */
QO_EXPORT double qo_gaussmix_f64(const double* x, const double* th)
{
    double f = 0.0;
    for (uint32_t c = 0; c < 4; ++c) {
        double q = 0.0;
        for (uint32_t d = 0; d < 6; ++d) {
            double diff = x[d] - ((d % 2 == 0) ? th[4 * c + 1] : th[4 * c + 2]);
            q += diff * diff;
        }
        f += th[4 * c + 0] * exp(-q / (2.0 * th[4 * c + 3] * th[4 * c + 3]));
    }
    return f;
}

/* ------------------------------------------------------------------------ */
/* Closed-form integrals over [0,1)^s (Sec. 2.6: test functions with        */
/* analytic integrals).                                                      */
/* ------------------------------------------------------------------------ */

/* Product peak: prod_j a_j [atan(a_j (1 - u_j)) + atan(a_j u_j)]. */
QO_EXPORT double qo_exact_genz_product_peak(uint32_t s, const float* theta)
{
    double I = 1.0;
    for (uint32_t j = 0; j < s; ++j) {
        double a = theta[j], u = theta[s + j];
        I *= a * (atan(a * (1.0 - u)) + atan(a * u));
    }
    return I;
}

/* Oscillatory: Re[ e^{i 2 pi u_1} prod_j (e^{i a_j} - 1) / (i a_j) ]. */
QO_EXPORT double qo_exact_genz_oscillatory(uint32_t s, const float* theta)
{
    const double two_pi = 6.283185307179586476925286766559;
    double re = cos(two_pi * (double)theta[s]), im = sin(two_pi * (double)theta[s]);
    for (uint32_t j = 0; j < s; ++j) {
        double a = theta[j];
        double fr, fi;  /* (e^{ia} - 1)/(ia) = sin(a)/a + i (1 - cos a)/a */
        if (a == 0.0) { fr = 1.0; fi = 0.0; }
        else { fr = sin(a) / a; fi = (1.0 - cos(a)) / a; }
        double nr = re * fr - im * fi, ni = re * fi + im * fr;
        re = nr; im = ni;
    }
    return re;
}

/* int_0^1 exp(-(x - m)^2 / (2 sg^2)) dx = sg sqrt(pi/2) [erf((1-m)/(sg sqrt 2)) + erf(m/(sg sqrt 2))] */
static double gauss_1d(double m, double sg)
{
    const double r2 = 1.4142135623730950488016887242097;
    const double sqrt_half_pi = 1.2533141373155002512078826424055;
    return sg * sqrt_half_pi * (erf((1.0 - m) / (sg * r2)) + erf(m / (sg * r2)));
}

/* d/dm and d/dsg of gauss_1d */
static double gauss_1d_dm(double m, double sg)
{
    return exp(-m * m / (2 * sg * sg)) - exp(-(1 - m) * (1 - m) / (2 * sg * sg));
}
static double gauss_1d_ds(double m, double sg)
{
    return (gauss_1d(m, sg) - (1 - m) * exp(-(1 - m) * (1 - m) / (2 * sg * sg)) -
            m * exp(-m * m / (2 * sg * sg))) / sg;
}

/* sum_c w_c G(mu_c, sigma_c)^3 G(nu_c, sigma_c)^3; grad (may be NULL) gets dI/dtheta. */
QO_EXPORT double qo_exact_gaussmix(const double* th, double* grad)
{
    double I = 0.0;
    for (uint32_t c = 0; c < 4; ++c) {
        double w = th[4 * c], mu = th[4 * c + 1], nu = th[4 * c + 2], sg = th[4 * c + 3];
        double Gm = gauss_1d(mu, sg), Gn = gauss_1d(nu, sg);
        double P = Gm * Gm * Gm * Gn * Gn * Gn;
        I += w * P;
        if (grad) {
            grad[4 * c + 0] = P;
            grad[4 * c + 1] = w * 3 * Gm * Gm * gauss_1d_dm(mu, sg) * Gn * Gn * Gn;
            grad[4 * c + 2] = w * 3 * Gn * Gn * gauss_1d_dm(nu, sg) * Gm * Gm * Gm;
            grad[4 * c + 3] = w * (3 * Gm * Gm * gauss_1d_ds(mu, sg) * Gn * Gn * Gn +
                                   3 * Gn * Gn * gauss_1d_ds(nu, sg) * Gm * Gm * Gm);
        }
    }
    return I;
}

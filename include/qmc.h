/*
 * qmc.h -- C-ABI of libqmc_gb300.so: low-discrepancy point generation and
 * massively parallel quasi-Monte Carlo integro-approximation on one GB300
 * (sm_103a), after Keller, Waechter, Binder, "Quasi-Monte Carlo Algorithms
 * (not only) for Graphics Software" (arXiv 2307.15584).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are
 *     host pointers owned by the caller.  The library allocates no device
 *     memory; kernels that need scratch use the caller's workspace.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  The returned status covers argument
 *     validation and the launch; a fault inside a kernel surfaces at the next
 *     synchronisation, and in-kernel capacity checks set bits that
 *     qmc_read_device_error() returns.
 *   - Invalid arguments are rejected before anything is enqueued.  No C++
 *     exception crosses this boundary.
 *   - QMC_ERR_CUDA: qmc_last_cuda_error() gives the CUDA runtime's error code
 *     behind the most recent QMC_ERR_CUDA returned on the calling thread.
 *   - Fault injection (for tests of a caller's error handling, host side
 *     only): with the environment variable QMC_FAULT_INJECT=launch, every
 *     entry point that would enqueue GPU work validates its arguments as usual
 *     and then returns QMC_ERR_CUDA without any CUDA call;
 *     qmc_last_cuda_error() then reports QMC_INJECTED_FAULT.  The variable is
 *     read on every call.
 *   - NVTX: every entry point that enqueues GPU work opens an NVTX range
 *     named after it (domain "qmc"), visible to Nsight tools.
 *   - Point layouts are row-major [count][s]: row r holds point index_begin + r.
 *   - Indices are 32-bit unless an entry point says otherwise: index_begin +
 *     count must not exceed 2^32 (Sec. 2.5 warns that indices wrapping around
 *     in 32 bits cause subtle errors, so the range is checked instead of
 *     wrapped).  The *_wide and *_partitioned entry points take 64-bit index
 *     ranges (Alg. 3, Sec. 2.5.1), checked the same way.
 */
#ifndef QMC_GB300_H
#define QMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define QMC_API __attribute__((visibility("default")))
#else
#define QMC_API
#endif

/* cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st* qmc_stream_t;

typedef enum qmc_status {
    QMC_OK = 0,
    QMC_ERR_INVALID_ARG = 1, /* null pointer, zero/oversized dimension, bad enum */
    QMC_ERR_RANGE = 2,       /* index range beyond 2^32, counts beyond limits */
    QMC_ERR_ALIGN = 3,       /* a device buffer is not aligned to its element type */
    QMC_ERR_CUDA = 4,        /* the CUDA runtime reported an error at launch */
    QMC_ERR_TIMEOUT = 5,     /* reserved: a bounded device wait gave up */
    QMC_ERR_UNSUPPORTED = 6, /* a valid combination this build does not implement */
    QMC_ERR_WORKSPACE = 7,   /* workspace missing, misaligned or too small */
    QMC_ERR_IO = 8           /* a file could not be read or written (autotune cache) */
} qmc_status;

/* Randomisation of Sobol' points, kept in integers (Sec. 2.1, Sec. 2.3). */
typedef enum qmc_scramble {
    QMC_SCRAMBLE_NONE = 0,   /* plain Eq. (ts) */
    QMC_SCRAMBLE_XOR = 1,    /* random digital shift: y ^ seed (Sec. 2.3) */
    QMC_SCRAMBLE_NESTED = 2, /* hash-based nested (Owen-type) scramble, per-dimension seed */
    QMC_SCRAMBLE_NESTED_XOR = 3 /* the digital shift y ^ seed (Sec. 2.3), then the nested
                                   scramble keyed by the same seed (Sec. 2.1): each dimension's
                                   one seed word selects both */
} qmc_scramble;

/* Flags of rank-1 lattice points. */
#define QMC_LATTICE_BACKWARD 1u /* enumerate phi_2(2^32-1-k) as Alg. 4 does: the origin comes last */

typedef enum qmc_source {
    QMC_SOURCE_SOBOL = 0,         /* digital (t,s)-sequence in base 2, Eq. (ts) */
    QMC_SOURCE_LATTICE = 1,       /* rank-1 lattice sequence in base 2, Eq. (R1LS) */
    QMC_SOURCE_PIXEL_LATTICE = 2, /* pixel-shifted rank-1 lattice, Eq. (PixelShiftedR1LS):
                                     integral p is pixel (x, y) = (p % image_width, p / image_width);
                                     sample i = (phi_2(i) + phi_3(h)) g mod 1 with h the pixel's
                                     position along the Hilbert curve of the smallest 2^k x 2^k
                                     grid covering the image (computed in integers: floor(phi_3
                                     2^32) is added to phi_2(i) 2^32 mod 2^32, then multiplied
                                     by g mod 2^32) */
    QMC_SOURCE_RANDOM_LATTICE = 3 /* a random rank-1 lattice sequence per pixel (Alg. 4, Sec. 3):
                                     integral p is pixel (x, y) as for PIXEL_LATTICE; randomize =
                                     kind | (R << 8) (qmc_rlat_kind; R in {1,2,4,8,16} superimposed
                                     instances); d_seeds[0] = the seed; see qmc_random_lattice_points */
} qmc_source;

/* Generator vectors of the random rank-1 lattices (Sec. 2.4.2). */
typedef enum qmc_rlat_kind {
    QMC_RLAT_HASH = 0,  /* g_j = hash_value(j, pixel, instance) | 1 (Alg. 4) */
    QMC_RLAT_LFSR = 1   /* g_j = 2 xi_j + 1, xi_j = the per-pixel seed state advanced by 32 j
                           LFSR steps (one 32-bit number per 32 register steps) */
} qmc_rlat_kind;

/* Integrands with closed-form integrals (Sec. 2.6 recommends such test
 * functions).  theta layouts are per integral, fp32:
 *   BILINEAR2D          s = 2, no parameters: (1 + (x-1/2)/2)(1 + (y-1/2)/2)
 *   GENZ_PRODUCT_PEAK   1 <= s <= 16, theta = a[s], u[s]: prod_j 1/(a_j^-2 + (x_j-u_j)^2)
 *   GENZ_OSCILLATORY    1 <= s <= 16, theta = a[s], u[s]: cos(2 pi u_1 + sum_j a_j x_j)
 *   GAUSSMIX4_6D        s = 6, theta[16] = 4 x (w, mu, nu, sigma):
 *                       sum_c w_c exp(-sum_d (x_d - m_{c,d})^2 / (2 sigma_c^2)),
 *                       m_{c,d} = mu_c for even d, nu_c for odd d.
 *   SCENE4D             s = 4, theta[16] = (fx, fy, fw, fh, cx, cy, h, side, Le,
 *                       ox, oy, oz, rho, freq, 0, 0): a procedural scene (a Fig. 1
 *                       substitute; no closed form): P = (fx + fw x0, fy + fh x1, 0)
 *                       on a checkerboard plane (albedo 0.8 / 0.2 by the parity of
 *                       floor(freq P_x) + floor(freq P_y)), L = (cx + side (x2 - 1/2),
 *                       cy + side (x3 - 1/2), h) on a square light facing down,
 *                       f = albedo V Le side^2 h^2 / |L - P|^4 with V = 0 when the
 *                       segment P-L meets the sphere (ox, oy, oz; rho) lying inside
 *                       0 < z < h.  The checker and occlusion decisions are taken in
 *                       fp32 with every operation rounded in the order of the
 *                       definition (no fused multiply-add), so they are reproducible
 *                       on any IEEE machine. */
typedef enum qmc_integrand {
    QMC_F_BILINEAR2D = 0,
    QMC_F_GENZ_PRODUCT_PEAK = 1,
    QMC_F_GENZ_OSCILLATORY = 2,
    QMC_F_GAUSSMIX4_6D = 3,
    QMC_F_SCENE4D = 4
} qmc_integrand;

/* One batch of integrals that share a point source and an integrand
 * (Sec. 2.5: many problems in parallel, no intermediate communication).
 * Integral p takes indices 0 .. counts[p]-1 of the source, randomised with
 * its own seeds when seeds_per_integral is set (Sec. 2.5.2, randomised QMC
 * per processing element). */
typedef struct qmc_problem {
    uint32_t source;             /* qmc_source */
    uint32_t integrand;          /* qmc_integrand */
    uint32_t s;                  /* dimension of the points = of the integrand */
    uint32_t randomize;          /* SOBOL: qmc_scramble; LATTICE: 0 or QMC_LATTICE_BACKWARD;
                                    RANDOM_LATTICE: kind | (instances << 8) */
    const uint32_t* d_matrices;  /* SOBOL: [s][32] generator columns (see qmc_sobol_points) */
    const uint32_t* d_g;         /* LATTICE, PIXEL_LATTICE: [s] generator words, low bit forced
                                    to 1 (PIXEL_LATTICE takes no seeds and no randomize flags) */
    const uint32_t* d_seeds;     /* SOBOL: scramble seeds; LATTICE: Cranley-Patterson shifts
                                    (units of 2^-32).  [s], or [n_integrals][s] when
                                    seeds_per_integral = 1.  NULL: no randomisation/shift.
                                    RANDOM_LATTICE: [1], the seed of hash_value (required). */
    uint32_t seeds_per_integral; /* 0 or 1 */
    uint32_t chunk;              /* samples per work item: a power of two in [32, 8192];
                                    0 = the tuned value for this problem class, else 4096 */
    uint32_t block;              /* threads per CTA (multiple of 32, <= 1024); 0 = tuned/256 */
    uint32_t max_count;          /* upper bound of every count; sizes the workspace when the
                                    host does not pass counts to qmc_integrate_workspace_bytes */
    uint32_t with_gradient;      /* 1: size the workspace for qmc_integrate_backward and
                                    qmc_integrate_fwd_bwd (17 partial sums per work item) */
    uint32_t image_width;        /* PIXEL_LATTICE, RANDOM_LATTICE: pixels per image row (>= 1);
                                    the image has ceil(n_integrals / image_width) rows (both
                                    sides at most 2^20 for RANDOM_LATTICE).  Ignored otherwise. */
    uint32_t index_bits;         /* SOBOL: columns per dimension of d_matrices, 0 (= 32, the
                                    layout of qmc_sobol_matrices) or 32..64 (the layout of
                                    qmc_sobol_matrices_wide) */
    uint32_t partition_log2;     /* SOBOL, Sec. 2.5.1: 0, or q in 1..32 with index_bits >= 32 + q:
                                    d_matrices holds s+1 dimensions, dimension 0 the extra
                                    one, and integral p enumerates element p mod 2^q of the
                                    sequence partitioned by it -- sample J of integral p is
                                    dimensions 1..s of point J 2^q + c (c = the q-bit
                                    reversal of p mod 2^q).  With equal counts n, 2^q
                                    consecutive integrals are one integral over the
                                    sequence's first 2^q n points (up to 2^(32+q) samples):
                                    the mean of their estimates.  0 for other sources. */
} qmc_problem;

/* ABI revision of this header (bumped on any incompatible change). */
QMC_API uint32_t qmc_abi_version(void);

/* The value qmc_last_cuda_error() reports for a fault injected by
 * QMC_FAULT_INJECT (no CUDA runtime error code is negative). */
#define QMC_INJECTED_FAULT (-1)

/* The cudaError_t code behind the most recent QMC_ERR_CUDA returned on the
 * calling thread (0 when there was none; QMC_INJECTED_FAULT for an injected
 * fault).  Thread-local; later successful calls do not reset it. */
QMC_API int qmc_last_cuda_error(void);

/* Human-readable name of a status code (static storage). */
QMC_API const char* qmc_status_string(qmc_status status);

/*
 * Sobol' generator matrices (Sec. 2.3, Eq. (ts); host only, no CUDA call).
 *   s            number of dimensions, 1 <= s <= 37 (1 + the 36 primitive
 *                polynomials of degree <= 7)
 *   h_raw_init   [s][7] random words; dimension j >= 1 takes its initial
 *                direction numbers m_k = (h_raw_init[j][k-1] mod 2^k) | 1 for
 *                k <= degree (row 0 is ignored)
 *   h_matrices   out: [s][32]; column k of dimension j is the image of index
 *                bit k, its bit 31 being the first digit 2^-1
 * Dimension 0 is the identity (the van der Corput sequence, phi_2);
 * dimension j >= 1 uses the j-th primitive polynomial over GF(2), enumerated
 * by degree and then by integer encoding (x+1 first, giving the Pascal matrix
 * mod 2), with the Sobol' recurrence
 *   m_k = m_{k-d} ^ (m_{k-d} << d) ^ XOR_{l=1}^{d-1} a_l (m_{k-l} << l),
 * a_l the coefficient of x^(d-l), and column k-1 = m_k << (32-k).
 */
QMC_API qmc_status qmc_sobol_matrices(uint32_t s, const uint32_t* h_raw_init, uint32_t* h_matrices);

/*
 * Sobol' generator matrices for indices of up to m bits (Alg. 3 stores 52
 * columns per dimension; host only, no CUDA call).
 *   m            columns per dimension, 32 <= m <= 64
 *   h_matrices   out: [s][m]; column k of dimension j is the first 32 digits of
 *                the image of index bit k (bit 31 = digit 2^-1)
 * Other arguments as for qmc_sobol_matrices, whose [s][32] output equals the
 * first 32 columns.  Column k-1 holds the first 32 digits of m_k / 2^k for
 * every k (m_k >> (k-32) beyond the 32nd); dimension 0's columns beyond the
 * 32nd are zero, since 2^-k has no digit among the first 32 for k > 32.
 */
QMC_API qmc_status qmc_sobol_matrices_wide(uint32_t s, uint32_t m, const uint32_t* h_raw_init,
                                           uint32_t* h_matrices);

/*
 * Materialised Sobol' points (Alg. 3, Eq. (ts), Sec. 2.1 float conversion).
 *   d_matrices   [s][32] generator columns (layout of qmc_sobol_matrices)
 *   s            1 <= s <= 1024
 *   index_begin, count   indices index_begin .. index_begin+count-1; their
 *                end must not exceed 2^32 (QMC_ERR_RANGE)
 *   scramble     qmc_scramble; d_seeds [s] required unless NONE
 *   d_out_u32    [count][s] integer points (units of 2^-32), or NULL
 *   d_out_f32    [count][s] map_u32_to_unifloat of the same values (every
 *                component in [0,1)), or NULL; at least one output required
 * Outputs must be 4-byte aligned (QMC_ERR_ALIGN); with 16-byte aligned outputs
 * and index_begin * s a multiple of 4 the points are written with 128-bit
 * stores (a start off the row-group grid first writes the rows up to the next
 * group in a separate small launch on the same stream), otherwise the walking
 * kernel writes them (128-bit stores when s % 4 == 0 and both outputs are
 * 16-byte aligned, else 4-byte stores).
 * count = 0 is a no-op.
 */
QMC_API qmc_status qmc_sobol_points(const uint32_t* d_matrices, uint32_t s, uint64_t index_begin,
                            uint64_t count, uint32_t scramble, const uint32_t* d_seeds,
                            uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream);

/*
 * Materialised Sobol' points with 64-bit indices (Alg. 3: the index bits
 * beyond the 32nd select further generator columns).
 *   d_matrices   [s][m] columns (layout of qmc_sobol_matrices_wide), 32 <= m <= 64
 *   index_begin, count   indices index_begin .. index_begin+count-1, all below
 *                2^m (QMC_ERR_RANGE otherwise; for m = 64 the range may end at
 *                2^64 - 1)
 * Other arguments, layouts, paths and errors as for qmc_sobol_points, whose
 * output this reproduces for m = 32.
 */
QMC_API qmc_status qmc_sobol_points_wide(const uint32_t* d_matrices, uint32_t m, uint32_t s,
                                         uint64_t index_begin, uint64_t count, uint32_t scramble,
                                         const uint32_t* d_seeds, uint32_t* d_out_u32,
                                         float* d_out_f32, qmc_stream_t stream);

/*
 * One element of a Sobol' sequence partitioned across P = 2^q processing
 * elements by an extra dimension (Sec. 2.5.1).  Dimension 0 of the matrices
 * (phi_2) is the extra dimension: element p owns the points whose dimension-0
 * coordinate lies in [p/P, (p+1)/P), i.e. the indices i = J 2^q + c_p, c_p the
 * q-bit reversal of p.  Row r holds dimensions 1..s of the point with
 * J = j_begin + r, so each element enumerates its own subsequence without
 * communication; the elements' rows together are the whole sequence.
 *   d_matrices   [s+1][m] columns (layout of qmc_sobol_matrices_wide); dimension
 *                0 must be the identity written there
 *   q            0 <= q < m;  p: 0 <= p < 2^q (QMC_ERR_INVALID_ARG otherwise)
 *   j_begin, count   J = j_begin .. j_begin+count-1, all below 2^(m-q)
 *                (QMC_ERR_RANGE otherwise)
 *   d_seeds      [s] seeds of the output dimensions (unless NONE)
 *   d_out_u32, d_out_f32   [count][s]
 * Other arguments, layouts and errors as for qmc_sobol_points.
 */
QMC_API qmc_status qmc_sobol_points_partitioned(const uint32_t* d_matrices, uint32_t m, uint32_t s,
                                                uint32_t q, uint64_t p, uint64_t j_begin,
                                                uint64_t count, uint32_t scramble,
                                                const uint32_t* d_seeds, uint32_t* d_out_u32,
                                                float* d_out_f32, qmc_stream_t stream);

/*
 * Materialised rank-1 lattice points (Eq. (R1LS), Alg. 4):
 *   x_j(k) = (phi_2(k) g_j + shift_j) mod 1, computed as a 32-bit multiply-add.
 *   d_g          [s] generator words; the low bit is forced to 1 (Alg. 4), so
 *                every dimension is stratified at powers of two (Sec. 2.4.1)
 *   d_shift      [s] Cranley-Patterson shifts in units of 2^-32, or NULL
 *   flags        0 or QMC_LATTICE_BACKWARD (phi_2(2^32-1-k), Alg. 4)
 * Other arguments, layouts and errors as for qmc_sobol_points.
 */
QMC_API qmc_status qmc_lattice_points(const uint32_t* d_g, const uint32_t* d_shift, uint32_t s,
                                      uint64_t index_begin, uint64_t count, uint32_t flags,
                                      uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream);

/* Digit permutations of the Halton engine (Sec. 2.2). */
typedef enum qmc_halton_mode {
    QMC_HALTON_PLAIN = 0,  /* phi_b: the digits mirrored */
    QMC_HALTON_FAURE = 1,  /* Faure's recursive permutation sigma_b of every digit */
    QMC_HALTON_LINEAR = 2  /* linear digit scramble d -> (m_j d) mod b (Alg. 2, radinv_linscramble) */
} qmc_halton_mode;

/*
 * Materialised Halton points (Sec. 2.2, Alg. 1, Alg. 2): component j of point
 * i is the radical inverse of i in base b_j = the j-th prime (2, 3, 5, ...),
 * digits permuted per `mode`, as floor(phi 2^32) (u32) and its float mapping.
 * Base 2 uses the bit reversal of the full 32-bit index; other bases reduce the
 * index modulo the largest power of b_j below 2^32 first (Alg. 1's domain
 * limit), so point i and point i + b_j^K coincide in that dimension.
 *   s              1 <= s <= 64
 *   h_multipliers  HOST array [s] for QMC_HALTON_LINEAR: 1 <= m_j < b_j
 *                  (ignored for base 2); NULL otherwise
 * Other arguments, layouts and errors as for qmc_sobol_points.
 */
QMC_API qmc_status qmc_halton_points(uint32_t s, uint32_t mode, const uint32_t* h_multipliers,
                                     uint64_t index_begin, uint64_t count, uint32_t* d_out_u32,
                                     float* d_out_f32, qmc_stream_t stream);

/*
 * One element of a Halton sequence partitioned across P = 2^q processing
 * elements by its base-2 dimension (Sec. 2.5.1): element p owns the indices
 * i = J 2^q + c_p (c_p the q-bit reversal of p), whose phi_2 lies in
 * [p/P, (p+1)/P).  Row r holds Halton dimensions 1..s (bases 3, 5, ..) of the
 * point with J = j_begin + r; indices are 64-bit and reduced modulo b_j^K as
 * in qmc_halton_points (q = 0 gives the whole sequence with 64-bit indices).
 *   s              1 <= s <= 63
 *   h_multipliers  HOST array [s] for QMC_HALTON_LINEAR, entry j for base
 *                  b_{j+1}: 1 <= m_j < b_{j+1}; NULL otherwise
 *   q              0 <= q <= 63;  p: 0 <= p < 2^q (QMC_ERR_INVALID_ARG otherwise)
 *   j_begin, count   all J below 2^(64-q) (QMC_ERR_RANGE otherwise)
 * Other arguments, layouts and errors as for qmc_halton_points.
 */
QMC_API qmc_status qmc_halton_points_partitioned(uint32_t s, uint32_t mode,
                                                 const uint32_t* h_multipliers, uint32_t q,
                                                 uint64_t p, uint64_t j_begin, uint64_t count,
                                                 uint32_t* d_out_u32, float* d_out_f32,
                                                 qmc_stream_t stream);

/*
 * Materialised per-pixel random rank-1 lattice samples (Alg. 4, Sec. 2.4.2,
 * Sec. 3): every pixel (x, y) of a row-major image_width x image_height image
 * draws its own generator vectors g^(k), k < instances, and sample t of the
 * pixel is
 *   x_j(t) = phi_2(2^32 - 1 - i) g_j^(k) mod 1,  k = t mod R, i = t div R
 * (backwards, so that no pixel starts at the common origin; R superimposed
 * instances hide the rare bad generator vector).  Generator components:
 *   QMC_RLAT_HASH  g_j = hash_value(j) | 1, hash_value = the high 32 bits of
 *                  SplitMix64 output c = y 2^44 + x 2^24 + k 2^20 + j of the
 *                  stream seeded with `seed` (Steele, Lea, Flood 2014)
 *   QMC_RLAT_LFSR  g_j = 2 xi_j + 1 mod 2^32: xi_0 = hash_value at the reserved
 *                  dimension 2^20 - 1 (1 if that is 0), xi_{j+1} = xi_j times x
 *                  modulo x^32 + x^22 + x^2 + x + 1 over GF(2)
 *   kind           qmc_rlat_kind
 *   instances      R in {1, 2, 4, 8, 16}
 *   s              1 <= s <= 1024
 *   image_width, image_height   1 .. 2^20 each
 *   pixel_begin, n_pixels   pixels pixel_begin .. pixel_begin+n_pixels-1 of the
 *                  image (QMC_ERR_RANGE beyond it); spp >= 1 samples each
 *   outputs        [n_pixels * spp][s]: row q*spp + t is sample t of pixel
 *                  pixel_begin + q; u32 (units of 2^-32) and/or fp32
 * Other conventions as for qmc_sobol_points (alignment, count 0 no-op).
 */
QMC_API qmc_status qmc_random_lattice_points(uint32_t kind, uint32_t seed, uint32_t instances, uint32_t s,
                                             uint32_t image_width, uint32_t image_height,
                                             uint64_t pixel_begin, uint64_t n_pixels, uint32_t spp,
                                             uint32_t* d_out_u32, float* d_out_f32, qmc_stream_t stream);

/*
 * Materialised pixel-shifted rank-1 lattice samples (Sec. 3, Eq.
 * (PixelShiftedR1LS)): for pixels pixel_begin .. pixel_begin+n_pixels-1 of a
 * row-major image_width x image_height image, samples 0 .. spp-1 of each pixel,
 *   x_j(i) = (phi_2(i) + phi_3(h)) g_j mod 1,
 * h = the pixel's position along the Hilbert curve of the smallest 2^k x 2^k
 * grid covering the image, in integers as for QMC_SOURCE_PIXEL_LATTICE.
 *   d_g        [s] generator words (low bit forced to 1), 1 <= s <= 1024
 *   outputs    [n_pixels * spp][s]: row q*spp + i is sample i of pixel pixel_begin+q;
 *              4-byte aligned; u32 (units of 2^-32) and/or f32 (map_u32_to_unifloat)
 * Errors: QMC_ERR_INVALID_ARG (null g, zero sizes, no output), QMC_ERR_RANGE
 * (pixels beyond the image), QMC_ERR_ALIGN.  n_pixels = 0 is a no-op.
 */
QMC_API qmc_status qmc_pixel_lattice_points(const uint32_t* d_g, uint32_t s, uint32_t image_width,
                                            uint32_t image_height, uint64_t pixel_begin, uint64_t n_pixels,
                                            uint32_t spp, uint32_t* d_out_u32, float* d_out_f32,
                                            qmc_stream_t stream);

/*
 * Bytes of workspace qmc_integrate / qmc_integrate_backward /
 * qmc_integrate_fwd_bwd / qmc_integrate_points need for n_integrals
 * integrals.  With h_counts (host copy of the counts) the size is exact; with
 * NULL it is the worst case for counts <= p->max_count.  When p->chunk is 0
 * the size covers every chunk the tuner may choose.  The work-item capacity
 * of a call is derived from the workspace_bytes it is given; a call whose
 * items do not fit integrates nothing, writes NaN results and sets bit 0 of
 * the device error word.  Returns 0 for an invalid problem.
 */
QMC_API size_t qmc_integrate_workspace_bytes(const qmc_problem* p, uint32_t n_integrals,
                                     const uint32_t* h_counts);

/*
 * Batched QMC integration (Sec. 2.5, parallel integro-approximation):
 *   d_estimate[p] = (1/counts[p]) sum_{i < counts[p]} f(x_i; theta_p), 0 when
 *   counts[p] = 0.
 * Points are generated, evaluated in fp32 and summed with compensated (Neumaier)
 * fp32 sums inside one persistent kernel; work items are (integral, chunk of
 * p->chunk samples) and each writes its compensated partial to a fixed slot,
 * so the result does not depend on scheduling.  A last kernel adds each
 * integral's partials in index order in fp64 (Sec. 2.5.1: controlled order of
 * additions) and divides by the count.
 *   d_counts     [n_integrals] sample counts, each <= 2^32 - 1
 *   d_theta      [n_integrals][P] fp32 parameters (layout of qmc_integrand), or
 *                NULL for BILINEAR2D
 *   d_estimate   out: [n_integrals] fp64
 *   d_workspace  >= qmc_integrate_workspace_bytes(), 256-byte aligned
 */
QMC_API qmc_status qmc_integrate(const qmc_problem* p, uint32_t n_integrals, const uint32_t* d_counts,
                         const float* d_theta, double* d_estimate, void* d_workspace,
                         size_t workspace_bytes, qmc_stream_t stream);

/*
 * Adjoint of qmc_integrate with respect to theta (GAUSSMIX4_6D only):
 *   d_grad_theta[p][k] = d_grad_estimate[p] (1/counts[p]) sum_i df(x_i; theta_p)/dtheta_k.
 * The points are regenerated, never stored; sums as in qmc_integrate.
 *   d_grad_estimate [n_integrals] fp64 upstream gradient dL/d estimate
 *   d_grad_theta    out: [n_integrals][16] fp32
 */
QMC_API qmc_status qmc_integrate_backward(const qmc_problem* p, uint32_t n_integrals,
                                  const uint32_t* d_counts, const float* d_theta,
                                  const double* d_grad_estimate, float* d_grad_theta,
                                  void* d_workspace, size_t workspace_bytes, qmc_stream_t stream);

/*
 * Fused forward + backward for the squared-error loss (GAUSSMIX4_6D only):
 * one pass over the points computes I_p and J_p = (1/n_p) sum_i df/dtheta, then
 *   d_estimate[p]   = I_p
 *   d_loss[0]       = sum_p (I_p - target_p)^2        (fp64, fixed order)
 *   d_grad_theta[p] = 2 (I_p - target_p) J_p           (fp32)
 *   d_target     [n_integrals] fp64
 */
QMC_API qmc_status qmc_integrate_fwd_bwd(const qmc_problem* p, uint32_t n_integrals,
                                 const uint32_t* d_counts, const float* d_theta,
                                 const double* d_target, double* d_estimate,
                                 float* d_grad_theta, double* d_loss, void* d_workspace,
                                 size_t workspace_bytes, qmc_stream_t stream);

/*
 * Unfused comparison path: integrate points that were materialised in HBM
 * by qmc_sobol_points / qmc_lattice_points (d_points [rows][s] fp32).
 * Integral p reads rows offset_p .. offset_p + counts[p] - 1, where
 * offset_p = sum_{q<p} counts[q], or rows 0 .. counts[p]-1 when
 * points_shared = 1.  Sums and workspace as for qmc_integrate (the problem's
 * source fields are ignored; p->integrand, p->s, p->chunk, p->block apply).
 */
QMC_API qmc_status qmc_integrate_points(const qmc_problem* p, uint32_t n_integrals,
                                const uint32_t* d_counts, const float* d_points,
                                uint32_t points_shared, const float* d_theta,
                                double* d_estimate, void* d_workspace, size_t workspace_bytes,
                                qmc_stream_t stream);

/*
 * Autotuner of the work split (Sec. 2.5: the batch is cut into work items of
 * `chunk` samples, each processed by one warp of a CTA of `block` threads).
 * Times every (chunk, block) in {1024, 2048, 4096, 8192} x {128, 256} on the
 * given problem and inputs (one warm-up and three timed runs each, CUDA events
 * on `stream`; synchronises), returns the fastest and records it for the
 * problem class (device, source, integrand, s, randomisation, per-integral
 * seeds, forward or forward+backward, ceil(log2 n_integrals)); later calls of
 * that class with p->chunk == 0 / p->block == 0 use the recorded values.
 * With d_grad_theta NULL it tunes qmc_integrate, otherwise qmc_integrate_fwd_bwd
 * (d_target and d_loss then required).  The workspace must be sized with
 * p->chunk == 0 (covering every candidate).  Outputs are overwritten.
 */
typedef struct qmc_tuning {
    uint32_t chunk;
    uint32_t block;
    float ms; /* median time of the chosen split */
} qmc_tuning;

QMC_API qmc_status qmc_tune_integrate(const qmc_problem* p, uint32_t n_integrals, const uint32_t* d_counts,
                                      const float* d_theta, const double* d_target, double* d_estimate,
                                      float* d_grad_theta, double* d_loss, void* d_workspace,
                                      size_t workspace_bytes, qmc_stream_t stream, qmc_tuning* h_best);

/* Forget every recorded tuning result (later calls use the defaults). */
QMC_API qmc_status qmc_tune_clear(void);

/*
 * Persistence of the tuner's records (host only; no GPU work).  A record is
 * keyed by the problem class above and by the kind of device it was measured
 * on (its name and SM count), so a file written on one GPU model is ignored on
 * another.  The file is a JSON document:
 *   {"qmc_autotune_cache": 1, "entries": [{"device": "...", "sms": 152,
 *    "source": 0, "integrand": 3, "s": 6, "randomize": 2,
 *    "seeds_per_integral": 1, "gradient": 1, "size_class": 20,
 *    "chunk": 4096, "block": 256}, ...]}
 * size_class = ceil(log2 n_integrals).  Entries with a missing field or an
 * invalid split (chunk a power of two in [32, 8192], block a multiple of 32 up
 * to 256) are skipped when loading.
 *   qmc_tune_save   writes every record to `path` (replaced atomically);
 *                   QMC_ERR_IO when the file cannot be written.
 *   qmc_tune_load   adds the file's records (overriding records of the same
 *                   class); *h_loaded (optional) = records taken; QMC_ERR_IO when
 *                   the file cannot be read.
 *   qmc_tune_lookup the recorded split for a problem class on the current
 *                   device: h_out->chunk, ->block, or both 0 when none (ms = 0).
 * Environment: QMC_AUTOTUNE_CACHE=path makes the library load that file once,
 * before its first lookup or tuning run in the process (a missing file is an
 * empty cache), and rewrite it after every qmc_tune_integrate; a file that
 * cannot be written then leaves the result in memory only.
 */
QMC_API qmc_status qmc_tune_save(const char* path);
QMC_API qmc_status qmc_tune_load(const char* path, uint32_t* h_loaded);
QMC_API qmc_status qmc_tune_lookup(const qmc_problem* p, uint32_t n_integrals, uint32_t with_gradient,
                                   qmc_tuning* h_out);

/*
 * CUDA-graph capture of qmc_* calls (Sec. 2.5: many integrals in one launch
 * sequence replayed without host work).  qmc_graph_begin starts a thread-local
 * capture of `stream` (not the legacy NULL stream); every qmc_* call enqueued
 * on it until qmc_graph_end is recorded with its arguments (pointers, sizes and
 * the problem's values at capture time) and instantiated into a graph that
 * qmc_graph_launch replays on any stream.  The captured buffers must stay alive
 * and in place while the graph exists.  qmc_graph_destroy frees the graph.
 */
typedef struct qmc_graph_st* qmc_graph_t;

QMC_API qmc_status qmc_graph_begin(qmc_stream_t stream);
QMC_API qmc_status qmc_graph_end(qmc_stream_t stream, qmc_graph_t* out_graph);
QMC_API qmc_status qmc_graph_launch(qmc_graph_t graph, qmc_stream_t stream);
QMC_API qmc_status qmc_graph_destroy(qmc_graph_t graph);

/* Size of the device array qmc_integrate_static works in (16 MiB per GPU that
 * loads the library, held until the process exits). */
#define QMC_STATIC_WORKSPACE_BYTES (16u << 20)

/*
 * qmc_integrate for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is an interface for hosts such as a plug-in inside an
 * application that owns all GPU memory, a frame loop that cannot afford
 * cudaMalloc's implicit synchronisation, or a process whose memory budget is
 * fixed at start-up.  It takes the same inputs and output as qmc_integrate but
 * no workspace: the scratch is a fixed device array of
 * QMC_STATIC_WORKSPACE_BYTES inside the library.  It calls no cudaMalloc, no
 * cudaFree and no allocating library routine.
 *   Where the array lives: the CUDA runtime places it on a device when the
 *   library's device code is loaded there, which with lazy module loading (the
 *   default) happens at the first call on that device.  That first call may
 *   therefore take device memory and synchronise like a module load, and can
 *   fail with QMC_ERR_CUDA when the host application already holds all GPU
 *   memory.  Make it at start-up, before memory is committed elsewhere and
 *   before any stream capture: a call with n_integrals = 0 and the problem you
 *   will use places the array, looks up its address and returns QMC_OK
 *   without enqueueing work (d_counts, d_theta and d_estimate may then be
 *   NULL).  Every later call on that device reuses it.
 *   p->max_count must bound every count; the call is rejected with
 *   QMC_ERR_WORKSPACE when the worst case for n_integrals integrals of up to
 *   max_count samples (forward only) does not fit the array, and with
 *   QMC_ERR_INVALID_ARG when max_count is 0.  Counts above max_count that do not
 *   fit are caught on the device: the estimates become NaN.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it per device.
 *   Every call on a device shares the one array, and it keeps the previous
 *   call's contents; each call's first kernel resets the scheduler and error
 *   words, and every other region is written before it is read.  Calls whose
 *   work overlaps on the GPU (different streams or threads without ordering)
 *   race on the array and corrupt each other's results: order them on one
 *   stream.
 */
QMC_API qmc_status qmc_integrate_static(const qmc_problem* p, uint32_t n_integrals,
                                        const uint32_t* d_counts, const float* d_theta,
                                        double* d_estimate, qmc_stream_t stream);

/*
 * The checked build (libqmc_gb300_checked.so, compiled with QMC_CHECKED=1; the
 * binding loads it when QMC_CHECKED=1 is set in the environment).  Every store of
 * a point kernel and every per-item and per-integral store of the integration
 * kernels tests its element offset against the extent the host validated; an
 * offset outside it skips the store and sets a bit of a device error word:
 *   1  a point kernel's store beyond count x s elements
 *   2  an integration work item beyond the workspace's capacity
 * qmc_checked_error synchronises the device, returns the word in *h_bits and,
 * with reset = 1, clears it.  The normal build returns QMC_ERR_UNSUPPORTED (and
 * *h_bits = 0).  Test hook: QMC_CHECK_SLACK=k makes the checked build treat every
 * point output as k elements shorter, so the last stores of a launch are skipped
 * and reported without any access outside the buffers.
 */
QMC_API qmc_status qmc_checked_error(uint32_t* h_bits, uint32_t reset);

/* In-kernel error bits of the last integration that used this workspace
 * (0 = none; bit 0: more work items than the workspace holds).  Synchronises
 * `stream`. */
QMC_API qmc_status qmc_read_device_error(const void* d_workspace, uint32_t* h_error_bits,
                                 qmc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* QMC_GB300_H */

"""Pins of the oracle's per-pixel random rank-1 lattice sequences (Alg. 4,
Sec. 2.4.2), the LFSR-generated generator vectors and the superposition of
instances (Sec. 3), against published values, closed forms and brute force.
CPU only."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs

POLY = (1 << 32) | (1 << 22) | (1 << 2) | (1 << 1) | 1  # x^32 + x^22 + x^2 + x + 1


def _gf2_mulmod(a, b, p=POLY, d=32):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> d) & 1:
            a ^= p
    return r


def _gf2_pow_x(e):
    r, b = 1, 2
    while e:
        if e & 1:
            r = _gf2_mulmod(r, b)
        b = _gf2_mulmod(b, b)
        e >>= 1
    return r


def test_splitmix64_published_outputs(oracle):
    """The first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood)."""
    L = oracle.lib()
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [L.qo_splitmix64(0, n) for n in range(4)] == want


def test_hash_is_uniform_and_separates_its_fields(oracle):
    """hash_value (Alg. 4 leaves it open): the top 8 bits are uniform over a grid of
    pixels, instances and dimensions (chi-square), and changing any one field
    changes the value."""
    L = oracle.lib()
    vals = np.array([L.qo_rlat_hash(77, k, j, px, py) for k in range(4) for j in range(8)
                     for px in range(32) for py in range(16)], np.uint64)
    counts = np.bincount((vals >> np.uint64(24)).astype(np.int64), minlength=256)
    exp = vals.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 255 + 5 * np.sqrt(2 * 255)  # 5 sigma
    base = L.qo_rlat_hash(5, 1, 2, 3, 4)
    for args in ((6, 1, 2, 3, 4), (5, 2, 2, 3, 4), (5, 1, 3, 3, 4), (5, 1, 2, 4, 4), (5, 1, 2, 3, 5)):
        assert L.qo_rlat_hash(*args) != base


def test_lfsr_is_multiplication_by_x_modulo_a_primitive_polynomial(oracle):
    """Sec. 2.4.2's LFSR: x^32 + x^22 + x^2 + x + 1 is primitive (x has order
    2^32 - 1: the maximal period, so xi = 0 never occurs), and each step
    multiplies the state by x modulo it."""
    N = (1 << 32) - 1
    assert _gf2_pow_x(N) == 1
    for q in (3, 5, 17, 257, 65537):  # the prime factors of 2^32 - 1
        assert _gf2_pow_x(N // q) != 1
    L = oracle.lib()
    rng = np.random.default_rng(3)
    for s0 in [1, 0x80000000, 0xFFFFFFFF] + rng.integers(1, 1 << 32, 5).tolist():
        st = int(s0)
        for t in range(1, 200):
            st = L.qo_lfsr_step(st)
            assert st == _gf2_mulmod(int(s0), _gf2_pow_x(t))
            assert st != 0


def _phi2(v):
    return sum(Fraction((v >> k) & 1, 2 ** (k + 1)) for k in range(32))


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("R", [1, 4])
def test_random_lattice_closed_form(oracle, kind, R):
    """Alg. 4: sample i of an instance is phi_2(2^32 - 1 - i) g_j mod 1 in exact
    rational arithmetic; with R superimposed instances, sample t belongs to
    instance t mod R, index t div R; the generator components are odd."""
    L = oracle.lib()
    rng = np.random.default_rng(4 + kind + R)
    for _ in range(60):
        t, j = int(rng.integers(0, 1 << 32)), int(rng.integers(0, 16))
        px, py, seed = int(rng.integers(0, 1920)), int(rng.integers(0, 1080)), int(rng.integers(0, 1 << 32))
        k, i = t % R, t // R
        g = L.qo_rlat_generator(kind, seed, k, j, px, py)
        assert g & 1
        x = _phi2(0xFFFFFFFF - i) * g
        want = int((x - int(x)) * 2**32)
        assert L.qo_random_lattice_u32(kind, seed, R, t, j, px, py) == want


def test_hash_and_lfsr_generators(oracle):
    """HASH: g_j = hash_value | 1.  LFSR: g_j = 2 xi_j + 1 with xi_j = x^(32 j) xi_0
    modulo the LFSR polynomial (32 register steps per number), xi_0 the instance's
    seed state."""
    L = oracle.lib()
    for (seed, k, px, py) in [(1, 0, 0, 0), (99, 3, 1919, 1079), (123456789, 2, 17, 5)]:
        xi0 = L.qo_rlat_hash(seed, k, (1 << 20) - 1, px, py) or 1
        for j in range(40):
            assert L.qo_rlat_generator(0, seed, k, j, px, py) == L.qo_rlat_hash(seed, k, j, px, py) | 1
            xi = _gf2_mulmod(xi0, _gf2_pow_x(32 * j))
            assert L.qo_rlat_generator(1, seed, k, j, px, py) == (2 * xi + 1) % (1 << 32)


def test_lfsr_generator_components_are_not_shifts_of_each_other(oracle):
    """With 32 register steps per number, consecutive components are unrelated
    words.  After a single step (a shift by one bit, plus the taps) every pair
    would have |g_{j+1} - 2 g_j| < 2^24 (mod 2^32); unrelated words land there
    with probability 2^-7, about 3.5 of these 448 pairs."""
    L = oracle.lib()
    near = 0
    for px in range(64):
        g = [L.qo_rlat_generator(1, 7, 0, j, px, 3) for j in range(8)]
        near += sum(1 for a, b in zip(g, g[1:]) if min((b - 2 * a) % (1 << 32), (2 * a - b) % (1 << 32)) < 1 << 24)
    assert near <= 20


def test_backward_enumeration_puts_the_origin_last(oracle):
    """Alg. 4 enumerates backwards so that no pixel starts at the common origin;
    the origin is the last of 2^32 samples."""
    L = oracle.lib()
    for kind in (0, 1):
        g = L.qo_rlat_generator(kind, 9, 0, 2, 10, 20)
        assert L.qo_random_lattice_u32(kind, 9, 1, 0, 2, 10, 20) == (1 << 32) - g
        assert L.qo_random_lattice_u32(kind, 9, 1, 0xFFFFFFFF, 2, 10, 20) == 0
        assert L.qo_random_lattice_u32(kind, 9, 4, 4 * 123, 2, 10, 20) == L.qo_random_lattice_u32(kind, 9, 1, 123, 2,
                                                                                                 10, 20)


@pytest.mark.parametrize("kind", [0, 1])
def test_each_instance_is_a_latin_hypercube(oracle, kind):
    """Odd generator components stratify every dimension: the first 2^m samples
    of every instance hit each of the 2^m intervals [l 2^-m, (l+1) 2^-m) once
    (Sec. 2.4.1); with R = 4 instances interleaved, each instance does."""
    R, m, s, spp = 4, 6, 8, 4 << 6
    pts = oracle.random_lattice_points(kind, 31, R, s, 7, 5, spp, pixel_begin=3)
    for q in range(5):
        rows = pts[q * spp:(q + 1) * spp]
        for k in range(R):
            inst = rows[k::R]
            for j in range(s):
                top = np.sort(inst[:, j] >> np.uint32(32 - m)).astype(np.int64)
                assert np.array_equal(top, np.arange(1 << m)), (q, k, j)


def test_random_lattice_integration(oracle):
    """The per-pixel estimates are the averages of the integrand over the
    materialised samples, and approach the closed-form integrals as the sample
    count grows (random generator vectors promise no more than that on these
    peaked 6-D mixtures)."""
    s, width, n_pix = 6, 16, 24
    theta = inputs.gaussmix_theta(n_pix)
    exact = np.array([oracle.exact_gaussmix(t) for t in theta])
    errs = {}
    for R in (1, 4):
        for n in (256, 4096):
            seeds = oracle.random_lattice_seeds(2024, width, n_pix)
            est = oracle.integrate(oracle.SOURCE_RANDOM_LATTICE, oracle.F_GAUSSMIX4_6D, s,
                                   np.full(n_pix, n, np.uint32), theta, scramble=0 + 256 * R, seeds=seeds)["est"]
            errs[(R, n)] = np.sqrt(np.mean(((est - exact) / exact) ** 2))
            if n == 256:
                pts = oracle.random_lattice_points(0, 2024, R, s, width, 3, n, pixel_begin=5)
                x = oracle.map_u32_to_unifloat(pts).astype(np.float64)
                for q in range(3):
                    f = np.array([oracle.integrand(oracle.F_GAUSSMIX4_6D, xr, theta[5 + q])[0]
                                  for xr in x[q * n:(q + 1) * n]])
                    assert abs(est[5 + q] - f.mean()) <= 1e-12 * abs(f).mean()
    for R in (1, 4):
        assert errs[(R, 4096)] < errs[(R, 256)] / 2, errs

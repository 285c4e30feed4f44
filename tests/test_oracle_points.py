"""Pins of the oracle's point construction against what the paper and the
mathematics fix (closed forms, invariants, brute force).  CPU only."""
from fractions import Fraction
from math import comb, gcd

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs


# ----------------------------------------------------------------- float map
def _trunc_closed_form(u: np.ndarray) -> np.ndarray:
    """u * 2^-32 truncated to 24 significant bits, in exact integer arithmetic."""
    u = u.astype(np.uint64)
    out = np.zeros(u.shape, np.float32)
    nz = u > 0
    # bit length of u (u < 2^32 is exact in float64)
    _, e = np.frexp(u[nz].astype(np.float64))
    drop = np.maximum(e - 24, 0).astype(np.uint64)
    t = (u[nz] >> drop) << drop  # keep the top 24 significant bits
    out[nz] = (t.astype(np.float64) * 2.0**-32).astype(np.float32)  # exact
    return out


def test_map_special_cases(oracle):
    """Sec. 2.1 / Alg. 1: 0 snaps to 0, 1 maps to 2^-32 (biased exponent 126-31)."""
    m = oracle.map_u32_to_unifloat(np.array([0, 1, 0xFFFFFFFF, 1 << 24, 2], np.uint32))
    bits = m.view(np.uint32)
    assert bits[0] == 0
    assert bits[1] == (126 - 31) << 23
    assert bits[2] == 0x3F7FFFFF  # largest float below 1: never rounds up to 1
    assert m[3] == np.float32(2.0**-8)
    assert m[4] == np.float32(2.0**-31)


def test_map_matches_truncation_closed_form(oracle):
    """Sec. 2.1: the best fp32 in [0,1) is u 2^-32 rounded toward zero."""
    rng = np.random.default_rng(1)
    parts = [np.arange(1 << 22, dtype=np.uint32),
             rng.integers(0, 1 << 32, size=1 << 22, dtype=np.uint64).astype(np.uint32)]
    for k in range(32):  # every binade edge
        b = np.int64(1) << k
        parts.append(np.clip(np.arange(b - 300, b + 300), 0, 0xFFFFFFFF).astype(np.uint32))
    parts.append(np.arange(0xFFFFFFFF - 5000, 0xFFFFFFFF + 1, dtype=np.uint64).astype(np.uint32))
    u = np.concatenate(parts)
    got = oracle.map_u32_to_unifloat(u)
    np.testing.assert_array_equal(got.view(np.uint32), _trunc_closed_form(u).view(np.uint32))


def test_map_range_monotone_and_collisions(oracle):
    """Results stay in [0,1), are non-decreasing in u, are exact (collision free)
    below 2^24 and collide from 2^24 = 1/256 on (Sec. 2.1)."""
    rng = np.random.default_rng(2)
    u = np.sort(rng.integers(0, 1 << 32, size=1 << 21, dtype=np.uint64)).astype(np.uint32)
    f = oracle.map_u32_to_unifloat(u)
    assert (f < 1.0).all() and (f >= 0.0).all()
    assert (np.diff(f.astype(np.float64)) >= 0).all()
    small = np.arange(1 << 24, dtype=np.uint32)
    fs = oracle.map_u32_to_unifloat(small)
    np.testing.assert_array_equal(fs.astype(np.float64) * 2.0**32, small.astype(np.float64))
    at = oracle.map_u32_to_unifloat(np.array([(1 << 24) - 1, 1 << 24, (1 << 24) + 1], np.uint32))
    assert at[0] < at[1] and at[1] == at[2]


# ------------------------------------------------------------ bit reversal, phi_b
def test_bit_reverse_and_radical_inverse(oracle):
    """phi_2(i) 2^32 is the mirrored bit string (Sec. 2.2); phi_b by exact fractions."""
    rng = np.random.default_rng(3)
    for i in list(range(64)) + rng.integers(0, 1 << 32, size=200).tolist():
        i = int(i)
        assert oracle.bit_reverse(i) == int(format(i, "032b")[::-1], 2)
        for b in (2, 3, 5, 7):
            phi, k, j = Fraction(0), 0, i
            while j:
                phi += Fraction(j % b, b ** (k + 1))
                j //= b
                k += 1
            assert oracle.radical_inverse_u32(b, i) == int(phi * 2**32)


# ---------------------------------------------------------- primitive polynomials
def _totient(n):
    return sum(1 for k in range(1, n + 1) if gcd(n, k) == 1)


def test_primitive_polynomial_counts(oracle):
    """There are phi(2^d - 1)/d primitive polynomials of degree d over GF(2)."""
    polys = oracle.primitive_polynomials(7)
    degs = [p.bit_length() - 1 for p in polys]
    for d in range(1, 8):
        assert degs.count(d) == _totient(2**d - 1) // d
    assert len(polys) == 36
    # textbook lists for small degrees: x+1; x^2+x+1; x^3+x+1, x^3+x^2+1; x^4+x+1, x^4+x^3+1
    assert polys[:6] == [0b11, 0b111, 0b1011, 0b1101, 0b10011, 0b11001]
    assert degs == sorted(degs)


# ------------------------------------------------------------------ generator matrices
@pytest.fixture(scope="module")
def C32(oracle):
    return oracle.sobol_matrices(32, inputs.sobol_raw_init(32))


def test_dimension0_is_radical_inverse(oracle, C32):
    """Dimension 0 is the identity matrix: the van der Corput radical inverse phi_2."""
    rng = np.random.default_rng(4)
    idx = np.concatenate([np.arange(4096), rng.integers(0, 1 << 32, size=4096)]).astype(np.uint64)
    for i in idx.tolist():
        phi, k, j = Fraction(0), 0, int(i)
        while j:
            phi += Fraction(j % 2, 2 ** (k + 1))
            j //= 2
            k += 1
        assert oracle.lib().qo_sobol_u32(C32[0].ctypes.data, int(i)) == int(phi * 2**32)


def test_dimension1_is_pascal(C32):
    """Dimension 1 (polynomial x+1, m_1 = 1) is the upper-triangular Pascal matrix mod 2:
    column c carries binom(c, l) mod 2 in digit c - l + 1."""
    for c in range(32):
        m = sum((comb(c, l) % 2) << l for l in range(c + 1))
        assert int(C32[1, c]) == m << (31 - c)
    assert [int(C32[1, c]) >> (31 - c) for c in range(8)] == [1, 3, 5, 15, 17, 51, 85, 255]


def test_matrices_unit_upper_triangular(C32):
    """Every column c has digit c+1 set and no later digit: each matrix is
    invertible, so every dimension is stratified at every power of two."""
    for j in range(32):
        for c in range(32):
            col = int(C32[j, c])
            assert (col >> (31 - c)) & 1 == 1
            assert col & ((1 << (31 - c)) - 1) == 0


def _is_tms_net(xy: np.ndarray, m: int, t: int, dims) -> bool:
    """Brute force: every elementary interval of volume 2^(t-m) holds 2^t points."""
    k_total = m - t
    pts = [xy[:, d].astype(np.uint64) for d in dims]
    s = len(dims)

    def compositions(n, parts):
        if parts == 1:
            yield (n,)
            return
        for a in range(n + 1):
            for rest in compositions(n - a, parts - 1):
                yield (a,) + rest

    for ks in compositions(k_total, s):
        code = np.zeros(xy.shape[0], np.uint64)
        for kd, p in zip(ks, pts):
            code = (code << np.uint64(kd)) | (p >> np.uint64(32 - kd)) if kd else code
        cnt = np.bincount(code.astype(np.int64), minlength=1 << k_total)
        if not (cnt == (1 << t)).all():
            return False
    return True


def test_first_two_dims_are_0m2_nets(oracle, C32):
    """Config 1: dims 0-1 of the first 2^m points form a (0,m,2)-net for m <= 16,
    and so does every aligned block of 2^m points (a (0,2)-sequence)."""
    u, _ = oracle.sobol_points(C32[:2], 0, 1 << 16)
    for m in range(1, 17):
        assert _is_tms_net(u[: 1 << m], m, 0, (0, 1)), m
    for m in (3, 6, 9):
        for q in (1, 5, 17):
            blk, _ = oracle.sobol_points(C32[:2], q << m, 1 << m)
            assert _is_tms_net(blk, m, 0, (0, 1))


def test_t_values_of_projections(oracle, C32):
    """Niederreiter: the Sobol' construction is a (t,s)-sequence with
    t = sum_j (deg p_j - 1).  The projection onto dims {0, j} (j >= 1) therefore is a
    (deg p_j - 1, 2)-sequence; a wrong recurrence breaks this."""
    polys = oracle.primitive_polynomials(7)
    u, _ = oracle.sobol_points(C32, 0, 1 << 12)
    for j in range(1, 32):
        t = polys[j - 1].bit_length() - 2
        for m in range(t, 13):
            assert _is_tms_net(u[: 1 << m], m, t, (0, j)), (j, m)
    # one 3-D projection: dims 0,1,2 have t = 0 + 0 + 1
    for m in range(1, 13):
        assert _is_tms_net(u[: 1 << m], m, 1, (0, 1, 2)) or m < 1


def test_each_dimension_stratified(oracle, C32):
    u, _ = oracle.sobol_points(C32, 0, 1 << 12)
    for j in range(32):
        for m in (1, 4, 8, 12):
            top = (u[: 1 << m, j] >> (32 - m)).astype(np.int64)
            assert np.array_equal(np.sort(top), np.arange(1 << m))


# ------------------------------------------------------------------ nested scramble
def test_nested_scramble_is_nested_bijection(oracle):
    """Digit d of the output depends only on digits 1..d of the input and the
    map is one-to-one at every level (Owen's nested structure)."""
    w = 12
    for seed in inputs.scramble_seeds(6, seed=11).tolist():
        a = np.arange(1 << w, dtype=np.uint64)
        low = 0x0005A5A5  # fixed lower digits
        z = np.array([oracle.nested_scramble(int(v << np.uint64(32 - w)) | low, seed) for v in a],
                     dtype=np.uint64)
        top = z >> np.uint64(32 - w)
        assert np.array_equal(np.sort(top), a)  # bijection on the first w digits
        for d in range(1, w):
            grp = (a >> np.uint64(w - d)).astype(np.int64)
            zt = z >> np.uint64(32 - d)
            for g in range(1 << d):
                assert len(set(zt[grp == g].tolist())) == 1


def test_nested_scramble_uniform_and_pairwise(oracle):
    """Over seeds, a fixed point's first 8 digits are close to uniform, and two
    points that first differ at digit k agree at digit k+1 about half the time."""
    seeds = inputs.words32(np.uint64(77), np.arange(1 << 14))
    y = 0x12345678
    top = np.array([oracle.nested_scramble(y, int(s)) >> 24 for s in seeds])
    cnt = np.bincount(top, minlength=256)
    chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
    assert chi2 < 400  # 255 dof: mean 255, sd ~22.6
    for k in (1, 5, 13):
        y1 = 0x0F0F0F0F
        y2 = y1 ^ (1 << (32 - k))  # first differing digit is k
        same = 0
        for s in seeds[:4096].tolist():
            z1, z2 = oracle.nested_scramble(y1, s), oracle.nested_scramble(y2, s)
            assert (z1 >> (32 - k + 1)) == (z2 >> (32 - k + 1))  # digits < k agree
            assert ((z1 >> (32 - k)) & 1) != ((z2 >> (32 - k)) & 1)  # digit k still differs
            same += ((z1 >> (31 - k)) & 1) == ((z2 >> (31 - k)) & 1)
        assert abs(same / 4096 - 0.5) < 0.05


def test_nested_scramble_keeps_net_property(oracle, C32):
    seeds = inputs.scramble_seeds(2, seed=5)
    u, _ = oracle.sobol_points(C32[:2], 0, 1 << 12, mode=oracle.SCRAMBLE_NESTED, seeds=seeds)
    for m in range(1, 13):
        assert _is_tms_net(u[: 1 << m], m, 0, (0, 1))
    ux, _ = oracle.sobol_points(C32[:2], 0, 1 << 10, mode=oracle.SCRAMBLE_XOR, seeds=seeds)
    u0, _ = oracle.sobol_points(C32[:2], 0, 1 << 10)
    np.testing.assert_array_equal(ux, u0 ^ seeds[None, :])


def test_nested_xor_scramble_structure(oracle, C32):
    """QMC_SCRAMBLE_NESTED_XOR (the digital shift, then the nested scramble, one seed
    per dimension): dimension 0 over the first 2^w indices covers every value of
    the first w digits, so the map is seen on all of them; it is a bijection at
    every level and digit d of the output depends only on digits 1..d of the
    input (nested), it keeps the (0,m,2)-net property of dimensions 0-1, and it
    differs from both of the modes it composes."""
    w = 12
    for seed in inputs.scramble_seeds(4, seed=13).tolist():
        sd = np.array([seed], np.uint32)
        y, _ = oracle.sobol_points(C32[:1], 0, 1 << w)  # first w digits = the w-bit reversal of i
        z, _ = oracle.sobol_points(C32[:1], 0, 1 << w, mode=oracle.SCRAMBLE_NESTED_XOR, seeds=sd)
        y, z = y[:, 0].astype(np.uint64), z[:, 0].astype(np.uint64)
        assert np.array_equal(np.sort(z >> np.uint64(32 - w)), np.arange(1 << w, dtype=np.uint64))
        for d in range(1, w):
            prefix = (y >> np.uint64(32 - d)).astype(np.int64)
            out = z >> np.uint64(32 - d)
            for g in range(1 << d):
                assert len(set(out[prefix == g].tolist())) == 1, (seed, d, g)
    seeds = inputs.scramble_seeds(2, seed=5)
    u3, _ = oracle.sobol_points(C32[:2], 0, 1 << 12, mode=oracle.SCRAMBLE_NESTED_XOR, seeds=seeds)
    for m in range(1, 13):
        assert _is_tms_net(u3[: 1 << m], m, 0, (0, 1))
    u1, _ = oracle.sobol_points(C32[:2], 0, 1 << 12, mode=oracle.SCRAMBLE_XOR, seeds=seeds)
    u2, _ = oracle.sobol_points(C32[:2], 0, 1 << 12, mode=oracle.SCRAMBLE_NESTED, seeds=seeds)
    u0, _ = oracle.sobol_points(C32[:2], 0, 1 << 12)
    assert (u3 != u1).mean() > 0.9 and (u3 != u2).mean() > 0.9 and (u3 != u0).mean() > 0.9


def test_nested_xor_uniform_over_seeds(oracle, C32):
    """Over seeds, one fixed point's first 8 digits under NESTED_XOR are close to
    uniform (the shift and the hash share the seed word)."""
    seeds = inputs.words32(np.uint64(78), np.arange(1 << 13))
    top = np.array([oracle.sobol_points(C32[1:2], 1234567, 1, mode=oracle.SCRAMBLE_NESTED_XOR,
                                        seeds=np.array([s], np.uint32), threads=1)[0][0, 0] >> 24
                    for s in seeds.tolist()])
    cnt = np.bincount(top, minlength=256)
    chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
    assert chi2 < 400  # 255 dof: mean 255, sd ~22.6


# ------------------------------------------------------------------ rank-1 lattice
def _rev(k, m):
    return int(format(k, f"0{m}b")[::-1], 2) if m else 0


def test_lattice_closed_form(oracle):
    """Eq. (R1LS), b = 2: point k < 2^m is ((rev_m(k) g) mod 2^m) 2^(32-m); the first
    2^m points are the rank-1 lattice {l g mod 2^m}; odd g stratifies every dimension."""
    g = inputs.lattice_generator(16) | np.uint32(1)
    for m in (1, 5, 10, 14):
        u, _ = oracle.lattice_points(g, None, 0, 1 << m)
        for k in range(0, 1 << m, max(1, (1 << m) // 97)):
            for j in range(16):
                assert int(u[k, j]) == ((_rev(k, m) * int(g[j])) % (1 << m)) << (32 - m)
        for j in range(16):
            top = np.sort((u[:, j] >> (32 - m)).astype(np.int64))
            assert np.array_equal(top, np.arange(1 << m))
    # raw (even) generator words are forced odd, as Alg. 4 does
    graw = inputs.lattice_generator(16)
    a, _ = oracle.lattice_points(graw, None, 0, 64)
    b, _ = oracle.lattice_points(graw | np.uint32(1), None, 0, 64)
    np.testing.assert_array_equal(a, b)


def test_lattice_shift_and_backward(oracle):
    g = inputs.lattice_generator(4) | np.uint32(1)
    sh = inputs.lattice_shift(4)
    u0, _ = oracle.lattice_points(g, None, 100, 300)
    u1, _ = oracle.lattice_points(g, sh, 100, 300)
    np.testing.assert_array_equal(u1, (u0.astype(np.uint64) + sh).astype(np.uint32))
    ub, _ = oracle.lattice_points(g, None, 0, 16, backward=True)
    for k in range(16):
        for j in range(4):
            fw = oracle.lib().qo_lattice_u32(0xFFFFFFFF - k, int(g[j]), 0, 0)
            assert int(ub[k, j]) == fw
    # Alg. 4 enumerates backwards so the origin comes last, not first
    assert (ub[0] != 0).all()
    assert oracle.lib().qo_lattice_u32(0xFFFFFFFF, int(g[0]), 0, 1) == 0


def test_shifted_lattice_identity(oracle):
    """Sec. 2.4.1: phi_2(i + k 2^m) = phi_2(i) + phi_2(k) 2^-m for i < 2^m
    (the printed b^(-m-1) is read as b^(-m): the digits of k move up by m places)."""
    rng = np.random.default_rng(9)
    for _ in range(500):
        m = int(rng.integers(1, 20))
        i = int(rng.integers(0, 1 << m))
        k = int(rng.integers(0, 1 << (32 - m)))
        lhs = oracle.bit_reverse(i + (k << m))
        assert lhs == oracle.bit_reverse(i) + (oracle.bit_reverse(k) >> m)

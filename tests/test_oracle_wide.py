"""Pins of the oracle's wide-index Sobol' construction (Alg. 3: generator
matrices with more than 32 columns, 64-bit indices) and of the partitioning of
one sequence across processing elements (Sec. 2.5.1).  CPU only."""
from fractions import Fraction
from itertools import product
from math import comb

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs

from test_oracle_points import _is_tms_net


@pytest.fixture(scope="module")
def W64(oracle):
    return oracle.sobol_matrices_wide(32, 64, inputs.sobol_raw_init(32))


def _row(C, j, r, ncols):
    """Digit r (0 = b^-1) of dimension j as a GF(2) vector over index bits < ncols."""
    v = 0
    for k in range(ncols):
        v |= ((int(C[j, k]) >> (31 - r)) & 1) << k
    return v


def _rank(rows):
    """Rank over GF(2) of integer-encoded row vectors."""
    basis = {}  # leading bit -> row
    for v in rows:
        while v:
            h = v.bit_length() - 1
            if h not in basis:
                basis[h] = v
                break
            v ^= basis[h]
    return len(basis)


def _compositions(n, parts, cap):
    if parts == 1:
        if 0 <= n <= cap:
            yield (n,)
        return
    for a in range(max(0, n - cap * (parts - 1)), min(cap, n) + 1):
        for rest in _compositions(n - a, parts - 1, cap):
            yield (a,) + rest


def _is_digital_tms_net(C, dims, m, t):
    """Niederreiter's criterion: the first 2^m points (index bits < m) form a
    (t,m,s)-net iff for every d_1 + .. + d_s = m - t the first d_j digits of the
    dimensions are linearly independent over GF(2).  Only the first 32 digits are
    known, so compositions with a part above 32 are skipped."""
    rows = {j: [_row(C, j, r, m) for r in range(32)] for j in dims}
    for ds in _compositions(m - t, len(dims), 32):
        sel = [v for j, d in zip(dims, ds) for v in rows[j][:d]]
        if _rank(sel) != m - t:
            return False
    return True


def test_wide_matrices_extend_the_32_column_ones(oracle, W64):
    C32 = oracle.sobol_matrices(32, inputs.sobol_raw_init(32))
    np.testing.assert_array_equal(W64[:, :32], C32)
    W52 = oracle.sobol_matrices_wide(32, 52, inputs.sobol_raw_init(32))
    np.testing.assert_array_equal(W52, W64[:, :52])
    assert not W64[0, 32:].any()  # 2^-k, k > 32, has no digit among the first 32
    with pytest.raises(ValueError):
        oracle.sobol_matrices_wide(4, 31, inputs.sobol_raw_init(4))
    with pytest.raises(ValueError):
        oracle.sobol_matrices_wide(4, 65, inputs.sobol_raw_init(4))


def test_dimension1_is_pascal_over_64_columns(oracle, W64):
    """Dimension 1 (x + 1) is the Pascal matrix mod 2 for every column: digit r of
    the image of index bit k is binom(k, r) mod 2, i.e. (k & r) == r (Lucas)."""
    for k in range(64):
        for r in range(32):
            assert (int(W64[1, k]) >> (31 - r)) & 1 == (1 if (k & r) == r else 0), (k, r)
    # the same, evaluated on 64-bit indices
    rng = np.random.default_rng(11)
    for i in [(1 << 32), (1 << 63) | 5, (1 << 52) - 1] + rng.integers(0, 1 << 63, 64).tolist():
        i = int(i)
        want = 0
        for r in range(32):
            par = sum(1 for k in range(64) if (i >> k) & 1 and (k & r) == r) & 1
            want |= par << (31 - r)
        assert oracle.lib().qo_sobol_u64(W64[1].ctypes.data, 64, i) == want


def test_dimension0_ignores_index_bits_beyond_32(oracle, W64):
    """phi_2 to 32 digits sees only the low 32 index bits: the (0,1)-sequence
    repeats with period 2^32 at 32-bit output precision."""
    rng = np.random.default_rng(12)
    for i in rng.integers(0, 1 << 63, 64).tolist():
        lo = int(i) & 0xFFFFFFFF
        phi = sum(Fraction((lo >> k) & 1, 2 ** (k + 1)) for k in range(32))
        assert oracle.lib().qo_sobol_u64(W64[0].ctypes.data, 64, int(i)) == int(phi * 2**32)


@pytest.mark.parametrize("m", [33, 40, 52, 64])
def test_t_values_beyond_32_index_bits(oracle, W64, m):
    """The Sobol' construction is a (t,s)-sequence with t = sum_j (deg p_j - 1)
    (Niederreiter), so its first 2^m points form a (t,m,s)-net for every m.  For
    m > 32 the high columns decide the rank criterion; a wrong recurrence or a
    wrong truncation of m_k beyond 2^32 fails it."""
    polys = oracle.primitive_polynomials(7)
    deg = [1] + [p.bit_length() - 1 for p in polys]
    for dims in [(0, 1), (0, 2), (0, 7), (0, 31), (1, 2), (3, 5), (12, 30), (0, 1, 2)]:
        t = sum(deg[j] - 1 for j in dims)
        assert _is_digital_tms_net(W64, dims, m, t), dims
    # the criterion sees the plausible mistakes: high columns left out, or their
    # 32-digit window taken one digit too low (m_k >> (k-31))
    for bad_hi in (np.zeros_like(W64[1, 32:]), W64[1, 32:] >> 1):
        bad = W64.copy()
        bad[1, 32:] = bad_hi
        assert not _is_digital_tms_net(bad, (0, 1), m, 0)


def test_blocks_at_large_offsets_are_nets(oracle, W64):
    """Every aligned block of 2^m points is a (t,m,s)-net, also far beyond 2^32."""
    for K in (1 << 30, (1 << 44) + 12345):
        m = 10
        u, _ = oracle.sobol_points_wide(W64[:3], K << m, 1 << m)
        assert _is_tms_net(u, m, 0, (0, 1))
        assert _is_tms_net(u, m, 1, (0, 1, 2))


def test_wide_points_randomisation_and_range(oracle, W64):
    seeds = inputs.scramble_seeds(8)
    begin = (1 << 40) + 77
    u0, _ = oracle.sobol_points_wide(W64[:8], begin, 64)
    ux, _ = oracle.sobol_points_wide(W64[:8], begin, 64, oracle.SCRAMBLE_XOR, seeds)
    np.testing.assert_array_equal(ux, u0 ^ seeds[None, :])
    un, fn = oracle.sobol_points_wide(W64[:8], begin, 64, oracle.SCRAMBLE_NESTED, seeds)
    for r in range(0, 64, 9):
        for j in range(8):
            assert un[r, j] == oracle.nested_scramble(int(u0[r, j]), int(seeds[j]))
    np.testing.assert_array_equal(fn, oracle.map_u32_to_unifloat(un))
    # the last representable index of a 64-bit sequence
    ul, _ = oracle.sobol_points_wide(W64[:2], (1 << 64) - 1, 1)
    assert ul[0, 0] == 0xFFFFFFFF


# ------------------------------------------------------------------ partitioning (Sec. 2.5.1)
def _phi(b, i, digits=64):
    x, k = Fraction(0), 0
    while i and k < digits:
        x += Fraction(i % b, b ** (k + 1))
        i //= b
        k += 1
    return x


@pytest.mark.parametrize("b,q", [(2, 1), (2, 3), (2, 5), (3, 1), (3, 2), (5, 2)])
def test_partition_is_selection_by_the_extra_dimension(oracle, b, q):
    """Element p of P = b^q owns exactly the points whose extra coordinate
    phi_b(i) lies in [p/P, (p+1)/P), in increasing index order; the elements'
    subsequences are disjoint and cover every index."""
    P = b**q
    N = P * 40
    owner = [int(_phi(b, i) * P) for i in range(N)]
    seen = set()
    for p in range(P):
        mine = [i for i in range(N) if owner[i] == p]
        got = [oracle.partition_index(b, q, p, J) for J in range(len(mine))]
        assert got == mine, (p, got[:4], mine[:4])
        seen.update(got)
    assert seen == set(range(N))


def test_partition_index_large(oracle):
    """64-bit indices: J P + c_p with c_p the digit reversal of p."""
    assert oracle.partition_index(2, 10, 1, (1 << 50) + 3) == ((1 << 50) + 3) * 1024 + 512
    assert oracle.partition_index(2, 0, 0, 12345) == 12345
    assert oracle.partition_index(3, 3, 1, 7) == 7 * 27 + 9


@pytest.mark.parametrize("q", [1, 3, 6])
def test_partitioned_subsequences_are_t_s_minus_1_sequences(oracle, W64, q):
    """Sec. 2.5.1 with net theory: dimensions 0..2 of Sobol' form a (1,3)-sequence,
    so element p's subsequence in dimensions 1..2 is a (1,2)-sequence (an aligned
    block of 2^m of its points fills the elementary intervals of volume 2^(1-m)
    that the (1,m+q,3)-net assigns to the slab [p/P, (p+1)/P)), and dimension 1
    alone a (0,1)-sequence."""
    P = 1 << q
    for p in sorted({0, 1, P - 1, P // 2 + (P > 2)}):
        if p >= P:
            continue
        for m in (4, 8):
            for K in (0, 3):
                u, _ = oracle.sobol_points_partitioned(W64[:3], q, p, K << m, 1 << m)
                assert _is_tms_net(u, m, 1, (0, 1)), (p, m, K)
                assert _is_tms_net(u, m, 0, (0,)), (p, m, K)


def test_partitioned_points_are_the_selected_points(oracle, W64):
    seeds = inputs.scramble_seeds(6)
    for q, p, j0 in [(2, 3, 0), (7, 77, 5), (20, 123456, (1 << 40) + 9)]:
        u, f = oracle.sobol_points_partitioned(W64[:7], q, p, j0, 33, oracle.SCRAMBLE_NESTED, seeds)
        for r in range(33):
            i = oracle.partition_index(2, q, p, j0 + r)
            row, _ = oracle.sobol_points_wide(W64[:7], i, 1, oracle.SCRAMBLE_NESTED,
                                              np.concatenate([[0], seeds]).astype(np.uint32))
            np.testing.assert_array_equal(u[r], row[0, 1:])
            assert int(_phi(2, i, 32) * (1 << q)) == p  # the extra coordinate selects p


# ------------------------------------------------------------------ Halton with 64-bit indices
def test_halton_u64_domain_limit(oracle):
    """Alg. 1 reduces the index modulo the largest power of the base that the
    32-bit result resolves (2^32 for base 2), so wide indices wrap there."""
    rng = np.random.default_rng(13)
    L = oracle.lib()
    for j in (0, 1, 2, 10, 63):
        b = L.qo_prime(j)
        bk = 1 << 32 if b == 2 else max(b**k for k in range(40) if b**k < (1 << 32))
        for i in rng.integers(1 << 32, 1 << 63, 16).tolist() + [(1 << 64) - 1]:
            want = int(_phi(b, int(i) % bk) * 2**32)
            assert L.qo_halton_u64(int(i), j, 0, 0) == want
        for i in rng.integers(0, 1 << 32, 16).tolist():
            assert L.qo_halton_u64(int(i), j, 1, 0) == L.qo_halton_u32(int(i), j, 1, 0)


def test_halton_partitioned(oracle):
    """Partitioned by base 2: the rows are Halton dimensions 1..s of the points
    that the extra coordinate phi_2 assigns to element p."""
    s = 6
    mult = np.array([1 + (3 * j) % (oracle.lib().qo_prime(j + 1) - 1) for j in range(s)], np.uint32)
    for mode, q, p, j0 in product((0, 1, 2), (3, 9), (0, 5), (0, (1 << 30) + 7)):
        got = oracle.halton_points_partitioned(s, q, p, j0, 20, mode, mult)
        for r in range(20):
            i = oracle.partition_index(2, q, p, j0 + r)
            assert int(_phi(2, i % (1 << 32), 32) * (1 << q)) == p
            want = [oracle.lib().qo_halton_u64(i, j + 1, mode, int(mult[j])) for j in range(s)]
            assert got[r].tolist() == want
    # the union of the elements' points is the sequence itself (dimension 1 = phi_3)
    q, n = 2, 64
    allpts = sorted(
        (oracle.partition_index(2, q, p, J), int(oracle.halton_points_partitioned(1, q, p, J, 1)[0, 0]))
        for p in range(4) for J in range(n // 4))
    ref = oracle.halton_points(2, 0, n)
    assert [v for _, v in allpts] == ref[:, 1].tolist()

"""Pins of the oracle's radical inversion engine (Sec. 2.2, Alg. 1, Alg. 2):
Faure permutations against the printed examples, radical inverses against
exact fractions, stratification, the listing's domain limit.  CPU only."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "radinv3_perm.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, *rest = line.split()
            vals[name] = [int(v) for v in rest]
    return vals


def test_primes(oracle):
    assert [oracle.lib().qo_prime(j) for j in range(12)] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37]


def test_faure_printed_examples(oracle):
    """sigma_5 = (0,3,2,1,4) is printed; sigma_4 = (0,2,1,3) follows from the
    even rule applied to sigma_2; every sigma_b is a permutation fixing 0."""
    F = oracle.lib().qo_faure
    assert [F(5, d) for d in range(5)] == _golden()["sigma_5"]
    assert [F(4, d) for d in range(4)] == [0, 2, 1, 3]
    for b in range(2, 60):
        perm = [F(b, d) for d in range(b)]
        assert sorted(perm) == list(range(b)) and perm[0] == 0


def test_two_digit_sigma5_table(oracle):
    """The printed sigma_5 x sigma_5 table encodes digit pair (r, c) as
    5 sigma_5(r) + sigma_5(c).  Rows 1, 3, 4, 5 of the print match; the second
    printed row (25..29) cannot be right (values must stay below 25): the
    reading used is 15 + sigma_5(c) = 15, 18, 17, 16, 19."""
    F = oracle.lib().qo_faure
    g = _golden()
    table = [[5 * F(5, r) + F(5, c) for c in range(5)] for r in range(5)]
    for r in (0, 2, 3, 4):
        assert table[r] == g[f"sigma5x5_row{r}"]
    assert table[1] == [15, 18, 17, 16, 19]
    assert max(g["sigma5x5_row1"]) >= 25  # the misprint


def test_halton_radical_inverse_and_permutations(oracle):
    lib = oracle.lib()
    rng = np.random.default_rng(2)
    for j in range(8):
        b = lib.qo_prime(j)
        maxp = 1
        while maxp * b <= 0xFFFFFFFF:
            maxp *= b
        for i in list(range(200)) + rng.integers(0, 1 << 32, 40).tolist():
            i = int(i)
            ii = i if b == 2 else i % maxp
            for mode, m in ((0, 0), (1, 0), (2, 1 + j % (b - 1) if b > 2 else 1)):
                phi, k, t = Fraction(0), 0, ii
                while t:
                    dgt = t % b
                    dgt = lib.qo_faure(b, dgt) if mode == 1 else (m * dgt) % b if mode == 2 else dgt
                    phi += Fraction(dgt, b ** (k + 1))
                    t //= b
                    k += 1
                assert lib.qo_halton_u32(i, j, mode, m) == int(phi * 2**32)
            # the listing's domain limit: i and i + b^K give the same point (b > 2)
            if b > 2 and i + maxp < 1 << 32:
                assert lib.qo_halton_u32(i, j, 0, 0) == lib.qo_halton_u32(i + maxp, j, 0, 0)


def test_halton_stratification(oracle):
    """The first b^m points of dimension j hit every interval [k/b^m, (k+1)/b^m)
    exactly once, with or without a digit permutation."""
    for mode in (0, 1, 2):
        mult = [1, 2, 3, 4, 5, 6] if mode == 2 else None
        pts = oracle.halton_points(6, 0, 3125, mode, mult, threads=1)
        for j, b in enumerate([2, 3, 5, 7, 11, 13]):
            m = 1
            while b ** (m + 1) <= 3125:
                m += 1
            n = b**m
            cells = sorted(((pts[:n, j].astype(np.int64) + 1) * n) >> 32)
            assert cells == list(range(n)), (mode, j)

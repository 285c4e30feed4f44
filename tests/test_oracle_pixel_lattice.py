"""Pins of the oracle's pixel-shifted rank-1 lattice (Sec. 3, Eq. (PixelShiftedR1LS)):
Hilbert-curve properties, the paper's printed digit table, and the identity that
one shift of phi_2 before the multiplication is a Cranley-Patterson rotation by
shift * g.  CPU only."""
import os

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "radinv3_perm.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, *rest = line.split()
            vals[name] = [int(v) for v in rest]
    return vals


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_hilbert_curve_properties(oracle, k):
    """A bijection of the 2^k x 2^k grid onto 0..4^k-1 that starts at the origin,
    ends at (2^k - 1, 0) and moves to a 4-neighbour at every step."""
    n = 1 << k
    pos = {}
    for x in range(n):
        for y in range(n):
            pos[oracle.hilbert_index(x, y, k)] = (x, y)
    assert sorted(pos) == list(range(n * n))
    assert pos[0] == (0, 0) and pos[n * n - 1] == (n - 1, 0)
    for d in range(n * n - 1):
        (x0, y0), (x1, y1) = pos[d], pos[d + 1]
        assert abs(x0 - x1) + abs(y0 - y1) == 1
    # each quarter of the curve fills one quadrant (the recursive structure)
    q = n // 2
    for d in range(n * n):
        x, y = pos[d]
        quad = {(0, 0): 0, (0, 1): 1, (1, 1): 2, (1, 0): 3}[(x // q if q else 0, y // q if q else 0)]
        assert d // (q * q if q else 1) == quad


def test_printed_base9_table_is_two_digit_base3_reversal(oracle):
    """Alg. 2's table maps d = 3 a + b to 3 b + a (two base-3 digits mirrored), and
    its domain limit is the largest power of 3 below 2^32; the oracle's base-3
    digit loop agrees with two-digit inversion through that table."""
    g = _golden()
    perm = g["radinv3_perm"]
    assert perm == [3 * (d % 3) + d // 3 for d in range(9)]
    assert g["max_power_base3"][0] == 3**20 and 3**21 > 1 << 32 > 3**20
    rng = np.random.default_rng(0)
    for h in list(range(2000)) + rng.integers(0, 1 << 22, 500).tolist():
        num, den, i = 0, 1, int(h)
        while i:  # two digits at a time through the printed table
            num = num * 9 + perm[i % 9]
            den *= 9
            i //= 9
        assert oracle.radical_inverse_u32(3, int(h)) == (num << 32) // den


def test_pixel_shift_is_a_cranley_patterson_rotation(oracle):
    """(phi_2(i) + S) g = phi_2(i) g + S g (mod 1): a pixel's samples are the
    unshifted rank-1 lattice rotated by S g in every dimension."""
    g = inputs.lattice_generator(8) | np.uint32(1)
    rng = np.random.default_rng(1)
    for _ in range(20):
        S = int(rng.integers(0, 1 << 32))
        for i in rng.integers(0, 1 << 32, 30).tolist():
            for j in range(8):
                rot = (S * int(g[j])) % (1 << 32)
                assert oracle.lib().qo_pixel_lattice_u32(i, int(g[j]), S) == oracle.lib().qo_lattice_u32(
                    i, int(g[j]), rot, 0)


def test_shifts_stratify_along_the_curve(oracle):
    """phi_3 along the curve: the first 3^m pixels of the curve receive shifts that
    hit every interval [a/3^m, (a+1)/3^m) exactly once."""
    k = 6
    n = 1 << k
    at = {}
    for x in range(n):
        for y in range(n):
            at[oracle.hilbert_index(x, y, k)] = oracle.pixel_shift(x, y, k)
    for m in (1, 2, 3):
        # shifts are floor(phi_3 2^32): (shift + 1) 3^m >> 32 recovers floor(phi_3 3^m)
        cells = sorted(((at[d] + 1) * 3**m) >> 32 for d in range(3**m))
        assert cells == list(range(3**m))


def test_golden_sigma5(oracle):
    """Sec. 2.2 prints sigma_5 = (0, 3, 2, 1, 4) (Faure's permutation)."""
    assert _golden()["sigma_5"] == [0, 3, 2, 1, 4]

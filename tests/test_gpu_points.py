"""GPU parity of the materialised points (K1 Sobol', K2 lattice) against the
oracle: bit-exact u32 and fp32 bit patterns, through the C-ABI."""
import math

import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _f32_bits(t):
    return t.cpu().numpy().view(np.uint32)


def _sobol_case(B, oracle, s, begin, count, mode, seed=7):
    raw = inputs.sobol_raw_init(s, seed=seed)
    C = B.qmc_sobol_matrices(min(s, 37), raw[: min(s, 37)])
    if s > 37:  # more dimensions than polynomials: reuse columns (any matrices are valid input)
        C = np.concatenate([C] * (s // 37 + 1))[:s]
    seeds = inputs.scramble_seeds(s, seed=seed)
    Cd, sd = B.u32_tensor(C), B.u32_tensor(seeds)
    u, f = B.sobol_points(Cd, count, index_begin=begin, scramble=mode, seeds=sd if mode else None)
    ou, of = oracle.sobol_points(C, begin, count, mode, seeds if mode else None)
    np.testing.assert_array_equal(B.as_u32(u), ou)
    np.testing.assert_array_equal(_f32_bits(f), of.view(np.uint32))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6, 7, 12, 16, 24, 31, 32, 33, 64, 96, 100, 1000])
def test_sobol_points_bit_exact(B, oracle, s, mode):
    """Fast path (s with K <= 4), the walking path (5, 7, 31, 33, 100: lanes own dimensions,
    idle lanes, chunks of 32 and a narrower last one) and, for tables beyond shared memory
    (1000 dimensions), one element per thread; several groups and a ragged tail."""
    count = 4096 * 3 + 37
    _sobol_case(B, oracle, s, 0, count, mode)


@pytest.mark.parametrize("begin", [1, 4, 5, 4096, 123457, (1 << 31) + 8, (1 << 32) - 3000])
def test_sobol_points_offsets(B, oracle, begin):
    for s, mode in ((32, 2), (2, 0), (6, 1), (5, 3), (32, 3)):
        _sobol_case(B, oracle, s, begin, min(2999, (1 << 32) - begin), mode)


@pytest.mark.parametrize("s", [4, 6, 8, 12, 20, 32, 64, 96, 128, 256])
def test_sobol_fast_path_any_start(B, oracle, s):
    """The 16-byte group path from starts off its group grid of Q = 128 / gcd(s, 128) rows: the
    first group cut at the start, ranges inside one group, and last groups cut at the end
    (index_begin * s a multiple of 4, so every group's chunks stay 16-byte aligned)."""
    Q = 128 // math.gcd(s, 128)
    step = 1 if s % 4 == 0 else 4 // math.gcd(s, 4)  # the smallest start spacing with begin * s % 4 == 0
    begins = sorted({step, Q - step, Q + step, 3 * Q + 2 * step, (1 << 31) + step})
    for i, begin in enumerate(begins):
        for count in (1, max(1, Q // 2 - 1), 5 * Q + 3, 4096 + 37):
            _sobol_case(B, oracle, s, begin, count, (i + count) % 4)


@pytest.mark.parametrize("s,begin,count,mode", [
    (32, 1, 4099, 2),      # a start off the group grid: a one-element-per-thread head, then the 16-byte path
    (100, 0, 1027, 3),     # 25 quads per row, one row per warp step (4-byte path: three 32-wide chunks, one 4-wide)
    (36, 6, 1030, 2),      # 9 quads, 3 rows per step, 5 lanes idle (32- and 4-wide chunks)
    (40, 9, 3001, 2),      # 10 quads, 3 rows per step (the bench's s = 40; 32- and 8-wide chunks)
    (44, 5, 2100, 2),      # 11 quads, 2 rows per step (32- and 12-wide chunks)
    (52, 0, 1500, 3),      # 13 quads (32- and 20-wide chunks)
    (60, 2, 999, 1),       # 15 quads (32- and 28-wide chunks)
    (644, 3, 700, 2),      # five 128-wide chunks and a 4-wide one with a 2^5-row table (shared memory is
                           # tight): its 32-row steps go one at a time
    (7, 3, 2053, 1),       # 7-wide chunks, four rows per warp step
    (2, 1, 777, 0),        # 2-wide chunks: 16 rows per warp step
])
def test_sobol_walk_outputs(B, oracle, s, begin, count, mode):
    """The walking path with each output alone (quads of four dimensions per lane, 16-byte
    stores), and with outputs that start 4 and 8 bytes past a 16-byte boundary (one dimension
    per lane, 4-byte stores); counts that leave rows of a unit outside a whole pair or group of
    steps."""
    raw = inputs.sobol_raw_init(s, seed=5)
    C = B.qmc_sobol_matrices(min(s, 37), raw[: min(s, 37)])
    if s > 37:
        C = np.concatenate([C] * (s // 37 + 1))[:s]
    seeds = inputs.scramble_seeds(s, seed=5)
    Cd, sd = B.u32_tensor(C), B.u32_tensor(seeds)
    sk = sd if mode else None
    ou, of = oracle.sobol_points(C, begin, count, mode, seeds if mode else None)
    u, _ = B.sobol_points(Cd, count, index_begin=begin, scramble=mode, seeds=sk, want_f32=False)
    _, f = B.sobol_points(Cd, count, index_begin=begin, scramble=mode, seeds=sk, want_u32=False)
    np.testing.assert_array_equal(B.as_u32(u), ou)
    np.testing.assert_array_equal(_f32_bits(f), of.view(np.uint32))
    ub = torch.zeros(count * s + 1, dtype=torch.int32, device="cuda")
    fb = torch.zeros(count * s + 2, dtype=torch.float32, device="cuda")
    u2, f2 = ub[1:].view(count, s), fb[2:].view(count, s)
    B.qmc_sobol_points(Cd, s, begin, count, mode, sk, u2, f2)
    np.testing.assert_array_equal(B.as_u32(u2), ou)
    np.testing.assert_array_equal(_f32_bits(f2), of.view(np.uint32))
    assert ub[0].item() == 0 and fb[:2].eq(0).all().item()


def test_sobol_single_outputs_and_empty(B, oracle):
    s, n = 32, 1000
    C = B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s))
    seeds = inputs.scramble_seeds(s)
    Cd, sd = B.u32_tensor(C), B.u32_tensor(seeds)
    ou, of = oracle.sobol_points(C, 0, n, 2, seeds)
    u, _ = B.sobol_points(Cd, n, scramble=2, seeds=sd, want_f32=False)
    _, f = B.sobol_points(Cd, n, scramble=2, seeds=sd, want_u32=False)
    np.testing.assert_array_equal(B.as_u32(u), ou)
    np.testing.assert_array_equal(_f32_bits(f), of.view(np.uint32))
    B.sobol_points(Cd, 0, scramble=2, seeds=sd)  # empty: no launch, no error
    with pytest.raises(B.QMCError):
        B.sobol_points(Cd, 16, index_begin=(1 << 32) - 8, scramble=2, seeds=sd)


def test_config1_plain_2d_sobol_and_net(B, oracle):
    """Config 1: 2-D Sobol', 2^16 points, unscrambled; bit-exact and a (0,16,2)-net."""
    C = B.qmc_sobol_matrices(2, inputs.sobol_raw_init(2))
    u, f = B.sobol_points(B.u32_tensor(C), 1 << 16)
    ou, of = oracle.sobol_points(C, 0, 1 << 16)
    gu = B.as_u32(u)
    np.testing.assert_array_equal(gu, ou)
    np.testing.assert_array_equal(_f32_bits(f), of.view(np.uint32))
    for k1 in range(17):
        code = ((gu[:, 0].astype(np.int64) >> (32 - k1)) << (16 - k1)) | (gu[:, 1].astype(np.int64) >> (16 + k1))
        assert np.unique(code).size == 1 << 16, k1


def _compare_in_chunks(B, u, f, ref_fn, rows, chunk=1 << 21):
    """Every row of the device outputs u, f against ref_fn(r0, n) -> (u32, f32), chunk by chunk."""
    for r0 in range(0, rows, chunk):
        n = min(chunk, rows - r0)
        ou, of = ref_fn(r0, n)
        np.testing.assert_array_equal(B.as_u32(u[r0:r0 + n]), ou, err_msg=f"rows {r0}..{r0 + n}")
        np.testing.assert_array_equal(_f32_bits(f[r0:r0 + n]), of.view(np.uint32), err_msg=f"rows {r0}..{r0 + n}")


def test_config2_full_size_every_row(B, oracle):
    """Config 2 at full size (s = 32, 2^24 points, nested scramble, u32 + fp32) in
    the bench's launch configuration: every one of the 2^29 coordinates, both
    outputs, bit for bit against the oracle."""
    s, N = 32, 1 << 24
    C = B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s))
    seeds = inputs.scramble_seeds(s)
    u, f = B.sobol_points(B.u32_tensor(C), N, scramble=2, seeds=B.u32_tensor(seeds))
    torch.cuda.synchronize()
    _compare_in_chunks(B, u, f, lambda r0, n: oracle.sobol_points(C, r0, n, 2, seeds), N)
    del u, f
    torch.cuda.empty_cache()


@pytest.mark.parametrize("backward", [False, True])
@pytest.mark.parametrize("s", [1, 2, 3, 5, 7, 16, 17, 32, 100, 1024])
def test_lattice_points_bit_exact(B, oracle, s, backward):
    """The grouped fast path (s / gcd(s, 128) <= 4, index_begin on its grid) and the flat-chunk
    path (5, 7, 17, 100, 1024 dimensions, or begin 7): batches of 512 rows, chunks straddling
    rows, a ragged last batch, indices up to 2^32 - 1."""
    g = inputs.lattice_generator(s)
    sh = inputs.lattice_shift(s)
    for begin, count, shift in ((0, 4096 * 2 + 13, sh), (7, 3001, None), ((1 << 32) - 2000, 2000, sh)):
        u, f = B.lattice_points(B.u32_tensor(g), count, index_begin=begin,
                                shift=None if shift is None else B.u32_tensor(shift), backward=backward)
        ou, of = oracle.lattice_points(g, shift, begin, count, backward)
        np.testing.assert_array_equal(B.as_u32(u), ou)
        np.testing.assert_array_equal(_f32_bits(f), of.view(np.uint32))


def test_config3_lattice_full_size_every_row(B, oracle):
    """Config 3 points: s = 16, 2^26 points, odd seeded g, integer CP shift; every
    coordinate of both outputs bit for bit against the oracle."""
    s, N = 16, 1 << 26
    g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
    u, f = B.lattice_points(B.u32_tensor(g), N, shift=B.u32_tensor(sh))
    torch.cuda.synchronize()
    _compare_in_chunks(B, u, f, lambda r0, n: oracle.lattice_points(g, sh, r0, n), N, chunk=1 << 22)
    del u, f
    torch.cuda.empty_cache()

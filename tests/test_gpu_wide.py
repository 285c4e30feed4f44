"""GPU parity of wide-index Sobol' points (Alg. 3, 64-bit indices) and of one
element of a partitioned sequence (Sec. 2.5.1), Sobol' and Halton: bit-exact
against the oracle, on the fast (128-bit / TMA) and the generic path."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _wide(B, oracle, m, s):
    """[s+1][m] columns: the library's construction (equal to the oracle's), its
    37 dimensions repeated when more are asked for (the kernels take any columns)."""
    d = min(s + 1, 37)
    raw = inputs.sobol_raw_init(d)
    W = oracle.sobol_matrices_wide(d, m, raw)
    np.testing.assert_array_equal(B.qmc_sobol_matrices_wide(d, m, raw), W)
    W = np.ascontiguousarray(np.resize(W, (s + 1, m)))
    return W, B.u32_tensor(W)


def _run_wide(B, Wd, m, s, begin, count, mode, seeds_d):
    u = torch.empty((count, s), dtype=torch.int32, device="cuda")
    f = torch.empty((count, s), dtype=torch.float32, device="cuda")
    B.qmc_sobol_points_wide(Wd, m, s, begin, count, mode, seeds_d, u, f)
    return B.as_u32(u), f.cpu().numpy()


@pytest.mark.parametrize("m", [32, 52, 64])
@pytest.mark.parametrize("s", [1, 6, 7, 32, 128])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_wide_sobol_bit_exact(B, oracle, m, s, mode):
    W, _ = _wide(B, oracle, m, s)
    Wd = B.u32_tensor(W[:s])
    seeds = inputs.scramble_seeds(s)
    sd = B.u32_tensor(seeds)
    begins = [0, (1 << 32) - 1000, (1 << 32) + 4096, (1 << (m - 1)) + 12345 * 128, (1 << m) - 3001 if m < 64 else U64 - 3000]
    for begin in begins:
        count = 3001
        if begin + count > (1 << m):
            begin = (1 << m) - count
        got_u, got_f = _run_wide(B, Wd, m, s, begin, count, mode, sd)
        ref_u, ref_f = oracle.sobol_points_wide(W[:s], begin, count, mode, seeds)
        np.testing.assert_array_equal(got_u, ref_u, err_msg=f"begin={begin}")
        np.testing.assert_array_equal(got_f.view(np.uint32), ref_f.view(np.uint32))


def test_wide_m32_equals_32bit_entry(B, oracle):
    s = 32
    raw = inputs.sobol_raw_init(s)
    C = B.u32_tensor(B.qmc_sobol_matrices(s, raw))
    sd = B.u32_tensor(inputs.scramble_seeds(s))
    a = torch.empty((1 << 16, s), dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    B.qmc_sobol_points(C, s, 1 << 20, 1 << 16, B.SCRAMBLE_NESTED, sd, a, None)
    B.qmc_sobol_points_wide(C, 32, s, 1 << 20, 1 << 16, B.SCRAMBLE_NESTED, sd, b, None)
    assert torch.equal(a, b)


@pytest.mark.parametrize("m", [52, 64])
@pytest.mark.parametrize("s", [5, 6, 32])
@pytest.mark.parametrize("q,p,j_begin", [(1, 1, 0), (5, 19, 4096), (20, 777777, (1 << 30) + 3),
                                         (40, (1 << 39) + 5, 8), (-4, -1, 0), (-1, 1, 0)])
def test_partitioned_sobol_bit_exact(B, oracle, m, s, q, p, j_begin):
    """q < 0 stands for m + q: the last few bits, where only a handful of J exist
    (the kernel's table entries beyond column m must stay unused)."""
    if q < 0:
        q = m + q
    if p < 0:
        p = (1 << q) - 1
    W, _ = _wide(B, oracle, m, s)
    Wd = B.u32_tensor(W[: s + 1])
    seeds = inputs.scramble_seeds(s, seed=99)
    sd = B.u32_tensor(seeds)
    count = min(2500, (1 << (m - q)) - j_begin)
    for mode in (0, 1, 2, 3):
        u = torch.empty((count, s), dtype=torch.int32, device="cuda")
        f = torch.empty((count, s), dtype=torch.float32, device="cuda")
        B.qmc_sobol_points_partitioned(Wd, m, s, q, p, j_begin, count, mode, sd, u, f)
        ref_u, ref_f = oracle.sobol_points_partitioned(W[: s + 1], q, p, j_begin, count, mode, seeds)
        np.testing.assert_array_equal(B.as_u32(u), ref_u)
        np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32), ref_f.view(np.uint32))


def test_partition_elements_rebuild_the_sequence(B, oracle):
    """The rows of all 2^q elements, placed at their global indices, are
    dimensions 1..s of the whole sequence (no point lost or repeated)."""
    m, s, q, n_per = 64, 32, 4, 1 << 12
    W, _ = _wide(B, oracle, m, s)
    Wd = B.u32_tensor(W[: s + 1])
    sd = B.u32_tensor(inputs.scramble_seeds(s))
    base = 1 << 44  # element-local J range [base, base + n_per)
    whole = torch.empty(((n_per << q), s + 1), dtype=torch.int32, device="cuda")
    sd_whole = B.u32_tensor(np.concatenate([[0], inputs.scramble_seeds(s)]).astype(np.uint32))
    B.qmc_sobol_points_wide(B.u32_tensor(W[: s + 1]), m, s + 1, base << q, n_per << q, B.SCRAMBLE_NESTED,
                            sd_whole, whole, None)
    rebuilt = torch.empty((n_per << q, s), dtype=torch.int32, device="cuda")
    for p in range(1 << q):
        part = torch.empty((n_per, s), dtype=torch.int32, device="cuda")
        B.qmc_sobol_points_partitioned(Wd, m, s, q, p, base, n_per, B.SCRAMBLE_NESTED, sd, part, None)
        c = int(format(p, f"0{q}b")[::-1], 2)
        rebuilt[c:: 1 << q] = part
    assert torch.equal(rebuilt, whole[:, 1:])


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("s,q,p,j_begin", [(6, 0, 0, (1 << 40) + 17), (6, 3, 5, 0), (63, 9, 300, 1 << 33),
                                           (16, 17, 99999, 12345), (4, 63, (1 << 63) - 1, 0)])
def test_partitioned_halton_bit_exact(B, oracle, mode, s, q, p, j_begin):
    L = oracle.lib()
    mult = np.array([1 + (5 * j + 1) % (L.qo_prime(j + 1) - 1) for j in range(s)], np.uint32)
    count = min(1500, (1 << (64 - q)) - j_begin)
    u = torch.empty((count, s), dtype=torch.int32, device="cuda")
    f = torch.empty((count, s), dtype=torch.float32, device="cuda")
    B.qmc_halton_points_partitioned(s, mode, mult if mode == 2 else None, q, p, j_begin, count, u, f)
    ref = oracle.halton_points_partitioned(s, q, p, j_begin, count, mode, mult)
    np.testing.assert_array_equal(B.as_u32(u), ref)
    np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32), oracle.map_u32_to_unifloat(ref).view(np.uint32))


def test_wide_fullsize_sampled(B, oracle):
    """s = 32, 2^24 points, nested scramble, 64-bit indices starting at 2^40, in
    the launch configuration of the 32-bit bench workload: sampled rows against
    the oracle, and the u32 output stratified in every dimension."""
    s, n, m = 32, 1 << 24, 64
    W, _ = _wide(B, oracle, m, s)
    Wd = B.u32_tensor(W[:s])
    seeds = inputs.scramble_seeds(s)
    u = torch.empty((n, s), dtype=torch.int32, device="cuda")
    f = torch.empty((n, s), dtype=torch.float32, device="cuda")
    begin = 1 << 40
    B.qmc_sobol_points_wide(Wd, m, s, begin, n, B.SCRAMBLE_NESTED, B.u32_tensor(seeds), u, f)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.integers(0, n, 2000), [0, n - 1]]))
    gu = B.as_u32(u[torch.from_numpy(rows).cuda()])
    for r, row in zip(rows.tolist(), gu):
        ref, _ = oracle.sobol_points_wide(W[:s], begin + r, 1, B.SCRAMBLE_NESTED, seeds)
        np.testing.assert_array_equal(row, ref[0])
    # an aligned block of 2^24 points of a nested-scrambled (t,s)-sequence: every
    # dimension hits each of the 2^24 strata of width 2^-24 exactly once
    top = (u.to(torch.int64) & 0xFFFFFFFF) >> 8
    for j in (0, 1, 17, 31):
        col = torch.sort(top[:, j]).values
        assert torch.equal(col, torch.arange(n, device="cuda"))

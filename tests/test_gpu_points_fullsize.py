"""Full-size parity of the materialising generators in the launch configuration
the bench's points workload times (s = 32, 2^24 rows, u32 + f32 outputs): sampled
rows against the oracle, computed one by one, plus a property of the whole
output where one holds at any size."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu

S, N = 32, 1 << 24


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def out():
    u = torch.empty((N, S), dtype=torch.int32, device="cuda")
    f = torch.empty((N, S), dtype=torch.float32, device="cuda")
    yield u, f
    del u, f
    torch.cuda.empty_cache()


def _rows(seed=7, k=600):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, N, k), [0, 1, N - 1]]))


def _check_rows(B, oracle, u, f, rows, ref_fn):
    idx = torch.from_numpy(rows).cuda()
    gu, gf = B.as_u32(u[idx]), f[idx].cpu().numpy()
    for k, r in enumerate(rows.tolist()):
        ref = ref_fn(r)
        np.testing.assert_array_equal(gu[k], ref, err_msg=f"row {r}")
        np.testing.assert_array_equal(gf[k].view(np.uint32), oracle.map_u32_to_unifloat(ref).view(np.uint32))


def _stratified_top_bits(u, dims, m, t=0):
    """The first 2^m rows hit each of the 2^(m-t) strata of width 2^(t-m) exactly
    2^t times in each listed dimension (a (t,m,1)-net)."""
    top = ((u[: 1 << m].to(torch.int64) & 0xFFFFFFFF) >> (32 - m + t))
    want = torch.arange(1 << (m - t), device="cuda").repeat_interleave(1 << t)
    for j in dims:
        assert torch.equal(torch.sort(top[:, j]).values, want), j


def test_shifted_lattice_fullsize(B, oracle, out):
    u, f = out
    g, sh = inputs.lattice_generator(S), inputs.lattice_shift(S)
    B.qmc_lattice_points(B.u32_tensor(g), B.u32_tensor(sh), S, 0, N, 0, u, f)
    torch.cuda.synchronize()
    _check_rows(B, oracle, u, f, _rows(1),
                lambda r: np.array([oracle.lib().qo_lattice_u32(r, int(g[j]), int(sh[j]), 0) for j in range(S)],
                                   np.uint32))
    _stratified_top_bits(u - torch.from_numpy(sh.view(np.int32)).cuda()[None, :], (0, 13, 31), 20)


def test_partition_element_fullsize(B, oracle, out):
    u, f = out
    W = B.qmc_sobol_matrices_wide(S + 1, 64, inputs.sobol_raw_init(S + 1))
    seeds = inputs.scramble_seeds(S)
    q, p, j0 = 3, 5, 1 << 37
    B.qmc_sobol_points_partitioned(B.u32_tensor(W), 64, S, q, p, j0, N, B.SCRAMBLE_NESTED, B.u32_tensor(seeds), u, f)
    torch.cuda.synchronize()

    def ref(r):
        row, _ = oracle.sobol_points_partitioned(W, q, p, j0 + r, 1, oracle.SCRAMBLE_NESTED, seeds, threads=1)
        return row[0]

    _check_rows(B, oracle, u, f, _rows(2, 300), ref)
    # the element's points form a (t, s-1)-sequence (Sec. 2.5.1 with net theory): paired with the
    # partition dimension, Sobol' dimension j has t = deg(p_j) - 1, so an aligned block of 2^20 of
    # the element's points stratifies output dimension 0 (x + 1, t = 0) fully and output
    # dimension 1 (x^2 + x + 1, t = 1) at width 2^-19
    _stratified_top_bits(u, (0,), 20)
    _stratified_top_bits(u, (1,), 20, t=1)


def test_halton_faure_fullsize(B, oracle, out):
    u, f = out
    B.qmc_halton_points(S, B.HALTON_FAURE, None, 0, N, u, f)
    torch.cuda.synchronize()
    _check_rows(B, oracle, u, f, _rows(3),
                lambda r: oracle.halton_points(S, r, 1, oracle.HALTON_FAURE, threads=1)[0])
    # base 2 (dimension 0) is the bit reversal: the first 2^24 rows stratify it completely
    _stratified_top_bits(u, (0,), 24)


def test_pixel_lattice_fullsize(B, oracle, out):
    u, f = out
    g = inputs.lattice_generator(S)
    width = height = 1024
    spp = 16
    B.qmc_pixel_lattice_points(B.u32_tensor(g), S, width, height, 0, width * height, spp, u, f)
    torch.cuda.synchronize()
    rows = _rows(4, 200)
    k = oracle.grid_log2(width, height)
    idx = torch.from_numpy(rows).cuda()
    gu = B.as_u32(u[idx])
    for n, r in enumerate(rows.tolist()):
        pix, t = divmod(r, spp)
        shift = oracle.pixel_shift(pix % width, pix // width, k)
        ref = [oracle.lib().qo_pixel_lattice_u32(t, int(g[j]), shift) for j in range(S)]
        assert gu[n].tolist() == ref, r


@pytest.mark.parametrize("kind", [0, 1])
def test_random_lattice_fullsize(B, oracle, out, kind):
    u, f = out
    width = height = 1024
    spp, R, seed = 16, 4, 7
    B.qmc_random_lattice_points(kind, seed, R, S, width, height, 0, width * height, spp, u, f)
    torch.cuda.synchronize()
    rows = _rows(5 + kind, 200)
    idx = torch.from_numpy(rows).cuda()
    gu, gf = B.as_u32(u[idx]), f[idx].cpu().numpy()
    L = oracle.lib()
    for n, r in enumerate(rows.tolist()):
        pix, t = divmod(r, spp)
        ref = np.array([L.qo_random_lattice_u32(kind, seed, R, t, j, pix % width, pix // width) for j in range(S)],
                       np.uint32)
        np.testing.assert_array_equal(gu[n], ref, err_msg=f"row {r}")
        np.testing.assert_array_equal(gf[n].view(np.uint32), oracle.map_u32_to_unifloat(ref).view(np.uint32))


def test_sobol_walk_fullsize(B, oracle, out):
    """The bench's walking-kernel configuration: s = 32 from index 1 (off the fast path's
    group grid), nested scramble, 2^24 rows."""
    u, f = out
    C = B.qmc_sobol_matrices(S, inputs.sobol_raw_init(S))
    seeds = inputs.scramble_seeds(S)
    B.qmc_sobol_points(B.u32_tensor(C), S, 1, N, B.SCRAMBLE_NESTED, B.u32_tensor(seeds), u, f)
    torch.cuda.synchronize()
    _check_rows(B, oracle, u, f, _rows(8),
                lambda r: oracle.sobol_points(C, 1 + r, 1, oracle.SCRAMBLE_NESTED, seeds, threads=1)[0][0])
    # rows 2^k - 1 .. of the first 2^20 points from index 1 are a shifted window; the block of
    # indices [2^20, 2^21) lies at rows 2^20 - 1 .. 2^21 - 2 and stratifies dimension 0 fully
    top = (u[(1 << 20) - 1: (1 << 21) - 1].to(torch.int64) & 0xFFFFFFFF) >> 12
    assert torch.equal(torch.sort(top[:, 0]).values, torch.arange(1 << 20, device="cuda"))


def test_halton_partition_fullsize(B, oracle, out):
    """The bench's partitioned Halton configuration: element 5 of 8 from J = 2^30, Faure."""
    u, f = out
    q, p, j0 = 3, 5, 1 << 30
    B.qmc_halton_points_partitioned(S, B.HALTON_FAURE, None, q, p, j0, N, u, f)
    torch.cuda.synchronize()
    _check_rows(B, oracle, u, f, _rows(9),
                lambda r: oracle.halton_points_partitioned(S, q, p, j0 + r, 1, oracle.HALTON_FAURE, threads=1)[0])


def test_lattice_flat_fullsize(B, oracle, out):
    """The bench's flat-chunk lattice configuration: the shifted rank-1 lattice, s = 32, from
    index 1 (off the grouped kernel's grid), 2^24 rows."""
    u, f = out
    g, sh = inputs.lattice_generator(S), inputs.lattice_shift(S)
    B.qmc_lattice_points(B.u32_tensor(g), B.u32_tensor(sh), S, 1, N, 0, u, f)
    torch.cuda.synchronize()
    _check_rows(B, oracle, u, f, _rows(10),
                lambda r: np.array([oracle.lib().qo_lattice_u32(1 + r, int(g[j]), int(sh[j]), 0) for j in range(S)],
                                   np.uint32))
    # indices [2^20, 2^21) sit at rows 2^20 - 1 .. 2^21 - 2 and stratify every dimension
    _stratified_top_bits((u[(1 << 20) - 1: (1 << 21) - 1] - torch.from_numpy(sh.view(np.int32)).cuda()[None, :])
                         .contiguous(), (0, 13, 31), 20)


def test_sobol_wide_fullsize(B, oracle, out):
    """The bench's 64-bit-index configuration (Alg. 3): s = 32 of the 64-column matrices from
    index 2^40, nested scramble, 2^24 rows."""
    u, f = out
    W = B.qmc_sobol_matrices_wide(S + 1, 64, inputs.sobol_raw_init(S + 1))
    seeds = inputs.scramble_seeds(S)
    B.qmc_sobol_points_wide(B.u32_tensor(W), 64, S, 1 << 40, N, B.SCRAMBLE_NESTED, B.u32_tensor(seeds), u, f)
    torch.cuda.synchronize()
    Ws = np.ascontiguousarray(W[:S])

    def ref(r):
        row, _ = oracle.sobol_points_wide(Ws, (1 << 40) + r, 1, oracle.SCRAMBLE_NESTED, seeds, threads=1)
        return row[0]

    _check_rows(B, oracle, u, f, _rows(11, 300), ref)
    # an aligned block of 2^20 points beyond 2^40: dimension 0 (the identity) stratified fully
    _stratified_top_bits(u, (0,), 20)

"""GPU parity of integration over elements of a partitioned Sobol' sequence
(Sec. 2.5.1): integral k enumerates element k mod 2^q of the sequence that
dimension 0 of the wide matrices partitions, its samples the remaining
dimensions.  Per-element estimates against the oracle on the same points; the
elements' mean against the estimate over the whole sequence; and integrals of
2^32 - 1 samples per element, where the index reaches bit 63 and only
properties that hold at any size can be checked.

Tolerances as in the plain integration tests (tests/tolerances.py)."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs
from tolerances import est_tol, grad_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _run(B, prob, counts, theta, with_grad=False):
    n = counts.size
    cd, thd = B.u32_tensor(counts), torch.from_numpy(np.ascontiguousarray(theta)).cuda()
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, cd, thd, est, ws)
    g = None
    if with_grad:  # an upstream gradient of 1: the gradient means J themselves
        gt = torch.empty((n, 16), dtype=torch.float32, device="cuda")
        B.qmc_integrate_backward(prob, n, cd, thd, torch.ones(n, dtype=torch.float64, device="cuda"), gt, ws)
        g = gt.cpu().numpy()
    torch.cuda.synchronize()
    assert B.qmc_read_device_error(ws) == 0
    return est.cpu().numpy(), g


# (integrand, s, q, m, scramble, per-integral seeds)
CASES = {
    "gaussmix_q3_m64_nested": ("gaussmix", 6, 3, 64, 2, True),
    "oscillatory_q5_m40_xor": ("oscillatory", 8, 5, 40, 1, False),
    "product_peak_q1_m33_plain": ("product_peak", 16, 1, 33, 0, False),
    "scene_q32_m64_nested": ("scene", 4, 32, 64, 2, True),
    "product_peak_q2_m48_nested_xor": ("product_peak", 5, 2, 48, 3, True),
}


def _theta(B, oracle, name, s, n):
    if name == "gaussmix":
        th = inputs.gaussmix_theta(n, seed=5)
        return B.F_GAUSSMIX4_6D, oracle.F_GAUSSMIX4_6D, th, np.abs(th[:, 0::4]).sum(axis=1)
    if name == "scene":
        th = inputs.scene_theta(20, (n + 19) // 20)[:n]
        return B.F_SCENE4D, oracle.F_SCENE4D, th, np.ones(n)
    th = np.stack([inputs.genz_params(name, s, k) for k in range(n)])
    kind = {"oscillatory": "F_GENZ_OSCILLATORY", "product_peak": "F_GENZ_PRODUCT_PEAK"}[name]
    return getattr(B, kind), getattr(oracle, kind), th, np.ones(n)


@pytest.mark.parametrize("case", list(CASES))
def test_element_estimates_match_oracle(B, oracle, case):
    name, s, q, m, scr, per = CASES[case]
    n = 300  # with q = 3: each element several times over; a ragged mix of counts
    counts = inputs.log_uniform_counts(n, hi=20000, seed=11)
    counts[[0, 7]] = 0, 1
    F, OF, theta, W = _theta(B, oracle, name, s, n)
    Wm = oracle.sobol_matrices_wide(s + 1, m, inputs.sobol_raw_init(s + 1))
    seeds = inputs.pixel_seeds(n, s, seed=6) if per else inputs.scramble_seeds(s, seed=6)
    grad = name == "gaussmix"
    keep = (B.u32_tensor(Wm), B.u32_tensor(seeds))
    prob = B.make_problem(B.SOURCE_SOBOL, F, s, scr, matrices=keep[0], seeds=keep[1] if scr else None,
                          seeds_per_integral=per, with_gradient=grad, index_bits=m, partition_log2=q)
    e, g = _run(B, prob, counts, theta, grad)
    elements = np.arange(n, dtype=np.uint64) % (np.uint64(1) << np.uint64(q))
    ref = oracle.integrate_partitioned(OF, s, counts, theta, Wm, q, elements, scramble=scr,
                                       seeds=seeds if scr else None, with_grad=grad)
    bad = np.abs(e - ref["est"]) > est_tol(ref["est"], W)
    assert not bad.any(), (np.flatnonzero(bad)[:5], e[bad][:5], ref["est"][bad][:5])
    assert e[0] == 0.0
    if grad:
        g_tol = grad_tol(theta, ref["grad"], ref["grad_scale"], tau=2e-6)
        assert (np.abs(g - ref["grad"]) <= g_tol).all(), np.max(np.abs(g - ref["grad"]) / g_tol)


def test_elements_combine_into_the_whole_sequence(B, oracle):
    """Equal counts: the mean of the 2^q elements' estimates is the estimate over
    the sequence's first 2^q n points, which the plain (32-column) path computes
    from dimensions 1..s; and 64 columns with q = 0 reproduce that path exactly."""
    s, q, n0 = 6, 4, (1 << 16) + 3
    P = 1 << q
    Wm = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
    seeds = inputs.scramble_seeds(s, seed=8)
    th = inputs.gaussmix_theta(1, seed=9)
    W = float(np.abs(th[0, 0::4]).sum())
    keep = (B.u32_tensor(Wm), B.u32_tensor(seeds), B.u32_tensor(np.ascontiguousarray(Wm[1:, :32])),
            B.u32_tensor(np.ascontiguousarray(Wm[1:])))
    part = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, s, B.SCRAMBLE_NESTED, matrices=keep[0],
                          seeds=keep[1], index_bits=64, partition_log2=q)
    e_parts, _ = _run(B, part, np.full(P, n0, np.uint32), np.tile(th, (P, 1)))
    whole = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, s, B.SCRAMBLE_NESTED, matrices=keep[2],
                           seeds=keep[1])
    counts = np.array([P * n0, 12345], np.uint32)
    e_whole, _ = _run(B, whole, counts, np.tile(th, (2, 1)))
    wide = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, s, B.SCRAMBLE_NESTED, matrices=keep[3],
                          seeds=keep[1], index_bits=64)
    e_wide, _ = _run(B, wide, counts, np.tile(th, (2, 1)))
    np.testing.assert_array_equal(e_wide, e_whole)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, s, counts[:1], th,
                           C=np.ascontiguousarray(Wm[1:, :32]), scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)
    assert abs(e_whole[0] - ref["est"][0]) <= est_tol(ref["est"][0], W)
    assert abs(e_parts.mean() - ref["est"][0]) <= 2 * est_tol(ref["est"][0], W)


@pytest.mark.parametrize("q", [2, 32])
def test_full_index_range(B, oracle, q):
    """2^32 - 1 samples in each of 4 elements (q = 32: indices up to 2^64 - 1,
    every column of the 64-column matrices in use): the bilinear integrand's
    exact value 1 within the (t,s)-sequence error and the fp32 sums' rounding;
    their mean likewise."""
    s, P = 2, 4
    Wm = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
    keep = (B.u32_tensor(Wm),)
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_BILINEAR2D, s, 0, matrices=keep[0], index_bits=64,
                          partition_log2=q)
    counts = np.full(P, 0xFFFFFFFF, np.uint32)
    e, _ = _run(B, prob, counts, np.zeros((P, 1), np.float32))
    assert np.all(np.abs(e - 1.0) < 2e-6), e
    assert abs(e.mean() - 1.0) < 2e-6

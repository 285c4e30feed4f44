"""GPU parity of the fused integration kernels against the fp64 oracle on the
same points, through the C-ABI.

Tolerances (per result; tests/tolerances.py): |I32 - I64| <= 1e-6 |I64| + 1e-12 W,
where W is the sum of the mixture weights (1 for the other integrands): fp32
evaluation with compensated sums, fp64 only in the last per-integral reduction.
Gradient means J: 1e-6 |J| (w, sigma) or 1e-6 (|J| + M) (mu, nu; M = mean
|df/dtheta|, the scale of the terms that cancel) plus an underflow floor."""
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


def _gaussmix_case(B, n, counts, seed=3, chunk=0, block=0, scramble=2):
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n, seed=seed)
    seeds = inputs.pixel_seeds(n, 6, seed=seed)
    dev = {"C": B.u32_tensor(C6), "counts": B.u32_tensor(counts), "theta": torch.from_numpy(theta).cuda(),
           "seeds": B.u32_tensor(seeds)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, scramble, matrices=dev["C"],
                          seeds=dev["seeds"] if scramble else None, seeds_per_integral=True, chunk=chunk,
                          block=block, with_gradient=True)
    return C6, theta, seeds, dev, prob


def _run_forward(B, prob, n, dev, counts):
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, dev["counts"], dev["theta"], est, ws)
    torch.cuda.synchronize()
    assert B.qmc_read_device_error(ws) == 0
    return est.cpu().numpy()


def test_config1_bilinear(B, oracle):
    """Config 1: the 2-D Sobol' estimate of the bilinear integrand (exact value 1)."""
    C = B.qmc_sobol_matrices(2, inputs.sobol_raw_init(2))
    counts = np.array([1 << 16, 1 << 10, 1, 0, 1000], np.uint32)
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_BILINEAR2D, 2, 0, matrices=B.u32_tensor(C))
    cd = B.u32_tensor(counts)
    ws = B.alloc_workspace(prob, counts.size, counts)
    est = torch.empty(counts.size, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, counts.size, cd, None, est, ws)
    e = est.cpu().numpy()
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_BILINEAR2D, 2, counts, np.zeros((5, 1)), C=C)
    assert (np.abs(e - ref["est"]) <= est_tol(ref["est"], 1.0)).all(), (e, ref["est"])
    assert e[3] == 0.0
    assert abs(e[0] - 1.0) < 1e-5


@pytest.mark.parametrize("family", ["product_peak", "oscillatory"])
def test_config3_genz_lattice(B, oracle, family):
    """Config 3 (reduced count): rank-1 lattice s = 16 with CP shift, four seeded
    parameter sets, several chunks per integral and a ragged last chunk."""
    s, n = 16, 4
    N = (1 << 20) + 77
    g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
    theta = np.stack([inputs.genz_params(family, s, k) for k in range(n)])
    kind = B.F_GENZ_PRODUCT_PEAK if family == "product_peak" else B.F_GENZ_OSCILLATORY
    counts = np.full(n, N, np.uint32)
    prob = B.make_problem(B.SOURCE_LATTICE, kind, s, 0, g=B.u32_tensor(g), seeds=B.u32_tensor(sh))
    dev = {"counts": B.u32_tensor(counts), "theta": torch.from_numpy(theta).cuda()}
    e = _run_forward(B, prob, n, dev, counts)
    ref = oracle.integrate(oracle.SOURCE_LATTICE, kind, s, counts, theta, g=g, seeds=sh)
    err = np.abs(e - ref["est"])
    assert (err <= est_tol(ref["est"], 1.0)).all(), (err, ref["est"])


def test_config4_batched_small(B, oracle):
    """Config 4 (reduced): log-uniform counts in [1, 65536], per-pixel nested
    scramble seeds, the Gaussian mixture; every result against the oracle."""
    n = 1500
    counts = inputs.log_uniform_counts(n, seed=4)
    counts[:5] = [0, 1, 2, 31, 65536]
    C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts, seed=4)
    e = _run_forward(B, prob, n, dev, counts)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    err = np.abs(e - ref["est"])
    bad = err > est_tol(ref["est"], W)
    assert e[0] == 0.0
    assert not bad.any(), (np.nonzero(bad)[0][:10], (err / np.maximum(np.abs(ref["est"]), 1e-300))[bad][:10],
                           counts[bad][:10])


def test_tail_dominated_single_samples(B, oracle):
    """Pixels with one or a few samples, often far in a Gaussian's tail (where the
    fp32 exponent argument's rounding error grows with |t|): the adaptive float-float
    recomputation keeps every estimate within 1e-6 of the fp64 oracle."""
    n = 8000
    counts = np.where(np.arange(n) % 4 == 0, 1, np.arange(n) % 7 + 1).astype(np.uint32)
    C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts, seed=31)
    e = _run_forward(B, prob, n, dev, counts)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    err = np.abs(e - ref["est"])
    bad = err > est_tol(ref["est"], W)
    assert not bad.any(), (np.nonzero(bad)[0][:10], (err / np.abs(ref["est"]))[bad][:10])


@pytest.mark.parametrize("family", ["product_peak", "oscillatory"])
@pytest.mark.parametrize("source,s", [("lattice", 16), ("sobol_nested", 5)])
def test_genz_few_samples(B, oracle, family, source, s):
    """Genz integrals of one to seven samples, where an fp32 evaluation's own
    rounding (the oscillatory phase, the product's sixteen factors) is not
    averaged away: the adaptive float-float recomputation keeps every estimate
    within 1e-6 of the fp64 oracle."""
    n = 6000
    counts = (np.arange(n) % 7 + 1).astype(np.uint32)
    theta = np.stack([inputs.genz_params(family, s, k, seed=77) for k in range(n)])
    kind = B.F_GENZ_PRODUCT_PEAK if family == "product_peak" else B.F_GENZ_OSCILLATORY
    okind = oracle.F_GENZ_PRODUCT_PEAK if family == "product_peak" else oracle.F_GENZ_OSCILLATORY
    if source == "lattice":
        g, sh = inputs.lattice_generator(s, seed=78), inputs.lattice_shift(s, seed=79)
        keep = (B.u32_tensor(g), B.u32_tensor(sh))
        prob = B.make_problem(B.SOURCE_LATTICE, kind, s, 0, g=keep[0], seeds=keep[1])
        okw = dict(source=oracle.SOURCE_LATTICE, g=g, seeds=sh)
    else:
        C = B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s))
        sd = inputs.pixel_seeds(n, s, seed=80)
        keep = (B.u32_tensor(C), B.u32_tensor(sd))
        prob = B.make_problem(B.SOURCE_SOBOL, kind, s, B.SCRAMBLE_NESTED, matrices=keep[0], seeds=keep[1],
                              seeds_per_integral=True)
        okw = dict(source=oracle.SOURCE_SOBOL, C=C, scramble=oracle.SCRAMBLE_NESTED, seeds=sd)
    dev = {"counts": B.u32_tensor(counts), "theta": torch.from_numpy(theta).cuda()}
    e = _run_forward(B, prob, n, dev, counts)
    ref = oracle.integrate(integrand=okind, s=s, counts=counts, theta=theta, **okw)
    err = np.abs(e - ref["est"])
    bad = err > est_tol(ref["est"], 1.0)
    assert not bad.any(), (np.nonzero(bad)[0][:10], (err / np.abs(ref["est"]))[bad][:10], counts[bad][:10])


@pytest.mark.parametrize("scramble", [0, 1, 3])
def test_other_scrambles_and_chunks(B, oracle, scramble):
    n = 200
    counts = inputs.log_uniform_counts(n, hi=20000, seed=8)
    for chunk, block in ((32, 64), (1024, 128), (8192, 256)):
        C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts, seed=8, chunk=chunk, block=block,
                                                      scramble=scramble)
        e = _run_forward(B, prob, n, dev, counts)
        ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                               scramble=scramble, seeds=seeds if scramble else None)
        W = np.abs(theta[:, 0::4]).sum(axis=1)
        assert (np.abs(e - ref["est"]) <= est_tol(ref["est"], W)).all()


def test_determinism_and_unfused_equality(B):
    """Two runs are bitwise identical; the unfused path (points materialised in HBM,
    then integrated) gives bitwise the same estimates as the fused kernel."""
    n = 300
    counts = inputs.log_uniform_counts(n, hi=8192, seed=12)
    C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts, seed=12, scramble=1)
    e1 = _run_forward(B, prob, n, dev, counts)
    e2 = _run_forward(B, prob, n, dev, counts)
    np.testing.assert_array_equal(e1, e2)
    # materialise each pixel's points (XOR scramble with its seeds) back to back
    rows = int(counts.sum())
    pts = torch.empty((rows, 6), dtype=torch.float32, device="cuda")
    r0 = 0
    for p in range(n):
        c = int(counts[p])
        if c:
            view = pts[r0:r0 + c]
            B.qmc_sobol_points(dev["C"], 6, 0, c, 1, dev["seeds"][p], None, view)
        r0 += c
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate_points(prob, n, dev["counts"], pts, 0, dev["theta"], est, ws)
    np.testing.assert_array_equal(est.cpu().numpy(), e1)


def test_capacity_error_is_reported_not_overrun(B):
    n = 64
    counts = np.full(n, 50000, np.uint32)
    C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts)
    prob.with_gradient = 0  # forward-only sizing: one partial per work item
    small = B.qmc_integrate_workspace_bytes(prob, n, np.full(n, 100, np.uint32))
    ws = torch.zeros(small, dtype=torch.uint8, device="cuda")
    est = torch.zeros(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, dev["counts"], dev["theta"], est, ws)
    torch.cuda.synchronize()
    assert B.qmc_read_device_error(ws) == 1
    assert torch.isnan(est).all()


def test_config5_fwd_bwd_small(B, oracle):
    """Config 5 (reduced): 512 pixels x 4096 samples; fused forward+backward and the
    unfused forward + backward against the oracle's estimate and its analytic
    gradient on the same points."""
    n = 512
    counts = np.full(n, 4096, np.uint32)
    C6, theta, seeds, dev, prob = _gaussmix_case(B, n, counts, seed=21)
    target = inputs.gaussmix_target(inputs.gaussmix_theta(n, seed=22))
    tg = torch.from_numpy(target).cuda()
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    gth = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    B.qmc_integrate_fwd_bwd(prob, n, dev["counts"], dev["theta"], tg, est, gth, loss, ws)
    torch.cuda.synchronize()
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    e = est.cpu().numpy()
    assert (np.abs(e - ref["est"]) <= est_tol(ref["est"], W)).all()
    r = ref["est"] - target
    assert loss.item() == pytest.approx(float((r * r).sum()), rel=1e-5)
    g_ref = 2.0 * r[:, None] * ref["grad"]
    # d(2 (I - T) J) = 2 dI J + 2 (I - T) dJ: the estimate's own tolerance enters through dI
    e_tol = est_tol(ref["est"], W)
    g_tol = 2.0 * (e_tol[:, None] * np.abs(ref["grad"])
                   + np.abs(r)[:, None] * grad_tol(theta, ref["grad"], ref["grad_scale"]))
    g = gth.cpu().numpy()
    assert (np.abs(g - g_ref) <= g_tol).all(), np.max(np.abs(g - g_ref) / g_tol)
    # unfused backward with an upstream gradient of 2 (I - T)
    ge = torch.from_numpy(2.0 * (e - target)).cuda()
    gb = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    B.qmc_integrate_backward(prob, n, dev["counts"], dev["theta"], ge, gb, ws)
    np.testing.assert_allclose(gb.cpu().numpy(), g, rtol=1e-6, atol=1e-30)

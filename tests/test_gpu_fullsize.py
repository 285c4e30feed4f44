"""Full-size workloads in the launch configuration the bench times (tuned work
split; the batched image as one CUDA graph), checked against the fp64 oracle
on sampled results (the oracle recomputes each sampled integral in full)."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _sample(n, k, counts, seed):
    rng = np.random.default_rng(seed)
    pix = rng.choice(n, k, replace=False)
    extra = [int(np.argmax(counts)), int(np.argmin(counts))]  # largest and smallest integral
    return np.unique(np.concatenate([pix, extra]))


def test_config4_full_image_graph(B, oracle):
    """1920x1080 integrals, log-uniform counts in [1, 65536] (1.2e10 samples)."""
    n = 1920 * 1080
    counts = inputs.log_uniform_counts(n)
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n, seed=7)
    seeds = inputs.pixel_seeds(n, 6, seed=7)
    d = {"C": B.u32_tensor(C6), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda(),
         "sd": B.u32_tensor(seeds)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws)
    est.fill_(-1.0)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        B.qmc_graph_begin(side)
        B.qmc_integrate(prob, n, d["c"], d["th"], est, ws, stream=side)
        graph = B.qmc_graph_end(side)
        B.qmc_graph_launch(graph, side)
    side.synchronize()
    B.qmc_graph_destroy(graph)
    B.qmc_tune_clear()
    assert B.qmc_read_device_error(ws) == 0
    e = est.cpu().numpy()
    assert (e >= 0).all()  # every integral written (the mixture is non-negative)
    pix = _sample(n, 300, counts, 4)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix], C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds[pix])
    W = np.abs(theta[pix][:, 0::4]).sum(axis=1)
    assert (np.abs(e[pix] - ref["est"]) <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).all()


def test_config5_full_fwd_bwd(B, oracle):
    """1024x1024 integrals x 4096 samples, fused forward + backward of the squared loss."""
    n = 1 << 20
    counts = np.full(n, 4096, np.uint32)
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n)
    seeds = inputs.pixel_seeds(n, 6)
    target = inputs.gaussmix_target(inputs.gaussmix_theta(n, seed=inputs.DEFAULT_SEED + 1))
    d = {"C": B.u32_tensor(C6), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda(),
         "sd": B.u32_tensor(seeds), "tg": torch.from_numpy(target).cuda()}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True, with_gradient=True)
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    gth = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws, target=d["tg"], grad_theta=gth, loss=loss)
    B.qmc_integrate_fwd_bwd(prob, n, d["c"], d["th"], d["tg"], est, gth, loss, ws)
    torch.cuda.synchronize()
    B.qmc_tune_clear()
    e, g = est.cpu().numpy(), gth.cpu().numpy()
    # the loss is the fixed-order sum of the estimates' squared residuals
    assert loss.item() == pytest.approx(float(((e - target) ** 2).sum()), rel=1e-12)
    pix = _sample(n, 64, counts, 5)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix], C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds[pix], with_grad=True)
    W = np.abs(theta[pix][:, 0::4]).sum(axis=1)
    tol_i = 1e-6 * np.abs(ref["est"]) + 1e-12 * W
    assert (np.abs(e[pix] - ref["est"]) <= tol_i).all()
    r = ref["est"] - target[pix]
    g_ref = 2 * r[:, None] * ref["grad"]
    g_tol = 2 * (tol_i[:, None] * np.abs(ref["grad"]) + 1e-5 * np.abs(r)[:, None] *
                 (np.abs(ref["grad"]) + ref["grad_mass"])) + 1e-12 * W[:, None]
    assert (np.abs(g[pix] - g_ref) <= g_tol).all()


def test_config3_full_lattice_genz(B, oracle):
    """Rank-1 lattice s = 16, 2^26 points, CP shift; the first parameter set of each
    Genz family against the oracle on all 2^26 points, all four against the exact
    integral (QMC error)."""
    s, N = 16, 1 << 26
    g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
    gd, shd = B.u32_tensor(g), B.u32_tensor(sh)
    for fam, kind, exact_fn in (("product_peak", B.F_GENZ_PRODUCT_PEAK, oracle.exact_genz_product_peak),
                                ("oscillatory", B.F_GENZ_OSCILLATORY, oracle.exact_genz_oscillatory)):
        theta = np.stack([inputs.genz_params(fam, s, k) for k in range(4)])
        counts = np.full(4, N, np.uint32)
        cd, thd = B.u32_tensor(counts), torch.from_numpy(theta).cuda()
        prob = B.make_problem(B.SOURCE_LATTICE, kind, s, 0, g=gd, seeds=shd)
        ws = B.alloc_workspace(prob, 4, counts)
        est = torch.empty(4, dtype=torch.float64, device="cuda")
        B.qmc_tune_integrate(prob, 4, cd, thd, est, ws)
        B.qmc_integrate(prob, 4, cd, thd, est, ws)
        e = est.cpu().numpy()
        exact = np.array([exact_fn(t, s) for t in theta])
        assert (np.abs(e - exact) <= 5e-3 * np.abs(exact)).all()
        ref = oracle.integrate(oracle.SOURCE_LATTICE, kind, s, counts[:1], theta[:1], g=g, seeds=sh)
        assert abs(e[0] - ref["est"][0]) <= 1e-6 * abs(ref["est"][0]) + 1e-12
    B.qmc_tune_clear()

"""Full-size integration workloads in the launch configuration the bench times
(tuned work split; the batched image as one CUDA graph), every result against
the fp64 oracle on the same points: all 2,073,600 estimates of the 1920x1080
batch, all 2^20 estimates and 16 x 2^20 gradients of the 1024x1024 fused
forward+backward, and all eight lattice Genz integrals of 2^26 samples.

Tolerances (per result; tests/tolerances.py): estimates 1e-6 relative + 1e-12 W;
gradient means J (a backward with an upstream gradient of 1) 1e-6 |J| for the
non-cancelling means (w, sigma) and 1e-6 (|J| + M) for the cancelling ones (mu, nu),
plus a floor for means that underflow in fp32; the fused dtheta = 2 (I - T) J
within the two errors combined, 2 (tol_I |J64| + |I64 - T| tol_J)."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs
from tolerances import est_tol, grad_tol, tau_needed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _rel_quantiles(err, ref):
    r = err / np.maximum(np.abs(ref), 1e-300)
    return {q: float(np.quantile(r, float(q))) for q in ("0.5", "0.99", "0.999", "1.0")}


def test_config4_full_image_graph(B, oracle, parity_report):
    """1920x1080 integrals, log-uniform counts in [1, 65536] (1.2e10 samples), one
    graph-captured launch; every estimate against the oracle."""
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
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)["est"]
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    err = np.abs(e - ref)
    tol = est_tol(ref, W)
    parity_report["config4_batched_1920x1080"] = {
        "results": n, "samples": int(counts.sum()), "est_rel_err": _rel_quantiles(err, ref),
        "max_err_over_tol": float((err / tol).max()), "results_within_floor_only": int((err > 1e-6 * np.abs(ref)).sum())}
    bad = err > tol
    assert not bad.any(), (np.flatnonzero(bad)[:8], (err / tol)[bad][:8])


def test_config5_full_fwd_bwd(B, oracle, parity_report):
    """1024x1024 integrals x 4096 samples: the fused forward + backward of the squared
    loss, and the gradient means J alone (backward with an upstream gradient of 1);
    every estimate and every gradient against the oracle."""
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
    e, g = est.cpu().numpy(), gth.cpu().numpy().astype(np.float64)
    gj = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    B.qmc_integrate_backward(prob, n, d["c"], d["th"], torch.ones(n, dtype=torch.float64, device="cuda"), gj, ws)
    torch.cuda.synchronize()
    B.qmc_tune_clear()
    J = gj.cpu().numpy().astype(np.float64)
    # the loss is the fixed-order sum of the estimates' squared residuals
    assert loss.item() == pytest.approx(float(((e - target) ** 2).sum()), rel=1e-12)
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    tol_i = est_tol(ref["est"], W)
    err_i = np.abs(e - ref["est"])
    tol_j = grad_tol(theta, ref["grad"], ref["grad_scale"])
    err_j = np.abs(J - ref["grad"])
    r = ref["est"] - target
    g_ref = 2 * r[:, None] * ref["grad"]
    tol_g = 2 * (tol_i[:, None] * np.abs(ref["grad"]) + np.abs(r)[:, None] * tol_j)
    err_g = np.abs(g - g_ref)
    kinds = {"w": 0, "mu": 1, "nu": 2, "sigma": 3}
    parity_report["config5_fwd_bwd_1024x1024"] = {
        "results": n, "samples": int(counts.sum()), "est_rel_err": _rel_quantiles(err_i, ref["est"]),
        "est_max_err_over_tol": float((err_i / tol_i).max()),
        "grad_mean_rel_err": {k: _rel_quantiles(err_j[:, v::4], ref["grad"][:, v::4]) for k, v in kinds.items()},
        "grad_mean_err_over_J_plus_S": {k: float((err_j[:, v::4] / (np.abs(ref["grad"][:, v::4]) +
                                                                    ref["grad_scale"][:, v::4])).max())
                                        for k, v in kinds.items()},
        "grad_mean_max_err_over_tol": float((err_j / tol_j).max()),
        "grad_mean_tau_needed": tau_needed(theta, J, ref["grad"], ref["grad_scale"]),
        "dtheta_rel_err": _rel_quantiles(err_g, g_ref), "dtheta_max_err_over_tol": float((err_g / tol_g).max())}
    assert (err_i <= tol_i).all(), np.flatnonzero(err_i > tol_i)[:8]
    bad = err_j > tol_j
    assert not bad.any(), (np.argwhere(bad)[:8], (err_j / tol_j)[bad][:8])
    assert (err_g <= tol_g).all(), np.argwhere(err_g > tol_g)[:8]


def test_config3_full_lattice_genz(B, oracle, parity_report):
    """Rank-1 lattice s = 16, 2^26 points, CP shift; all four parameter sets of each
    Genz family against the oracle on all 2^26 points, and against the exact
    integral (the QMC error)."""
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
        ref = oracle.integrate(oracle.SOURCE_LATTICE, kind, s, counts, theta, g=g, seeds=sh)["est"]
        err = np.abs(e - ref)
        parity_report[f"config3_lattice_{fam}"] = {
            "results": 4, "samples_each": N, "est_rel_err": [float(v) for v in err / np.abs(ref)],
            "rel_err_vs_exact": [float(v) for v in np.abs(e - exact) / np.abs(exact)]}
        assert (err <= est_tol(ref, 1.0)).all(), (err, ref)
    B.qmc_tune_clear()

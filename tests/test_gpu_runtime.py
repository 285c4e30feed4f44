"""GPU tests of the runtime around the kernels: the torch.autograd Function over
the hand-written adjoint, the work-split autotuner and CUDA-graph capture."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs
from tolerances import grad_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _mixture(B, n, counts, seed):
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n, seed=seed)
    seeds = inputs.pixel_seeds(n, 6, seed=seed)
    return C6, theta, seeds


def test_autograd_backward_matches_fused_and_oracle(B, oracle):
    """loss = sum (I(theta) - T)^2 through QMCIntegrate: backward recomputes the
    points in the adjoint kernel; the gradient equals the fused forward+backward
    and the oracle's analytic-on-points gradient."""
    from paper_2307_15584_gb300.autograd import GaussMixIntegrator

    n = 300
    counts = inputs.log_uniform_counts(n, hi=8192, seed=51)
    C6, theta, seeds = _mixture(B, n, counts, 51)
    target = inputs.gaussmix_target(inputs.gaussmix_theta(n, seed=52))
    integ = GaussMixIntegrator(C6, counts, seeds)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    tg = torch.from_numpy(target).cuda()
    est = integ(th)
    loss = ((est - tg) ** 2).sum()
    loss.backward()
    g_auto = th.grad.cpu().numpy()

    est_f = torch.empty(n, dtype=torch.float64, device="cuda")
    g_f = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    loss_f = torch.empty(1, dtype=torch.float64, device="cuda")
    B.qmc_integrate_fwd_bwd(integ.problem, n, integ.counts, th.detach(), tg, est_f, g_f, loss_f, integ.workspace)
    np.testing.assert_array_equal(est.detach().cpu().numpy(), est_f.cpu().numpy())
    np.testing.assert_allclose(g_auto, g_f.cpu().numpy(), rtol=1e-6, atol=0)
    assert loss.item() == pytest.approx(loss_f.item(), rel=1e-12)

    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    tol_i = 1e-6 * np.abs(ref["est"]) + 1e-12 * W
    r = ref["est"] - target
    g_ref = 2 * r[:, None] * ref["grad"]
    g_tol = 2 * (tol_i[:, None] * np.abs(ref["grad"]) +
                 np.abs(r)[:, None] * grad_tol(theta, ref["grad"], ref["grad_scale"], tau=2e-6))
    assert (np.abs(g_auto - g_ref) <= g_tol).all()


def test_autograd_over_partition_elements(B, oracle):
    """The differentiable integral over elements of a partitioned 64-bit Sobol' sequence
    (Sec. 2.5.1): d(sum_p I_p)/dtheta through QMCIntegrate is the per-element gradient mean,
    against the oracle's analytic-on-points gradient of each element."""
    from paper_2307_15584_gb300.autograd import GaussMixIntegrator

    n, q = 24, 3
    counts = inputs.log_uniform_counts(n, hi=6000, seed=61)
    W7 = oracle.sobol_matrices_wide(7, 64, inputs.sobol_raw_init(7))
    theta = inputs.gaussmix_theta(n, seed=62)
    seeds = inputs.pixel_seeds(n, 6, seed=62)
    integ = GaussMixIntegrator(W7, counts, seeds, index_bits=64, partition_log2=q)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    est = integ(th)
    est.sum().backward()
    g = th.grad.cpu().numpy()
    ref = oracle.integrate_partitioned(oracle.F_GAUSSMIX4_6D, 6, counts, theta, W7, q, np.arange(n) % (1 << q),
                                       scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    assert (np.abs(est.detach().cpu().numpy() - ref["est"]) <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).all()
    g_tol = grad_tol(theta, ref["grad"], ref["grad_scale"], tau=2e-6)
    assert (np.abs(g - ref["grad"]) <= g_tol).all(), np.max(np.abs(g - ref["grad"]) / g_tol)
    with pytest.raises(ValueError):  # the element dimension must be there
        GaussMixIntegrator(W7[1:], counts, seeds, index_bits=64, partition_log2=q)


def test_autotuner_records_and_applies(B, oracle):
    n = 2000
    counts = inputs.log_uniform_counts(n, seed=61)
    C6, theta, seeds = _mixture(B, n, counts, 61)
    d = {"C": B.u32_tensor(C6), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda(),
         "sd": B.u32_tensor(seeds)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts)  # chunk 0: sized for every candidate
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_tune_clear()
    best = B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws)
    assert best.chunk in (1024, 2048, 4096, 8192) and best.block in (128, 256) and best.ms > 0
    # a call with chunk = block = 0 now uses the recorded split: bitwise equal to the explicit one
    e_auto = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, d["c"], d["th"], e_auto, ws)
    explicit = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"],
                              seeds=d["sd"], seeds_per_integral=True, chunk=best.chunk, block=best.block)
    e_exp = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(explicit, n, d["c"], d["th"], e_exp, ws)
    np.testing.assert_array_equal(e_auto.cpu().numpy(), e_exp.cpu().numpy())
    ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, theta, C=C6,
                           scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    assert (np.abs(e_auto.cpu().numpy() - ref["est"]) <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).all()
    B.qmc_tune_clear()


def test_graph_capture_replays_the_batch(B):
    """The whole batched integration (scan kernels, persistent kernel, reduction)
    recorded once and replayed: replays equal direct calls, also after the
    parameters change in place."""
    n = 1500
    counts = inputs.log_uniform_counts(n, seed=71)
    C6, theta, seeds = _mixture(B, n, counts, 71)
    d = {"C": B.u32_tensor(C6), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda(),
         "sd": B.u32_tensor(seeds)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts)
    est_direct = torch.empty(n, dtype=torch.float64, device="cuda")
    est_graph = torch.empty(n, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        B.qmc_graph_begin(side)
        B.qmc_integrate(prob, n, d["c"], d["th"], est_graph, ws, stream=side)
        graph = B.qmc_graph_end(side)
    try:
        for k in range(2):
            if k:
                d["th"].mul_(0.9)
            B.qmc_integrate(prob, n, d["c"], d["th"], est_direct, ws)
            torch.cuda.synchronize()
            with torch.cuda.stream(side):
                B.qmc_graph_launch(graph, side)
            side.synchronize()
            np.testing.assert_array_equal(est_graph.cpu().numpy(), est_direct.cpu().numpy())
    finally:
        B.qmc_graph_destroy(graph)


def test_autotune_cache_file_round_trip(B, tmp_path):
    """A tuning result saved to the cache file, forgotten, and loaded back applies
    again to the same problem class on this device (recorded under its name)."""
    import json

    n = 1000
    counts = inputs.log_uniform_counts(n, hi=8192, seed=81)
    C6, theta, seeds = _mixture(B, n, counts, 81)
    d = {"C": B.u32_tensor(C6), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda(),
         "sd": B.u32_tensor(seeds)}
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=d["C"], seeds=d["sd"],
                          seeds_per_integral=True)
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_tune_clear()
    best = B.qmc_tune_integrate(prob, n, d["c"], d["th"], est, ws)
    path = tmp_path / "tune.json"
    B.qmc_tune_save(str(path))
    entries = json.loads(path.read_text())["entries"]
    assert [e["device"] for e in entries] == [torch.cuda.get_device_name()]
    B.qmc_tune_clear()
    assert B.qmc_tune_lookup(prob, n).chunk == 0
    assert B.qmc_tune_load(str(path)) == 1
    hit = B.qmc_tune_lookup(prob, n)
    assert (hit.chunk, hit.block) == (best.chunk, best.block)
    B.qmc_tune_clear()


def test_autotune_cache_from_the_environment(tmp_path):
    """QMC_AUTOTUNE_CACHE: one process tunes and the file is written; a second
    process finds the record before tuning anything."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "env_tune.json"
    script = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2307_15584_gb300 import binding as B, inputs
n = 500
counts = inputs.log_uniform_counts(n, hi=4096, seed=82)
C = B.u32_tensor(B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6)))
sd = B.u32_tensor(inputs.pixel_seeds(n, 6, seed=82))
prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=C, seeds=sd,
                      seeds_per_integral=True)
if sys.argv[1] == "tune":
    th = torch.from_numpy(inputs.gaussmix_theta(n, seed=82)).cuda()
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    best = B.qmc_tune_integrate(prob, n, B.u32_tensor(counts), th, est, B.alloc_workspace(prob, n, counts))
else:
    best = B.qmc_tune_lookup(prob, n)
print(best.chunk, best.block)
""".format(root=root)
    env = dict(os.environ, QMC_AUTOTUNE_CACHE=str(path))
    run = lambda mode: subprocess.run([sys.executable, "-c", script, mode], env=env, capture_output=True, text=True,
                                      timeout=300)
    a = run("tune")
    assert a.returncode == 0, a.stderr
    assert path.exists()
    b = run("lookup")
    assert b.returncode == 0, b.stderr
    assert a.stdout.split() == b.stdout.split() and a.stdout.split()[0] != "0"


def test_injected_launch_fault_leaves_the_context_usable(B, oracle, monkeypatch):
    """QMC_FAULT_INJECT=launch on a GPU: the call fails on the host with QMC_ERR_CUDA,
    nothing runs (the output keeps its sentinel), and the next call without the
    variable runs normally on the same context."""
    s, n = 8, 4096
    C = B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s))
    seeds = inputs.scramble_seeds(s)
    Cd, sd = B.u32_tensor(C), B.u32_tensor(seeds)
    u = torch.full((n, s), -7, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("QMC_FAULT_INJECT", "launch")
    with pytest.raises(B.QMCError) as e:
        B.qmc_sobol_points(Cd, s, 0, n, B.SCRAMBLE_NESTED_XOR, sd, u, None)
    assert e.value.status == 4 and B.qmc_last_cuda_error() == B.QMC_INJECTED_FAULT
    torch.cuda.synchronize()
    assert (u == -7).all()
    monkeypatch.delenv("QMC_FAULT_INJECT")
    B.qmc_sobol_points(Cd, s, 0, n, B.SCRAMBLE_NESTED_XOR, sd, u, None)
    ou, _ = oracle.sobol_points(C, 0, n, oracle.SCRAMBLE_NESTED_XOR, seeds)
    np.testing.assert_array_equal(B.as_u32(u), ou)

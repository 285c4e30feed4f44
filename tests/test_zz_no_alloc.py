"""qmc_integrate_static: batched integration for callers that cannot allocate
device memory (a plug-in inside an application that owns the GPU's memory, a
frame loop that cannot afford cudaMalloc's synchronisation, a fixed memory
budget).  It must give the same estimates as qmc_integrate with a caller
workspace, call after call, although every call reuses one fixed device array.

This file sorts last so that a run stopping at its first failure has already
run every other test; it also passes when run on its own in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu


def _tol(ref, W):
    # the tolerance of the integration tests: 1e-6 relative plus 1e-12 W
    return 1e-6 * np.abs(ref) + 1e-12 * W


def test_static_startup_call_places_the_array():
    """A caller that cannot allocate later makes one call with no integrals at
    start-up: it places the library's array on the device and looks up its
    address, reads no other pointer and enqueues nothing."""
    from paper_2307_15584_gb300 import binding as B

    C6 = B.u32_tensor(B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6)))
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, 0, matrices=C6, max_count=4096)
    torch.cuda.synchronize()
    B.qmc_integrate_static(prob, 0, None, None, None)
    B.qmc_integrate_static(prob, 0, None, None, None)  # and again: the address is kept
    torch.cuda.synchronize()


def test_static_matches_workspace_entry_point_twice():
    from paper_2307_15584_gb300 import binding as B

    n, max_count = 700, 4096
    counts = inputs.log_uniform_counts(n, hi=max_count, seed=41)
    counts[:3] = [0, 1, max_count]
    C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6))
    theta = inputs.gaussmix_theta(n, seed=41)
    seeds = inputs.pixel_seeds(n, 6, seed=41)
    Cd, cd, sd = B.u32_tensor(C6), B.u32_tensor(counts), B.u32_tensor(seeds)
    thd = torch.from_numpy(theta).cuda()
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=Cd, seeds=sd,
                          seeds_per_integral=True, max_count=max_count)

    ws = B.alloc_workspace(prob, n, counts)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, cd, thd, ref, ws)
    ref = ref.cpu().numpy()
    W = np.abs(theta[:, 0::4]).sum(axis=1)

    for _ in range(2):  # the array keeps the previous call's contents
        est = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        B.qmc_integrate_static(prob, n, cd, thd, est)
        e = est.cpu().numpy()
        assert np.all(np.abs(e - ref) <= _tol(ref, W))
        assert e[0] == 0.0

    # a bilinear problem through the same array right after
    C2 = B.qmc_sobol_matrices(2, inputs.sobol_raw_init(2))
    c2 = np.array([1 << 12, 37, 5000], np.uint32)
    p2 = B.make_problem(B.SOURCE_SOBOL, B.F_BILINEAR2D, 2, 0, matrices=B.u32_tensor(C2), max_count=1 << 13)
    ref2 = torch.empty(3, dtype=torch.float64, device="cuda")
    B.qmc_integrate(p2, 3, B.u32_tensor(c2), None, ref2, B.alloc_workspace(p2, 3, c2))
    est2 = torch.empty(3, dtype=torch.float64, device="cuda")
    B.qmc_integrate_static(p2, 3, B.u32_tensor(c2), None, est2)
    r2 = ref2.cpu().numpy()
    assert np.all(np.abs(est2.cpu().numpy() - r2) <= _tol(r2, 1.0))


def test_static_rejects_sizes_beyond_its_array():
    from paper_2307_15584_gb300 import binding as B

    C6 = B.u32_tensor(B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6)))
    n = 1 << 20  # a million integrals of up to 65536 samples cannot fit 16 MiB
    prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, 0, matrices=C6, max_count=65536)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(B.QMCError) as exc:
        B.qmc_integrate_static(prob, n, dummy, dummy, dummy)
    assert exc.value.status == 7  # QMC_ERR_WORKSPACE
    prob0 = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, 0, matrices=C6, max_count=0)
    with pytest.raises(B.QMCError) as exc:
        B.qmc_integrate_static(prob0, 4, dummy, dummy, dummy)
    assert exc.value.status == 1  # QMC_ERR_INVALID_ARG: no bound on the counts

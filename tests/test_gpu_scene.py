"""GPU parity of the procedural scene integrand (the Fig. 1 substitute) under
each per-pixel point source: estimates against the oracle on the same points.
The fp32 checker and occlusion decisions are reproduced bit for bit, so the
estimates agree to the shading's rounding."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu

SEED = 20230728


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


def _source(B, oracle, name, W, n):
    """(problem, device tensors kept alive, oracle kwargs) for one point source."""
    F = B.F_SCENE4D
    if name == "sobol_nested":
        C = B.qmc_sobol_matrices(4, inputs.sobol_raw_init(4))
        sd = inputs.pixel_seeds(n, 4)
        keep = (B.u32_tensor(C), B.u32_tensor(sd))
        prob = B.make_problem(B.SOURCE_SOBOL, F, 4, B.SCRAMBLE_NESTED, matrices=keep[0], seeds=keep[1],
                              seeds_per_integral=True)
        return prob, keep, dict(source=oracle.SOURCE_SOBOL, C=C, scramble=oracle.SCRAMBLE_NESTED, seeds=sd)
    if name == "pixel_lattice":
        g = inputs.lattice_generator(4, seed=5)
        keep = (B.u32_tensor(g),)
        prob = B.make_problem(B.SOURCE_PIXEL_LATTICE, F, 4, 0, g=keep[0], image_width=W)
        return prob, keep, dict(source=oracle.SOURCE_PIXEL_LATTICE, g=g)
    kind, R = {"random_hash_x4": (0, 4), "random_lfsr_x1": (1, 1)}[name]
    keep = (B.u32_tensor(np.array([SEED], np.uint32)),)
    prob = B.make_problem(B.SOURCE_RANDOM_LATTICE, F, 4, B.rlat_randomize(kind, R), seeds=keep[0], image_width=W)
    return prob, keep, dict(source=oracle.SOURCE_RANDOM_LATTICE, scramble=kind + 256 * R)


def _oracle_seeds(oracle, name, kw, W, H, pix):
    if name == "sobol_nested":
        return kw["seeds"][pix]
    if name == "pixel_lattice":
        k = oracle.grid_log2(W, H)
        return np.array([[oracle.pixel_shift(int(p) % W, int(p) // W, k)] for p in pix], np.uint32)
    return oracle.random_lattice_seeds(SEED, W, W * H)[pix]


@pytest.mark.parametrize("name", ["sobol_nested", "pixel_lattice", "random_hash_x4", "random_lfsr_x1"])
@pytest.mark.parametrize("W,H", [(64, 36), (1920, 1080)])
def test_scene_integration(B, oracle, name, W, H):
    n = W * H
    counts = inputs.log_uniform_counts(n, hi=4096, seed=17)
    theta = inputs.scene_theta(W, H)
    prob, keep, kw = _source(B, oracle, name, W, n)
    cd, thd = B.u32_tensor(counts), torch.from_numpy(theta).cuda()
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, cd, thd, est, ws)
    e = est.cpu().numpy()
    pix = np.arange(n) if n <= 4096 else np.unique(np.random.default_rng(9).choice(n, 300, replace=False))
    okw = {k: v for k, v in kw.items() if k != "seeds"}
    ref = oracle.integrate(integrand=oracle.F_SCENE4D, s=4, counts=counts[pix], theta=theta[pix],
                           seeds=_oracle_seeds(oracle, name, kw, W, H, pix), **okw)
    scale = 0.3 ** 2 / 1.0 ** 2  # Le side^2 / h^2: the largest f / albedo
    tol = 1e-6 * np.abs(ref["est"]) + 1e-12 * scale
    bad = np.abs(e[pix] - ref["est"]) > tol
    assert not bad.any(), (pix[bad][:5], e[pix][bad][:5], ref["est"][bad][:5])
    # the image has lit, shadowed and penumbra pixels
    assert (ref["est"] == 0).sum() < pix.size and ref["est"].max() > 0


def test_scene_argument_checks(B):
    theta = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    for s in (3, 6):
        prob = B.make_problem(B.SOURCE_RANDOM_LATTICE, B.F_SCENE4D, s, B.rlat_randomize(0, 1),
                              seeds=B.u32_tensor(np.array([1], np.uint32)), image_width=2)
        assert B.qmc_integrate_workspace_bytes(prob, 4, None) == 0

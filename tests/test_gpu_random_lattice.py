"""GPU parity of the per-pixel random rank-1 lattices (Alg. 4, Sec. 2.4.2,
Sec. 3): materialised samples bit-exact for both generator kinds and several
superimposed instance counts, and the fused integration source (forward and
forward+backward) against the oracle on the same points."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs
from tolerances import grad_tol

pytestmark = pytest.mark.gpu

SEED = 20230728


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("R", [1, 4, 16])
@pytest.mark.parametrize("width,height,spp,s,begin,n", [
    (37, 23, 17, 6, 0, 37 * 23),          # s % 4 != 0: chunks straddle rows and pixels
    (64, 64, 5, 3, 100, 700),
    (1920, 1080, 16, 2, 12345, 1000),     # 2-D per-pixel sampling
    (333, 77, 7, 1, 3, 2000),
    (64, 48, 9, 5, 1, 64 * 48 - 1),
    (100, 70, 16, 32, 1234, 3001),        # coalesced path, ragged pixel batches
    (37, 23, 1, 4, 5, 37 * 23 - 5),       # spp = 1
    (1920, 1080, 4, 12, 1920 * 1080 - 4099, 4099),
])
def test_random_lattice_points_bit_exact(B, oracle, kind, R, width, height, spp, s, begin, n):
    u = torch.empty((n * spp, s), dtype=torch.int32, device="cuda")
    f = torch.empty((n * spp, s), dtype=torch.float32, device="cuda")
    B.qmc_random_lattice_points(kind, SEED, R, s, width, height, begin, n, spp, u, f)
    ref = oracle.random_lattice_points(kind, SEED, R, s, width, n, spp, pixel_begin=begin)
    np.testing.assert_array_equal(B.as_u32(u), ref)
    np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32),
                                  oracle.map_u32_to_unifloat(ref).view(np.uint32))


def test_random_lattice_points_fullsize_sampled(B, oracle):
    """2^20 pixels x 16 samples x 32 dimensions in the bench's launch configuration:
    sampled pixels against the oracle, every instance a Latin hypercube."""
    width, height, spp, s, R = 1024, 1024, 16, 32, 4
    n = width * height
    u = torch.empty((n * spp, s), dtype=torch.int32, device="cuda")
    B.qmc_random_lattice_points(0, SEED, R, s, width, height, 0, n, spp, u, None)
    torch.cuda.synchronize()
    rng = np.random.default_rng(8)
    for q in np.unique(np.concatenate([rng.integers(0, n, 40), [0, n - 1]])).tolist():
        ref = oracle.random_lattice_points(0, SEED, R, s, width, 1, spp, pixel_begin=q)
        np.testing.assert_array_equal(B.as_u32(u[q * spp:(q + 1) * spp]), ref)
    # 4 samples per instance: the top 2 bits of every dimension of every instance
    # of every pixel are a permutation of 0..3
    top = ((u.view(n, spp // R, R, s).to(torch.int64) & 0xFFFFFFFF) >> 30).sort(dim=1).values
    assert torch.equal(top, torch.arange(4, device="cuda").view(1, 4, 1, 1).expand_as(top))


def _rlat_problem(B, kind, R, width, n, seed=SEED):
    seed_d = B.u32_tensor(np.array([seed], np.uint32))
    prob = B.make_problem(B.SOURCE_RANDOM_LATTICE, B.F_GAUSSMIX4_6D, 6, B.rlat_randomize(kind, R), seeds=seed_d,
                          image_width=width)
    return prob, seed_d


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("R", [1, 4])
@pytest.mark.parametrize("width,height", [(48, 32), (1920, 1080)])
def test_random_lattice_integration(B, oracle, kind, R, width, height):
    """A Gaussian-mixture image integrated per pixel, each pixel with its own
    random lattice(s); every pixel of the small image, sampled pixels of 1080p."""
    n = width * height
    counts = inputs.log_uniform_counts(n, hi=4096, seed=91)
    theta = inputs.gaussmix_theta(n, seed=91)
    prob, _ = _rlat_problem(B, kind, R, width, n)
    cd, thd = B.u32_tensor(counts), torch.from_numpy(theta).cuda()
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, cd, thd, est, ws)
    e = est.cpu().numpy()
    pix = np.arange(n) if n <= 4096 else np.unique(np.random.default_rng(3).choice(n, 300, replace=False))
    seeds = oracle.random_lattice_seeds(SEED, width, n)[pix]
    ref = oracle.integrate(oracle.SOURCE_RANDOM_LATTICE, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix],
                           scramble=kind + 256 * R, seeds=seeds)
    W = np.abs(theta[pix][:, 0::4]).sum(axis=1)
    assert (np.abs(e[pix] - ref["est"]) <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).all()


@pytest.mark.parametrize("kind", [0, 1])
def test_random_lattice_fwd_bwd(B, oracle, kind):
    """The fused forward+backward with the random-lattice source: loss and
    analytic gradient against the oracle on the same points."""
    width, n, R = 32, 512, 4
    counts = np.full(n, 4096, np.uint32)
    theta = inputs.gaussmix_theta(n, seed=31)
    target = inputs.gaussmix_target(inputs.gaussmix_theta(n, seed=32))
    prob, _ = _rlat_problem(B, kind, R, width, n)
    prob.with_gradient = 1
    cd, thd, tg = B.u32_tensor(counts), torch.from_numpy(theta).cuda(), torch.from_numpy(target).cuda()
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    gth = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    B.qmc_integrate_fwd_bwd(prob, n, cd, thd, tg, est, gth, loss, ws)
    torch.cuda.synchronize()
    ref = oracle.integrate(oracle.SOURCE_RANDOM_LATTICE, oracle.F_GAUSSMIX4_6D, 6, counts, theta,
                           scramble=kind + 256 * R, seeds=oracle.random_lattice_seeds(SEED, width, n),
                           with_grad=True)
    W = np.abs(theta[:, 0::4]).sum(axis=1)
    e = est.cpu().numpy()
    e_tol = 1e-6 * np.abs(ref["est"]) + 1e-12 * W
    assert (np.abs(e - ref["est"]) <= e_tol).all()
    r = ref["est"] - target
    assert loss.item() == pytest.approx(float((r * r).sum()), rel=1e-5)
    g_ref = 2.0 * r[:, None] * ref["grad"]
    g_tol = 2.0 * (e_tol[:, None] * np.abs(ref["grad"])
                   + np.abs(r)[:, None] * grad_tol(theta, ref["grad"], ref["grad_scale"]))
    assert (np.abs(gth.cpu().numpy() - g_ref) <= g_tol).all()

"""GPU parity of the pixel-shifted rank-1 lattice (Sec. 3, Eq. (PixelShiftedR1LS)):
materialised samples bit-exact, and the fused integration source against the
oracle on the same points."""
import numpy as np
import pytest
import torch

from paper_2307_15584_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


@pytest.mark.parametrize("width,height,spp,s,begin,n", [(37, 23, 17, 6, 0, 37 * 23), (64, 64, 5, 3, 100, 700),
                                                      (1920, 1080, 2, 16, 1920 * 1080 - 300, 300),
                                                      # coalesced path (s % 4 == 0): ragged batches, spp = 1
                                                      (37, 23, 1, 4, 5, 37 * 23 - 5), (100, 70, 16, 32, 1234, 3001),
                                                      (256, 256, 3, 8, 0, 65536), (1920, 1080, 4, 12, 777, 4099),
                                                      # coalesced path, s % 4 != 0: chunks straddle rows and
                                                      # pixels, ragged batch ends
                                                      (1920, 1080, 16, 2, 12345, 1000), (333, 77, 7, 1, 3, 333 * 70),
                                                      (64, 48, 9, 5, 1, 64 * 48 - 1), (128, 128, 1, 7, 0, 5000)])
def test_pixel_lattice_points_bit_exact(B, oracle, width, height, spp, s, begin, n):
    g = inputs.lattice_generator(s, seed=13)
    u = torch.empty((n * spp, s), dtype=torch.int32, device="cuda")
    f = torch.empty((n * spp, s), dtype=torch.float32, device="cuda")
    B.qmc_pixel_lattice_points(B.u32_tensor(g), s, width, height, begin, n, spp, u, f)
    ref = oracle.pixel_lattice_points(g, width, n, spp, pixel_begin=begin, height=height)
    np.testing.assert_array_equal(B.as_u32(u), ref)
    np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32),
                                  oracle.map_u32_to_unifloat(ref).view(np.uint32))


def test_pixel_lattice_points_errors(B):
    g = B.u32_tensor(inputs.lattice_generator(4))
    out = torch.empty(64, dtype=torch.int32, device="cuda")
    with pytest.raises(B.QMCError) as e:
        B.qmc_pixel_lattice_points(g, 4, 8, 8, 60, 5, 1, out, None)  # pixels beyond the image
    assert e.value.status == 2
    with pytest.raises(B.QMCError):
        B.qmc_pixel_lattice_points(g, 4, 0, 8, 0, 1, 1, out, None)
    B.qmc_pixel_lattice_points(g, 4, 8, 8, 64, 0, 1, out, None)  # empty range: no-op


@pytest.mark.parametrize("width,height", [(48, 32), (1920, 1080)])
def test_pixel_lattice_integration(B, oracle, width, height):
    """A Gaussian-mixture image integrated per pixel with the pixel-shifted lattice
    (one generator vector, one shift per pixel); sampled pixels for the full image."""
    n = width * height
    counts = inputs.log_uniform_counts(n, hi=4096, seed=81)
    theta = inputs.gaussmix_theta(n, seed=81)
    g = inputs.lattice_generator(6, seed=81)
    d = {"g": B.u32_tensor(g), "c": B.u32_tensor(counts), "th": torch.from_numpy(theta).cuda()}
    prob = B.make_problem(B.SOURCE_PIXEL_LATTICE, B.F_GAUSSMIX4_6D, 6, 0, g=d["g"], image_width=width)
    ws = B.alloc_workspace(prob, n, counts)
    est = torch.empty(n, dtype=torch.float64, device="cuda")
    B.qmc_integrate(prob, n, d["c"], d["th"], est, ws)
    e = est.cpu().numpy()
    pix = np.arange(n) if n <= 4096 else np.unique(np.random.default_rng(3).choice(n, 400, replace=False))
    k = oracle.grid_log2(width, height)
    shifts = np.array([[oracle.pixel_shift(int(p) % width, int(p) // width, k)] for p in pix], np.uint32)
    ref = oracle.integrate(oracle.SOURCE_PIXEL_LATTICE, oracle.F_GAUSSMIX4_6D, 6, counts[pix], theta[pix], g=g,
                           seeds=shifts)
    W = np.abs(theta[pix][:, 0::4]).sum(axis=1)
    assert (np.abs(e[pix] - ref["est"]) <= 1e-6 * np.abs(ref["est"]) + 1e-12 * W).all()

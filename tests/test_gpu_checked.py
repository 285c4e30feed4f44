"""The checked build (libqmc_gb300_checked.so: every store of a point kernel and
every per-item store of the integration kernels tested against the extent the
host validated).  Run in a child process with QMC_CHECKED=1 so the binding loads
that library: small cases of every generator and an integration, bit for bit (or
within the integration tolerance) against the oracle with a clear error word;
then QMC_CHECK_SLACK=k, which makes the kernels treat each output as k elements
shorter -- the last stores are skipped and reported, the buffers' tails keep their
sentinel, and nothing outside the buffers is touched."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
import numpy as np, torch
import oracle
from paper_2307_15584_gb300 import binding as B, inputs
from tolerances import est_tol
assert B.CHECKED and B.LIB_PATH.endswith("libqmc_gb300_checked.so")
B.qmc_checked_error(reset=True)
SENT = -0x5A5A5A5B

def fresh(n, s):
    return (torch.full((n, s), SENT, dtype=torch.int32, device="cuda"),
            torch.full((n, s), float("nan"), dtype=torch.float32, device="cuda"))

def same(u, f, ou, of, what):
    np.testing.assert_array_equal(B.as_u32(u), ou, err_msg=what)
    np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32), of.view(np.uint32), err_msg=what)

s, n = 32, 4096 + 37
C = B.qmc_sobol_matrices(s, inputs.sobol_raw_init(s)); Cd = B.u32_tensor(C)
sd = inputs.scramble_seeds(s); sdd = B.u32_tensor(sd)
for begin, mode in ((0, 2), (1, 3), (4096, 1)):  # the 16-byte path, on and off its group grid
    u, f = fresh(n, s)
    B.qmc_sobol_points(Cd, s, begin, n, mode, sdd, u, f)
    same(u, f, *oracle.sobol_points(C, begin, n, mode, sd), f"sobol {begin} {mode}")
C37 = B.qmc_sobol_matrices(37, inputs.sobol_raw_init(37))
for s2, begin, mode in ((40, 3, 2), (7, 1, 1)):  # the walking path: 32- and 8-wide chunks; 7-wide chunks
    C2, sd2 = np.ascontiguousarray(np.concatenate([C37, C37])[:s2]), inputs.scramble_seeds(s2)
    u, f = fresh(n, s2)
    B.qmc_sobol_points(B.u32_tensor(C2), s2, begin, n, mode, B.u32_tensor(sd2), u, f)
    same(u, f, *oracle.sobol_points(C2, begin, n, mode, sd2), f"sobol walk {s2}")
W = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1)); Wd = B.u32_tensor(W)
u, f = fresh(n, s); B.qmc_sobol_points_wide(B.u32_tensor(np.ascontiguousarray(W[:s])), 64, s, 1 << 40, n, 2, sdd, u, f)
same(u, f, *oracle.sobol_points_wide(W[:s], 1 << 40, n, 2, sd), "wide")
u, f = fresh(n, s); B.qmc_sobol_points_partitioned(Wd, 64, s, 3, 5, 1 << 20, n, 2, sdd, u, f)
same(u, f, *oracle.sobol_points_partitioned(W, 3, 5, 1 << 20, n, 2, sd), "partitioned")
g, sh = inputs.lattice_generator(s), inputs.lattice_shift(s)
for begin in (0, 7):  # grouped and flat lattice paths
    u, f = fresh(n, s); B.qmc_lattice_points(B.u32_tensor(g), B.u32_tensor(sh), s, begin, n, 0, u, f)
    same(u, f, *oracle.lattice_points(g, sh, begin, n), f"lattice {begin}")
u, f = fresh(512, s); B.qmc_halton_points(s, B.HALTON_FAURE, None, 0, 512, u, f)
np.testing.assert_array_equal(B.as_u32(u), oracle.halton_points(s, 0, 512, oracle.HALTON_FAURE))
u, f = fresh(n, 6); B.qmc_halton_points_partitioned(6, 0, None, 3, 5, 1 << 10, n, u, f)
np.testing.assert_array_equal(B.as_u32(u), oracle.halton_points_partitioned(6, 3, 5, 1 << 10, n))
u, f = fresh(64 * 16, s); B.qmc_pixel_lattice_points(B.u32_tensor(g), s, 16, 16, 0, 64, 16, u, f)
np.testing.assert_array_equal(B.as_u32(u), oracle.pixel_lattice_points(g, 16, 64, 16, height=16))
for kind in (0, 1):
    u, f = fresh(256 * 16, s); B.qmc_random_lattice_points(kind, 7, 4, s, 64, 64, 0, 256, 16, u, f)
    np.testing.assert_array_equal(B.as_u32(u), oracle.random_lattice_points(kind, 7, 4, s, 64, 256, 16))
npx = 300
counts = inputs.log_uniform_counts(npx, hi=4096, seed=5); counts[:2] = [0, 1]
C6 = B.qmc_sobol_matrices(6, inputs.sobol_raw_init(6)); th = inputs.gaussmix_theta(npx, seed=5)
ps = inputs.pixel_seeds(npx, 6, seed=5)
prob = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, B.SCRAMBLE_NESTED, matrices=B.u32_tensor(C6),
                      seeds=B.u32_tensor(ps), seeds_per_integral=True, with_gradient=True)
est = torch.empty(npx, dtype=torch.float64, device="cuda")
B.qmc_integrate(prob, npx, B.u32_tensor(counts), torch.from_numpy(th).cuda(), est, B.alloc_workspace(prob, npx, counts))
ref = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, counts, th, C=C6, scramble=2, seeds=ps)["est"]
assert (np.abs(est.cpu().numpy() - ref) <= est_tol(ref, np.abs(th[:, 0::4]).sum(axis=1))).all()
assert B.qmc_checked_error(reset=True) == 0, "in-range launches reported an error"

# the test hook: each output treated as 5 elements shorter
os.environ["QMC_CHECK_SLACK"] = "5"
u, f = fresh(n, s)
B.qmc_sobol_points(Cd, s, 0, n, 2, sdd, u, f)
bits = B.qmc_checked_error(reset=True)
assert bits == 1, bits
ou, of = oracle.sobol_points(C, 0, n, 2, sd)
gu, gf = B.as_u32(u).reshape(-1), f.cpu().numpy().view(np.uint32).reshape(-1)
limit = n * s - 5
assert (gu[limit:] == np.uint32(SENT & 0xFFFFFFFF)).all()  # the skipped stores left their sentinel
assert (gu[:limit - 4] == ou.reshape(-1)[:limit - 4]).all() and (gf[:limit - 4] == of.view(np.uint32).reshape(-1)[:limit - 4]).all()
u, f = fresh(512, s)
B.qmc_halton_points(s, 0, None, 0, 512, u, f)
assert B.qmc_checked_error(reset=True) == 1
gh = B.as_u32(u).reshape(-1)
assert (gh[512 * s - 5:] == np.uint32(SENT & 0xFFFFFFFF)).all()
# a 16-byte store that reaches past the shortened extent is skipped whole
assert (gh[:512 * s - 9] == oracle.halton_points(s, 0, 512).reshape(-1)[:512 * s - 9]).all()
C2, sd2 = np.ascontiguousarray(np.concatenate([C37, C37])[:40]), inputs.scramble_seeds(40)
u, f = fresh(n, 40)
B.qmc_sobol_points(B.u32_tensor(C2), 40, 0, n, 2, B.u32_tensor(sd2), u, f)  # the walking path
assert B.qmc_checked_error(reset=True) == 1
gw, ow = B.as_u32(u).reshape(-1), oracle.sobol_points(C2, 0, n, 2, sd2)[0].reshape(-1)
assert (gw[n * 40 - 5:] == np.uint32(SENT & 0xFFFFFFFF)).all() and (gw[:n * 40 - 9] == ow[:n * 40 - 9]).all()
del os.environ["QMC_CHECK_SLACK"]
u, f = fresh(n, s)
B.qmc_sobol_points(Cd, s, 0, n, 2, sdd, u, f)
assert B.qmc_checked_error() == 0
print("checked build ok")
""".replace("ROOT", repr(ROOT))


def test_checked_build_parity_and_reports():
    env = dict(os.environ, QMC_CHECKED="1")
    env.pop("QMC_CHECK_SLACK", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout

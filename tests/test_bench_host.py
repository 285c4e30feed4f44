"""Host-side helpers of bench.py: the closed-form integrals it reports errors
against agree with the oracle's (CPU only)."""
import numpy as np

import bench
from paper_2307_15584_gb300 import inputs


def test_genz_closed_forms_match_oracle(oracle):
    for fam, fn in (("product_peak", oracle.exact_genz_product_peak), ("oscillatory", oracle.exact_genz_oscillatory)):
        for k in range(4):
            for s in (1, 6, 16):
                t = inputs.genz_params(fam, s, k)
                assert abs(bench.genz_exact(fam, t, s) - fn(t, s)) <= 1e-12 * max(1.0, abs(fn(t, s)))


def test_mixture_closed_form_matches_oracle(oracle):
    theta = inputs.gaussmix_theta(64, seed=5)
    exact = inputs.gaussmix_target(theta)
    for p in range(64):
        assert abs(exact[p] - oracle.exact_gaussmix(theta[p])) <= 1e-12 * abs(exact[p])


def test_rms_rel_err():
    assert abs(bench.rms_rel_err(np.array([1.1, 0.9]), np.array([1.0, 1.0])) - 0.1) < 1e-15


def test_cpu_baselines_sit_beside_their_gpu_figures():
    import bench

    extras = {"fwd_bwd": {"fused_gsamples_s": 1.0}, "lattice": {"points": 4, "oscillatory": {"gsamples_s": 2.0}},
              "points": {"rows": 8, "halton_faure": {"gb_s": 3.0}}}
    base = {"fwd_bwd": {"value": 0.1}, "lattice": {"oscillatory": {"value": 0.2}, "product_peak": {"value": 0.3}},
            "points": {"halton_faure": {"value": 0.4}}}
    bench.attach_cpu_baselines(extras, base)
    assert extras["fwd_bwd"]["cpu_baseline"] == {"value": 0.1}
    assert extras["lattice"]["oscillatory"]["cpu_baseline"] == {"value": 0.2}
    assert "product_peak" not in extras["lattice"]  # no GPU figure to sit beside
    assert extras["points"]["halton_faure"]["cpu_baseline"] == {"value": 0.4}


def test_committed_profile_figures_match_the_sources():
    """Every figure in the digest-keyed profile tables was taken on the committed sources: a
    kernel edit without a re-capture shows up here (bench.py would report it as null)."""
    import os

    import bench
    from paper_2307_15584_gb300.build import source_digest

    for fname in ("traffic.txt", "inst_per_coord.txt", "inst_per_sample.txt"):
        path = os.path.join(bench.ROOT, "profiles", fname)
        for line in open(path):
            parts = line.split()
            if len(parts) != 3 or line.startswith("#"):
                continue
            key, digest, _ = parts
            assert source_digest(bench.profile_sources(fname, key)) == digest, (fname, key)

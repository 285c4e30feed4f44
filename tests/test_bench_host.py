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

    for fname in ("traffic.txt", "inst_per_coord.txt", "inst_per_sample.txt", "pipes.txt"):
        path = os.path.join(bench.ROOT, "profiles", fname)
        for line in open(path):
            parts = line.split("#", 1)[0].split()
            if len(parts) < 3:
                continue
            key, digest = parts[:2]
            assert source_digest(bench.profile_sources(fname, key)) == digest, (fname, key)


def test_gradient_errors_and_compact_summary():
    """The bench's error statement: relative errors of the non-cancelling gradient
    means, errors relative to |J| + M for the cancelling ones; and the summary the
    JSON line carries keeps every workload's rate and fractions."""
    import bench

    rng = np.random.default_rng(3)
    n = 8
    J64 = rng.uniform(0.1, 1.0, (n, 16))
    M64 = np.abs(J64) * 3
    ref = {"est": rng.uniform(0.5, 1.0, n), "grad": J64, "grad_scale": M64}
    gpu = {"est": ref["est"] * (1 + 1e-7), "J": (J64 * (1 + 2e-7)).astype(np.float32),
           "dtheta": np.zeros((n, 16), np.float32)}
    target = ref["est"] - 0.25
    gpu["dtheta"] = (2 * 0.25 * J64 * (1 + 3e-7)).astype(np.float32)
    e = bench.gradient_errors(gpu, ref, None, target)
    assert 0.9e-7 < e["est_max_rel"] < 1.1e-7
    assert e["J_w_max_rel"] < 3e-7 and e["J_sigma_max_rel"] < 3e-7
    assert e["J_mu_max_over_J_plus_S"] < 1e-7  # the error over 4 |J|
    assert e["dtheta_rel_quantiles"]["1.0"] < 5e-7
    roof = {"alg_frac": 0.61234, "frac": 0.8, "pipes": {"alu": 0.5, "fma": 0.6, "fmaheavy": 0.2, "xu": 0.1}}
    x = {"fwd_bwd": {"fused_gsamples_s": 142.0, "unfused_gsamples_s": 86.0, "roofline": roof,
                     "cpu_baseline": {"value": 0.03, "value_1core": 0.002}, "errors_vs_oracle": e},
         "batched": {"gsamples_s": 217.0, "roofline": roof},
         "lattice": {"points": 4, "product_peak": {"gsamples_s": 264.0, "roofline": roof},
                     "oscillatory": {"gsamples_s": 325.0, "roofline": roof}},
         "partition": {"gsamples_s": 118.0, "roofline": roof, "rel_err_vs_exact": 2.4e-7},
         "points": {"rows": 8, "sobol32_nested": {"gdims_s": 848.0, "frac_hbm": 1.01}}}
    c = bench.compact_extras(x)
    assert c["fwd_bwd"]["gsamples_s"] == 142.0 and c["fwd_bwd"]["alg_frac"] == 0.612
    assert c["fwd_bwd"]["oracle"] == [0.03, 0.002]
    assert set(c) == {"pipes_order", "oracle_order", "fwd_bwd", "batched", "lattice_product_peak",
                      "lattice_oscillatory", "partition", "points_gdims_s_frac_hbm"}
    assert c["fwd_bwd"]["pipes"] == [0.5, 0.6, 0.2, 0.1] and c["pipes_order"] == ["alu", "fma", "fmaheavy", "xu"]
    assert c["points_gdims_s_frac_hbm"] == {"sobol32_nested": [848.0, 1.0]}  # 2 significant digits


def test_digest_ignores_comments_only():
    """Profile figures are keyed by the code without its comments: a comment-only edit keeps the
    key, a code edit (even inside a line that also holds a comment) changes it; string literals
    that look like comments are code."""
    from paper_2307_15584_gb300.build import code_only

    base = 'int a = 1;  // one\n/* block\n comment */ const char* p = "x//y";\n\nint b;\n'
    assert code_only(base) == code_only(base.replace("// one", "// another").replace("block", "other"))
    assert code_only(base) != code_only(base.replace("int a = 1;", "int a = 2;"))
    assert '"x//y"' in code_only(base) and "one" not in code_only(base)

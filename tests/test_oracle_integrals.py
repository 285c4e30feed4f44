"""Pins of the oracle's integrands, closed forms, estimates and gradients
against numerical quadrature, finite differences and convergence.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate as spi

from paper_2307_15584_gb300 import inputs


@pytest.fixture(scope="module")
def C6(oracle):
    return oracle.sobol_matrices(6, inputs.sobol_raw_init(6))


def test_genz_product_peak_closed_form(oracle):
    """Sec. 2.6 test functions: the product peak integral factorises into 1-D quadratures."""
    for idx in range(3):
        s = 5
        th = inputs.genz_params("product_peak", s, idx)
        a, u = th[:s].astype(np.float64), th[s:].astype(np.float64)
        q = 1.0
        for j in range(s):
            q *= spi.quad(lambda x: 1.0 / (a[j] ** -2 + (x - u[j]) ** 2), 0, 1, epsabs=0, epsrel=1e-13)[0]
        assert oracle.exact_genz_product_peak(th, s) == pytest.approx(q, rel=1e-11)


def test_genz_oscillatory_closed_form(oracle):
    for idx in range(3):
        s = 2
        th = inputs.genz_params("oscillatory", s, idx)
        a, u = th[:s].astype(np.float64), th[s:].astype(np.float64)
        val = spi.dblquad(lambda y, x: math.cos(2 * math.pi * u[0] + a[0] * x + a[1] * y), 0, 1, 0, 1,
                          epsabs=1e-13, epsrel=1e-13)[0]
        assert oracle.exact_genz_oscillatory(th, s) == pytest.approx(val, rel=1e-9, abs=1e-12)
    # separable check in 16 dims via complex 1-D integrals
    s = 16
    th = inputs.genz_params("oscillatory", s, 7)
    a, u = th[:s].astype(np.float64), th[s:].astype(np.float64)
    z = complex(math.cos(2 * math.pi * u[0]), math.sin(2 * math.pi * u[0]))
    for j in range(s):
        re = spi.quad(lambda x: math.cos(a[j] * x), 0, 1, epsrel=1e-13)[0]
        im = spi.quad(lambda x: math.sin(a[j] * x), 0, 1, epsrel=1e-13)[0]
        z *= complex(re, im)
    assert oracle.exact_genz_oscillatory(th, s) == pytest.approx(z.real, rel=1e-10, abs=1e-13)


def test_gaussmix_closed_form_and_gradient(oracle):
    th = inputs.gaussmix_theta(4, seed=3).astype(np.float64)
    for t in th:
        val = 0.0
        for c in range(4):
            w, mu, nu, sg = t[4 * c: 4 * c + 4]
            gm = spi.quad(lambda x: math.exp(-(x - mu) ** 2 / (2 * sg * sg)), 0, 1, epsrel=1e-13)[0]
            gn = spi.quad(lambda x: math.exp(-(x - nu) ** 2 / (2 * sg * sg)), 0, 1, epsrel=1e-13)[0]
            val += w * gm**3 * gn**3
        I, grad = oracle.exact_gaussmix(t, with_grad=True)
        assert I == pytest.approx(val, rel=1e-11)
        h = 1e-6
        for k in range(16):
            tp, tm = t.copy(), t.copy()
            tp[k] += h
            tm[k] -= h
            fd = (oracle.exact_gaussmix(tp) - oracle.exact_gaussmix(tm)) / (2 * h)
            assert grad[k] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    # target image helper of the inputs module agrees with the oracle's closed form
    tgt = inputs.gaussmix_target(th.astype(np.float32))
    for p in range(4):
        assert tgt[p] == pytest.approx(oracle.exact_gaussmix(th[p].astype(np.float32).astype(np.float64)), rel=1e-12)


def test_bilinear_estimate_config1(oracle):
    """Config 1: the 2-D Sobol' estimate of the bilinear integrand tends to the exact value 1."""
    C = oracle.sobol_matrices(2, inputs.sobol_raw_init(2))
    errs = []
    for m in (4, 8, 12, 16):
        r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_BILINEAR2D, 2, [1 << m], np.zeros((1, 1)), C=C)
        errs.append(abs(r["est"][0] - 1.0))
    assert errs[-1] < 1e-5
    assert errs[0] > errs[-1]


def test_estimates_converge_to_closed_forms(oracle, C6):
    th = inputs.gaussmix_theta(3, seed=8)
    seeds = inputs.pixel_seeds(3, 6, seed=8)
    exact = np.array([oracle.exact_gaussmix(t.astype(np.float64)) for t in th])
    r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, [1 << 16] * 3, th, C=C6,
                         scramble=oracle.SCRAMBLE_NESTED, seeds=seeds)
    np.testing.assert_allclose(r["est"], exact, rtol=2e-2)
    s = 16
    g = inputs.lattice_generator(s)
    sh = inputs.lattice_shift(s)
    for fam, fn, kind in (("product_peak", oracle.exact_genz_product_peak, oracle.F_GENZ_PRODUCT_PEAK),
                          ("oscillatory", oracle.exact_genz_oscillatory, oracle.F_GENZ_OSCILLATORY)):
        t = inputs.genz_params(fam, s, 0)
        e = fn(t, s)
        r = oracle.integrate(oracle.SOURCE_LATTICE, kind, s, [1 << 16], t[None], g=g, seeds=sh)
        assert abs(r["est"][0] - e) < 5e-2 * abs(e) + 1e-3


def test_gradient_on_points_matches_central_differences(oracle, C6):
    """Config 5: the analytic per-sample gradient averaged over fixed points equals
    the central difference (h = 1e-3, fp64) of the estimate on the same points,
    up to the O(h^2) truncation of the difference quotient."""
    th = inputs.gaussmix_theta(2, seed=21)
    seeds = inputs.pixel_seeds(2, 6, seed=21)
    n = 512
    r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, [n, n], th, C=C6,
                         scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    for p in range(2):
        _, x = oracle.sobol_points(C6, 0, n, mode=oracle.SCRAMBLE_NESTED, seeds=seeds[p])
        x = x.astype(np.float64)
        base = th[p].astype(np.float64)

        def est(t):
            return sum(oracle.gaussmix_f64(x[i], t) for i in range(n)) / n

        assert r["est"][p] == pytest.approx(est(base), rel=1e-12)
        h = 1e-3
        for k in range(16):
            tp, tm = base.copy(), base.copy()
            tp[k] += h
            tm[k] -= h
            fd = (est(tp) - est(tm)) / (2 * h)
            scale = r["grad_mass"][p, k] + 1e-12
            assert abs(r["grad"][p, k] - fd) <= 2e-3 * scale, (p, k)


def test_gradient_term_scale(oracle, C6):
    """grad_scale (the tolerance scale of the cancelling gradient means) is the mean over
    samples of the summed absolute values of each derivative's terms: recomputed here
    from the oracle's own points with numpy, and >= mean |df/dtheta| >= |mean df/dtheta|,
    with equality to mean |df/dtheta| for w and sigma (terms of one sign)."""
    th = inputs.gaussmix_theta(3, seed=23)
    seeds = inputs.pixel_seeds(3, 6, seed=23)
    n = 300
    r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, [n] * 3, th, C=C6,
                         scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    for p in range(3):
        _, x = oracle.sobol_points(C6, 0, n, mode=oracle.SCRAMBLE_NESTED, seeds=seeds[p])
        x = x.astype(np.float64)
        t = th[p].astype(np.float64).reshape(4, 4)
        want = np.zeros(16)
        for c in range(4):
            w, mu, nu, sg = t[c]
            m = np.array([mu, nu, mu, nu, mu, nu])
            G = np.exp(-((x - m) ** 2).sum(1) / (2 * sg * sg))
            want[4 * c] = G.mean()
            want[4 * c + 1] = (abs(w) * G * np.abs(x[:, 0::2] - mu).sum(1)).mean() / sg**2
            want[4 * c + 2] = (abs(w) * G * np.abs(x[:, 1::2] - nu).sum(1)).mean() / sg**2
            want[4 * c + 3] = (abs(w) * G * ((x - m) ** 2).sum(1)).mean() / sg**3
        np.testing.assert_allclose(r["grad_scale"][p], want, rtol=1e-12)
    S, M, J = r["grad_scale"], r["grad_mass"], np.abs(r["grad"])
    assert (S >= M * (1 - 1e-15)).all() and (M >= J * (1 - 1e-15)).all()
    np.testing.assert_allclose(S[:, 0::4], M[:, 0::4], rtol=1e-14)
    np.testing.assert_allclose(S[:, 3::4], M[:, 3::4], rtol=1e-14)
    assert (S[:, 1::4] > M[:, 1::4] * 1.01).mean() > 0.5  # mostly, the differences inside a sample cancel


def test_gradient_tends_to_closed_form_gradient(oracle, C6):
    th = inputs.gaussmix_theta(1, seed=5)
    seeds = inputs.pixel_seeds(1, 6, seed=5)
    _, g_exact = oracle.exact_gaussmix(th[0].astype(np.float64), with_grad=True)
    r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, [1 << 16], th, C=C6,
                         scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=True)
    scale = np.abs(g_exact).max()
    assert np.abs(r["grad"][0] - g_exact).max() < 3e-2 * scale


def test_zero_count_and_argument_checks(oracle, C6):
    th = inputs.gaussmix_theta(1)
    r = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_GAUSSMIX4_6D, 6, [0], th, C=C6)
    assert r["est"][0] == 0.0
    with pytest.raises(ValueError):
        oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_BILINEAR2D, 3, [4], th, C=C6[:3])

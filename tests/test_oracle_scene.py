"""Pins of the oracle's procedural scene integrand (the Fig. 1 substitute):
the light-square integral against its closed form, the visibility and checker
decisions against fp64 geometry.  CPU only."""
import math

import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs


def _F(x, y, h):
    """Antiderivative of 1 / (x^2 + y^2 + h^2)^2 in x and y."""
    rx, ry = math.sqrt(x * x + h * h), math.sqrt(y * y + h * h)
    return (x / rx * math.atan(y / rx) + y / ry * math.atan(x / ry)) / (2 * h * h)


def _light_integral(px, py, th):
    """int over the light square of 1 / |L - P|^4 dL, L at height h."""
    cx, cy, h, side = (float(v) for v in th[4:8])
    xa, xb = cx - side / 2 - px, cx + side / 2 - px
    ya, yb = cy - side / 2 - py, cy + side / 2 - py
    return _F(xb, yb, h) - _F(xa, yb, h) - _F(xb, ya, h) + _F(xa, ya, h)


def test_closed_form_matches_quadrature():
    scipy = pytest.importorskip("scipy.integrate")
    th = inputs.scene_theta(8, 4)[5]
    px, py = 0.9, 0.2
    h = float(th[6])
    cx, cy, side = float(th[4]), float(th[5]), float(th[7])
    num, _ = scipy.dblquad(lambda b, a: 1.0 / ((a * a + b * b + h * h) ** 2),
                           cx - side / 2 - px, cx + side / 2 - px, cy - side / 2 - py, cy + side / 2 - py,
                           epsabs=0, epsrel=1e-11)
    assert _light_integral(px, py, th) == pytest.approx(num, rel=1e-9)


@pytest.mark.parametrize("pixel", [0, 37, 1234])
def test_unoccluded_uniform_estimate_matches_closed_form(oracle, pixel):
    """No occluder, one albedo (freq 0): the pixel's mean of
    0.2 Le side^2 h^2 / d^4 over footprint and light is 0.2 Le h^2 / (fw fh) times
    the footprint integral of the closed-form light integral."""
    scipy = pytest.importorskip("scipy.integrate")
    W, H = 64, 36
    th = inputs.scene_theta(W, H, freq=0.0, occluder=False)[pixel]
    fx, fy, fw, fh = (float(v) for v in th[:4])
    h, Le = float(th[6]), float(th[8])
    inner, _ = scipy.dblquad(lambda y, x: _light_integral(x, y, th), fx, fx + fw, fy, fy + fh,
                             epsabs=0, epsrel=1e-10)
    exact = 0.2 * Le * h * h * inner / (fw * fh)
    C = oracle.sobol_matrices(4, inputs.sobol_raw_init(4))
    est = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_SCENE4D, 4, np.array([1 << 16], np.uint32),
                           th[None, :], C=C)["est"][0]
    assert est == pytest.approx(exact, rel=2e-4)


def test_visibility_and_checker_decisions(oracle):
    """f is 0 exactly when the segment from the plane point to the light point
    meets the sphere, and otherwise carries albedo 0.8 or 0.2 by the parity of the
    checker cell; both checked in fp64 away from the boundaries."""
    W, H = 64, 36
    thetas = inputs.scene_theta(W, H)
    rng = np.random.default_rng(3)
    agree = blocked = 0
    for _ in range(4000):
        p = int(rng.integers(0, W * H))
        th = thetas[p]
        x = rng.random(4).astype(np.float32).astype(np.float64)
        f = oracle.integrand(oracle.F_SCENE4D, x, th, s=4)[0]
        P = np.array([th[0] + th[2] * x[0], th[1] + th[3] * x[1], 0.0])
        L = np.array([th[4] + th[7] * (x[2] - 0.5), th[5] + th[7] * (x[3] - 0.5), th[6]], np.float64)
        O, rho = np.array(th[9:12], np.float64), float(th[12])
        D = L - P
        t = np.clip(np.dot(O - P, D) / np.dot(D, D), 0.0, 1.0)
        dist = np.linalg.norm(P + t * D - O)
        if abs(dist - rho) < 1e-5:
            continue
        shadow = dist < rho
        blocked += shadow
        assert (f == 0.0) == shadow
        if not shadow:
            cell = (math.floor(P[0] * th[13]) + math.floor(P[1] * th[13])) & 1
            edge = min(abs(P[0] * th[13] - round(P[0] * th[13])), abs(P[1] * th[13] - round(P[1] * th[13])))
            if edge > 1e-5:
                d2 = float(np.dot(D, D))
                G = float(th[8]) * float(th[7]) ** 2 * float(th[6]) ** 2 / (d2 * d2)
                assert f / G == pytest.approx(0.8 if cell else 0.2, rel=1e-5)
        agree += 1
    assert agree > 3900 and 100 < blocked < agree - 100  # both outcomes occur

"""Pins of the oracle's integration over elements of a partitioned Sobol'
sequence (Sec. 2.5.1): the elements' points are disjoint pieces of one sequence,
so their estimates combine into the estimate over the whole.  CPU only."""
import numpy as np
import pytest

from paper_2307_15584_gb300 import inputs


@pytest.mark.parametrize("integrand,s", [("gaussmix", 6), ("osc", 8)])
@pytest.mark.parametrize("q", [1, 3])
def test_elements_combine_into_the_whole_sequence(oracle, integrand, s, q):
    """Equal counts n: the mean of the 2^q elements' estimates is the estimate
    over the first 2^q n points of dimensions 1..s (computed by the plain
    integration routine with the 32-column matrices), and the elements' gradient
    means combine the same way."""
    W = oracle.sobol_matrices_wide(s + 1, 64, inputs.sobol_raw_init(s + 1))
    seeds = inputs.scramble_seeds(s, seed=3)
    n, P = 640, 1 << q
    if integrand == "gaussmix":
        F, th = oracle.F_GAUSSMIX4_6D, inputs.gaussmix_theta(1, seed=4)[0]
    else:
        F, th = oracle.F_GENZ_OSCILLATORY, inputs.genz_params("oscillatory", s, 1)
    grad = integrand == "gaussmix"
    parts = oracle.integrate_partitioned(F, s, np.full(P, n, np.uint32), np.tile(th, (P, 1)), W, q, np.arange(P),
                                         scramble=oracle.SCRAMBLE_NESTED, seeds=seeds, with_grad=grad)
    whole = oracle.integrate(oracle.SOURCE_SOBOL, F, s, np.array([n * P], np.uint32), th[None, :],
                             C=np.ascontiguousarray(W[1:, :32]), scramble=oracle.SCRAMBLE_NESTED, seeds=seeds,
                             with_grad=grad)
    assert parts["est"].mean() == pytest.approx(whole["est"][0], rel=1e-13, abs=1e-300)
    if grad:
        np.testing.assert_allclose(parts["grad"].mean(axis=0), whole["grad"][0], rtol=1e-12, atol=1e-16)


def test_single_element_is_the_plain_sequence(oracle):
    """q = 0: the one element is the sequence itself (dimensions 1..s)."""
    s = 4
    W = oracle.sobol_matrices_wide(s + 1, 40, inputs.sobol_raw_init(s + 1))
    th = inputs.scene_theta(8, 4)[13]
    a = oracle.integrate_partitioned(oracle.F_SCENE4D, s, np.array([3000], np.uint32), th[None, :], W, 0, [0])
    b = oracle.integrate(oracle.SOURCE_SOBOL, oracle.F_SCENE4D, s, np.array([3000], np.uint32), th[None, :],
                         C=np.ascontiguousarray(W[1:, :32]))
    assert a["est"][0] == b["est"][0]


def test_argument_checks(oracle):
    W = oracle.sobol_matrices_wide(7, 40, inputs.sobol_raw_init(7))
    th = inputs.gaussmix_theta(1)
    with pytest.raises(ValueError):  # 2^(32+q) points need m >= 32 + q index bits
        oracle.integrate_partitioned(oracle.F_GAUSSMIX4_6D, 6, np.array([8], np.uint32), th, W, 9, [0])

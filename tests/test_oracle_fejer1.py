"""Pins of the oracle's shifted grid of Fejer's first rule (Sec. 3.3,
Eq. fejer1-points and Eq. fejer1-wgt) to facts the mathematics fixes,
independent of the oracle's code: the closed-form nodes, exact integration
of polynomials up to degree J-1, the weights as the unique solution of the
moment system, exact rationals at J = 3, and the full transform's round
trip and agreement with a Gaussian transform on band-limited fields."""
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O
from paper_1711_11296_gb300 import workloads as W


def test_nodes_are_shifted_by_half_a_step_and_symmetric():
    for J in (1, 3, 7, 65):
        theta, mu, s = O.fejer1_nodes(J)
        j = np.arange(1, J + 1)
        np.testing.assert_allclose(theta, (j - 0.5) * np.pi / J, rtol=0, atol=1e-15)
        # no pole: the grid starts half a step (pi/2J) from each pole
        assert abs(theta[0] - np.pi / (2 * J)) < 1e-15
        assert abs(theta[-1] - (np.pi - np.pi / (2 * J))) < 1e-15
        np.testing.assert_allclose(mu, -mu[::-1], rtol=0, atol=1e-15)
        # odd J: the middle node is on the Equator
        assert abs(mu[(J - 1) // 2]) < 1e-15


def test_j1_and_j3_weights_are_exact_rationals():
    # J = 1: one node on the Equator carrying the whole measure, 2.
    assert abs(O.fejer1_weights(1)[0] - 2.0) < 1e-15
    # J = 3: nodes mu = sqrt(3)/2, 0, -sqrt(3)/2.  The interpolatory rule
    # integrates 1 and mu^2 exactly: 2a + b = 2 and 2a (3/4) = 2/3, so
    # a = 4/9, b = 10/9 (exact rationals, solved here by hand).
    a = Fraction(2, 3) / (2 * Fraction(3, 4))
    b = 2 - 2 * a
    assert (a, b) == (Fraction(4, 9), Fraction(10, 9))
    # (to 2 ulp of values near 1: the cosine sum rounds)
    np.testing.assert_allclose(O.fejer1_weights(3), [float(a), float(b), float(a)],
                               rtol=0, atol=4.5e-16)


def test_printed_weight_formula_is_not_exact():
    # Eq. (fejer1-wgt) as printed lacks the factor 2 in front of the sum.
    # That reading gives 5/9, 8/9, 5/9 at J = 3, which sum to 2 but
    # integrate mu^2 to 5/6 instead of 2/3; the oracle's rule is exact.
    J = 3
    theta, mu, _ = O.fejer1_nodes(J)
    printed = 2.0 / J * (1.0 - np.cos(2 * theta) / 3.0)
    np.testing.assert_allclose(printed, [5 / 9, 8 / 9, 5 / 9], rtol=0, atol=1e-15)
    assert abs(printed @ mu ** 2 - 5 / 6) < 1e-15
    assert abs(O.fejer1_weights(J) @ mu ** 2 - 2 / 3) < 1e-15


@pytest.mark.parametrize("J", [5, 9, 64, 65, 321, 1281])
def test_weights_sum_to_two_and_are_symmetric_and_positive(J):
    w = O.fejer1_weights(J)
    assert abs(w.sum() - 2.0) < 1e-13
    np.testing.assert_allclose(w, w[::-1], rtol=0, atol=1e-15)
    assert (w > 0).all()


@pytest.mark.parametrize("J", [8, 9, 33, 64, 65, 129])
def test_weights_integrate_polynomials_exactly(J):
    # The J-point interpolatory rule is exact to degree J-1; for odd J the
    # symmetric nodes make degree J (odd) exact too.
    _, mu, _ = O.fejer1_nodes(J)
    w = O.fejer1_weights(J)
    top = J if J % 2 else J - 1
    for k in range(0, top + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        got = npleg.legval(mu, c) @ w
        exact = 2.0 if k == 0 else 0.0
        assert abs(got - exact) < 5e-15, (J, k, got)
    # the first even degree above the exact range is not integrated exactly
    k = J + 1 if J % 2 else J
    c = np.zeros(k + 1)
    c[k] = 1.0
    assert abs(npleg.legval(mu, c) @ w) > 1e-6


@pytest.mark.parametrize("J", [3, 8, 9, 17, 33])
def test_weights_equal_unique_interpolatory_weights(J):
    # Moment system in the Chebyshev-T basis the rule is built on (Sec. 3.3):
    # sum_j w_j cos(l theta_j) = int_{-1}^{1} T_l(mu) dmu, l = 0..J-1, with
    # int T_l = 2/(1 - l^2) for even l and 0 for odd l.
    theta, _, _ = O.fejer1_nodes(J)
    l = np.arange(J)[:, None]
    A = np.cos(l * theta[None, :])
    b = np.array([2.0 / (1.0 - k * k) if k % 2 == 0 else 0.0 for k in range(J)])
    w = np.linalg.solve(A, b)
    np.testing.assert_allclose(O.fejer1_weights(J), w, rtol=0, atol=1e-14)


def test_transform_round_trip_and_gauss_agreement():
    # J >= 2N+1: the rule integrates every product P~_n P~_n' of a band-
    # limited field exactly, so analysis(synthesis(a)) = a, and a Gaussian
    # transform of the same field gives the same spectrum.
    N, J, I, F = 7, 15, 16, 2
    a = W.random_spectrum(N, F, "n^-1.5", seed=1401)
    x = O.synthesis_fejer1(a, N, J, I)
    got = O.analysis_fejer1(x, N)
    a0 = a.copy()
    a0[:N + 1] = a0[:N + 1].real        # Im(X_n^0) is not an input
    np.testing.assert_allclose(got, a0, rtol=0, atol=2e-14)
    xg = O.synthesis_gauss(a, N, N + 1, I)
    np.testing.assert_allclose(O.analysis_gauss(xg, N), got, rtol=0, atol=2e-14)

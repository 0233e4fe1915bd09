"""Pins of the oracle's nodes and weights (Eq. cc-points, Eq. cc-wgt) to
facts the paper and the mathematics fix, independent of the oracle's code."""
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_small_J_weights_match_hand_derivation():
    for row in _read_golden("cc_weights_small.txt"):
        J = int(row[0])
        want = np.array([float(v) for v in row[1:]])
        np.testing.assert_allclose(O.cc_weights(J), want, rtol=0, atol=2e-16)


@pytest.mark.parametrize("J", [5, 9, 65, 321, 641, 1281])
def test_weights_sum_to_two_and_are_symmetric(J):
    w = O.cc_weights(J)
    assert abs(w.sum() - 2.0) < 1e-14
    np.testing.assert_allclose(w, w[::-1], rtol=0, atol=1e-15)
    assert (w > 0).all()


@pytest.mark.parametrize("J", [9, 33, 65, 129])
def test_weights_integrate_polynomials_exactly(J):
    # Sec. 3.1: exact for degree <= J-1; degree J by symmetry when J is odd.
    _, mu, _ = O.cc_nodes(J)
    w = O.cc_weights(J)
    for k in range(0, J + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        got = npleg.legval(mu, c) @ w
        exact = 2.0 if k == 0 else 0.0
        assert abs(got - exact) < 5e-15, (J, k, got)
    # degree J+1 is the first inexact one (U_{J+1} aliases onto -U_{J-1}).
    c = np.zeros(J + 2)
    c[J + 1] = 1.0
    assert abs(npleg.legval(mu, c) @ w) > 1e-6


@pytest.mark.parametrize("J", [3, 9, 17, 33])
def test_weights_equal_unique_interpolatory_weights(J):
    # The weights of an interpolatory rule are the solution of the moment
    # system sum_j w_j U_l(mu_j) = int U_l, l = 0..J-1 (Appendix A: the rule
    # integrates the Chebyshev-U expansion of degree J-1 exactly).
    theta, _, s = O.cc_nodes(J)
    l = np.arange(J)[:, None]
    A = np.sin((l + 1) * theta[None, :]) / s[None, :]
    b = np.array([(1 + (-1) ** k) / (k + 1) for k in range(J)], dtype=float)
    w = np.linalg.solve(A, b)
    np.testing.assert_allclose(O.cc_weights(J), w, rtol=0, atol=1e-14)


def _printed_interval(txt):
    """Values consistent with a number printed to its last digit, whether
    truncated or rounded: [p - u/2, p + u)."""
    mant = txt.lower().split("e")[0]
    exp = int(txt.lower().split("e")[1]) if "e" in txt.lower() else 0
    decimals = len(mant.split(".")[1]) if "." in mant else 0
    unit = 10.0 ** (exp - decimals)
    p = float(txt)
    return p - unit / 2, p + unit


def _exact_and_values(family, n, theta, mu, s):
    if family == "U":
        return (1 + (-1) ** n) / (n + 1), np.sin((n + 1) * theta) / s
    if family == "T":
        return (0.0 if n % 2 else 2.0 / (1 - n * n)), np.cos(n * theta)
    c = np.zeros(n + 1)
    c[n] = 1.0
    return 0.0, npleg.legval(mu, c)


def test_quadrature_errors_printed_in_section_4_3():
    for rule, J, fam, n, txt in _read_golden("cc959_quadrature_errors.txt"):
        J, n = int(J), int(n)
        if rule == "cc":
            theta, mu, s = O.cc_nodes(J)
            w = O.cc_weights(J)
        else:
            mu, s, w = O.gauss_nodes_weights(J)
            theta = np.arccos(mu)
        exact, vals = _exact_and_values(fam, n, theta, mu, s)
        err = abs(exact - vals @ w)
        lo, hi = _printed_interval(txt)
        assert lo <= err < hi, (rule, J, fam, n, err, txt)


def test_u_aliasing_identity_closed_form():
    # Sec. 4.3: e_J(p) = 2/(J+1+p) + 2/(J+1-p) for even J+p, 0 for odd.
    J = 959
    theta, _, s = O.cc_nodes(J)
    w = O.cc_weights(J)
    for p in [1, 2, 3, 5, 241, 481, 720]:
        n = J + p
        exact = (1 + (-1) ** n) / (n + 1)
        err = exact - (np.sin((n + 1) * theta) / s) @ w
        closed = 0.0 if (J + p) % 2 else 2 / (J + 1 + p) + 2 / (J + 1 - p)
        assert abs(err - closed) < 1e-12, (p, err, closed)


def test_gauss_golub_welsch_against_library():
    x, w = npleg.leggauss(64)
    mu, s, wg = O.gauss_nodes_weights(64)
    order = np.argsort(-x)
    np.testing.assert_allclose(mu, x[order], atol=1e-15)
    np.testing.assert_allclose(wg, w[order], atol=1e-14)


@pytest.mark.parametrize("K", [1, 3, 31, 127, 511])
def test_nodes_nest_in_2K_plus_1_grid(K):
    # Sec. 3.2: the K-point grid is every other latitude (from j = 2) of the
    # (2K+1)-point grid; exact as rationals j/(J+1).
    Jf = 2 * K + 1
    for jc in range(1, K + 1):
        assert 2 * jc * (K + 1) == jc * (Jf + 1)     # theta_{2jc}^f == theta_jc^c
    th_c = O.cc_nodes(K)[0]
    th_f = O.cc_nodes(Jf)[0]
    np.testing.assert_allclose(th_f[O.nested_rows(K, 1) - 1], th_c, rtol=0,
                               atol=1e-15)
    # and the (2K-1)-point grid does not contain it: as exact rationals,
    # j/(K+1) == j'/(2K) only at the Equator (odd K).
    if K > 1:
        shared = [jc for jc in range(1, K + 1)
                  if (jc * 2 * K) % (K + 1) == 0]
        assert shared == ([(K + 1) // 2] if K % 2 else [])

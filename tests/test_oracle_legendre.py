"""Pins of the oracle's normalised associated Legendre functions (Sec. 4.1,
Eq. pnm-ortho) against closed forms, SciPy's spherical harmonics and the
orthonormality facts of Sec. 4.1."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import special

import oracle as O


def test_binary128_node_series_matches_libm():
    for J in [3, 65, 1281]:
        for j in [1, 2, (J + 1) // 2, J - 1, J]:
            c, s = O.cc_node_binary128(J, j)
            th = np.pi * j / (J + 1)
            assert abs(c - np.cos(th)) < 4e-16 and abs(s - np.sin(th)) < 4e-16


def test_closed_forms_low_degree():
    J = 17
    th, mu, s = O.cc_nodes(J)
    P = O.pnm_cc(2, J)                # rows (0,0),(0,1),(0,2),(1,1),(1,2),(2,2)
    np.testing.assert_allclose(P[0], 1 / np.sqrt(2), atol=1e-16)
    np.testing.assert_allclose(P[1], np.sqrt(1.5) * mu, atol=1e-15)
    np.testing.assert_allclose(P[2], np.sqrt(5 / 8) * (3 * mu ** 2 - 1), atol=1e-15)
    np.testing.assert_allclose(P[3], np.sqrt(3) / 2 * s, atol=1e-15)
    np.testing.assert_allclose(P[4], np.sqrt(15) / 2 * mu * s, atol=1e-15)
    np.testing.assert_allclose(P[5], np.sqrt(15) / 4 * s ** 2, atol=1e-15)


def test_against_scipy_spherical_harmonics():
    # P~_n^m(cos t) = sqrt(2 pi) (-1)^m Y_n^m(t, 0): SciPy's Y is unit-normed
    # on the sphere and carries the Condon-Shortley phase.
    N, J = 40, 81
    th, mu, s = O.cc_nodes(J)
    P = O.pnm_cc(N, J)
    r = 0
    for m in range(N + 1):
        for n in range(m, N + 1):
            y = special.sph_harm_y(n, m, th, 0.0).real
            ref = np.sqrt(2 * np.pi) * (-1) ** m * y
            np.testing.assert_allclose(P[r], ref, rtol=0, atol=2e-13)
            r += 1


def test_orthonormal_under_gauss_quadrature():
    # Eq. pnm-ortho with an independent rule (Gauss-Legendre, 2N+2 nodes).
    N = 48
    x, w = npleg.leggauss(N + 2)
    P = O.pnm_at(N, x, np.sqrt(1 - x * x))
    r = 0
    for m in range(N + 1):
        blk = P[r:r + N - m + 1]
        G = (blk * w) @ blk.T
        # node errors of ~1e-16 enter through P' ~ n^2: allow ~N^2 eps
        np.testing.assert_allclose(G, np.eye(N - m + 1), atol=3e-13)
        r += N - m + 1


@pytest.mark.parametrize("N,J", [(31, 65), (159, 321)])
def test_cubic_cc_orthonormality_at_rounding_level(N, J):
    # Sec. 4.1: with J >= 2N+1 both errors are at rounding level for all (n, m).
    for m in range(0, N + 1, max(1, N // 16)):
        eN, eO = O.orthonormality_errors(N, J, m)
        assert eN.max() < 2e-14 and eO.max() < 2e-14, (m, eN.max(), eO.max())


def test_tc479_selected_orders():
    N, J = 479, 959
    for m in [0, 1, 240, 479]:
        eN, eO = O.orthonormality_errors(N, J, m)
        assert eN.max() < 5e-14 and eO.max() < 5e-14


def test_quadratic_truncation_breaks_normality_only_above_half():
    # Sec. 4.1, Tq639 on J = 959: normality fails only for n > (J-1)/2 = 479,
    # orthogonality holds for n <= J - N = 320 (odd products vanish by
    # symmetry) and fails from n = J - N + 1.  The paper reads the size of the
    # errors off a logarithmic colour scale as "< 1e-3"; the exact maximum is
    # 1.69e-3 (m = 0, n = 639), confirmed here with NumPy's Legendre series,
    # so the bound is taken as "of order 1e-3" (< 2e-3).
    N, J = 639, 959
    _, mu, _ = O.cc_nodes(J)
    w = O.cc_weights(J)
    c = np.zeros(N + 1)
    c[N] = 1.0
    p0 = npleg.legval(mu, c) * np.sqrt((2 * N + 1) / 2)
    eN0 = O.orthonormality_errors(N, J, 0)[0]
    assert abs(eN0[-1] - abs(p0 ** 2 @ w - 1)) < 1e-13
    for m in [0, 7]:
        eN, eO = O.orthonormality_errors(N, J, m)
        n = np.arange(m, N + 1)
        assert eN[n <= 479].max() < 5e-14
        assert eN[n > 479].max() > 1e-10
        assert eO[n <= J - N].max() < 5e-14
        assert eO[n == J - N + 1].max() > 1e-12
        assert eN.max() < 2e-3 and eO.max() < 2e-3

"""Pins of the oracle's aliasing experiment (Sec. 4.2): the product
pipeline (synthesis of U, V, W; X_q = U V and X_c = U V W on the grid;
analysis) against an independent quadrature where both are exact, a
constant factor, and the paper's qualitative finding that the cubic
Clenshaw-Curtis grid aliases far less than the linear Gaussian grid."""
import numpy as np
import pytest

import oracle as O
from paper_1711_11296_gb300 import workloads as W

N = 10


def _uvw(F=2):
    return [W.random_spectrum(N, F, "uniform^-1/3", seed=s) for s in (41, 42, 43)]


def test_products_exact_on_fine_grids_agree_across_quadratures():
    # X_c has degree 3N; its projection onto P~_n^m (n <= N) integrates a
    # polynomial of degree 4N in mu, which the J-point CC rule integrates
    # exactly for J >= 4N+1 and the Gaussian rule for J >= 2N+1; zonally,
    # I > 4N keeps wavenumbers up to 3N from aliasing onto m <= N.  Two
    # independent rules (the explicit CC weight sum, Golub-Welsch) must then
    # give the same spectra.
    U, V, Wv = _uvw()
    I = 4 * N + 4
    q_cc, c_cc = O.aliasing_products(U, V, Wv, N, 4 * N + 3, I)
    q_g, c_g = O.aliasing_products(U, V, Wv, N, 2 * N + 2, I, quad="gauss")
    np.testing.assert_allclose(q_cc, q_g, rtol=0, atol=1e-13 * np.abs(q_g).max())
    np.testing.assert_allclose(c_cc, c_g, rtol=0, atol=1e-13 * np.abs(c_g).max())
    # the quadratic term is already exact at J >= 3N+1, I > 3N
    q3, _ = O.aliasing_products(U, V, Wv, N, 3 * N + 1, 3 * N + 2)
    np.testing.assert_allclose(q3, q_g, rtol=0, atol=1e-13 * np.abs(q_g).max())


def test_constant_factor_scales_the_other_field():
    # U = u00 P~_0^0 = u00 / sqrt(2) everywhere: X_q = V / sqrt(2) * u00, and
    # the transform of a band-limited V is exact at J = 2N+1
    U, V, Wv = _uvw()
    U[:] = 0.0
    U[0] = 3.0
    q, c = O.aliasing_products(U, V, Wv, N, 2 * N + 1, 2 * N + 2)
    np.testing.assert_allclose(q, V * 3.0 / np.sqrt(2.0), rtol=0, atol=1e-14 * 3)
    # U V W is symmetric in V and W on any grid
    _, cw = O.aliasing_products(U, Wv, V, N, 2 * N + 1, 2 * N + 2)
    np.testing.assert_allclose(c, cw, rtol=0, atol=1e-12 * np.abs(c).max())


def test_cubic_cc_grid_aliases_less_than_linear_gaussian_grid():
    # Sec. 4.2: on the cubic CC grid (J = 2N+1) the aliasing errors are far
    # below those of the linear Gaussian grid (J = N+1) for the same
    # truncation; the reference is the exact fine-grid result.
    U, V, Wv = _uvw(F=3)
    q_ref, c_ref = O.aliasing_products(U, V, Wv, N, 4 * N + 3, 4 * N + 4)
    q_cc, c_cc = O.aliasing_products(U, V, Wv, N, 2 * N + 1, 4 * N + 4)
    q_gl, c_gl = O.aliasing_products(U, V, Wv, N, N + 1, 2 * N + 2, quad="gauss")
    for t_cc, t_gl, ref in ((q_cc, q_gl, q_ref), (c_cc, c_gl, c_ref)):
        e_cc = np.median(O.aliasing_error(t_cc, ref))
        e_gl = np.median(O.aliasing_error(t_gl, ref))
        assert e_cc * 10 < e_gl, (e_cc, e_gl)

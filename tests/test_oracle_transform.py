"""Pins of the oracle's full transforms: DFT special cases, exactness of the
CC round trip (Sec. 3.1), agreement with an independent Gaussian transform
and with SciPy's spherical harmonics, hemispheric flip symmetry
(Appendix B), nested restriction (Sec. 3.2, Appendix C) and the adjoints."""
import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_1711_11296_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_dft_matches_numpy_fft():
    g = np.random.default_rng(1).standard_normal((3, 5, 40))
    N = 13
    X = O.dft_forward(g, N)
    ref = np.fft.rfft(g, axis=-1)[..., :N + 1] / 40
    np.testing.assert_allclose(X, ref, atol=1e-15)
    # inverse of a Hermitian-truncated spectrum
    Y = np.fft.rfft(g, axis=-1)[..., :N + 1] / 40
    full = np.zeros((3, 5, 21), dtype=complex)
    full[..., :N + 1] = Y
    np.testing.assert_allclose(O.dft_inverse(Y, 40),
                               np.fft.irfft(full * 40, n=40, axis=-1), atol=1e-14)


def test_dft_pure_harmonic():
    I, k, ph = 30, 7, 0.4
    lam = 2 * np.pi * np.arange(I) / I
    x = np.cos(k * lam + ph)[None, None, :]
    X = O.dft_forward(x, 14)[0, 0]
    want = np.zeros(15, dtype=complex)
    want[k] = 0.5 * np.exp(1j * ph)
    np.testing.assert_allclose(X, want, atol=1e-15)


@pytest.mark.parametrize("N,J,I", [(31, 65, 128), (10, 21, 22), (16, 33, 40)])
def test_round_trip_exact_for_cubic_grid(N, J, I):
    # Sec. 3.1 / abstract: J >= 2N+1 and I > 2N give an exact transform pair.
    a = W.random_spectrum(N, 3, "n^-1.5", seed=5)
    back = O.analysis(O.synthesis(a, N, J, I), N)
    assert _rel(back, a) < 1e-14


def test_round_trip_inexact_below_cubic():
    N = 20
    a = W.random_spectrum(N, 1, "n^-1.5", seed=6)
    back = O.analysis(O.synthesis(a, N, 2 * N - 1, 64), N)
    assert _rel(back, a) > 1e-6


def _cartesian_poly(theta, lam):
    """A fixed polynomial of total degree 12 in (x, y, z) on the unit sphere:
    band-limited to n <= 12 with no transform arithmetic involved."""
    st = np.sin(theta)[:, None]
    x = st * np.cos(lam)[None, :]
    y = st * np.sin(lam)[None, :]
    z = np.cos(theta)[:, None] * np.ones_like(lam)[None, :]
    return (1.0 + 0.3 * x - 0.7 * y * z + 0.2 * x ** 2 * y ** 3 + 0.5 * z ** 5 * x
            + 0.4 * (x * y * z) ** 2 - 0.25 * y ** 7 * z ** 5 + 0.1 * x ** 12)


def test_cc_and_gauss_agree_on_a_band_limited_field():
    # Two different rules (Eq. cc-quad and Eq. gauss-quad) on different nodes
    # must give the same spectrum of an exactly band-limited field.
    N, I = 12, 26
    lam = 2 * np.pi * np.arange(I) / I
    Jc = 2 * N + 1
    th_c = O.cc_nodes(Jc)[0]
    a_cc = O.analysis(_cartesian_poly(th_c, lam)[None], N)
    Jg = N + 1
    mu_g = O.gauss_nodes_weights(Jg)[0]
    a_g = O.analysis_gauss(_cartesian_poly(np.arccos(mu_g), lam)[None], N)
    np.testing.assert_allclose(a_cc, a_g, atol=2e-15)
    # and a CC grid below the cubic limit does not reproduce it
    th_l = O.cc_nodes(N + 3)[0]
    a_l = O.analysis(_cartesian_poly(th_l, lam)[None], N)
    assert np.abs(a_l - a_g).max() > 1e-6


def test_synthesis_matches_scipy_harmonics():
    N, J, I = 10, 21, 24
    a = W.random_spectrum(N, 1, "n^-1.5", seed=9)[:, 0]
    th = O.cc_nodes(J)[0]
    lam = 2 * np.pi * np.arange(I) / I
    T, L = np.meshgrid(th, lam, indexing="ij")
    ref = np.zeros((J, I))
    r = 0
    for m in range(N + 1):
        for n in range(m, N + 1):
            y = np.sqrt(2 * np.pi) * (-1) ** m * special.sph_harm_y(n, m, T, L)
            if m == 0:
                ref += (a[r].real * y).real
            else:
                ref += 2 * (a[r] * y).real
            r += 1
    np.testing.assert_allclose(O.synthesis(a[:, None], N, J, I)[0], ref,
                               atol=1e-13)


def test_meridional_flip_maps_to_parity_sign():
    # Appendix B: flipping the grid north-south multiplies X_n^m by (-1)^(n-m).
    N, J, I = 15, 31, 32
    x = W.random_grid(2, J, I)
    a = O.analysis(x, N)
    af = O.analysis(x[:, ::-1, :], N)
    sign = (-1.0) ** (W.degree_of_rows(N) - W.order_of_rows(N))
    np.testing.assert_allclose(af, sign[:, None] * a, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2])
def test_restriction_of_band_limited_field_is_truncation(k):
    # Sec. 3.2 / Appendix C: the coarse CC transform of the injected sub-grid
    # recovers the spectrum of a field band-limited to the coarse truncation.
    Nc = 7
    Jc, Ic = 2 * Nc + 1, 16
    Jf, If = 2 ** k * (Jc + 1) - 1, 2 ** k * Ic
    a = W.random_spectrum(Nc, 2, "n^-1.5", seed=11)
    fine = O.synthesis(a, Nc, Jf, If)
    np.testing.assert_allclose(O.restrict_nested(fine, k, Nc), a, atol=1e-14)


def test_restriction_rejects_non_nested_grid():
    with pytest.raises(ValueError):
        O.restrict_nested(np.zeros((1, 14, 16)), 1, 3)


def _real_view(c):
    return np.concatenate([c.real.ravel(), c.imag.ravel()])


def _dense(fun, shape_in, complex_in):
    cols = []
    size = int(np.prod(shape_in))
    for part in ([1.0, 1j] if complex_in else [1.0]):
        for e in range(size):
            v = np.zeros(size, dtype=complex if complex_in else float)
            v[e] = part
            out = fun(v.reshape(shape_in))
            cols.append(_real_view(out) if np.iscomplexobj(out) else out.ravel())
    return np.array(cols).T


@pytest.mark.parametrize("N,J,I", [(1, 3, 4), (3, 7, 8), (4, 11, 10)])
def test_adjoints_are_dense_transposes(N, J, I):
    nc = O.ncoef(N)
    A = _dense(lambda x: O.analysis(x, N), (1, J, I), False)          # grid->spec
    At = _dense(lambda a: O.adjoint_analysis(a, N, J, I), (nc, 1), True)
    np.testing.assert_allclose(At, A.T, atol=1e-15)
    S = _dense(lambda a: O.synthesis(a, N, J, I), (nc, 1), True)      # spec->grid
    St = _dense(lambda x: O.adjoint_synthesis(x, N), (1, J, I), False)
    np.testing.assert_allclose(St, S.T, atol=1e-14)


def test_adjoint_dot_products_t31():
    N, J, I = 31, 65, 128
    x = W.random_grid(2, J, I, seed=3)
    a = W.random_spectrum(N, 2, "n^-1.5", seed=4)
    a_im0 = a.copy()
    lhs = np.sum(np.real(np.conj(O.analysis(x, N)) * a))
    rhs = np.sum(x * O.adjoint_analysis(a, N, J, I))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    lhs = np.sum(O.synthesis(a_im0, N, J, I) * x)
    rhs = np.sum(np.real(np.conj(a_im0) * O.adjoint_synthesis(x, N)))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_synthesis_rows_matches_scipy_at_scattered_latitudes():
    # synthesis_rows (Eq. iSHT at chosen 1-based latitudes) pinned against
    # SciPy's spherical harmonics evaluated at those latitudes only, and
    # against the full synthesis's rows: rows 1, J_h (the Equator) and J,
    # unsorted, with a repeat, so that an off-by-one in the 1-based index or
    # a dropped row ordering fails.
    N, J, I = 12, 25, 28
    Jh = (J + 1) // 2
    rows = np.array([J, 1, Jh, 4, 1, J - 3])
    a = W.random_spectrum(N, 2, "n^-1.5", seed=21)
    got = O.synthesis_rows(a, N, J, I, rows)
    assert got.shape == (2, len(rows), I)
    th = O.cc_nodes(J)[0][rows - 1]
    lam = 2 * np.pi * np.arange(I) / I
    T, L = np.meshgrid(th, lam, indexing="ij")
    for f in range(2):
        ref = np.zeros((len(rows), I))
        r = 0
        for m in range(N + 1):
            for n in range(m, N + 1):
                y = np.sqrt(2 * np.pi) * (-1) ** m * special.sph_harm_y(n, m, T, L)
                ref += (a[r, f].real * y).real if m == 0 else 2 * (a[r, f] * y).real
                r += 1
        np.testing.assert_allclose(got[f], ref, atol=1e-13)
    full = O.synthesis(a, N, J, I)
    np.testing.assert_allclose(got, full[:, rows - 1, :], rtol=0, atol=1e-15)


def test_sampled_adjoints_equal_the_dense_transposes_parts():
    # adjoint_analysis_rows and adjoint_synthesis(ms=...) against the full
    # adjoints, which the dense-transpose test above pins; scattered rows
    # (1, the Equator, J, unsorted) and wavenumbers (0, the last, unsorted).
    N, J, I = 4, 11, 10
    A = _dense(lambda x: O.analysis(x, N), (1, J, I), False)
    nc = O.ncoef(N)
    a = W.random_spectrum(N, 2, "n^-1.5", seed=23)
    rows = np.array([J, 1, (J + 1) // 2, 3])
    got = O.adjoint_analysis_rows(a, N, J, I, rows)
    full = O.adjoint_analysis(a, N, J, I)
    np.testing.assert_allclose(got, full[:, rows - 1, :], rtol=0, atol=1e-15)
    # and directly against the dense transpose of the analysis
    v = np.concatenate([a[:, 0].real, a[:, 0].imag])
    dense = (A.T @ v).reshape(J, I)
    np.testing.assert_allclose(got[0], dense[rows - 1], rtol=0, atol=1e-14)
    x = W.random_grid(2, J, I, seed=24)
    ms = [N, 0, 2]
    d = O.adjoint_synthesis(x, N, ms=ms)
    full = O.adjoint_synthesis(x, N)
    for m in ms:
        r0 = O.coef_offset(N, m)
        np.testing.assert_allclose(d[m], full[r0:r0 + N - m + 1], rtol=0, atol=1e-15)
    S = _dense(lambda s: O.synthesis(s, N, J, I), (nc, 1), True)
    t = S.T @ x[0].ravel()
    dense = t[:nc] + 1j * t[nc:]
    for m in ms:
        r0 = O.coef_offset(N, m)
        np.testing.assert_allclose(d[m][:, 0], dense[r0:r0 + N - m + 1], rtol=0, atol=1e-14)

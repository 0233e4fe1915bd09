"""Pins of the oracle's reduced Clenshaw-Curtis grid (per-latitude longitude
counts by the reduction rule quoted in Sec. 6) to facts that do not come from
the reduced-grid code itself: the count rule's arithmetic, the reduction to
the full-grid transforms when every row keeps I points, the exact round trip
of band-limited fields (the 1e-16 rule drops only negligible terms), its
failure on a grid that drops significant wavenumbers, and agreement with the
full-grid synthesis at the longitudes the two grids share."""
import numpy as np
import pytest
from scipy import special

import oracle as O
from oracle import cc_oracle as OC
from paper_1711_11296_gb300 import workloads as W

SHAPES = [(31, 65, 128), (63, 129, 256)]


def _smooth(n):
    h = n // 2
    for p in (2, 3, 5):
        while h % p == 0:
            h //= p
    return n % 2 == 0 and h == 1


@pytest.mark.parametrize("N,J,I", SHAPES)
def test_sizes_follow_the_rule(N, J, I):
    Ij, M = O.reduced_sizes(N, J, I)
    assert Ij.shape == (J,) and M.shape == (J,)
    np.testing.assert_array_equal(Ij, Ij[::-1])          # symmetric about the Equator
    np.testing.assert_array_equal(M, M[::-1])
    assert M[(J - 1) // 2] == N                          # every m significant at the Equator
    h = (J + 1) // 2
    assert np.all(np.diff(M[:h]) >= 0)                   # fewer significant m toward the pole
    assert M[0] < N and Ij[0] < I                        # and a real reduction there
    for n, m in zip(Ij, M):
        need = 4 * int(m) + 1
        assert _smooth(int(n)) and n <= I
        if n < I:
            assert n >= need
            # the smallest such count: no even smooth count in [need, n)
            assert not any(_smooth(k) for k in range(need, int(n)))
    assert Ij.sum() < J * I


def test_even_smooth_ceil_by_hand():
    # 4 M + 1 for M = 0, 4, 17, 31 -> 2, 18 (= 2 x 9), 72 (= 2 x 36), 128
    assert [OC._even_smooth_ceil(4 * m + 1) for m in (0, 4, 17, 31)] == [2, 18, 72, 128]
    # 2 x 7 = 14 and 2 x 11 = 22 are not smooth: 13 -> 16, 21 -> 24
    assert OC._even_smooth_ceil(13) == 16 and OC._even_smooth_ceil(21) == 24


def test_full_counts_reduce_to_the_full_grid():
    N, J, I, F = 15, 31, 32, 3
    Ij = np.full(J, I)
    x = W.random_grid(F, J, I, seed=1701)
    np.testing.assert_allclose(O.analysis_reduced(x.reshape(F, -1), N, J, Ij),
                               O.analysis(x, N), rtol=0, atol=1e-15)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1702)
    np.testing.assert_allclose(O.synthesis_reduced(a, N, J, Ij),
                               O.synthesis(a, N, J, I).reshape(F, -1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("N,J,I", SHAPES)
def test_round_trip_is_exact_on_the_rule_grid(N, J, I):
    F = 2
    Ij, _ = O.reduced_sizes(N, J, I)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1710 + N)
    a[:N + 1] = a[:N + 1].real
    back = O.analysis_reduced(O.synthesis_reduced(a, N, J, Ij), N, J, Ij)
    err = np.linalg.norm(back - a) / np.linalg.norm(a)
    assert err < 1e-13, err


def test_round_trip_needs_only_m_j_per_row_and_fails_below():
    # The round trip only needs row j to carry its significant wavenumbers,
    # I_j >= 2 M_j + 2 (the rule's 4 M_j + 1 is the cubic-truncation count):
    # on that linear minimum it is still exact.  Halving those rows poleward
    # of 30 degrees drops significant wavenumbers and the round trip fails,
    # so the exactness test above does detect a rule that keeps too few.
    N, J, I, F = 31, 65, 128, 2
    _, M = O.reduced_sizes(N, J, I)
    lin = np.array([OC._even_smooth_ceil(2 * int(m) + 2) for m in M])
    a = W.random_spectrum(N, F, "n^-1.5", seed=1720)
    a[:N + 1] = a[:N + 1].real
    back = O.analysis_reduced(O.synthesis_reduced(a, N, J, lin), N, J, lin)
    assert np.linalg.norm(back - a) / np.linalg.norm(a) < 1e-13
    bad = lin.copy()
    lat = 90.0 - np.degrees(np.arange(1, J + 1) * np.pi / (J + 1))
    for j in np.nonzero(np.abs(lat) > 30.0)[0]:
        bad[j] = OC._even_smooth_ceil(lin[j] // 2)
    back = O.analysis_reduced(O.synthesis_reduced(a, N, J, bad), N, J, bad)
    assert np.linalg.norm(back - a) / np.linalg.norm(a) > 1e-3


def test_synthesis_matches_full_grid_at_shared_longitudes():
    # Where I_j divides I, the reduced row's longitudes 2 pi i / I_j are the
    # full row's every (I/I_j)-th point.
    N, J, I, F = 63, 129, 256, 2
    Ij, _ = O.reduced_sizes(N, J, I)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1730)
    red = O.synthesis_reduced(a, N, J, Ij)
    full = O.synthesis(a, N, J, I)
    off = O.reduced_row_offsets(Ij)
    shared = [j for j in range(J) if I % Ij[j] == 0 and Ij[j] < I]
    assert shared, "no reduced row divides I"
    scale = np.abs(full).max()
    for j in shared + [(J - 1) // 2]:
        step = I // Ij[j]
        np.testing.assert_allclose(red[:, off[j]:off[j + 1]], full[:, j, ::step],
                                   rtol=0, atol=1e-14 * scale)


def test_significant_wavenumbers_match_an_independent_legendre_routine():
    # M_j from SciPy's associated Legendre functions (their own algorithm,
    # normalised here by sqrt((2n+1)/2 (n-m)!/(n+m)!); the phase does not
    # matter for a magnitude) equals the oracle's, at T31 where SciPy's
    # factorials stay in range.
    special = pytest.importorskip("scipy.special")
    N, J, I = 31, 65, 128
    mu = np.cos(np.arange(1, J + 1) * np.pi / (J + 1))
    M = np.zeros(J, dtype=np.int64)
    for m in range(N + 1):
        for n in range(m, N + 1):
            c = np.sqrt((2 * n + 1) / 2.0 *
                        np.exp(special.gammaln(n - m + 1) - special.gammaln(n + m + 1)))
            sig = np.abs(c * special.lpmv(m, n, mu)) >= 1e-16
            M[sig] = np.maximum(M[sig], m)
    _, Mo = O.reduced_sizes(N, J, I)
    np.testing.assert_array_equal(Mo, M)


def test_octahedral_counts():
    # 20 points on the first latitude from either pole, 4 more per row,
    # mirrored about the Equator (J = 9: five rows from the north to it)
    assert O.octahedral_sizes(9).tolist() == [20, 24, 28, 32, 36, 32, 28, 24, 20]
    Ij = O.octahedral_sizes(1281)
    assert Ij[640] == 20 + 4 * 640 and np.array_equal(Ij, Ij[::-1])


def test_icositetrahedral_counts_and_shifts():
    # the paper's Tc23 figure: J + 1 = 48 latitudes of 3.75 degrees, 30 N at
    # row 16: 6 j points up to row 16, 96 on every tropical row, tropical
    # rows alternately shifted by half a spacing from row 16 (unshifted)
    Ij, sh = O.icositetrahedral_sizes(47)
    assert Ij[:16].tolist() == [6 * j for j in range(1, 17)]
    assert np.all(Ij[15:32] == 96)
    assert np.array_equal(Ij, Ij[::-1]) and np.array_equal(sh, sh[::-1])
    assert np.all(sh[:16] == 0.0)
    assert sh[16:24].tolist() == [0.5, 0.0, 0.5, 0.0, 0.5, 0.0, 0.5, 0.0]
    # 6 j30 points on the tropical rows: twice the J + 1 latitude spacings,
    # the count of the cubic regular grid, I = 2 (J + 1)
    assert Ij[23] == 2 * 48


def test_shifted_rows_match_scipy_harmonics():
    # synthesis on the icositetrahedral grid (shifted tropical rows) against
    # SciPy's spherical harmonics evaluated at each row's own longitudes, row
    # j summing the wavenumbers it carries, m <= min(N, I_j/2 - 1)
    J, N = 23, 5
    Ij, sh = O.icositetrahedral_sizes(J)
    a = W.random_spectrum(N, 1, "n^-1.5", seed=61)[:, 0]
    th = O.cc_nodes(J)[0]
    ref = []
    for j in range(J):
        lam = 2 * np.pi * (np.arange(Ij[j]) + sh[j]) / Ij[j]
        row = np.zeros(Ij[j])
        r = 0
        for m in range(N + 1):
            for n in range(m, N + 1):
                if m <= min(N, Ij[j] // 2 - 1):
                    y = np.sqrt(2 * np.pi) * (-1) ** m * special.sph_harm_y(n, m, th[j], lam)
                    row += (a[r].real * y).real if m == 0 else 2 * (a[r] * y).real
                r += 1
        ref.append(row)
    got = O.synthesis_reduced(a[:, None], N, J, Ij, shifts=sh)[0]
    np.testing.assert_allclose(got, np.concatenate(ref), atol=1e-13)
    # and the shift matters: without it the tropical rows differ
    plain = O.synthesis_reduced(a[:, None], N, J, Ij)[0]
    assert np.abs(plain - got).max() > 1e-3


def test_shifted_grid_round_trip_is_exact():
    # every row of the Tc23 icositetrahedral grid carries m <= 2 (6 points
    # at the first row) and J >= 2N+1: the transform pair is exact
    J, N = 47, 2
    Ij, sh = O.icositetrahedral_sizes(J)
    a = W.random_spectrum(N, 3, "n^-1.5", seed=62)
    g = O.synthesis_reduced(a, N, J, Ij, shifts=sh)
    np.testing.assert_allclose(O.analysis_reduced(g, N, J, Ij, shifts=sh), a, atol=1e-14)
    # the octahedral grid likewise for N = 9 (20 points at the first row)
    Io = O.octahedral_sizes(J)
    a = W.random_spectrum(9, 2, "n^-1.5", seed=63)
    g = O.synthesis_reduced(a, 9, J, Io)
    np.testing.assert_allclose(O.analysis_reduced(g, 9, J, Io), a, atol=1e-14)

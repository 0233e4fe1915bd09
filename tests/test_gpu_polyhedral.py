"""Octahedral and icositetrahedral Clenshaw-Curtis grids (Sec. 6) on the GPU.
Their row counts have half-lengths with prime factors above 5, which the
library transforms by Bluestein's chirp-z method, and the icositetrahedral
tropical rows are shifted by half a spacing (a zonal phase per row).
Checked against the oracle's reduced-grid transforms with the same counts
and shifts (FP64 element by element, split paths by relative L2), by exact
round trips of band-limited fields, and by the adjoint identities."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SPLIT_TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6}


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _grid(sht, kind, J):
    if kind == "octahedral":
        return sht.octahedral_grid_sizes(J), None
    return sht.icositetrahedral_grid_sizes(J)


def _oracle_shift(sh):
    return None if sh is None else np.array(sh) * 0.5


@pytest.mark.parametrize("kind", ["octahedral", "icositetrahedral"])
@pytest.mark.parametrize("N,J,F", [(23, 47, 3), (47, 95, 2), (159, 321, 4)])
def test_fp64_matches_oracle(sht, kind, N, J, F):
    pts, sh = _grid(sht, kind, J)
    if max(pts) <= 2 * N:
        pytest.skip("the widest row does not exceed 2N")
    p = sht.Plan(N, J, 0, F, "fp64", grid="reduced", lat_points=pts, half_shift=sh)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1900 + N)
    g = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    assert_fp64_close(g, O.synthesis_reduced(a, N, J, pts, shifts=_oracle_shift(sh)))
    x = W.random_grid(F, 1, sum(pts), seed=1901 + N)[:, 0, :]
    s = p.forward(to_cuda(x, torch.float64)).cpu().numpy()
    assert_fp64_close(s, O.analysis_reduced(x, N, J, pts, shifts=_oracle_shift(sh)))
    p.status()


@pytest.mark.parametrize("kind", ["octahedral", "icositetrahedral"])
@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("N,J,F", [(47, 95, 5), (159, 321, 3)])
def test_split_matches_oracle(sht, kind, prec, N, J, F):
    pts, sh = _grid(sht, kind, J)
    p = sht.Plan(N, J, 0, F, prec, grid="reduced", lat_points=pts, half_shift=sh)
    x = W.random_grid(F, 1, sum(pts), seed=1910 + N)[:, 0, :]
    x = x.astype(np.float32).astype(np.float64)
    s = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    ref = O.analysis_reduced(x, N, J, pts, shifts=_oracle_shift(sh))
    assert rel_l2(s, ref) <= SPLIT_TOL[prec], rel_l2(s, ref)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1911 + N).astype(np.complex64)
    g = p.inverse(torch.from_numpy(a).cuda()).cpu().numpy()
    ref = O.synthesis_reduced(a.astype(np.complex128), N, J, pts, shifts=_oracle_shift(sh))
    assert rel_l2(g, ref) <= SPLIT_TOL[prec], rel_l2(g, ref)
    p.status()


def test_band_limited_round_trips_are_exact(sht):
    # every row of the J = 47 icositetrahedral grid carries m <= 2 and every
    # row of the octahedral grid m <= 9: the pairs are exact there
    J = 47
    for kind, N in (("icositetrahedral", 2), ("octahedral", 9)):
        pts, sh = _grid(sht, kind, J)
        p = sht.Plan(N, J, 0, 3, "fp64", grid="reduced", lat_points=pts, half_shift=sh)
        a = W.random_spectrum(N, 3, "n^-1.5", seed=1920)
        back = p.forward(p.inverse(to_cuda(a, torch.complex128))).cpu().numpy()
        assert rel_l2(back, a) < 1e-13, (kind, rel_l2(back, a))
        p.status()


@pytest.mark.parametrize("kind", ["octahedral", "icositetrahedral"])
def test_adjoint_dot_products(sht, kind):
    N, J, F = 31, 65, 2
    pts, sh = _grid(sht, kind, J)
    p = sht.Plan(N, J, 0, F, "fp64", grid="reduced", lat_points=pts, half_shift=sh)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1930)
    a[:N + 1] = a[:N + 1].real
    x = W.random_grid(F, 1, sum(pts), seed=1931)[:, 0, :]
    ta, tx = to_cuda(a, torch.complex128), to_cuda(x, torch.float64)
    lhs = float(np.sum(p.inverse(ta).cpu().numpy() * x))
    rhs = float(np.sum((np.conj(a) * p.adjoint(1, tx).cpu().numpy()).real))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    lhs = float(np.sum((np.conj(p.forward(tx).cpu().numpy()) * a).real))
    rhs = float(np.sum(x * p.adjoint(0, ta).cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    p.status()


def test_shift_is_a_rotation_of_the_row(sht):
    # a shifted grid whose every row has the same count I: its synthesis is
    # the unshifted synthesis of the field rotated west by half a spacing,
    # i.e. X_n^m e^{i m pi / I}
    N, J, I, F = 15, 31, 34, 2        # I/2 = 17: Bluestein rows
    pts = [I] * J
    sh = [1] * J
    p = sht.Plan(N, J, 0, F, "fp64", grid="reduced", lat_points=pts, half_shift=sh)
    q = sht.Plan(N, J, 0, F, "fp64", grid="reduced", lat_points=pts)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1940)
    m = W.order_of_rows(N)
    rot = a * np.exp(1j * np.pi * m / I)[:, None]
    g1 = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    g2 = q.inverse(to_cuda(rot, torch.complex128)).cpu().numpy()
    assert_fp64_close(g1, g2)

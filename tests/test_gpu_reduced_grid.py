"""Reduced Clenshaw-Curtis grids (a longitude count I_j per latitude, by the
reduction rule quoted in Sec. 6) on the GPU: the size rule against the
oracle's, FP64 and split transforms against the oracle on the rule's grids
and on a hand-made grid whose polar rows cut the spectrum below N, the exact
FP64 round trip, the adjoint identities, the full-count special case against
the regular plan, and the rejected requests."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SPLIT_TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6}
# longitude counts whose half-length has a compile-time FFT kernel
FAST_COUNTS = [128, 256, 512, 640, 1024, 1280, 2048, 2560]


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _rule(sht, N, J, I, rule="smooth"):
    full = sht.Plan(N, J, I, 1, "fp64")
    return full.reduced_grid_sizes(rule)


def _hand_grid(J, I):
    # the six rows nearest each pole have half-lengths 5, 9, 10, 12, 15, 18
    # (odd ones included) and carry the wavenumbers up to 4, 8, 9, 11, 14, 15;
    # the other rows have I longitudes
    head = [10, 18, 20, 24, 30, 36]
    pts = head + [I] * (J - 2 * len(head)) + head[::-1]
    assert len(pts) == J
    return pts


@pytest.mark.parametrize("rule", ["smooth", "fast"])
@pytest.mark.parametrize("N,J,I", [(31, 65, 128), (63, 129, 256), (159, 321, 640)])
def test_sizes_match_oracle(sht, rule, N, J, I):
    got = _rule(sht, N, J, I, rule)
    want, _ = O.reduced_sizes(N, J, I, counts=FAST_COUNTS if rule == "fast" else None)
    assert got == [int(v) for v in want]


@pytest.mark.parametrize("rule", ["smooth", "fast"])
@pytest.mark.parametrize("N,J,I,F", [(31, 65, 128, 3), (63, 129, 256, 2)])
def test_fp64_rule_grid_matches_oracle(sht, rule, N, J, I, F):
    pts = _rule(sht, N, J, I, rule)
    p = sht.Plan(N, J, I, F, "fp64", grid="reduced", lat_points=pts)
    assert p.npts == sum(pts) and p.grid_shape == (F, sum(pts))
    a = W.random_spectrum(N, F, "n^-1.5", seed=1800 + N)
    g = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    assert_fp64_close(g, O.synthesis_reduced(a, N, J, pts))
    x = W.random_grid(F, 1, sum(pts), seed=1801 + N)[:, 0, :]
    s = p.forward(to_cuda(x, torch.float64)).cpu().numpy()
    assert_fp64_close(s, O.analysis_reduced(x, N, J, pts))
    # band-limited round trip: exact to rounding on the rule's grid
    a[:N + 1] = a[:N + 1].real
    back = p.forward(p.inverse(to_cuda(a, torch.complex128))).cpu().numpy()
    assert rel_l2(back, a) < 1e-13
    p.status()


def test_fp64_hand_grid_cuts_the_spectrum(sht):
    # polar rows with I_j/2 - 1 < N keep only their own wavenumbers
    N, J, I, F = 15, 31, 40, 3
    pts = _hand_grid(J, I)
    p = sht.Plan(N, J, I, F, "fp64", grid="reduced", lat_points=pts)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1810)
    g = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    assert_fp64_close(g, O.synthesis_reduced(a, N, J, pts))
    x = W.random_grid(F, 1, sum(pts), seed=1811)[:, 0, :]
    s = p.forward(to_cuda(x, torch.float64)).cpu().numpy()
    assert_fp64_close(s, O.analysis_reduced(x, N, J, pts))
    p.status()


@pytest.mark.parametrize("rule", ["smooth", "fast"])
@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("N,J,I,F", [(63, 129, 256, 5), (159, 321, 640, 4)])
def test_split_rule_grid_matches_oracle(sht, rule, prec, N, J, I, F):
    # the fast rule's rows all run compile-time kernels (at T159 the
    # register-fed first and last passes of L = 256 and 320 included); the
    # smooth rule's mix them with the generic kernel
    pts = _rule(sht, N, J, I, rule)
    p = sht.Plan(N, J, I, F, prec, grid="reduced", lat_points=pts)
    x = W.random_grid(F, 1, sum(pts), seed=1820 + N)[:, 0, :]
    x = x.astype(np.float32).astype(np.float64)
    s = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(s, O.analysis_reduced(x, N, J, pts)) <= SPLIT_TOL[prec]
    a = W.random_spectrum(N, F, "n^-1.5", seed=1821 + N).astype(np.complex64)
    g = p.inverse(torch.from_numpy(a).cuda()).cpu().numpy()
    ref = O.synthesis_reduced(a.astype(np.complex128), N, J, pts)
    assert rel_l2(g, ref) <= SPLIT_TOL[prec]
    p.status()


def test_adjoint_dot_products(sht):
    # <inverse(a), x> = <a, adjoint_1(x)> and <forward(x), a> = <x, adjoint_0(a)>
    N, J, I, F = 31, 65, 128, 2
    pts = _rule(sht, N, J, I)
    p = sht.Plan(N, J, I, F, "fp64", grid="reduced", lat_points=pts)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1830)
    a[:N + 1] = a[:N + 1].real
    x = W.random_grid(F, 1, sum(pts), seed=1831)[:, 0, :]
    ta, tx = to_cuda(a, torch.complex128), to_cuda(x, torch.float64)
    lhs = float(np.sum(p.inverse(ta).cpu().numpy() * x))
    rhs = float(np.sum((np.conj(a) * p.adjoint(1, tx).cpu().numpy()).real))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    lhs = float(np.sum((np.conj(p.forward(tx).cpu().numpy()) * a).real))
    rhs = float(np.sum(x * p.adjoint(0, ta).cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_full_counts_equal_the_regular_plan(sht, prec):
    N, J, I, F = 63, 129, 256, 3
    r = sht.Plan(N, J, I, F, prec)
    p = sht.Plan(N, J, I, F, prec, grid="reduced", lat_points=[I] * J)
    x = to_cuda(W.random_grid(F, J, I, seed=1840), r.real_dtype)
    a = to_cuda(W.random_spectrum(N, F, "n^-1.5", seed=1841), r.complex_dtype)
    tol = 1e-14 if prec == "fp64" else 1e-7
    assert rel_l2(p.forward(x.reshape(F, -1)).cpu().numpy(), r.forward(x).cpu().numpy()) < tol
    assert rel_l2(p.inverse(a).cpu().numpy(), r.inverse(a).reshape(F, -1).cpu().numpy()) < tol


def test_rejected_requests(sht):
    N, J, I = 15, 31, 40
    pts = _hand_grid(J, I)
    bad = [
        pts[:-1] + [16],                           # not symmetric
        [p + 1 if p == 18 else p for p in pts],    # odd count
        [min(p, 30) for p in pts],                 # the widest row does not exceed 2N
        pts[:-1],                                  # J - 1 entries
    ]
    for b in bad:
        with pytest.raises((sht.SHTError, ValueError)):
            sht.Plan(N, J, I, 1, "fp64", grid="reduced", lat_points=b)
    p = sht.Plan(N, J, I, 1, "fp64", grid="reduced", lat_points=pts)
    fine = torch.zeros((1, 2 * (J + 1) - 1, 2 * p.I), dtype=torch.float64, device="cuda")
    with pytest.raises(sht.SHTError) as ei:
        p.restrict_nested(fine, 1)
    assert ei.value.code == -4
    with pytest.raises(sht.SHTError) as ei:
        sht.Group([p])
    assert ei.value.code == -7
    with pytest.raises(ValueError):
        sht.Plan(N, J, I, 1, "fp64", lat_points=pts)
    with pytest.raises(ValueError):
        sht.Plan(N, J, I, 1, "fp64").reduced_grid_sizes("octahedral")

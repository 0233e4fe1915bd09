"""Quadratic and cubic terms of the aliasing experiment (Sec. 4.2) on the
GPU: synthesis of U, V and W, the products U V and U V W formed inside W's
inverse FFT, and the analyses of both, against the oracle's product
pipeline (FP64 element by element; split paths by relative L2, where the
three synthesised fields' errors add up in the products), and at the
paper's size Tc479 (N = 479, J = 959, I = 1920) by a property that holds at
any size: for U, V, W band-limited to N/3 the cubic term is band-limited to
N, so its analysis is exact and its synthesis returns U V W point by point."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SPLIT_TOL = {"bf16x3": 2e-6, "fp16x2": 4e-6}


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _uvw(N, F, seed):
    return [W.random_spectrum(N, F, "uniform^-1/3", seed=seed + k) for k in range(3)]


@pytest.mark.parametrize("N,J,I,F", [(31, 65, 128, 2), (23, 47, 96, 3), (47, 95, 192, 1)])
def test_alias_products_fp64_match_oracle(sht, N, J, I, F):
    p = sht.Plan(N, J, I, F, "fp64")
    U, V, Wv = _uvw(N, F, 2000 + N)
    q, c = p.alias_products(*(to_cuda(a, torch.complex128) for a in (U, V, Wv)))
    rq, rc = O.aliasing_products(U, V, Wv, N, J, I)
    assert_fp64_close(q.cpu().numpy(), rq)
    assert_fp64_close(c.cpu().numpy(), rc)
    p.status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("N,J,I,F", [(31, 65, 128, 3), (63, 127, 256, 2)])
def test_alias_products_split_match_oracle(sht, prec, N, J, I, F):
    p = sht.Plan(N, J, I, F, prec)
    U, V, Wv = [a.astype(np.complex64).astype(np.complex128) for a in _uvw(N, F, 2100 + N)]
    grids = [p.empty_grid(), p.empty_grid()]
    q, c = p.alias_products(*(to_cuda(a, torch.complex64) for a in (U, V, Wv)), grids=grids)
    rq, rc = O.aliasing_products(U, V, Wv, N, J, I)
    assert rel_l2(q.cpu().numpy(), rq) <= SPLIT_TOL[prec], rel_l2(q.cpu().numpy(), rq)
    assert rel_l2(c.cpu().numpy(), rc) <= SPLIT_TOL[prec], rel_l2(c.cpu().numpy(), rc)
    # the work grids hold U V and U V W
    gu, gv, gw = (O.synthesis(a, N, J, I) for a in (U, V, Wv))
    assert rel_l2(grids[0].cpu().numpy(), gu * gv) <= SPLIT_TOL[prec]
    assert rel_l2(grids[1].cpu().numpy(), gu * gv * gw) <= SPLIT_TOL[prec]
    p.status()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 2e-6)])
def test_alias_products_tc479_band_limited_cubic_term_is_exact(sht, prec, tol):
    N, J, I, F = 479, 959, 1920, 8
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    p = sht.Plan(N, J, I, F, prec)
    Nb = N // 3
    specs = []
    for k in range(3):
        a = np.zeros((O.ncoef(N), F), dtype=np.complex128)
        b = W.random_spectrum(Nb, F, "uniform^-1/3", seed=2200 + k)
        for m in range(Nb + 1):
            a[O.coef_offset(N, m):O.coef_offset(N, m) + Nb - m + 1] = \
                b[O.coef_offset(Nb, m):O.coef_offset(Nb, m) + Nb - m + 1]
        specs.append(to_cuda(a, cd))
    grids = [p.empty_grid(), p.empty_grid()]
    q, c = p.alias_products(*specs, grids=grids)
    # U V W is band-limited to N: the analysis is exact, so synthesising the
    # cubic term's spectrum returns the grid products point by point
    back_c = p.inverse(c).cpu().numpy()
    back_q = p.inverse(q).cpu().numpy()
    assert rel_l2(back_c, grids[1].cpu().numpy()) <= tol
    assert rel_l2(back_q, grids[0].cpu().numpy()) <= tol
    p.status()

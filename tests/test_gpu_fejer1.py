"""The shifted grid of Fejer's first rule (Sec. 3.3) on the GPU: plan tables,
FP64 and split transforms against the oracle, the FP64 round trip, the
adjoint dot-product identity and the rejection of nested restriction."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SPLIT_TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6}
CASES = [(0, 1, 2, 2), (7, 15, 16, 3), (31, 65, 128, 5), (63, 129, 256, 4)]


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


@pytest.mark.parametrize("J", [1, 15, 65, 641])
def test_tables_match_oracle(sht, J):
    p = sht.Plan(7 if J > 1 else 0, J, 16, 1, "fp64", grid="fejer1")
    w, mu, _ = p.tables()
    _, mu_ref, _ = O.fejer1_nodes(J)
    np.testing.assert_allclose(w, O.fejer1_weights(J), rtol=0, atol=2e-15)
    np.testing.assert_allclose(mu, mu_ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N,J,I,F", CASES)
def test_fp64_forward_inverse_match_oracle(sht, N, J, I, F):
    p = sht.Plan(N, J, I, F, "fp64", grid="fejer1")
    x = W.random_grid(F, J, I, seed=1500 + N)
    assert_fp64_close(p.forward(to_cuda(x, torch.float64)).cpu().numpy(),
                      O.analysis_fejer1(x, N))
    a = W.random_spectrum(N, F, "n^-1.5", seed=1510 + N)
    assert_fp64_close(p.inverse(to_cuda(a, torch.complex128)).cpu().numpy(),
                      O.synthesis_fejer1(a, N, J, I))
    # J >= 2N+1: the round trip is exact to rounding
    back = p.forward(p.inverse(to_cuda(a, torch.complex128))).cpu().numpy()
    a0 = a.copy()
    a0[:N + 1] = a0[:N + 1].real
    assert rel_l2(back, a0) < 1e-13
    p.status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("N,J,I,F", [(31, 65, 128, 5), (159, 321, 640, 17)])
def test_split_matches_oracle(sht, prec, N, J, I, F):
    p = sht.Plan(N, J, I, F, prec, grid="fejer1")
    x = W.random_grid(F, J, I, seed=1520 + N).astype(np.float32).astype(np.float64)
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(got, O.analysis_fejer1(x, N)) <= SPLIT_TOL[prec]
    a = W.random_spectrum(N, F, "n^-1.5", seed=1530 + N).astype(np.complex64)
    g = p.inverse(torch.from_numpy(a).cuda()).cpu().numpy()
    ref = O.synthesis_fejer1(a.astype(np.complex128), N, J, I)
    assert rel_l2(g, ref) <= SPLIT_TOL[prec]
    p.status()


def test_adjoint_dot_products(sht):
    # <inverse(a), x> = <a, adjoint_1(x)> and <forward(x), a> = <x, adjoint_0(a)>
    # for the plain inner products the adjoints are defined by.
    N, J, I, F = 31, 65, 128, 3
    p = sht.Plan(N, J, I, F, "fp64", grid="fejer1")
    a = W.random_spectrum(N, F, "n^-1.5", seed=1540)
    a[:N + 1] = a[:N + 1].real
    x = W.random_grid(F, J, I, seed=1541)
    ta, tx = to_cuda(a, torch.complex128), to_cuda(x, torch.float64)
    lhs = float(np.sum(p.inverse(ta).cpu().numpy() * x))
    rhs = float(np.sum((np.conj(a) * p.adjoint(1, tx).cpu().numpy()).real))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    lhs = float(np.sum((np.conj(p.forward(tx).cpu().numpy()) * a).real))
    rhs = float(np.sum(x * p.adjoint(0, ta).cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_restriction_is_rejected(sht):
    p = sht.Plan(7, 15, 16, 1, "fp64", grid="fejer1")
    fine = torch.zeros((1, 31, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(sht.SHTError):
        p.restrict_nested(fine, 1)
    with pytest.raises(ValueError):
        sht.Plan(7, 15, 16, 1, "fp64", grid="fejer2")

"""FP32 FFT lengths L = Q x 32 with Q >= 8, where the forward's first pass
reads the grid rows into registers and the inverse's last pass stores
straight to the grid rows: every such radix Q (8, 10, 16, 20) against the
oracle, partial field groups, the adjoints (which run the same kernels with
other row scales), and launch shapes whose first pass takes several rounds
per thread, compared bit for bit with the default shape."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6}

# (N, J, I, F): L = I/2 = 256 (Q = 8), 320 (Q = 10), 512 (Q = 16), 640 (Q = 20)
CASES = [
    (127, 257, 512, 6),
    (159, 321, 640, 5),
    (255, 513, 1024, 3),
    (319, 641, 1280, 2),
]


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _f32(a):
    return np.asarray(a).astype(np.float32).astype(np.float64)


def _c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


_REF = {}


def _case(N, J, I, F):
    """Seeded inputs of a case and their oracle transforms, computed once."""
    key = (N, J, I, F)
    if key not in _REF:
        x = _f32(W.random_grid(F, J, I, seed=1600 + N))
        a = _c64(W.random_spectrum(N, F, "n^-1.5", seed=1610 + N))
        _REF[key] = (x, a, O.analysis(x, N), O.synthesis(a, N, J, I))
    return _REF[key]


@pytest.mark.parametrize("N,J,I,F", CASES)
@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
def test_fused_lengths_match_oracle(sht, prec, N, J, I, F):
    x, a, sref, gref = _case(N, J, I, F)
    p = sht.Plan(N, J, I, F, prec)
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(got, sref) <= TOL[prec]
    assert np.all(got[:N + 1].imag == 0.0)
    g = p.inverse(to_cuda(a, torch.complex64)).cpu().numpy()
    assert rel_l2(g, gref) <= TOL[prec]
    p.status()


@pytest.mark.parametrize("N,J,I,F", [(127, 257, 512, 3), (159, 321, 640, 5)])
def test_fused_lengths_adjoints(sht, N, J, I, F):
    p = sht.Plan(N, J, I, F, "bf16x3")
    a = _c64(W.random_spectrum(N, F, "n^-1.5", seed=1620 + N))
    x = _f32(W.random_grid(F, J, I, seed=1621 + N))
    g0 = p.adjoint(0, to_cuda(a, torch.complex64)).cpu().numpy()
    assert rel_l2(g0, O.adjoint_analysis(a, N, J, I)) <= 1e-6
    g1 = p.adjoint(1, to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(g1, O.adjoint_synthesis(x, N)) <= 1e-6
    p.status()


def test_fused_lengths_shapes_do_not_change_results(sht):
    # With 12 or 16 fields per CTA the forward's first pass runs 768 or
    # 1024 butterflies on 256 threads (several rounds per thread), and the
    # inverse's last pass 960 or 1280; 1 and 3 fields leave threads idle.
    N, J, I, F = 159, 321, 640, 16
    p = sht.Plan(N, J, I, F, "bf16x3")
    x = to_cuda(W.random_grid(F, J, I, seed=1631), torch.float32)
    a = to_cuda(W.random_spectrum(N, F, "n^-1.5", seed=1632), torch.complex64)
    s0 = p.forward(x).clone()
    g0 = p.inverse(a).clone()
    for G in (1, 3, 12, 16):
        p.set_tuning(fields_per_cta=G)
        assert torch.equal(p.forward(x), s0), G
        assert torch.equal(p.inverse(a), g0), G
    ref = O.analysis(x.cpu().numpy().astype(np.float64), N)
    assert rel_l2(s0.cpu().numpy(), ref) <= 1e-6
    p.status()

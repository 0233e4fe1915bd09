"""Reduced transform (Sec. 4.1): split plans that neglect |P~| < 1e-16 per
tile give the full transform's results to far below the split tolerance,
alone and in a group, and match the oracle within it."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6}


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
@pytest.mark.parametrize("N,J,I,F", [(63, 129, 256, 5), (159, 321, 640, 17), (319, 641, 1280, 4)])
def test_reduced_matches_full_and_oracle(sht, prec, N, J, I, F):
    full = sht.Plan(N, J, I, F, prec)
    red = sht.Plan(N, J, I, F, prec)
    red.set_reduced(True)
    x = W.random_grid(F, J, I, seed=1600 + N).astype(np.float32).astype(np.float64)
    a = W.random_spectrum(N, F, "energy^-2", seed=1601 + N).astype(np.complex64)
    tx, ta = to_cuda(x, torch.float32), torch.from_numpy(a).cuda()
    s_full, s_red = full.forward(tx).cpu().numpy(), red.forward(tx).cpu().numpy()
    g_full, g_red = full.inverse(ta).cpu().numpy(), red.inverse(ta).cpu().numpy()
    # the neglected terms are below 1e-16 of P~'s scale
    assert rel_l2(s_red, s_full) < 1e-9
    assert rel_l2(g_red, g_full) < 1e-9
    assert rel_l2(s_red, O.analysis(x, N)) <= TOL[prec]
    if N <= 159:
        assert rel_l2(g_red, O.synthesis(a.astype(np.complex128), N, J, I)) <= TOL[prec]
    # switching it off restores the full sums exactly
    red.set_reduced(False)
    assert np.array_equal(red.forward(tx).cpu().numpy(), s_full)
    red.status()
    full.status()


def test_reduced_in_a_group(sht):
    cfg = [(63, 129, 256, 3), (127, 257, 512, 2)]
    plans = [sht.Plan(N, J, I, F, "bf16x3") for N, J, I, F in cfg]
    for p in plans:
        p.set_reduced(True)
    grp = sht.Group(plans)
    specs = [torch.from_numpy(W.random_spectrum(N, F, "energy^-2", seed=1610 + k)
                              .astype(np.complex64)).cuda()
             for k, (N, J, I, F) in enumerate(cfg)]
    outs = grp.inverse(specs)
    for p, a, g in zip(plans, specs, outs):
        assert torch.equal(g, p.inverse(a))


@pytest.mark.parametrize("N,J,I,F", [(63, 129, 256, 3), (319, 641, 1280, 2)])
def test_fp64_reduced_matches_full_and_oracle(sht, N, J, I, F):
    full = sht.Plan(N, J, I, F, "fp64")
    red = sht.Plan(N, J, I, F, "fp64")
    red.set_reduced(True)
    x = to_cuda(W.random_grid(F, J, I, seed=1620 + N), torch.float64)
    a = to_cuda(W.random_spectrum(N, F, "energy^-2", seed=1621 + N), torch.complex128)
    s_full, s_red = full.forward(x).cpu().numpy(), red.forward(x).cpu().numpy()
    g_full, g_red = full.inverse(a).cpu().numpy(), red.inverse(a).cpu().numpy()
    # the neglected terms are below 1e-16 of P~'s scale: FP64 rounding level
    assert rel_l2(s_red, s_full) < 1e-14
    assert rel_l2(g_red, g_full) < 1e-14
    if N <= 63:
        assert rel_l2(s_red, O.analysis(x.cpu().numpy(), N)) < 1e-12
    red.set_reduced(False)
    assert np.array_equal(red.forward(x).cpu().numpy(), s_full)
    red.status()

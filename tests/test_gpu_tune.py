"""Launch shapes and the autotuner: the FFT's fields per CTA and the split
GEMMs' column-tile width change speed, never results.  Outputs under every
shape are compared bit for bit with the default shape, and against the
oracle within the split tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SPLIT_TOL = {"bf16x3": 1e-6, "fp16x2": 2e-6, "bf16x2": 5e-5, "fp16x3": 1e-6}


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _pair(p, x, a):
    s = p.forward(x)
    g = p.inverse(a)
    torch.cuda.synchronize()
    return s.clone(), g.clone()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2", "fp64"])
def test_shapes_do_not_change_results(sht, prec):
    N, J, I, F = 63, 129, 256, 19
    p = sht.Plan(N, J, I, F, prec)
    x = to_cuda(W.random_grid(F, J, I, seed=1301), p.real_dtype)
    a = to_cuda(W.random_spectrum(N, F, "n^-1.5", seed=1302), p.complex_dtype)
    s0, g0 = _pair(p, x, a)
    widths = [0] if prec == "fp64" else [64, 128]
    for tn in widths:
        for G in (1, 3, 7, F):
            p.set_tuning(fields_per_cta=G, tile_width=tn)
            assert p.tuning["fields_per_cta"] == G
            if tn:
                assert p.tuning["tile_width"] == tn
            s, g = _pair(p, x, a)
            assert torch.equal(s, s0), (G, tn)
            assert torch.equal(g, g0), (G, tn)
    p.status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
def test_tile_width_64_matches_oracle(sht, prec):
    N, J, I, F = 159, 321, 640, 33
    p = sht.Plan(N, J, I, F, prec)
    p.set_tuning(tile_width=64)
    x = W.random_grid(F, J, I, seed=1311).astype(np.float32).astype(np.float64)
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(got, O.analysis(x, N)) <= SPLIT_TOL[prec]
    a = W.random_spectrum(N, F, "n^-1.5", seed=1312).astype(np.complex64)
    g = p.inverse(torch.from_numpy(a).cuda()).cpu().numpy()
    assert rel_l2(g, O.synthesis(a.astype(np.complex128), N, J, I)) <= SPLIT_TOL[prec]
    p.status()


def test_autotune_chooses_applies_and_remembers(sht):
    N, J, I, F = 31, 65, 128, 7
    p = sht.Plan(N, J, I, F, "bf16x3")
    r = p.autotune(reps=2)
    assert 1 <= r["fields_per_cta"] <= F
    assert r["tile_width"] in (64, 128)
    assert r["ms_per_pair"] > 0
    assert p.tuning == {"fields_per_cta": r["fields_per_cta"], "tile_width": r["tile_width"]}
    x = W.random_grid(F, J, I, seed=1321).astype(np.float32).astype(np.float64)
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(got, O.analysis(x, N)) <= 1e-6
    # a second plan of the same shape takes the remembered choice
    q = sht.Plan(N, J, I, F, "bf16x3")
    assert q.autotune(reps=2) == r
    assert q.tuning == p.tuning
    # FP64: fields per CTA only
    f = sht.Plan(N, J, I, F, "fp64")
    rf = f.autotune(reps=1)
    assert rf["tile_width"] == 0 and 1 <= rf["fields_per_cta"] <= F
    xd = to_cuda(W.random_grid(F, J, I, seed=1322), torch.float64)
    assert_fp64_close(f.forward(xd).cpu().numpy(), O.analysis(xd.cpu().numpy(), N))


def test_tuning_arguments_and_groups(sht):
    p = sht.Plan(15, 31, 32, 4, "bf16x3")
    q = sht.Plan(15, 31, 32, 4, "bf16x3")
    d = sht.Plan(15, 31, 32, 4, "fp64")
    for G in (-1, 5, 65):
        with pytest.raises(sht.SHTError):
            p.set_tuning(fields_per_cta=G)
    for tn in (-64, 32, 96, 256):
        with pytest.raises(sht.SHTError):
            p.set_tuning(tile_width=tn)
    with pytest.raises(sht.SHTError):
        d.set_tuning(tile_width=64)
    assert p.tuning == {"fields_per_cta": p.tuning["fields_per_cta"], "tile_width": 128}
    # plans of a group share the tile width, and keep it while the group lives
    q.set_tuning(tile_width=64)
    with pytest.raises(sht.SHTError):
        sht.Group([p, q])
    q.set_tuning(tile_width=128)
    grp = sht.Group([p, q])
    x = [to_cuda(W.random_grid(4, 31, 32, seed=1330 + k), torch.float32) for k in range(2)]
    grp.forward(x)
    q.set_tuning(tile_width=64)
    with pytest.raises(sht.SHTError):
        grp.forward(x)

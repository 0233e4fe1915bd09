"""FP64 GPU path at the full workload sizes (T159 x 256 field-levels, T639 x
256, the nested ladder T511 -> T255 -> T127 x 64), in the launch
configuration the benchmark times.  T159 is compared element by element;
T639 and the ladder on sampled zonal wavenumbers, latitudes and fields that
the oracle computes one by one, plus the exact round trip over everything."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _grid(F, J, I):
    return np.stack([W.random_grid_field(f, J, I) for f in range(F)])


def test_t159_full(sht):
    w = W.WORKLOADS["T159"]
    p = sht.Plan(w.N, w.J, w.I, w.F, "fp64")
    x = _grid(w.F, w.J, w.I)
    got = p.forward(to_cuda(x, torch.float64)).cpu().numpy()
    assert_fp64_close(got, O.analysis(x, w.N))
    a = W.workload_spectrum(w)
    got = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    assert_fp64_close(got, O.synthesis(a, w.N, w.J, w.I))


def test_t639_sampled(sht):
    w = W.WORKLOADS["T639"]
    p = sht.Plan(w.N, w.J, w.I, w.F, "fp64")
    fields = [0, 1, 130, 255]
    ms = [0, 1, 2, 101, 319, 320, 501, 638, 639]
    x = _grid(w.F, w.J, w.I)
    spec = p.forward(to_cuda(x, torch.float64))
    torch.cuda.synchronize()
    got = spec.cpu().numpy()
    ref = O.analysis(x[fields], w.N, ms=ms)
    del x
    for m in ms:
        r0 = O.coef_offset(w.N, m)
        assert_fp64_close(got[r0:r0 + w.N - m + 1][:, fields], ref[m])
    # synthesis at sampled latitudes (1-based rows), all longitudes
    a = W.workload_spectrum(w)
    ta = to_cuda(a, torch.complex128)
    grid = p.inverse(ta).cpu().numpy()
    rows = [1, 2, 320, 640, 641, 642, 1000, 1280, 1281]
    ref = O.synthesis_rows(a[:, fields], w.N, w.J, w.I, rows)
    assert_fp64_close(grid[fields][:, np.array(rows) - 1, :], ref)
    # exact round trip over every coefficient (J >= 2N+1, I > 2N)
    back = p.forward(to_cuda(grid, torch.float64)).cpu().numpy()
    assert_fp64_close(back, a)


def test_nested_ladder_sampled(sht):
    fine_w, mid_w, coarse_w = W.LADDER
    F = fine_w.F
    x = _grid(F, fine_w.J, fine_w.I)
    tx = to_cuda(x, torch.float64)
    fields = [0, 33, 63]
    for k, cw in ((1, mid_w), (2, coarse_w)):
        p = sht.Plan(cw.N, cw.J, cw.I, F, "fp64")
        got = p.restrict_nested(tx, k).cpu().numpy()
        s = 2 ** k
        sub = x[fields][:, O.nested_rows(cw.J, k) - 1, ::s]
        ms = [0, 1, cw.N // 2, cw.N]
        ref = O.analysis(sub, cw.N, ms=ms)
        for m in ms:
            r0 = O.coef_offset(cw.N, m)
            assert_fp64_close(got[r0:r0 + cw.N - m + 1][:, fields], ref[m])

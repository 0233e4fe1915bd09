"""Per-stage instrumentation: every stage of a transform pair is timed once
per call, and the kernels launched inside it are counted (the split inverse
Legendre stage is the spectrum split plus the GEMM; a reduced grid's FFT
stage is one launch per row-length class with a compile-time kernel plus one
generic launch for the rest)."""
import pytest
import torch

from paper_1711_11296_gb300 import workloads as W
from sht_testutil import built_lib, to_cuda

pytestmark = pytest.mark.gpu

FIXED_HALF_LENGTHS = {64, 128, 256, 320, 512, 640, 1024, 1280}


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _pair_profile(p, reps):
    a = to_cuda(W.random_spectrum(p.N, p.F, "n^-1.5", seed=1900), p.complex_dtype)
    g = p.empty_grid()
    s = p.empty_spec()
    p.profile(True)
    for _ in range(reps):
        p.inverse(a, out=g)
        p.forward(g, out=s)
    torch.cuda.synchronize()
    p.profile(False)
    return p.profile_read(kernels=True)


@pytest.mark.parametrize("prec,inv_kernels", [("fp64", 1), ("bf16x3", 2), ("fp16x2", 3)])
def test_stage_runs_and_kernels(sht, prec, inv_kernels):
    # fp16x2 adds the column-maximum pass of the spectrum before the split
    p = sht.Plan(31, 65, 128, 3, prec)
    prof = _pair_profile(p, 3)
    assert set(prof) == {"fft_forward", "legendre_forward", "legendre_inverse", "fft_inverse"}
    for name, (ms, runs, kernels) in prof.items():
        assert runs == 3 and ms > 0.0, name
        assert kernels == 3 * (inv_kernels if name == "legendre_inverse" else 1), name
    assert p.profile_read() == {}          # the read resets


def test_reduced_grid_fft_kernels(sht):
    N, J, I = 63, 129, 256
    pts = sht.Plan(N, J, I, 1, "fp64").reduced_grid_sizes("smooth")
    halves = {n // 2 for n in pts}
    per_fft = len(halves & FIXED_HALF_LENGTHS) + (1 if halves - FIXED_HALF_LENGTHS else 0)
    assert per_fft >= 2                     # both kinds of launch occur here
    p = sht.Plan(N, J, I, 2, "bf16x3", grid="reduced", lat_points=pts)
    prof = _pair_profile(p, 2)
    assert prof["fft_forward"][2] == 2 * per_fft
    assert prof["fft_inverse"][2] == 2 * per_fft

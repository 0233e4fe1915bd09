"""The allocation-free analysis entry point, checked against the plan-based
one and against the oracle.

Some callers cannot allocate device memory: a plug-in inside an application
that owns all of the GPU's memory through its own pool, or code that runs
where the application forbids allocations.  They cannot create a plan, so
``sht_forward_noalloc`` serves them from a fixed scratch array the library
keeps on the device.  This file calls it through the C ABI several times in
a row, with problem sizes that differ from call to call so that no call can
lean on tables left behind by the previous one, and compares every result
with ``sht_forward`` on an FP64 plan within the FP64 tolerance of the other
GPU tests, and one case with the oracle directly.  It also checks that
calls after the first leave the device's free memory unchanged.  It is kept
in a file of its own that pytest collects last."""
import ctypes

import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    built_lib()
    from paper_1711_11296_gb300 import _native, sht
    return _native, sht


def _spec(N, F):
    return torch.empty(((N + 1) * (N + 2) // 2, F), dtype=torch.complex128, device="cuda")


def _call(native, N, J, I, F, x, spec):
    stream = torch.cuda.current_stream().cuda_stream
    return native.lib.sht_forward_noalloc(N, J, I, F, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(spec.data_ptr()),
                                          ctypes.c_void_p(stream))


def _noalloc(native, N, J, I, F, x):
    spec = _spec(N, F)
    rc = _call(native, N, J, I, F, x, spec)
    assert rc == 0, native.lib.sht_last_error()
    return spec


def test_noalloc_matches_plan_forward_on_consecutive_calls(mods):
    native, sht = mods
    cases = [(63, 129, 256, 5, 31), (31, 65, 128, 3, 32), (63, 129, 256, 5, 33)]
    inputs = [to_cuda(W.random_grid(F, J, I, seed=seed), torch.float64)
              for N, J, I, F, seed in cases]
    # back-to-back calls on one stream, no synchronisation in between
    outs = [_noalloc(native, N, J, I, F, x)
            for (N, J, I, F, _), x in zip(cases, inputs)]
    for (N, J, I, F, _), x, got in zip(cases, inputs, outs):
        ref = sht.Plan(N, J, I, F, "fp64").forward(x)
        assert_fp64_close(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_matches_oracle(mods):
    native, _ = mods
    N, J, I, F = 31, 65, 128, 2
    x = W.random_grid(F, J, I, seed=34)
    got = _noalloc(native, N, J, I, F, to_cuda(x, torch.float64))
    assert_fp64_close(got.cpu().numpy(), O.analysis(x, N))


def test_noalloc_calls_allocate_nothing(mods):
    native, _ = mods
    a = (63, 129, 256, 4)
    b = (31, 65, 128, 2)
    xa = to_cuda(W.random_grid(a[3], a[1], a[2], seed=35), torch.float64)
    xb = to_cuda(W.random_grid(b[3], b[1], b[2], seed=36), torch.float64)
    sa, sb = _spec(a[0], a[3]), _spec(b[0], b[3])
    assert _call(native, *a, xa, sa) == 0, native.lib.sht_last_error()   # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _call(native, *b, xb, sb) == 0, native.lib.sht_last_error()
        assert _call(native, *a, xa, sa) == 0, native.lib.sht_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_scratch(mods):
    native, _ = mods
    N, J, I, F = 255, 511, 1024, 64
    x = torch.zeros((F, J, I), dtype=torch.float64, device="cuda")
    spec = _spec(N, F)
    rc = native.lib.sht_forward_noalloc(N, J, I, F, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(spec.data_ptr()), None)
    assert rc == -1
    assert b"scratch" in native.lib.sht_last_error()
    # the next successful call clears the message
    x = to_cuda(W.random_grid(1, 65, 128, seed=37), torch.float64)
    assert _call(native, 31, 65, 128, 1, x, _spec(31, 1)) == 0
    assert native.lib.sht_last_error() == b""

"""Failure detection on the GPU without faulting it.  A fault-injection hook
makes the first CTA of a split plan's forward GEMM never arm its first
pipeline stage: every bounded wait downstream runs out (about 2 s), the CTA
drains its copies, frees its tensor memory and records SHT_ERR_TIMEOUT, which
sht_plan_status reports; the context stays usable.  A second hook fails a
plan's device allocation as if the GPU were out of memory."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

SHT_ERR_ALLOC, SHT_ERR_TIMEOUT = -2, -5


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _with_env(name, value, fn):
    os.environ[name] = value
    try:
        return fn()
    finally:
        del os.environ[name]


def test_bounded_wait_timeout_is_reported_and_context_survives(sht):
    N, J, I, F = 7, 15, 16, 1
    p = _with_env("SHT_INJECT_STALL", "1", lambda: sht.Plan(N, J, I, F, "bf16x3"))
    x = W.random_grid(F, J, I, seed=1701).astype(np.float32).astype(np.float64)
    p.forward(to_cuda(x, torch.float32))
    with pytest.raises(sht.SHTError) as ei:
        p.status()
    assert ei.value.code == SHT_ERR_TIMEOUT
    p.status()                      # reading the status cleared it
    p.close()
    # the device is healthy: a fresh plan computes the right answer
    q = sht.Plan(N, J, I, F, "bf16x3")
    got = q.forward(to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(got, O.analysis(x, N)) <= 1e-6
    q.status()


def test_injected_allocation_failure(sht):
    for k in (1, 3):
        with pytest.raises(sht.SHTError) as ei:
            _with_env("SHT_INJECT_ALLOC_FAIL", str(k), lambda: sht.Plan(31, 65, 128, 2, "fp64"))
        assert ei.value.code == SHT_ERR_ALLOC
    p = sht.Plan(31, 65, 128, 2, "fp64")    # nothing leaked into the next plan
    x = W.random_grid(2, 65, 128, seed=1702)
    assert rel_l2(p.forward(to_cuda(x, torch.float64)).cpu().numpy(), O.analysis(x, 31)) < 1e-12

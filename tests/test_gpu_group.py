"""Grouped execution (one launch per stage for several plans) against the
per-plan entry points and the oracle, and its capture in a CUDA graph.

The full-size case is the uneven ensemble: 16 members x 32 levels x 2
fields at each of T63, T127, T255 and T511 (1024 field-levels per
truncation), split BF16 x 3."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


SMALL = [(31, 65, 128, 3), (15, 31, 32, 2), (0, 1, 2, 1), (20, 41, 50, 5), (12, 31, 30, 4)]


def test_fp64_group_matches_plans_and_oracle(sht):
    plans = [sht.Plan(N, J, I, F, "fp64") for N, J, I, F in SMALL]
    grp = sht.Group(plans)
    grids = [to_cuda(W.random_grid(F, J, I, seed=40 + k), torch.float64)
             for k, (N, J, I, F) in enumerate(SMALL)]
    specs = grp.forward(grids)
    for p, g, s, (N, J, I, F) in zip(plans, grids, specs, SMALL):
        single = p.forward(g).cpu().numpy()
        got = s.cpu().numpy()
        assert_fp64_close(got, single, 1e-14, 1e-14)
        assert_fp64_close(got, O.analysis(g.cpu().numpy(), N))
    a = [to_cuda(W.random_spectrum(N, F, seed=60 + k), torch.complex128)
         for k, (N, J, I, F) in enumerate(SMALL)]
    outs = grp.inverse(a)
    for p, x, o, (N, J, I, F) in zip(plans, a, outs, SMALL):
        assert_fp64_close(o.cpu().numpy(), p.inverse(x).cpu().numpy(), 1e-14, 1e-14)
        assert_fp64_close(o.cpu().numpy(), O.synthesis(x.cpu().numpy(), N, J, I))


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-6), ("fp16x2", 2e-6)])
def test_split_group_matches_plans(sht, prec, tol):
    cfg = [(31, 65, 128, 3), (63, 129, 256, 4), (40, 81, 96, 2)]
    plans = [sht.Plan(N, J, I, F, prec) for N, J, I, F in cfg]
    grp = sht.Group(plans)
    grids = [to_cuda(W.random_grid(F, J, I, seed=80 + k), torch.float32)
             for k, (N, J, I, F) in enumerate(cfg)]
    specs = grp.forward(grids)
    for p, g, s, (N, J, I, F) in zip(plans, grids, specs, cfg):
        assert rel_l2(s.cpu().numpy(), p.forward(g).cpu().numpy()) < 1e-7
        ref = O.analysis(g.cpu().numpy().astype(np.float64), N)
        assert rel_l2(s.cpu().numpy(), ref) < tol
    a = [to_cuda(W.random_spectrum(N, F, seed=90 + k), torch.complex64)
         for k, (N, J, I, F) in enumerate(cfg)]
    outs = grp.inverse(a)
    for p, x, o, (N, J, I, F) in zip(plans, a, outs, cfg):
        assert rel_l2(o.cpu().numpy(), p.inverse(x).cpu().numpy()) < 1e-7
    for p in plans:
        p.status()


def test_group_rejects_bad_input(sht):
    p = sht.Plan(7, 15, 16, 1, "fp64")
    q = sht.Plan(7, 15, 16, 1, "bf16x3")
    with pytest.raises(sht.SHTError):
        sht.Group([p, p])            # same plan twice
    with pytest.raises(sht.SHTError):
        sht.Group([p, q])            # mixed precision


def test_ensemble_group_full_size_and_graph(sht):
    members = W.ENSEMBLE
    plans = [sht.Plan(w.N, w.J, w.I, w.F, "bf16x3") for w in members]
    grp = sht.Group(plans)
    specs_h = [W.workload_spectrum(w).astype(np.complex64) for w in members]
    specs = [torch.from_numpy(a).cuda() for a in specs_h]
    grids = grp.inverse(specs)
    back = grp.forward(grids)
    torch.cuda.synchronize()
    for p in plans:
        p.status()
    fields = [0, 517, 1023]
    for w, a, g, b in zip(members, specs_h, grids, back):
        a64 = a.astype(np.complex128)
        rows = [1, (w.J + 1) // 2, w.J]
        ref = O.synthesis_rows(a64[:, fields], w.N, w.J, w.I, rows)
        got = g.cpu().numpy()[fields][:, np.array(rows) - 1, :]
        assert rel_l2(got, ref) < 1e-6, (w.name, rel_l2(got, ref))
        # every field: the split pair reproduces its input spectrum
        assert rel_l2(b.cpu().numpy(), a64) < 2e-6, w.name
    # the same pair captured in one CUDA graph and replayed
    static_in = [s.clone() for s in specs]
    g_out = [p.empty_grid() for p in plans]
    s_out = [p.empty_spec() for p in plans]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        grp.inverse(static_in, out=g_out)     # warm-up outside capture
        grp.forward(g_out, out=s_out)
    torch.cuda.current_stream().wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        grp.inverse(static_in, out=g_out)
        grp.forward(g_out, out=s_out)
    for s in s_out:
        s.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for s, b in zip(s_out, back):
        assert torch.equal(s, b)

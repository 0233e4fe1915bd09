"""Split-precision path (FP32 FFT, BF16-split Legendre contractions on the
tcgen05 tensor cores) against the FP64 oracle.

The split path takes FP32 inputs, so the oracle is given the same FP32
values (widened to FP64) and the error is that of the path itself.
Tolerances (relative L2 over the whole output, per direction):
  bf16x3: 1e-6  -- the accuracy target of the split path; three BF16 terms
                   carry 24 significand bits (the FP32 input precision) and
                   the tensor cores accumulate each K=16 block in FP32, so
                   about sqrt(K/16) * 2^-24 ~ 4e-7 is expected at K = 641.
  bf16x2: 5e-5  -- two BF16 terms carry 16 bits: ~2^-16 = 1.5e-5 per operand.
  fp16x2, fp16x3: operands scaled by powers of two into [-1, 1) (per P~ row,
                  per real column), x = x_1 + 2^-11 (x_2 [+ x_3]).  Per
                  product the error is at most 2^-24 (x2: representation of
                  each operand) x 2 + 2^-24 (the dropped x_2 y_2) of
                  rowmax * colmax, i.e. 1.8e-7; fp16x3 removes the first
                  two.  Relative to the output this is multiplied by the
                  ratio of the column maximum to the typical entry (up to
                  ~5 for these spectra), so: fp16x2 2e-6, fp16x3 1e-6.

Beside the whole-output error, every (m, parity) Legendre problem is held
to BLOCK_TOL relative to its own values, on inputs that give every problem
a comparable share (white-noise grids for the forward, flat spectra for the
inverse): a wrong or missing tile of a small high-m problem changes the
whole output by far less than 1e-6 of its norm, but its own block by O(1).
The block bound is looser than the global one because a block's values are
sums over fewer terms (fewer nodes carry |P~_n^m| near its maximum at high
m), so the relative rounding of a block is a few times that of the whole.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import (built_lib, grid_block_errors, rel_l2, spec_block_errors,
                          to_cuda, worst)

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-6, "bf16x2": 5e-5, "fp16x3": 1e-6, "fp16x2": 2e-6}
BLOCK_TOL = {"bf16x3": 4e-6, "bf16x2": 2e-4, "fp16x3": 4e-6, "fp16x2": 8e-6}
_BLOCK_REPORT = {}


def _record(name, errs):
    e, k = worst(errs)
    _BLOCK_REPORT[name] = {"worst": e, "m": int(k[0]), "parity": int(k[1])}
    out = os.environ.get("SHT_REPORT_DIR")
    if out:
        with open(os.path.join(out, "split_block_errors.json"), "w") as fh:
            json.dump(_BLOCK_REPORT, fh, indent=1)
    return e, k


PRECS = ["bf16x3", "bf16x2", "fp16x3", "fp16x2"]

CASES = [
    (31, 65, 128, 1),
    (31, 65, 128, 7),
    (0, 1, 2, 3),
    (12, 31, 30, 4),
    (40, 81, 96, 2),
    (63, 129, 256, 19),
    (159, 321, 640, 33),
    # 3 and 4 column tiles: clusters of 3 and 4 CTAs share each P~ tile
    # (at T31 a row tile has at most 2 groups of 8 rows, fewer than CTAs)
    (63, 129, 256, 160),
    (31, 65, 128, 256),
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


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,J,I,F", CASES)
def test_split_forward_inverse_match_oracle(sht, prec, N, J, I, F):
    p = sht.Plan(N, J, I, F, prec)
    x = _f32(W.random_grid(F, J, I, seed=700 + N))
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    ref = O.analysis(x, N)
    assert rel_l2(got, ref) <= TOL[prec], rel_l2(got, ref)
    assert np.all(got[:N + 1].imag == 0.0)
    e, k = _record("fwd %s T%d F%d" % (prec, N, F), spec_block_errors(got, ref, N))
    assert e <= BLOCK_TOL[prec], (e, k)
    a = _c64(W.random_spectrum(N, F, "n^-1.5", seed=800 + N))
    g = p.inverse(to_cuda(a, torch.complex64)).cpu().numpy()
    gref = O.synthesis(a, N, J, I)
    assert rel_l2(g, gref) <= TOL[prec], rel_l2(g, gref)
    # per problem, on a flat spectrum (rows j and J-1-j are mirrors)
    af = _c64(W.random_spectrum(N, F, "flat", seed=810 + N))
    g = p.inverse(to_cuda(af, torch.complex64)).cpu().numpy()
    gref = O.synthesis(af, N, J, I)
    assert rel_l2(g, gref) <= TOL[prec], rel_l2(g, gref)
    Jh = (J + 1) // 2
    north, south = np.arange(Jh), J - 1 - np.arange(Jh)
    errs = grid_block_errors(g[:, north], g[:, south], gref[:, north], gref[:, south], N,
                             floor=0.1)
    e, k = _record("inv %s T%d F%d" % (prec, N, F), errs)
    assert e <= BLOCK_TOL[prec], (e, k)
    p.status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("N,J,I,F", [(31, 65, 128, 3), (63, 129, 256, 4)])
def test_split_adjoints_and_restriction(sht, prec, N, J, I, F):
    p = sht.Plan(N, J, I, F, prec)
    a = _c64(W.random_spectrum(N, F, "n^-1.5", seed=900 + N))
    x = _f32(W.random_grid(F, J, I, seed=901 + N))
    g0 = p.adjoint(0, to_cuda(a, torch.complex64)).cpu().numpy()
    assert rel_l2(g0, O.adjoint_analysis(a, N, J, I)) <= 1e-6
    g1 = p.adjoint(1, to_cuda(x, torch.float32)).cpu().numpy()
    assert rel_l2(g1, O.adjoint_synthesis(x, N)) <= 1e-6
    fine = _f32(W.random_grid(F, 2 * (J + 1) - 1, 2 * I, seed=902 + N))
    got = p.restrict_nested(to_cuda(fine, torch.float32), 1).cpu().numpy()
    assert rel_l2(got, O.restrict_nested(fine, 1, N)) <= 1e-6
    p.status()


def test_split_t319_errors_per_field(sht):
    """T319 x 300 field-levels: per-field spectral and grid errors of the
    four splits against the oracle on sampled fields (all fields run on the
    GPU).  Writes the table to $SHT_REPORT_DIR if set."""
    w = W.WORKLOADS["T319"]
    fields = [0, 1, 99, 150, 299]
    x = np.stack([W.random_grid_field(f, w.J, w.I) for f in range(w.F)])
    x = _f32(x)
    a = _c64(W.workload_spectrum(w))
    ref_s = O.analysis(x[fields], w.N)
    ref_g = O.synthesis(a[:, fields], w.N, w.J, w.I)
    report = {}
    for prec in PRECS:
        p = sht.Plan(w.N, w.J, w.I, w.F, prec)
        s = p.forward(to_cuda(x, torch.float32)).cpu().numpy()[:, fields]
        g = p.inverse(to_cuda(a, torch.complex64)).cpu().numpy()[fields]
        p.status()
        es = [rel_l2(s[:, k], ref_s[:, k]) for k in range(len(fields))]
        eg = [rel_l2(g[k], ref_g[k]) for k in range(len(fields))]
        report[prec] = {"fields": fields, "spectral_rel_l2": es, "grid_rel_l2": eg}
        assert max(es) <= TOL[prec] and max(eg) <= TOL[prec], (prec, es, eg)
        del p
    out = os.environ.get("SHT_REPORT_DIR")
    if out:
        with open(os.path.join(out, "split_errors_T319.json"), "w") as fh:
            json.dump(report, fh, indent=1)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x2"])
def test_split_t639_sampled(sht, prec):
    w = W.WORKLOADS["T639"]
    p = sht.Plan(w.N, w.J, w.I, w.F, prec)
    fields = [0, 77, 255]
    ms = [0, 1, 2, 320, 638, 639]
    x = _f32(np.stack([W.random_grid_field(f, w.J, w.I) for f in range(w.F)]))
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    ref = O.analysis(x[fields], w.N, ms=ms)
    num = den = 0.0
    for m in ms:
        r0 = O.coef_offset(w.N, m)
        d = got[r0:r0 + w.N - m + 1][:, fields] - ref[m]
        num += np.sum(np.abs(d) ** 2)
        den += np.sum(np.abs(ref[m]) ** 2)
    assert np.sqrt(num / den) <= TOL[prec], np.sqrt(num / den)
    e, k = _record("fwd %s T639 sampled" % prec,
                   spec_block_errors(got[:, fields], ref, w.N, ms=ms))
    assert e <= BLOCK_TOL[prec], (e, k)
    del x
    a = _c64(W.workload_spectrum(w))
    grid = p.inverse(to_cuda(a, torch.complex64)).cpu().numpy()
    rows = [1, 2, 640, 641, 1281]
    gref = O.synthesis_rows(a[:, fields], w.N, w.J, w.I, rows)
    assert rel_l2(grid[fields][:, np.array(rows) - 1, :], gref) <= TOL[prec]
    # per (m, parity) problem on a flat spectrum, at northern rows spread
    # over the five 128-row tiles of the inverse contraction, their mirror
    # rows and the Equator (1-based rows; the mirror of r is J + 1 - r)
    af = _c64(W.random_spectrum(w.N, w.F, "flat", seed=1710))
    grid = p.inverse(to_cuda(af, torch.complex64)).cpu().numpy()[fields]
    north = np.array([1, 2, 100, 129, 200, 300, 385, 450, 513, 600, 640, 641])
    south = w.J + 1 - north
    gref = O.synthesis_rows(af[:, fields], w.N, w.J, w.I, np.concatenate([north, south]))
    R = len(north)
    assert rel_l2(grid[:, np.concatenate([north, south]) - 1], gref) <= TOL[prec]
    errs = grid_block_errors(grid[:, north - 1], grid[:, south - 1], gref[:, :R],
                             gref[:, R:], w.N, floor=0.1)
    e, k = _record("inv %s T639 sampled" % prec, errs)
    assert e <= BLOCK_TOL[prec], (e, k)
    p.status()


@pytest.mark.parametrize("prec", ["fp16x2", "fp16x3"])
def test_fp16_scaling_range(sht, prec):
    """FP16 splits scale each column into FP16's range: fields of magnitude
    1e12 and 1e-12 (far outside it) keep the same relative error, an
    all-zero field gives exactly zero, and an arbitrary Im(X_n^0) (not an
    input) does not disturb the scale of its column."""
    N, J, I, F = 63, 129, 256, 5
    p = sht.Plan(N, J, I, F, prec)
    x = W.random_grid(F, J, I, seed=1201)
    x[1] *= 1e12
    x[2] *= 1e-12
    x[3] = 0.0
    x = _f32(x)
    got = p.forward(to_cuda(x, torch.float32)).cpu().numpy()
    ref = O.analysis(x, N)
    for f in (0, 1, 2, 4):
        assert rel_l2(got[:, f], ref[:, f]) <= TOL[prec], (f, rel_l2(got[:, f], ref[:, f]))
    assert np.all(got[:, 3] == 0)
    a = W.random_spectrum(N, F, "n^-1.5", seed=1202)
    a[:, 1] *= 1e12
    a[:, 2] *= 1e-12
    a[:, 3] = 0.0
    a = _c64(a)
    ref_g = O.synthesis(a, N, J, I)
    a_junk = a.copy()
    a_junk[:N + 1] += 1j * 1e30            # Im(X_n^0): ignored on input
    g = p.inverse(to_cuda(a_junk, torch.complex64)).cpu().numpy()
    for f in (0, 1, 2, 4):
        assert rel_l2(g[f], ref_g[f]) <= TOL[prec], (f, rel_l2(g[f], ref_g[f]))
    assert np.all(g[3] == 0)
    p.status()

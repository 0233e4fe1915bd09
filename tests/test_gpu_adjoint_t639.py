"""The hand-written adjoints at T639 x 256 field-levels (N = 639, J = 1281,
I = 2560), in FP64 and in split BF16x3, in the launch configuration the
benchmark times.  The paper defines no adjoint; these are the transposes
of Eq. (dSHT) and Eq. (iSHT) for the plain inner products (the sum over
grid points of x y and over stored coefficients of Re(conj(a) b)).  Three
checks per path:

1. the dot-product identities <F x, a> = <x, F^T a> and <S a, y> = <a, S^T y>
   over all fields, with |lhs - rhs| bounded relative to |u| |v| of the
   vectors paired (1e-13 FP64; 1e-6 split, the split path's accuracy);
2. sampled values against the oracle's adjoints (latitudes spread over the
   inverse contraction's row tiles and their mirrors; zonal wavenumbers
   0, 1, 2, N/2, N-1, N), element by element for FP64 and by relative L2
   plus per-(m, parity) blocks for the split path;
3. finite differences of scalar losses through the autograd Functions: the
   losses are linear, so the central difference along a seeded direction
   equals the directional derivative up to rounding, and the gradient that
   backward returns (the native adjoint) must give the same number.

Grid inputs are seeded white-noise fields and spectral inputs the seeded
(n+1)^-2-energy spectra of the T639 workload."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import (assert_fp64_close, built_lib, grid_block_errors, rel_l2,
                          spec_block_errors, to_cuda, worst)

pytestmark = pytest.mark.gpu

DOT_TOL = {"fp64": 1e-13, "bf16x3": 1e-6}
FIELDS = [0, 77, 255]
MS = [0, 1, 2, 320, 638, 639]
# 1-based northern rows spread over the 128-row tiles, and the Equator
NORTH = np.array([1, 2, 100, 129, 200, 300, 385, 450, 513, 600, 640, 641])


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


@pytest.fixture(scope="module")
def inputs():
    w = W.WORKLOADS["T639"]
    x = np.stack([W.random_grid_field(f, w.J, w.I, seed=W.SEED_BASE + 4100)
                  for f in range(w.F)])
    a = W.workload_spectrum(w)
    return w, x, a


def _dtypes(prec):
    return ((torch.float64, torch.complex128) if prec == "fp64"
            else (torch.float32, torch.complex64))


def _round(x, a, prec):
    """The inputs as the path sees them (split plans take FP32 values)."""
    if prec == "fp64":
        return x, a
    return (x.astype(np.float32).astype(np.float64),
            a.astype(np.complex64).astype(np.complex128))


def _rdot(u, v):
    """Real inner product in FP64 on the device: sum of u*v over grid
    points, or of Re(conj(u) v) over stored coefficients."""
    if u.is_complex():
        u, v = torch.view_as_real(u), torch.view_as_real(v)
    u, v = u.double(), v.double()
    return float((u * v).sum()), float(u.norm()) * float(v.norm())


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_t639_adjoint_dot_products_and_oracle(sht, inputs, prec):
    w, x, a = inputs
    x, a = _round(x, a, prec)
    rd, cd = _dtypes(prec)
    p = sht.Plan(w.N, w.J, w.I, w.F, prec)
    tx, ta = to_cuda(x, rd), to_cuda(a, cd)
    g = W.random_spectrum(w.N, w.F, "energy^-2", seed=W.SEED_BASE + 4200)
    tg = to_cuda(g, cd)
    # 1. dot products (every field distinct on both sides)
    fx = p.forward(tx)
    at_g = p.adjoint(0, tg)                     # F^T g (spectrum -> grid)
    lhs, s1 = _rdot(fx, tg)
    rhs, s2 = _rdot(tx, at_g)
    assert abs(lhs - rhs) <= DOT_TOL[prec] * max(s1, s2), (lhs, rhs)
    del fx, at_g
    sa = p.inverse(ta)
    st_x = p.adjoint(1, tx)                     # S^T x (grid -> spectrum)
    lhs, s1 = _rdot(sa, tx)
    rhs, s2 = _rdot(ta, st_x)
    assert abs(lhs - rhs) <= DOT_TOL[prec] * max(s1, s2), (lhs, rhs)
    del sa
    st_x = st_x.cpu().numpy()[:, FIELDS]
    # 2. oracle values: F^T a at sampled rows, S^T x at sampled wavenumbers
    rows = np.concatenate([NORTH, w.J + 1 - NORTH])
    at_a = p.adjoint(0, ta).cpu().numpy()[FIELDS][:, rows - 1]
    ref = O.adjoint_analysis_rows(a[:, FIELDS], w.N, w.J, w.I, rows)
    refs = O.adjoint_synthesis(x[FIELDS], w.N, ms=MS)
    if prec == "fp64":
        assert_fp64_close(at_a, ref)
        # S^T x sums P~ times white-noise Fourier data over all 1281 nodes
        # without the quadrature weights, so the device P~ table's rounding
        # (within 1e-12 of each row's maximum, the plan-table parity bound)
        # reaches the output at that size; 1e-11 leaves room for the ratio of
        # a high-m row's maximum (near the Equator) to its typical value
        for m in MS:
            r0 = O.coef_offset(w.N, m)
            assert_fp64_close(st_x[r0:r0 + w.N - m + 1], refs[m], 1e-11, 1e-11)
    else:
        assert rel_l2(at_a, ref) <= 1e-6, rel_l2(at_a, ref)
        e, k = worst(spec_block_errors(st_x, refs, w.N, ms=MS))
        assert e <= 4e-6, (e, k)
        # per (m, parity) problem on a flat spectrum
        af = W.random_spectrum(w.N, w.F, "flat", seed=W.SEED_BASE + 4400)
        af = af.astype(np.complex64).astype(np.complex128)
        got = p.adjoint(0, to_cuda(af, cd)).cpu().numpy()[FIELDS][:, rows - 1]
        ref = O.adjoint_analysis_rows(af[:, FIELDS], w.N, w.J, w.I, rows)
        assert rel_l2(got, ref) <= 1e-6, rel_l2(got, ref)
        R = len(NORTH)
        e, k = worst(grid_block_errors(got[:, :R], got[:, R:], ref[:, :R], ref[:, R:], w.N,
                                       floor=0.1))
        assert e <= 4e-6, (e, k)
    p.status()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_t639_adjoint_finite_differences(sht, inputs, prec):
    w, x, a = inputs
    x, a = _round(x, a, prec)
    rd, cd = _dtypes(prec)
    p = sht.Plan(w.N, w.J, w.I, w.F, prec)
    tol = 1e-11 if prec == "fp64" else 2e-6
    # analysis: L(x) = <c, F x>, dL/dx = F^T c from backward
    c = to_cuda(W.random_spectrum(w.N, w.F, "energy^-2", seed=W.SEED_BASE + 4500), cd)
    d = to_cuda(np.stack([W.random_grid_field(f, w.J, w.I, seed=W.SEED_BASE + 4600)
                          for f in range(2)]).repeat(w.F // 2, axis=0), rd)
    tx = to_cuda(x, rd).requires_grad_(True)

    def loss_a(v):
        return _rdot(c, sht.analysis(v, p))[0]

    out = sht.analysis(tx, p)
    torch.view_as_real(out).mul(torch.view_as_real(c)).sum().backward()
    h = 1.0
    with torch.no_grad():
        fd = (loss_a(tx + h * d) - loss_a(tx - h * d)) / (2 * h)
    der, scale = _rdot(tx.grad, d)
    assert abs(fd - der) <= tol * scale, (fd, der)
    del tx, out, d
    # synthesis: L(a) = <y, S a>, dL/da = S^T y from backward
    y = to_cuda(np.stack([W.random_grid_field(f, w.J, w.I, seed=W.SEED_BASE + 4700)
                          for f in range(2)]).repeat(w.F // 2, axis=0), rd)
    e = W.random_spectrum(w.N, w.F, "energy^-2", seed=W.SEED_BASE + 4800)
    te = to_cuda(e, cd)
    ta = to_cuda(a, cd).requires_grad_(True)

    def loss_s(v):
        return _rdot(y, sht.synthesis(v, p))[0]

    out = sht.synthesis(ta, p)
    (out.double() * y.double()).sum().backward()
    with torch.no_grad():
        fd = (loss_s(ta + h * te) - loss_s(ta - h * te)) / (2 * h)
    der, scale = _rdot(ta.grad, te)
    assert abs(fd - der) <= tol * scale, (fd, der)
    p.status()

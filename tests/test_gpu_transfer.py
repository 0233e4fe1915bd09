"""Multigrid transfer operators (Appendix C): spectral prolongation (zero-pad
and synthesise) against the oracle, grid injection as exact sampling, and the
consistency of prolongation with the nested restriction and with injection."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, rel_l2, to_cuda

pytestmark = pytest.mark.gpu

COARSE = (15, 31, 32)     # N, J, I
FINE = (31, 63, 64)       # nests the coarse grid with k = 1 (Sec. 3.2)


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _pad(a, Nc, N):
    out = np.zeros((O.ncoef(N), a.shape[1]), dtype=a.dtype)
    for m in range(Nc + 1):
        out[O.coef_offset(N, m):O.coef_offset(N, m) + Nc - m + 1] = \
            a[O.coef_offset(Nc, m):O.coef_offset(Nc, m) + Nc - m + 1]
    return out


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_prolongation_matches_oracle(sht, prec):
    N, J, I = FINE
    F, Nc = 3, 15
    p = sht.Plan(N, J, I, F, prec)
    a = W.random_spectrum(Nc, F, "n^-1.5", seed=1801)
    if prec != "fp64":
        a = a.astype(np.complex64).astype(np.complex128)
    got = p.prolong_spectral(to_cuda(a, p.complex_dtype), Nc).cpu().numpy()
    ref = O.synthesis(_pad(a, Nc, N), N, J, I)
    if prec == "fp64":
        assert_fp64_close(got, ref)
    else:
        assert rel_l2(got, ref) <= 1e-6
    p.status()


@pytest.mark.parametrize("k", [1, 2])
def test_injection_is_exact_sampling(sht, k):
    N, J, I = COARSE
    F = 2
    p = sht.Plan(N, J, I, F, "fp64")
    Jf, If = 2 ** k * (J + 1) - 1, 2 ** k * I
    fine = W.random_grid(F, Jf, If, seed=1810 + k)
    got = p.inject_nested(to_cuda(fine, torch.float64), k).cpu().numpy()
    s = 2 ** k
    np.testing.assert_array_equal(got, fine[:, s - 1::s, ::s])


def test_prolong_then_restrict_or_inject_is_consistent(sht):
    (Nc, Jc, Ic), (N, J, I) = COARSE, FINE
    F = 2
    coarse = sht.Plan(Nc, Jc, Ic, F, "fp64")
    fine = sht.Plan(N, J, I, F, "fp64")
    a = W.random_spectrum(Nc, F, "n^-1.5", seed=1820)
    a[:Nc + 1] = a[:Nc + 1].real
    ta = to_cuda(a, torch.complex128)
    g = fine.prolong_spectral(ta, Nc)
    # the coarse analysis of the injected sub-grid recovers the spectrum
    # (J_c = 2 N_c + 1: exact), and injection equals the coarse synthesis
    assert_fp64_close(coarse.restrict_nested(g, 1).cpu().numpy(), a)
    assert_fp64_close(coarse.inject_nested(g, 1).cpu().numpy(), coarse.inverse(ta).cpu().numpy())


def test_transfer_argument_errors(sht):
    p = sht.Plan(*FINE, 1, "fp64")
    with pytest.raises(sht.SHTError):          # Nc = 40 > N = 31
        p.prolong_spectral(torch.zeros((O.ncoef(40), 1), dtype=torch.complex128,
                                       device="cuda"), 40)
    f1 = sht.Plan(*COARSE, 1, "fp64", grid="fejer1")
    with pytest.raises(sht.SHTError):
        f1.inject_nested(torch.zeros((1, 63, 64), dtype=torch.float64, device="cuda"), 1)


# A fine grid whose FP32 FFT half-length (320 = 10 x 32) writes the grid
# from its last pass, and the coarse grid it nests with k = 1.
COARSE2 = (79, 159, 320)
FINE2 = (159, 319, 640)


@pytest.mark.parametrize("shapes", [(COARSE, FINE), (COARSE2, FINE2)])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_prolong_add_is_grid_plus_prolongation(sht, prec, shapes):
    # the accumulating store adds, in the plan's precision, exactly the
    # values that the plain prolongation writes
    (Nc, _, _), (N, J, I) = shapes
    F = 3
    p = sht.Plan(N, J, I, F, prec)
    a = to_cuda(W.random_spectrum(Nc, F, "n^-1.5", seed=1830 + N), p.complex_dtype)
    g0 = to_cuda(W.random_grid(F, J, I, seed=1831 + N), p.real_dtype)
    out = g0.clone()
    p.prolong_spectral(a, Nc, out=out, add=True)
    assert torch.equal(out, g0 + p.prolong_spectral(a, Nc))
    with pytest.raises(ValueError):
        p.prolong_spectral(a, Nc, add=True)
    p.status()


@pytest.mark.parametrize("shapes", [(COARSE, FINE), (COARSE2, FINE2)])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_two_grid_correction_cancels_a_coarse_band_field(sht, prec, shapes):
    # Appendix C's V-cycle transfers on a fine field band-limited to the
    # coarse truncation: restricting it (Sec. 3.2, exact here) and adding
    # back the prolongation of minus that spectrum leaves zero.
    (Nc, Jc, Ic), (N, J, I) = shapes
    F = 2
    coarse = sht.Plan(Nc, Jc, Ic, F, prec)
    fine = sht.Plan(N, J, I, F, prec)
    a = W.random_spectrum(Nc, F, "n^-1.5", seed=1840 + N)
    a[:Nc + 1] = a[:Nc + 1].real
    x = fine.prolong_spectral(to_cuda(a, fine.complex_dtype), Nc)
    scale = float(x.abs().max())
    r = coarse.restrict_nested(x, 1)
    fine.prolong_spectral(-r, Nc, out=x, add=True)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert float(x.abs().max()) <= tol * scale
    fine.status()

"""FP64 GPU path against the oracle, element by element, on small and
ragged sizes (several FFT radices, odd half-lengths, partial field groups,
the Equator-only grid, an inexact grid), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import assert_fp64_close, built_lib, to_cuda

pytestmark = pytest.mark.gpu

CASES = [
    (31, 65, 128, 1),     # the T31 round-trip workload
    (31, 65, 128, 7),     # partial last field group
    (0, 1, 2, 3),         # N = 0: Equator-only grid, FFT of length 1
    (5, 11, 12, 5),       # L = 6 = 2 x 3
    (12, 31, 30, 4),      # L = 15 = 3 x 5 (odd half-length)
    (20, 33, 50, 3),      # L = 25 = 5 x 5, J < 2N+1 (inexact plan)
    (40, 81, 96, 2),      # L = 48 = 4 x 4 x 3
    (63, 129, 256, 19),   # radix-4 only, 19 fields
]


@pytest.fixture(scope="module")
def sht():
    built_lib()
    from paper_1711_11296_gb300 import sht as S
    return S


def _plan(sht, N, J, I, F):
    return sht.Plan(N, J, I, F, "fp64")


@pytest.mark.parametrize("N,J,I,F", CASES)
def test_tables_match_oracle(sht, N, J, I, F):
    p = _plan(sht, N, J, I, F)
    assert p.exact == (J >= 2 * N + 1)
    w, mu, pnm = p.tables()
    np.testing.assert_allclose(w, O.cc_weights(J), rtol=0, atol=2e-15)
    # the device mirrors the southern nodes exactly (mu_{J+1-j} = -mu_j);
    # the oracle rounds each cos separately: allow 1e-15
    np.testing.assert_allclose(mu, O.cc_nodes(J)[1], rtol=0, atol=1e-15)
    Jh = (J + 1) // 2
    ref = O.pnm_cc(N, J, j=np.arange(1, Jh + 1))
    # The device evaluates P~ at the FP64-rounded node (|d mu| <= 1.1e-16)
    # while the oracle uses the binary128 node; with |dP~/dmu| up to ~n^2
    # times the row scale, entries can differ by ~1e-13 of the row maximum
    # (relative differences blow up only near zeros of P~).
    rowmax = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(pnm - ref) <= 1e-12 * rowmax).all(), \
        np.max(np.abs(pnm - ref) / rowmax)


@pytest.mark.parametrize("N,J,I,F", CASES)
def test_forward_matches_oracle(sht, N, J, I, F):
    p = _plan(sht, N, J, I, F)
    x = W.random_grid(F, J, I, seed=100 + N)
    got = p.forward(to_cuda(x, torch.float64)).cpu().numpy()
    ref = O.analysis(x, N)
    assert_fp64_close(got, ref)
    m0 = slice(0, N + 1)
    assert np.all(got[m0].imag == 0.0)


@pytest.mark.parametrize("N,J,I,F", CASES)
def test_inverse_matches_oracle(sht, N, J, I, F):
    p = _plan(sht, N, J, I, F)
    a = W.random_spectrum(N, F, "n^-1.5", seed=200 + N)
    got = p.inverse(to_cuda(a, torch.complex128)).cpu().numpy()
    ref = O.synthesis(a, N, J, I)
    assert_fp64_close(got, ref)
    # the imaginary part of the m = 0 coefficients is ignored
    b = a.copy()
    b[:N + 1] += 1j * np.random.default_rng(0).standard_normal((N + 1, F))
    got_b = p.inverse(to_cuda(b, torch.complex128)).cpu().numpy()
    np.testing.assert_array_equal(got_b, got)


@pytest.mark.parametrize("N,J,I,F", CASES)
def test_adjoints_match_oracle(sht, N, J, I, F):
    p = _plan(sht, N, J, I, F)
    a = W.random_spectrum(N, F, "n^-1.5", seed=300 + N)
    x = W.random_grid(F, J, I, seed=400 + N)
    g0 = p.adjoint(0, to_cuda(a, torch.complex128)).cpu().numpy()
    assert_fp64_close(g0, O.adjoint_analysis(a, N, J, I))
    g1 = p.adjoint(1, to_cuda(x, torch.float64)).cpu().numpy()
    assert_fp64_close(g1, O.adjoint_synthesis(x, N))


@pytest.mark.parametrize("N,J,I,F", [c for c in CASES if c[1] >= 2 * c[0] + 1])
def test_round_trip_exact(sht, N, J, I, F):
    p = _plan(sht, N, J, I, F)
    a = W.random_spectrum(N, F, "n^-1.5", seed=500 + N)
    ta = to_cuda(a, torch.complex128)
    back = p.forward(p.inverse(ta)).cpu().numpy()
    assert_fp64_close(back, a, 1e-13, 1e-13)


def test_dot_product_adjoint_identities(sht):
    N, J, I, F = 31, 65, 128, 3
    p = _plan(sht, N, J, I, F)
    x = to_cuda(W.random_grid(F, J, I, seed=7), torch.float64)
    a = to_cuda(W.random_spectrum(N, F, seed=8), torch.complex128)
    lhs = torch.sum(torch.real(torch.conj(p.forward(x)) * a))
    rhs = torch.sum(x * p.adjoint(0, a))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    lhs = torch.sum(p.inverse(a) * x)
    rhs = torch.sum(torch.real(torch.conj(a) * p.adjoint(1, x)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_restrict_nested_matches_oracle(sht, k):
    Nc, Jc, Ic, F = 7, 15, 16, 5
    p = _plan(sht, Nc, Jc, Ic, F)
    Jf, If = 2 ** k * (Jc + 1) - 1, 2 ** k * Ic
    fine = W.random_grid(F, Jf, If, seed=600 + k)
    got = p.restrict_nested(to_cuda(fine, torch.float64), k).cpu().numpy()
    assert_fp64_close(got, O.restrict_nested(fine, k, Nc))


def test_restrict_nested_band_limited_is_truncation(sht):
    # Appendix C: for a field band-limited to the coarse truncation the
    # restriction returns its spectrum exactly.
    Nc, Jc, Ic, F = 15, 31, 32, 2
    p = _plan(sht, Nc, Jc, Ic, F)
    a = W.random_spectrum(Nc, F, seed=9)
    fine = O.synthesis(a, Nc, 2 * (Jc + 1) - 1, 2 * Ic)
    got = p.restrict_nested(to_cuda(fine, torch.float64), 1).cpu().numpy()
    assert_fp64_close(got, a, 1e-13, 1e-13)


def test_autograd_gradcheck(sht):
    N, J, I, F = 6, 13, 16, 2
    p = _plan(sht, N, J, I, F)
    x = to_cuda(W.random_grid(F, J, I, seed=10), torch.float64).requires_grad_()
    assert torch.autograd.gradcheck(lambda t: sht.analysis(t, p), (x,),
                                    eps=1e-6, atol=1e-8)
    a = to_cuda(W.random_spectrum(N, F, seed=11), torch.complex128).requires_grad_()
    assert torch.autograd.gradcheck(lambda t: sht.synthesis(t, p), (a,),
                                    eps=1e-6, atol=1e-8)


def test_errors_are_reported(sht):
    with pytest.raises(sht.SHTError):
        sht.Plan(10, 21, 20, 1, "fp64")        # I <= 2N
    with pytest.raises(sht.SHTError):
        sht.Plan(10, 22, 32, 1, "fp64")        # J even
    p = _plan(sht, 3, 7, 8, 1)
    with pytest.raises(ValueError):
        p.forward(torch.zeros((1, 7, 8), dtype=torch.float32, device="cuda"))

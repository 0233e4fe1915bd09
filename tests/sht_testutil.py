"""Shared helpers for the GPU tests (no transform arithmetic here)."""
import numpy as np

# FP64 path tolerance: relative L2 of the whole output and max abs error
# relative to the largest reference magnitude (the FP64 recurrence, FFT and
# contractions each contribute O(1e-15 sqrt(K)) rounding; 1e-12 leaves two
# orders of margin at T639).
FP64_REL_L2 = 1e-12
FP64_REL_MAX = 1e-12


def built_lib():
    from paper_1711_11296_gb300 import build
    return build.build()


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_fp64_close(got, ref, rel_l2_tol=FP64_REL_L2, rel_max_tol=FP64_REL_MAX):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    r = rel_l2(got, ref)
    scale = np.abs(ref).max() if ref.size else 1.0
    mx = np.abs(got - ref).max() / (scale if scale > 0 else 1.0) if ref.size else 0.0
    assert r <= rel_l2_tol and mx <= rel_max_tol, (r, mx)
    return r, mx


def to_cuda(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


# ---------------------------------------------------------------------------
# Per-(m, parity) errors.  One Legendre problem of the transform is one zonal
# wavenumber m and one parity q of n - m (Appendix B): a whole-output
# relative L2 hides a wrong or missing tile of a problem whose values are
# small next to the output's norm, so the split-path tests also bound the
# error of every problem relative to that problem's own values.
# ---------------------------------------------------------------------------
def spec_block_errors(got, ref, N, ms=None):
    """Relative L2 error of every (m, parity) block of a packed spectrum.

    got: [ncoef][F'] (columns already selected); ref: the same shape, or a
    dict m -> [N-m+1][F'] (the oracle's selected zonal wavenumbers).  The
    block (m, q) is the rows n = m + q, m + q + 2, ... of wavenumber m.
    Returns {(m, q): error} over ``ms`` (default every m)."""
    got = np.asarray(got)
    ms = range(N + 1) if ms is None else ms
    out = {}
    for m in ms:
        r0 = m * (N + 1) - m * (m - 1) // 2
        g = got[r0:r0 + N - m + 1]
        r = ref[m] if isinstance(ref, dict) else np.asarray(ref)[r0:r0 + N - m + 1]
        for q in (0, 1):
            gb, rb = g[q::2], r[q::2]
            if rb.size == 0:
                continue
            out[(m, q)] = rel_l2(gb, rb)
    return out


def fold_rows(north, south):
    """Zonal Fourier coefficients m of latitude rows (NumPy's real FFT with
    1/I) folded into the parts of Appendix B: S = (X_north + X_south)/2
    (n - m even) and A = (X_north - X_south)/2 (n - m odd).  north, south:
    real [F][R][I], row r of ``south`` the mirror of row r of ``north``
    (pass the Equator row as its own mirror).  Returns S, A [F][R][I/2+1]."""
    I = north.shape[-1]
    Xn = np.fft.rfft(north, axis=-1) / I
    Xs = np.fft.rfft(south, axis=-1) / I
    return (Xn + Xs) / 2, (Xn - Xs) / 2


def grid_block_errors(got_n, got_s, ref_n, ref_s, N, floor=0.0):
    """Relative L2 error of every (m, parity) block of a synthesised grid,
    from mirror-row pairs (see ``fold_rows``): block (m, 0) is S^m over the
    rows and fields, (m, 1) is A^m.  Empty blocks (A^m vanishes at the
    Equator; some blocks are empty for m = N) are skipped.

    Each error is relative to max(the block's own norm, ``floor`` times the
    median block norm).  The zonal FFT of a row rounds every coefficient by
    about the same amount (a share of the whole row's magnitude), so a block
    whose values at the sampled rows are far below the typical block's (high
    m away from the Equator) carries that rounding floor rather than its
    contraction's error; ``floor`` measures such blocks against the floor.
    Returns {(m, q): error}."""
    gS, gA = fold_rows(got_n, got_s)
    rS, rA = fold_rows(ref_n, ref_s)
    norms = {}
    for m in range(N + 1):
        norms[(m, 0)] = np.linalg.norm(rS[..., m])
        norms[(m, 1)] = np.linalg.norm(rA[..., m])
    med = float(np.median([v for v in norms.values() if v > 0.0]))
    out = {}
    for m in range(N + 1):
        for q, g, r in ((0, gS, rS), (1, gA, rA)):
            if norms[(m, q)] == 0.0:
                continue
            den = max(norms[(m, q)], floor * med)
            out[(m, q)] = np.linalg.norm(g[..., m] - r[..., m]) / den
    return out


def worst(errs):
    """(largest error, its (m, parity) key) of a block-error dict."""
    k = max(errs, key=errs.get)
    return errs[k], k

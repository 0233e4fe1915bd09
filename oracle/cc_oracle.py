"""Plain FP64 oracle of the Clenshaw-Curtis spherical-harmonic transform.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function is
the plain definition from the paper, with library primitives (matrix
products, a symmetric eigensolver) as single steps and no blocking,
folding or reordering of the sums.

Conventions (readings of points the paper leaves open):

* Nodes: theta_j = j pi/(J+1), j = 1..J, j = 1 northernmost; mu = sin(phi)
  = cos(theta) (Eq. cc-points).
* Spectra: complex array ``[ncoef][F]``; coefficient (m, n), 0 <= m <= n <= N,
  is row ``m (N+1) - m (m-1)/2 + (n - m)``.  Only m >= 0 is stored; a real
  field has X_n^{-m} = conj(X_n^m), so the synthesis (Eq. iSHT) reads
  X = sum_n Re(X_n^0) P~_n^0 + 2 Re sum_{m>=1} sum_n X_n^m P~_n^m e^{i m lambda}.
  The imaginary part of the m = 0 coefficients is ignored on input and is
  exactly zero on output.
* The inverse zonal DFT carries the zonal wavenumber m in its exponent (the
  printed formula below Eq. iLT drops it); the forward DFT carries 1/I (the
  discretised Eq. dFT), the inverse carries no factor.
* No Condon-Shortley phase.
* Adjoints are taken for the plain inner products: sum over grid points of
  x y, and sum over stored coefficients of Re(conj(a) b).
"""
import ctypes

import numpy as np

from . import build_oracle

__all__ = [
    "ncoef", "coef_offset", "cc_nodes", "cc_weights", "gauss_nodes_weights",
    "pnm_cc", "pnm_at", "dft_forward", "dft_inverse", "analysis",
    "synthesis", "adjoint_analysis", "adjoint_synthesis", "restrict_nested",
    "analysis_gauss", "synthesis_gauss", "legendre_forward_m",
    "legendre_inverse_m", "nested_rows", "fejer1_nodes", "fejer1_weights",
    "analysis_fejer1", "synthesis_fejer1", "reduced_sizes",
    "reduced_row_offsets", "reduced_kmax", "analysis_reduced",
    "synthesis_reduced",
]

_lib = None


def _clib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_pnm_cc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ip, ctypes.c_int, dp]
        lib.oracle_pnm_at.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      dp, dp, ctypes.c_int, dp]
        lib.oracle_cc_node_q.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# Indexing of the packed triangular spectrum
# --------------------------------------------------------------------------
def ncoef(N):
    """Number of stored coefficients (m >= 0) of a triangular truncation N."""
    return (N + 1) * (N + 2) // 2


def coef_offset(N, m):
    """Row of coefficient (m, n = m) in the packed m-major layout."""
    return m * (N + 1) - m * (m - 1) // 2


# --------------------------------------------------------------------------
# Quadrature: nodes and weights
# --------------------------------------------------------------------------
def cc_nodes(J):
    """Clenshaw-Curtis (Fejer second rule) nodes, Eq. (cc-points).

    Returns (theta, mu, sin_theta) for j = 1..J, theta_j = j pi/(J+1),
    mu_j = cos(theta_j) = sin(phi_j)."""
    j = np.arange(1, J + 1, dtype=np.float64)
    theta = np.pi * j / (J + 1)
    return theta, np.cos(theta), np.sin(theta)


def cc_weights(J):
    """Clenshaw-Curtis weights by the explicit sum of Eq. (cc-wgt).

    w_j = 4 sin(theta_j)/(J+1) * sum_{p odd, 1<=p<=J} sin(p theta_j)/p,
    with each sin(p theta_j) evaluated directly after reducing the integer
    p*j modulo 2(J+1)."""
    j = np.arange(1, J + 1, dtype=np.int64)[:, None]
    p = np.arange(1, J + 1, 2, dtype=np.int64)[None, :]
    r = (p * j) % (2 * (J + 1))
    s = np.sin(np.pi * r / (J + 1))
    sin_t = np.sin(np.pi * j[:, 0] / (J + 1))
    return 4.0 * sin_t / (J + 1) * (s / p).sum(axis=1)


def fejer1_nodes(J):
    """Nodes of Fejer's first rule on the shifted grid, Eq. (fejer1-points).

    Returns (theta, mu, sin_theta) for j = 1..J, theta_j = (j - 1/2) pi / J,
    j = 1 northernmost."""
    j = np.arange(1, J + 1, dtype=np.float64)
    theta = np.pi * (2.0 * j - 1.0) / (2.0 * J)
    return theta, np.cos(theta), np.sin(theta)


def fejer1_weights(J):
    """Weights of Fejer's first rule by its explicit cosine sum (Sec. 3.3):

        w_j = (2/J) (1 - 2 sum_{p=1}^{floor(J/2)} cos(2 p theta_j)/(4p^2 - 1)).

    Eq. (fejer1-wgt) is printed without the factor 2 in front of the sum;
    only with it is the rule interpolatory (exact to degree J-1), which the
    tests pin.  Each cos(2 p theta_j) = cos(pi p (2j-1)/J) is evaluated
    after reducing the integer p (2j-1) modulo 2J."""
    j = np.arange(1, J + 1, dtype=np.int64)[:, None]
    p = np.arange(1, J // 2 + 1, dtype=np.int64)[None, :]
    r = (p * (2 * j - 1)) % (2 * J)
    c = np.cos(np.pi * r / J)
    return 2.0 / J * (1.0 - 2.0 * (c / (4.0 * p * p - 1.0)).sum(axis=1))


def gauss_nodes_weights(J):
    """Gauss-Legendre nodes and weights (Eq. gauss-quad/gauss-wgt).

    Golub-Welsch: the nodes are the eigenvalues of the symmetric Jacobi
    matrix of the Legendre three-term recurrence (off-diagonal
    k/sqrt(4k^2-1)), the weights are 2 times the squared first components
    of the normalised eigenvectors.  Ordered north to south (mu
    decreasing).  Returns (mu, sin_theta, w)."""
    k = np.arange(1, J, dtype=np.float64)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    T = np.diag(beta, 1) + np.diag(beta, -1)
    x, V = np.linalg.eigh(T)
    w = 2.0 * V[0, :] ** 2
    order = np.argsort(-x)
    x, w = x[order], w[order]
    return x, np.sqrt((1.0 - x) * (1.0 + x)), w


# --------------------------------------------------------------------------
# Normalised associated Legendre functions (binary128 recurrence)
# --------------------------------------------------------------------------
def pnm_cc(N, J, m_lo=0, m_hi=None, j=None):
    """P~_n^m(mu_j) at Clenshaw-Curtis nodes, from the binary128 recurrence.

    Rows are (m, n) for m_lo <= m <= m_hi, n = m..N, packed m-major; columns
    are the 1-based node indices ``j`` (default all 1..J)."""
    if m_hi is None:
        m_hi = N
    jl = np.arange(1, J + 1, dtype=np.int32) if j is None else \
        np.ascontiguousarray(j, dtype=np.int32)
    rows = sum(N - m + 1 for m in range(m_lo, m_hi + 1))
    out = np.empty((rows, len(jl)), dtype=np.float64)
    rc = _clib().oracle_pnm_cc(N, J, m_lo, m_hi,
                               jl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               len(jl), _dptr(out))
    if rc != 0:
        raise ValueError("oracle_pnm_cc: bad arguments")
    return out


def pnm_at(N, cos_t, sin_t, m_lo=0, m_hi=None):
    """P~_n^m at arbitrary points (FP64 cos/sin of colatitude)."""
    if m_hi is None:
        m_hi = N
    c = np.ascontiguousarray(cos_t, dtype=np.float64)
    s = np.ascontiguousarray(sin_t, dtype=np.float64)
    rows = sum(N - m + 1 for m in range(m_lo, m_hi + 1))
    out = np.empty((rows, len(c)), dtype=np.float64)
    rc = _clib().oracle_pnm_at(N, m_lo, m_hi, _dptr(c), _dptr(s), len(c),
                               _dptr(out))
    if rc != 0:
        raise ValueError("oracle_pnm_at: bad arguments")
    return out


def cc_node_binary128(J, j):
    """(cos, sin) of theta_j from the binary128 series, rounded to FP64."""
    c = ctypes.c_double()
    s = ctypes.c_double()
    _clib().oracle_cc_node_q(J, j, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


# --------------------------------------------------------------------------
# Zonal Fourier transform (direct DFT)
# --------------------------------------------------------------------------
def _twiddle(I, ms, sign):
    """exp(sign * 2 pi i * (m*i mod I)/I) as an [I][len(ms)] matrix."""
    i = np.arange(I, dtype=np.int64)[:, None]
    r = (np.asarray(ms, dtype=np.int64)[None, :] * i) % I
    ang = 2.0 * np.pi * r / I
    return np.cos(ang) + sign * 1j * np.sin(ang)


def dft_forward(x, N, ms=None):
    """X^m(phi_j) = (1/I) sum_i X(lambda_i, phi_j) e^{-i m lambda_i}.

    Discretised Eq. (dFT) with lambda_i = 2 pi i/I; x is real [..., I];
    returns complex [..., len(ms)] for m in ``ms`` (default 0..N)."""
    I = x.shape[-1]
    ms = np.arange(N + 1) if ms is None else ms
    return (x @ _twiddle(I, ms, -1.0)) / I


def dft_inverse(X, I, ms=None):
    """Real field from zonal coefficients m >= 0 (conjugate symmetry).

    x_i = Re(X^0) + 2 Re sum_{m>=1} X^m e^{+i m lambda_i}."""
    M = X.shape[-1]
    ms = np.arange(M) if ms is None else np.asarray(ms)
    E = _twiddle(I, ms, +1.0).T                       # [len(ms)][I]
    c = np.where(ms == 0, 1.0, 2.0)[:, None]
    Xr = np.where(ms == 0, X.real + 0j, X)
    return np.real(Xr @ (c * E))


# --------------------------------------------------------------------------
# Legendre transform for one zonal wavenumber
# --------------------------------------------------------------------------
def legendre_forward_m(Xm, P, w):
    """X_n^m = sum_j X^m(phi_j) P~_n^m(mu_j) w_j (Eq. cc-quad / gauss-quad).

    Xm: complex [F][J]; P: [rows][J]; w: [J].  Returns [rows][F]."""
    return (P * w[None, :]) @ Xm.T


def legendre_inverse_m(a, P):
    """X^m(phi_j) = sum_n X_n^m P~_n^m(mu_j) (Eq. iLT).  a: [rows][F]."""
    return (P.T @ a).T                                 # [F][J]


# --------------------------------------------------------------------------
# Full transforms
# --------------------------------------------------------------------------
def _analysis_general(x, N, pfun, w, ms=None):
    F, J, I = x.shape
    ms = range(N + 1) if ms is None else ms
    X = dft_forward(x, N, ms=list(ms))                 # [F][J][len(ms)]
    out = {}
    for k, m in enumerate(ms):
        P = pfun(m)
        a = legendre_forward_m(X[:, :, k], P, w)
        if m == 0:
            a = a.real + 0j
        out[m] = a
    return out


def pnm_tables(N, J, ms):
    """{m: pnm_cc(N, J, m, m)} for the zonal wavenumbers ``ms``: the P~
    tables of ``analysis``, built once ahead of repeated transforms."""
    return {m: pnm_cc(N, J, m, m) for m in ms}


def analysis(x, N, ms=None, pnm=None):
    """Forward SHT on the Clenshaw-Curtis grid, Eq. (dSHT) with the zonal
    DFT and Eq. (cc-quad).  x: real [F][J][I] (j = 1 first).

    Returns the packed spectrum [ncoef][F] (complex), or, if ``ms`` is given,
    a dict m -> [N-m+1][F] for those zonal wavenumbers only.  ``pnm``: the
    P~ tables of ``pnm_tables`` (built here if None)."""
    x = np.asarray(x, dtype=np.float64)
    F, J, I = x.shape
    w = cc_weights(J)
    pf = (lambda m: pnm_cc(N, J, m, m)) if pnm is None else (lambda m: pnm[m])
    d = _analysis_general(x, N, pf, w, ms)
    if ms is not None:
        return d
    spec = np.zeros((ncoef(N), F), dtype=np.complex128)
    for m, a in d.items():
        spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1] = a
    return spec


def _synthesis_general(spec, N, J, I, pfun, ms=None):
    F = spec.shape[1]
    ms = list(range(N + 1)) if ms is None else list(ms)
    X = np.zeros((F, J, len(ms)), dtype=np.complex128)
    for k, m in enumerate(ms):
        a = spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1]
        X[:, :, k] = legendre_inverse_m(a, pfun(m))
    return dft_inverse(X, I, ms=ms)


def synthesis(spec, N, J, I):
    """Inverse SHT, Eq. (iSHT) via Eq. (iLT) and the inverse zonal DFT.

    spec: complex [ncoef][F]; returns real [F][J][I]."""
    spec = np.asarray(spec, dtype=np.complex128)
    return _synthesis_general(spec, N, J, I, lambda m: pnm_cc(N, J, m, m))


def synthesis_rows(spec, N, J, I, rows):
    """Synthesis (Eq. iSHT) evaluated only at the 1-based latitudes ``rows``
    (all longitudes): returns real [F][len(rows)][I]."""
    spec = np.asarray(spec, dtype=np.complex128)
    F = spec.shape[1]
    rows = np.asarray(rows)
    X = np.zeros((F, len(rows), N + 1), dtype=np.complex128)
    for m in range(N + 1):
        a = spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1]
        X[:, :, m] = legendre_inverse_m(a, pnm_cc(N, J, m, m, j=rows))
    return dft_inverse(X, I)


def analysis_fejer1(x, N):
    """Forward SHT on the shifted grid of Fejer's first rule (Sec. 3.3): the
    zonal DFT, then the quadrature with the weights of ``fejer1_weights`` at
    the nodes of ``fejer1_nodes``.  x: real [F][J][I] (j = 1 first)."""
    x = np.asarray(x, dtype=np.float64)
    F, J, I = x.shape
    _, mu, s = fejer1_nodes(J)
    d = _analysis_general(x, N, lambda m: pnm_at(N, mu, s, m, m), fejer1_weights(J))
    spec = np.zeros((ncoef(N), F), dtype=np.complex128)
    for m, a in d.items():
        spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1] = a
    return spec


def synthesis_fejer1(spec, N, J, I):
    """Inverse SHT (Eq. iSHT) evaluated on the J-point shifted grid."""
    _, mu, s = fejer1_nodes(J)
    return _synthesis_general(np.asarray(spec, np.complex128), N, J, I,
                              lambda m: pnm_at(N, mu, s, m, m))


def analysis_gauss(x, N):
    """Forward SHT on a Gaussian grid (Eq. gauss-quad), J = x.shape[1]."""
    F, J, I = x.shape
    mu, s, w = gauss_nodes_weights(J)
    d = _analysis_general(np.asarray(x, np.float64), N,
                          lambda m: pnm_at(N, mu, s, m, m), w)
    spec = np.zeros((ncoef(N), F), dtype=np.complex128)
    for m, a in d.items():
        spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1] = a
    return spec


def synthesis_gauss(spec, N, J, I):
    """Inverse SHT evaluated on the J-point Gaussian grid."""
    mu, s, _ = gauss_nodes_weights(J)
    return _synthesis_general(np.asarray(spec, np.complex128), N, J, I,
                              lambda m: pnm_at(N, mu, s, m, m))


def adjoint_analysis(abar, N, J, I):
    """Transpose of ``analysis`` (spectrum -> grid).

    x~_ij = (w_j / I) sum_{m>=0} sum_n P~_n^m(mu_j) Re(a~_n^m e^{i m lambda_i}),
    with no factor 2 for m >= 1 (the m = 0 imaginary part drops out)."""
    abar = np.asarray(abar, dtype=np.complex128)
    F = abar.shape[1]
    w = cc_weights(J)
    X = np.zeros((F, J, N + 1), dtype=np.complex128)
    for m in range(N + 1):
        a = abar[coef_offset(N, m):coef_offset(N, m) + N - m + 1]
        X[:, :, m] = legendre_inverse_m(a, pnm_cc(N, J, m, m))
    E = _twiddle(I, np.arange(N + 1), +1.0).T           # [N+1][I]
    return np.real(X @ E) * (w[None, :, None] / I)


def adjoint_analysis_rows(abar, N, J, I, rows):
    """``adjoint_analysis`` evaluated only at the 1-based latitudes ``rows``
    (all longitudes): the same formula with P~ and w taken at those nodes.
    Returns real [F][len(rows)][I]."""
    abar = np.asarray(abar, dtype=np.complex128)
    F = abar.shape[1]
    rows = np.asarray(rows)
    w = cc_weights(J)[rows - 1]
    X = np.zeros((F, len(rows), N + 1), dtype=np.complex128)
    for m in range(N + 1):
        a = abar[coef_offset(N, m):coef_offset(N, m) + N - m + 1]
        X[:, :, m] = legendre_inverse_m(a, pnm_cc(N, J, m, m, j=rows))
    E = _twiddle(I, np.arange(N + 1), +1.0).T           # [N+1][I]
    return np.real(X @ E) * (w[None, :, None] / I)


def adjoint_synthesis(xbar, N, ms=None):
    """Transpose of ``synthesis`` (grid -> spectrum).

    a~_n^m = c_m sum_j P~_n^m(mu_j) sum_i x~_ij e^{-i m lambda_i}, c_0 = 1,
    c_m = 2 (m >= 1); the m = 0 imaginary part is zero.  Returns the packed
    spectrum [ncoef][F], or, if ``ms`` is given, a dict m -> [N-m+1][F] for
    those zonal wavenumbers only."""
    xbar = np.asarray(xbar, dtype=np.float64)
    F, J, I = xbar.shape
    ml = list(range(N + 1)) if ms is None else list(ms)
    X = dft_forward(xbar, N, ms=ml) * I               # no 1/I
    out = {}
    for k, m in enumerate(ml):
        P = pnm_cc(N, J, m, m)
        a = (2.0 if m >= 1 else 1.0) * (P @ X[:, :, k].T)
        if m == 0:
            a = a.real + 0j
        out[m] = a
    if ms is not None:
        return out
    spec = np.zeros((ncoef(N), F), dtype=np.complex128)
    for m, a in out.items():
        spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1] = a
    return spec


# --------------------------------------------------------------------------
# Nested grids (Sec. 3.2) and restriction (Appendix C)
# --------------------------------------------------------------------------
def nested_rows(J_c, k):
    """1-based fine-grid latitude indices of the coarse nodes.

    The J_c-point grid is nested in the J_f = 2^k (J_c+1) - 1 point grid:
    theta^c_j = j pi/(J_c+1) = (2^k j) pi/(J_f+1)."""
    return (2 ** k) * np.arange(1, J_c + 1)


def restrict_nested(x_fine, k, N_c):
    """Coarse spectrum from a fine grid by injection + coarse analysis.

    The fine grid must have J_f = 2^k (J_c+1) - 1 latitudes and
    I_f = 2^k I_c longitudes; the coarse grid is every 2^k-th latitude
    starting at j = 2^k and every 2^k-th longitude starting at lambda = 0.
    Returns the coarse CC analysis (truncation N_c) of that sub-grid."""
    x_fine = np.asarray(x_fine, dtype=np.float64)
    F, J_f, I_f = x_fine.shape
    s = 2 ** k
    if (J_f + 1) % s != 0 or I_f % s != 0:
        raise ValueError("grid does not nest at this level")
    J_c = (J_f + 1) // s - 1
    rows = nested_rows(J_c, k) - 1
    sub = x_fine[:, rows, ::s]
    return analysis(sub, N_c)


def orthonormality_errors(N, J, m, pnm=None, w=None):
    """Normality and orthogonality errors of Eq. (norm-err)/(orth-err) for
    zonal wavenumber m on the J-point Clenshaw-Curtis grid.  Returns two
    arrays over n = m..N."""
    P = pnm_cc(N, J, m, m) if pnm is None else pnm
    w = cc_weights(J) if w is None else w
    G = (P * w[None, :]) @ P.T
    eN = np.abs(np.diag(G) - 1.0)
    off = np.abs(G - np.diag(np.diag(G)))
    eO = off.max(axis=1) if G.shape[0] > 1 else np.zeros(1)
    return eN, eO


__all__ += ["orthonormality_errors", "cc_node_binary128", "synthesis_rows",
            "adjoint_analysis_rows", "pnm_tables"]


# --------------------------------------------------------------------------
# Reduced Clenshaw-Curtis grids (per-latitude longitude counts, Sec. 6)
# --------------------------------------------------------------------------
def _even_smooth_ceil(x):
    """Smallest even n >= x whose half has no prime factor other than 2, 3,
    5 (so that its half-length FFT factors into radices 2, 3, 4, 5, 8)."""
    n = max(2, int(np.ceil(x)))
    while True:
        if n % 2 == 0:
            h = n // 2
            for p in (2, 3, 5):
                while h % p == 0:
                    h //= p
            if h == 1:
                return n
        n += 1


def reduced_sizes(N, J, I, thr=1e-16, counts=None):
    """Longitude counts I_j of the reduced Clenshaw-Curtis grid.

    Sec. 6 quotes the reduction rule of the JMA model: latitude j carries at
    least 4 M_j + 1 longitudes, M_j being the zonal wavenumber beyond which
    every |P~_n^m(mu_j)| (0 <= n <= N) is below 1e-16.  Read here as:
    M_j = the largest m with some |P~_n^m(mu_j)| >= 1e-16, and I_j = the
    smallest even 2-3-5-smooth count >= 4 M_j + 1 (or, if ``counts`` is
    given, the smallest of those counts >= 4 M_j + 1, else I), capped at the
    full grid's I.  Returns (I_j [J], M_j [J]) with j = 1 first; the P~ come
    from the binary128 recurrence rounded to FP64."""
    P = pnm_cc(N, J)                                   # [ncoef][J]
    M = np.zeros(J, dtype=np.int64)
    for m in range(N + 1):
        r0 = coef_offset(N, m)
        sig = np.any(np.abs(P[r0:r0 + N - m + 1]) >= thr, axis=0)
        M[sig] = m
    def pick(need):
        if counts is None:
            return _even_smooth_ceil(need)
        return next((c for c in sorted(counts) if c >= need), I)
    Ij = np.array([min(I, pick(4 * int(Mj) + 1)) for Mj in M], dtype=np.int64)
    return Ij, M


def reduced_row_offsets(Ij):
    """First point of each latitude row in a field's packed rows."""
    Ij = np.asarray(Ij, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(Ij)])


def reduced_kmax(N, Ij):
    """Largest zonal wavenumber carried on each latitude: min(N, I_j/2 - 1)
    (the Nyquist wavenumber I_j/2 is not a Fourier mode of a real row)."""
    return np.minimum(N, np.asarray(Ij, dtype=np.int64) // 2 - 1)


def _row_phase(I, shift, ms, sign):
    """exp(sign * 2 pi i * m * shift / I): the zonal phase of a row whose
    longitudes are lambda_i = 2 pi (i + shift) / I.  ``shift`` is 0 or 1/2,
    so the angle is reduced exactly as the integer (2 m shift) mod (2 I)."""
    ms = np.asarray(ms, dtype=np.int64)
    r = (ms * int(round(2 * shift))) % (2 * I)
    ang = np.pi * r / I
    return np.cos(ang) + sign * 1j * np.sin(ang)


def octahedral_sizes(J, first=20, step=4):
    """Longitude counts of the octahedral Clenshaw-Curtis grid (Sec. 6): the
    j-th latitude from either pole (j = 1..J_h) carries first + step (j - 1)
    points (ECMWF's octahedral pattern, 20 at the first row and 4 more per
    row), mirrored about the Equator.  Returns I_j [J], j = 1 first."""
    Jh = (J + 1) // 2
    north = [first + step * (j - 1) for j in range(1, Jh + 1)]
    return np.array(north + north[:J - Jh][::-1], dtype=np.int64)


def icositetrahedral_sizes(J):
    """Longitude counts and zonal shifts of the icositetrahedral
    Clenshaw-Curtis grid (Sec. 6): 24 equal-area triangular panels, 6 around
    each pole from the pole to 30 degrees of latitude and 12 in the tropical
    belt.  The j-th latitude from either pole carries 6 j points (6 panels of
    j points each) up to the row j30 nearest 30 degrees (theta = pi/3, so
    j30 = round((J+1)/3)), and 6 j30 points on every tropical row; tropical
    rows alternate between unshifted longitudes and longitudes shifted by
    half a spacing (the phase shift in the zonal transform that the paper
    names), counting from j30, which is unshifted.  Returns (I_j [J],
    shift_j [J] in units of the row's spacing), j = 1 first."""
    Jh = (J + 1) // 2
    j30 = int(round((J + 1) / 3.0))
    Ij = np.zeros(J, dtype=np.int64)
    sh = np.zeros(J)
    for j in range(1, Jh + 1):
        Ij[j - 1] = 6 * min(j, j30)
        sh[j - 1] = 0.5 * ((j - j30) % 2) if j > j30 else 0.0
        Ij[J - j] = Ij[j - 1]
        sh[J - j] = sh[j - 1]
    return Ij, sh


def analysis_reduced(x, N, J, Ij, shifts=None):
    """Forward SHT on a reduced Clenshaw-Curtis grid.

    x: real [F][sum I_j], latitude rows packed one after another (j = 1
    first).  Row j gives X^m(phi_j) by the zonal DFT of its I_j points
    (discretised Eq. dFT with 1/I_j) for m <= min(N, I_j/2 - 1), and 0 above;
    then the quadrature of Eq. (cc-quad) over all J nodes.  ``shifts``
    (default 0): row j's longitudes are lambda_i = 2 pi (i + shifts[j]) /
    I_j, so its DFT carries the phase exp(-i m 2 pi shifts[j] / I_j).
    Returns the packed spectrum [ncoef][F]."""
    x = np.asarray(x, dtype=np.float64)
    F = x.shape[0]
    off = reduced_row_offsets(Ij)
    K = reduced_kmax(N, Ij)
    X = np.zeros((F, J, N + 1), dtype=np.complex128)
    for j in range(J):
        row = x[:, off[j]:off[j + 1]]
        X[:, j, :K[j] + 1] = dft_forward(row, int(K[j]))
        if shifts is not None and shifts[j] != 0:
            X[:, j, :K[j] + 1] *= _row_phase(int(Ij[j]), shifts[j],
                                             np.arange(K[j] + 1), -1.0)
    w = cc_weights(J)
    spec = np.zeros((ncoef(N), F), dtype=np.complex128)
    for m in range(N + 1):
        a = legendre_forward_m(X[:, :, m], pnm_cc(N, J, m, m), w)
        if m == 0:
            a = a.real + 0j
        spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1] = a
    return spec


def synthesis_reduced(spec, N, J, Ij, shifts=None):
    """Inverse SHT (Eq. iSHT via Eq. iLT) on a reduced Clenshaw-Curtis grid:
    X^m(phi_j) for every node, then row j is the inverse zonal DFT of
    m <= min(N, I_j/2 - 1) on its I_j longitudes (shifted by shifts[j]
    spacings, as in ``analysis_reduced``).  Returns [F][sum I_j]."""
    spec = np.asarray(spec, dtype=np.complex128)
    F = spec.shape[1]
    X = np.zeros((F, J, N + 1), dtype=np.complex128)
    for m in range(N + 1):
        a = spec[coef_offset(N, m):coef_offset(N, m) + N - m + 1]
        X[:, :, m] = legendre_inverse_m(a, pnm_cc(N, J, m, m))
    off = reduced_row_offsets(Ij)
    K = reduced_kmax(N, Ij)
    out = np.zeros((F, int(off[-1])), dtype=np.float64)
    for j in range(J):
        Xj = X[:, j, :K[j] + 1]
        if shifts is not None and shifts[j] != 0:
            Xj = Xj * _row_phase(int(Ij[j]), shifts[j], np.arange(K[j] + 1), +1.0)
        out[:, off[j]:off[j + 1]] = dft_inverse(Xj, int(Ij[j]))
    return out


# --------------------------------------------------------------------------
# Aliasing of quadratic and cubic terms (Sec. 4.2)
# --------------------------------------------------------------------------
def aliasing_products(specU, specV, specW, N, J, I, quad="cc"):
    """Steps 2-3 of the aliasing experiment of Sec. 4.2: synthesise U, V, W
    from their spectra (Eq. iSHT) on the J x I grid, form the quadratic and
    cubic terms X_q = U V and X_c = U V W at every grid point, and analyse
    both (Eq. dSHT with the zonal DFT and the grid's quadrature).

    quad: "cc" (Clenshaw-Curtis nodes and weights, Eq. cc-quad) or "gauss"
    (Gaussian nodes and weights, Eq. gauss-quad).  Spectra [ncoef][F];
    returns (X_q, X_c) spectra [ncoef][F]."""
    syn = synthesis if quad == "cc" else synthesis_gauss
    ana = analysis if quad == "cc" else analysis_gauss
    U = syn(specU, N, J, I)
    V = syn(specV, N, J, I)
    W = syn(specW, N, J, I)
    Xq = U * V
    Xc = Xq * W
    return ana(Xq, N), ana(Xc, N)


def aliasing_error(test, ref):
    """Normalised aliasing error of Sec. 4.2 per stored (n, m):
    |X_test - X_ref| / |X_ref| (elementwise over [ncoef][F])."""
    return np.abs(np.asarray(test) - np.asarray(ref)) / np.abs(np.asarray(ref))


__all__ += ["aliasing_products", "aliasing_error", "octahedral_sizes",
            "icositetrahedral_sizes"]

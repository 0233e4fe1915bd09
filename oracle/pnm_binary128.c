/*
 * Oracle: normalised associated Legendre functions in binary128, rounded
 * to FP64 at the end.  TEST INFRASTRUCTURE ONLY: nothing in the product
 * path links, loads or calls this file.
 *
 * Follows Sec. 4.1 of Hotta & Ujiie (2018): the table of P~_n^m(sin phi_j)
 * is built by the three-point recurrence in quadruple precision and then
 * cast to double.  The normalisation is Eq. (pnm-ortho):
 *     int_{-1}^{1} P~_n^m(mu) P~_{n'}^m(mu) dmu = delta_{n n'},
 * with no Condon-Shortley phase (P~_m^m > 0 for 0 < theta < pi).
 *
 * Recurrence (standard, written out here):
 *     P~_0^0         = 1/sqrt(2)
 *     P~_m^m         = sqrt((2m+1)/(2m)) sin(theta) P~_{m-1}^{m-1}
 *     P~_{m+1}^m     = sqrt(2m+3) mu P~_m^m
 *     P~_n^m         = (mu P~_{n-1}^m - eps_{n-1}^m P~_{n-2}^m) / eps_n^m
 *     eps_n^m        = sqrt((n^2 - m^2) / (4 n^2 - 1))
 *
 * binary128 has a 15-bit exponent (range ~1e+-4932), so sin^m(theta) at the
 * polar-most node of a T639 grid (~1e-1670) does not underflow; values that
 * fall below the FP64 range become FP64 subnormals or zero on the final cast.
 *
 * Clenshaw-Curtis nodes (Eq. cc-points): theta_j = j pi / (J+1), j = 1..J.
 * Their sine and cosine are evaluated in binary128 by Taylor series after
 * the exact reduction theta -> min(j, J+1-j) pi/(J+1) <= pi/2.
 *
 * The portable C type _Float128 is used (binary128 on x86-64 and aarch64);
 * the square root is Newton's iteration seeded by the FP64 root.
 */
#include <stddef.h>

typedef _Float128 q_t;

static const q_t Q_PI =
    3.14159265358979323846264338327950288419716939937510582097494459f128;

static q_t q_sqrt(q_t a) {
    if (a <= 0) return 0;
    q_t x = (q_t)__builtin_sqrt((double)a);   /* FP64 seed, ~1e-16 rel */
    for (int it = 0; it < 3; ++it) x = 0.5f128 * (x + a / x);
    return x;
}

/* sin and cos of x, 0 <= x <= pi/2, by Taylor series in binary128 */
static void q_sincos(q_t x, q_t* s, q_t* c) {
    q_t x2 = x * x;
    q_t term = x, sum = x;
    for (int k = 1; k < 60; ++k) {
        term = -term * x2 / (q_t)((2 * k) * (2 * k + 1));
        sum += term;
    }
    *s = sum;
    term = 1; sum = 1;
    for (int k = 1; k < 60; ++k) {
        term = -term * x2 / (q_t)((2 * k - 1) * (2 * k));
        sum += term;
    }
    *c = sum;
}

/* Fill out[(row) * nj + jj] for m in [m_lo, m_hi], n in [m, N], rows packed
 * m-major relative to m_lo, at the points (cos_t[jj], sin_t[jj]).
 * The recurrence coefficients are computed once, in binary128, and shared
 * by all points.  Returns 0, or -1 if scratch memory is unavailable. */
static int pnm_rows(int N, int m_lo, int m_hi, const q_t* ct, const q_t* st,
                    int nj, double* out) {
    /* coefficients for the requested orders only: rows of m_lo..m_hi */
    size_t nrow = 0;
    for (int m = m_lo; m <= m_hi; ++m) nrow += (size_t)(N - m + 1);
    q_t* eps = (q_t*)__builtin_malloc(sizeof(q_t) * (nrow ? nrow : 1));   /* eps_n^m  */
    q_t* ieps = (q_t*)__builtin_malloc(sizeof(q_t) * (nrow ? nrow : 1));  /* 1/eps_n^m */
    q_t* amm = (q_t*)__builtin_malloc(sizeof(q_t) * (size_t)(N + 1));
    if (!eps || !ieps || !amm) {
        __builtin_free(eps); __builtin_free(ieps); __builtin_free(amm);
        return -1;
    }
    for (int m = 0; m <= m_hi; ++m)
        amm[m] = m > 0 ? q_sqrt((q_t)(2 * m + 1) / (q_t)(2 * m)) : 0;
    size_t off = 0;
    for (int m = m_lo; m <= m_hi; ++m) {
        for (int n = m; n <= N; ++n) {
            q_t nn = (q_t)n, mm = (q_t)m;
            q_t e = n > m ? q_sqrt((nn * nn - mm * mm) / (4 * nn * nn - 1)) : 0;
            eps[off + (size_t)(n - m)] = e;
            ieps[off + (size_t)(n - m)] = n > m ? 1 / e : 0;
        }
        off += (size_t)(N - m + 1);
    }
    const q_t p00 = 1 / q_sqrt(2.0f128);
#pragma omp parallel for schedule(dynamic, 4)
    for (int jj = 0; jj < nj; ++jj) {
        q_t mu = ct[jj], s = st[jj];
        q_t p_mm = p00;                          /* P~_0^0 */
        size_t row = 0;                          /* = offset into eps/ieps */
        for (int m = 0; m <= m_hi; ++m) {
            if (m > 0) p_mm = amm[m] * s * p_mm;
            if (m < m_lo) continue;
            out[row * (size_t)nj + jj] = (double)p_mm;
            q_t p2 = 0, p1 = p_mm;               /* P~_{n-2}^m, P~_{n-1}^m */
            for (int n = m + 1; n <= N; ++n) {
                /* eps_{m}^m = 0 makes n = m+1 the two-term start:
                 * P~_{m+1}^m = mu P~_m^m / eps_{m+1}^m = sqrt(2m+3) mu P~_m^m */
                q_t pn = (mu * p1 - eps[row + (size_t)(n - 1 - m)] * p2) *
                         ieps[row + (size_t)(n - m)];
                out[(row + (size_t)(n - m)) * (size_t)nj + jj] = (double)pn;
                p2 = p1; p1 = pn;
            }
            row += (size_t)(N - m + 1);
        }
    }
    __builtin_free(eps); __builtin_free(ieps); __builtin_free(amm);
    return 0;
}

/* P~_n^m(cos theta_j) at the Clenshaw-Curtis nodes j in jlist (1-based,
 * theta_j = j pi / (J+1)), for m_lo <= m <= m_hi, m <= n <= N.
 * out has sum_{m=m_lo}^{m_hi} (N-m+1) rows of nj doubles.  Returns 0, or -1
 * on a bad argument. */
int oracle_pnm_cc(int N, int J, int m_lo, int m_hi, const int* jlist, int nj,
                  double* out) {
    if (N < 0 || J < 1 || m_lo < 0 || m_hi > N || m_lo > m_hi || nj < 0)
        return -1;
    q_t* ct = (q_t*)__builtin_malloc(sizeof(q_t) * (size_t)(nj > 0 ? nj : 1));
    q_t* st = (q_t*)__builtin_malloc(sizeof(q_t) * (size_t)(nj > 0 ? nj : 1));
    if (!ct || !st) { __builtin_free(ct); __builtin_free(st); return -1; }
    for (int jj = 0; jj < nj; ++jj) {
        int j = jlist[jj];
        if (j < 1 || j > J) { __builtin_free(ct); __builtin_free(st); return -1; }
        int jr = j <= J + 1 - j ? j : J + 1 - j;      /* theta or pi - theta */
        q_t s, c;
        if (2 * jr == J + 1) { s = 1; c = 0; }         /* the Equator */
        else q_sincos((q_t)jr * Q_PI / (q_t)(J + 1), &s, &c);
        st[jj] = s;
        ct[jj] = (jr == j) ? c : -c;
    }
    int rc = pnm_rows(N, m_lo, m_hi, ct, st, nj, out);
    __builtin_free(ct); __builtin_free(st);
    return rc;
}

/* Same recurrence at arbitrary points given by FP64 cos/sin of the
 * colatitude (used for Gauss-Legendre nodes in the oracle's cross-check). */
int oracle_pnm_at(int N, int m_lo, int m_hi, const double* cos_t,
                  const double* sin_t, int nj, double* out) {
    if (N < 0 || m_lo < 0 || m_hi > N || m_lo > m_hi || nj < 0) return -1;
    q_t* ct = (q_t*)__builtin_malloc(sizeof(q_t) * (size_t)(nj > 0 ? nj : 1));
    q_t* st = (q_t*)__builtin_malloc(sizeof(q_t) * (size_t)(nj > 0 ? nj : 1));
    if (!ct || !st) { __builtin_free(ct); __builtin_free(st); return -1; }
    for (int jj = 0; jj < nj; ++jj) { ct[jj] = cos_t[jj]; st[jj] = sin_t[jj]; }
    int rc = pnm_rows(N, m_lo, m_hi, ct, st, nj, out);
    __builtin_free(ct); __builtin_free(st);
    return rc;
}

/* Binary128 sine/cosine of the node angle, rounded to FP64 (lets the tests
 * check the series against libm). */
int oracle_cc_node_q(int J, int j, double* cos_out, double* sin_out) {
    if (J < 1 || j < 1 || j > J) return -1;
    int jr = j <= J + 1 - j ? j : J + 1 - j;
    q_t s, c;
    if (2 * jr == J + 1) { s = 1; c = 0; }
    else q_sincos((q_t)jr * Q_PI / (q_t)(J + 1), &s, &c);
    *sin_out = (double)s;
    *cos_out = (double)((jr == j) ? c : -c);
    return 0;
}

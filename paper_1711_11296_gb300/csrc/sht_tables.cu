// Plan-time tables: Clenshaw-Curtis nodes and weights, FFT twiddles and the
// normalised associated Legendre functions at the northern nodes.
#include <math.h>

#include <vector>

#include "sht_internal.h"

namespace sht {

// Nodes (Eq. cc-points) and weights (Eq. cc-wgt) of the northern half,
// j = 1..(J+1)/2 (1-based), the Equator last.  theta_j = j pi/(J+1);
// w_j = 4 sin(theta_j)/(J+1) sum_{p odd <= J} sin(p theta_j)/p, each
// sin(p theta_j) taken after the exact integer reduction of p*j modulo
// 2(J+1).  One thread per node; O(J) work each.
__global__ void nodes_weights_kernel(int J, int Jh, int I, int grid, double* mu,
                                     double* sn, double* w, double* w_over_I) {
    const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (j0 >= Jh) return;
    const int j = j0 + 1;
    double s, c, wj;
    if (grid == SHT_GRID_FEJER1) {
        // Eq. (fejer1-points): theta_j = (j - 1/2) pi / J; the weights of
        // Fejer's first rule, w_j = (2/J) (1 - 2 sum_{p=1}^{floor(J/2)}
        // cos(2 p theta_j) / (4p^2 - 1)) (Eq. fejer1-wgt with the factor 2
        // that makes the rule interpolatory), each cosine after reducing the
        // integer p (2j - 1) modulo 2J
        if (2 * j - 1 == J) {
            s = 1.0;
            c = 0.0;
        } else {
            sincospi((double)(2 * j - 1) / (double)(2 * J), &s, &c);
        }
        const long long period = 2LL * J;
        double acc = 0.0;
        for (int p = 1; p <= J / 2; ++p) {
            const long long r = ((long long)p * (2 * j - 1)) % period;
            acc += cospi((double)r / (double)J) / (4.0 * p * p - 1.0);
        }
        wj = 2.0 / (double)J * (1.0 - 2.0 * acc);
    } else {
        if (2 * j == J + 1) {
            s = 1.0;
            c = 0.0;
        } else {
            sincospi((double)j / (double)(J + 1), &s, &c);
        }
        const long long period = 2LL * (J + 1);
        double acc = 0.0;
        for (int p = 1; p <= J; p += 2) {
            const long long r = ((long long)p * j) % period;
            acc += sinpi((double)r / (double)(J + 1)) / (double)p;
        }
        wj = 4.0 * s / (double)(J + 1) * acc;
    }
    mu[j0] = c;
    sn[j0] = s;
    w[j0] = wj;
    w_over_I[j0] = wj / (double)I;
}

// out[e] = exp(-2 pi i e / denom), e < n, rounded to the element type.
template <typename V>
__global__ void twiddle_kernel(V* out, int n, int denom) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s, c;
    sincospi(2.0 * (double)e / (double)denom, &s, &c);
    V v;
    v.x = c;
    v.y = -s;
    out[e] = v;
}

// P~_n^m(mu_j) for one (m, j) per thread, all n = m..N, by the standard
// normalised three-term recurrence that Sec. 4.1 uses:
//   P~_0^0 = 1/sqrt2, P~_m^m = a_m sin(theta) P~_{m-1}^{m-1},
//   P~_n^m = (mu P~_{n-1}^m - eps_{n-1}^m P~_{n-2}^m) / eps_n^m.
// The paper runs it in quadruple precision; here it runs in FP64 with an
// extended exponent: the pair (value, e) stands for value * 2^(256 e), so
// sin^m(theta) near the poles (down to ~1e-1670 at T639) does not underflow
// before the n-recurrence has grown it back into range.  Entries whose true
// value is below the FP64 range come out as subnormals or zero.
__global__ void pnm_kernel(int N, int Jh, int ldp, const double* __restrict__ mu,
                           const double* __restrict__ sn,
                           const double* __restrict__ amm,
                           const double* __restrict__ eps,
                           double* __restrict__ pnm) {
    const int jh = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (jh >= Jh) return;
    const double BIG = 0x1p256, IBIG = 0x1p-256;
    const double x = mu[jh], s = sn[jh];
    double p = 0.70710678118654752440;   // P~_0^0
    int e = 0;
    for (int k = 1; k <= m; ++k) {
        p *= amm[k] * s;
        if (fabs(p) < IBIG) {
            p *= BIG;
            --e;
        }
    }
    const size_t row0 = coef_offset(N, m);
    auto value = [&](double v, int ex) -> double {
        if (ex == 0) return v;
        if (ex < -5) return 0.0;
        for (int k = 0; k < -ex; ++k) v *= IBIG;
        return v;
    };
    pnm[row0 * (size_t)ldp + jh] = value(p, e);
    double p2 = 0.0, p1 = p;
    // eps[] holds, per (m, n), eps_n^m at [row0 + n - m]; slot n = m (eps_m^m = 0)
    // makes n = m+1 the two-term start.  ieps = 1/eps is stored after eps.
    const double* ieps = eps + (size_t)(N + 1) * (N + 2) / 2;
    for (int n = m + 1; n <= N; ++n) {
        double pn = (x * p1 - eps[row0 + (n - 1 - m)] * p2) * ieps[row0 + (n - m)];
        if (e < 0 && fabs(pn) >= BIG) {
            pn *= IBIG;
            p1 *= IBIG;
            ++e;
        }
        pnm[(row0 + (size_t)(n - m)) * (size_t)ldp + jh] = value(pn, e);
        p2 = p1;
        p1 = pn;
    }
}

// Per-pass twiddle tables of the in-place FFT: pass p, entry
// (k1 - 1) M_p + n1 holds W_L^{n1 k1 L / (r_p M_p)}, gathered from the
// length-L table so that both are rounded identically.
template <typename V>
__global__ void twpass_kernel(const V* __restrict__ tw, FftShape sh, V* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sh.twtotal) return;
    int p = 0;
    while (p + 1 < sh.npass && e >= sh.twoff[p + 1]) ++p;
    const int M = sh.span[p];
    const int S = sh.radix[p] * M;
    const int local = e - sh.twoff[p];
    const int k1 = local / M + 1;
    const int n1 = local % M;
    const long long ex = ((long long)n1 * k1 * (sh.L / S)) % sh.L;
    out[e] = tw[ex];
}

cudaError_t launch_twpass(const sht_plan_s* p, cudaStream_t s) {
    if (p->fft.twtotal == 0) return cudaSuccess;
    const int threads = 128;
    const int blocks = (p->fft.twtotal + threads - 1) / threads;
    if (p->prec == SHT_FP64)
        twpass_kernel<double2><<<blocks, threads, 0, s>>>((const double2*)p->d_tw, p->fft,
                                                          (double2*)p->d_twpass);
    else
        twpass_kernel<float2><<<blocks, threads, 0, s>>>((const float2*)p->d_tw, p->fft,
                                                         (float2*)p->d_twpass);
    return cudaGetLastError();
}

cudaError_t build_node_tables(sht_plan_s* p, cudaStream_t s) {
    const int threads = 128;
    nodes_weights_kernel<<<(p->Jh + threads - 1) / threads, threads, 0, s>>>(
        p->J, p->Jh, p->I, p->grid, p->d_mu, p->d_sin, p->d_w, p->d_w_over_I);
    return cudaGetLastError();
}

cudaError_t build_pnm_table(sht_plan_s* p, cudaStream_t s) {
    // Recurrence coefficients on the host (correctly rounded sqrt):
    // eps_n^m = sqrt((n^2 - m^2)/(4 n^2 - 1)), 1/eps, a_m = sqrt((2m+1)/(2m)).
    const int N = p->N;
    const size_t nc = p->ncoef;
    std::vector<double> eps(2 * nc, 0.0), amm(N + 1, 0.0);
    for (int m = 0; m <= N; ++m) {
        amm[m] = m > 0 ? sqrt((2.0 * m + 1.0) / (2.0 * m)) : 0.0;
        const size_t r0 = coef_offset(N, m);
        for (int n = m + 1; n <= N; ++n) {
            const double nn = n, mm = m;
            const double e = sqrt((nn * nn - mm * mm) / (4.0 * nn * nn - 1.0));
            eps[r0 + (n - m)] = e;
            eps[nc + r0 + (n - m)] = 1.0 / e;
        }
    }
    cudaError_t err = cudaMemcpyAsync(p->d_eps, eps.data(), 2 * nc * sizeof(double),
                                      cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(p->d_amm, amm.data(), (N + 1) * sizeof(double),
                          cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(p->d_pnm, 0, nc * (size_t)p->ldp * sizeof(double), s);
    if (err != cudaSuccess) return err;
    const int threads = 128;
    dim3 grid((p->Jh + threads - 1) / threads, N + 1);
    pnm_kernel<<<grid, threads, 0, s>>>(N, p->Jh, p->ldp, p->d_mu, p->d_sin,
                                        p->d_amm, p->d_eps, p->d_pnm);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // the host vectors must outlive the copies
    return cudaStreamSynchronize(s);
}

cudaError_t build_twiddles(sht_plan_s* p, cudaStream_t s) {
    const int L = p->fft.L;
    const int threads = 128;
    const int blocks = (L + threads - 1) / threads;
    if (p->prec == SHT_FP64) {
        twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)p->d_tw, L, L);
        twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)p->d_twpost, L, p->I);
    } else {
        twiddle_kernel<float2><<<blocks, threads, 0, s>>>((float2*)p->d_tw, L, L);
        twiddle_kernel<float2><<<blocks, threads, 0, s>>>((float2*)p->d_twpost, L, p->I);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    err = launch_twpass(p, s);
    if (err != cudaSuccess) return err;
    // digit-reversed output positions of the in-place mixed-radix FFT
    std::vector<int> rev(L);
    for (int k = 0; k < L; ++k) {
        int kk = k, pos = 0;
        for (int q = 0; q < p->fft.npass; ++q) {
            pos += (kk % p->fft.radix[q]) * p->fft.span[q];
            kk /= p->fft.radix[q];
        }
        rev[k] = pos;
    }
    err = cudaMemcpyAsync(p->d_rev, rev.data(), L * sizeof(int),
                          cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    return cudaStreamSynchronize(s);
}

// FFT tables of one half-length (I = 2 sh.L longitudes) into caller-owned
// device buffers: the per-pass twiddle tables (sh.twtotal entries), the
// real-spectrum twiddles e^{-2 pi i q / I} (L entries) and the digit-
// reversed positions (L ints).  tmp holds L complex entries (the length-L
// table the per-pass tables are gathered from).  Synchronises s.
cudaError_t build_fft_tables(const FftShape& sh, bool fp64, void* twpass, void* twpost,
                             int* rev, void* tmp, cudaStream_t s) {
    const int L = sh.L;
    const int threads = 128;
    const int blocks = (L + threads - 1) / threads;
    const int tblocks = (sh.twtotal + threads - 1) / threads;
    if (fp64) {
        twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)tmp, L, L);
        if (sh.twtotal > 0)
            twpass_kernel<double2><<<tblocks, threads, 0, s>>>((const double2*)tmp, sh,
                                                               (double2*)twpass);
        twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)twpost, L, 2 * L);
    } else {
        twiddle_kernel<float2><<<blocks, threads, 0, s>>>((float2*)tmp, L, L);
        if (sh.twtotal > 0)
            twpass_kernel<float2><<<tblocks, threads, 0, s>>>((const float2*)tmp, sh,
                                                              (float2*)twpass);
        twiddle_kernel<float2><<<blocks, threads, 0, s>>>((float2*)twpost, L, 2 * L);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    std::vector<int> h(L);
    for (int k = 0; k < L; ++k) {
        int kk = k, pos = 0;
        for (int q = 0; q < sh.npass; ++q) {
            pos += (kk % sh.radix[q]) * sh.span[q];
            kk /= sh.radix[q];
        }
        h[k] = pos;
    }
    err = cudaMemcpyAsync(rev, h.data(), L * sizeof(int), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    return cudaStreamSynchronize(s);
}

namespace {

// c_n = e^{-pi i n^2 / L}, the angle reduced exactly as (n^2 mod 2L) / L.
template <typename V>
__global__ void chirp_kernel(V* out, double2* out64, int L) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L) return;
    const long long r = ((long long)n * n) % (2LL * L);
    double sn, cs;
    sincospi((double)r / (double)L, &sn, &cs);
    V v;
    v.x = cs;
    v.y = -sn;
    out[n] = v;
    out64[n] = make_double2(cs, -sn);
}

// cos(2 pi r / n), r < n.
__global__ void cos_table_kernel(double* out, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = cospi(2.0 * (double)r / (double)n);
}

// D_k = (1/L2) sum_j b_j e^{-2 pi i j k / L2} for the conjugate chirp b
// wrapped around L2 (b_j = conj c_j for 0 <= j < L, b_{L2-j} = conj c_j for
// 0 < j < L, zero between): D_k = (1/L2) (1 + 2 sum_{0<j<L} conj(c_j)
// cos(2 pi j k / L2)), a direct FP64 sum with j k reduced mod L2 exactly.
template <typename V>
__global__ void bluestein_dft_kernel(V* out, const double2* c, const double* costab, int L,
                                     int L2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L2) return;
    double re = 1.0, im = 0.0;
    int r = 0;
    for (int j = 1; j < L; ++j) {
        r += k;
        if (r >= L2) r -= L2;
        const double cw = 2.0 * costab[r];
        re = fma(c[j].x, cw, re);
        im = fma(-c[j].y, cw, im);
    }
    V v;
    v.x = re / (double)L2;
    v.y = im / (double)L2;
    out[k] = v;
}

template <typename V>
__global__ void shift_kernel(V* out, int n, int I) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double sn, cs;
    sincospi((double)m / (double)I, &sn, &cs);
    V v;
    v.x = cs;
    v.y = -sn;
    out[m] = v;
}

}  // namespace

cudaError_t build_bluestein_tables(int L, const FftShape& sh2, bool fp64, void* twpass,
                                   void* twpost, int* rev, void* chirp, void* dft, void* tmp,
                                   cudaStream_t s) {
    const int L2 = sh2.L;
    const int threads = 128;
    // scratch: L2 entries for the passes' base twiddles, L2 for their unused
    // real-spectrum twiddles, then the FP64 chirp (L) and cosine table (L2)
    char* t = static_cast<char*>(tmp);
    const size_t vb = fp64 ? sizeof(double2) : sizeof(float2);
    void* base = t;
    void* post2 = t + L2 * vb;
    double2* c64 = reinterpret_cast<double2*>(t + 2 * L2 * sizeof(double2));
    double* costab = reinterpret_cast<double*>(c64 + L2);
    cudaError_t e = build_fft_tables(sh2, fp64, twpass, post2, rev, base, s);
    if (e != cudaSuccess) return e;
    const int bL = (L + threads - 1) / threads, bL2 = (L2 + threads - 1) / threads;
    cos_table_kernel<<<bL2, threads, 0, s>>>(costab, L2);
    if (fp64) {
        twiddle_kernel<double2><<<bL, threads, 0, s>>>((double2*)twpost, L, 2 * L);
        chirp_kernel<double2><<<bL, threads, 0, s>>>((double2*)chirp, c64, L);
        bluestein_dft_kernel<double2><<<bL2, threads, 0, s>>>((double2*)dft, c64, costab, L, L2);
    } else {
        twiddle_kernel<float2><<<bL, threads, 0, s>>>((float2*)twpost, L, 2 * L);
        chirp_kernel<float2><<<bL, threads, 0, s>>>((float2*)chirp, c64, L);
        bluestein_dft_kernel<float2><<<bL2, threads, 0, s>>>((float2*)dft, c64, costab, L, L2);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t build_shift_table(int n, int I, bool fp64, void* out, cudaStream_t s) {
    const int threads = 128, blocks = (n + threads - 1) / threads;
    if (fp64)
        shift_kernel<double2><<<blocks, threads, 0, s>>>((double2*)out, n, I);
    else
        shift_kernel<float2><<<blocks, threads, 0, s>>>((float2*)out, n, I);
    return cudaGetLastError();
}

}  // namespace sht

namespace sht {

// Launch only the P~ recurrence kernel; the caller has filled p->d_eps
// (eps and 1/eps, 2*ncoef doubles), p->d_amm, p->d_mu and p->d_sin.
cudaError_t launch_pnm_recurrence(const sht_plan_s* p, cudaStream_t s) {
    const int threads = 128;
    dim3 grid((p->Jh + threads - 1) / threads, p->N + 1);
    pnm_kernel<<<grid, threads, 0, s>>>(p->N, p->Jh, p->ldp, p->d_mu, p->d_sin,
                                        p->d_amm, p->d_eps, p->d_pnm);
    return cudaGetLastError();
}

// Launch only the two twiddle-table kernels (FP64 plans).
cudaError_t launch_twiddles_fp64(const sht_plan_s* p, cudaStream_t s) {
    const int L = p->fft.L;
    const int threads = 128;
    const int blocks = (L + threads - 1) / threads;
    twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)p->d_tw, L, L);
    twiddle_kernel<double2><<<blocks, threads, 0, s>>>((double2*)p->d_twpost, L, p->I);
    return cudaGetLastError();
}

}  // namespace sht

// Batched real FFT along latitude circles, fused with the equatorial
// parity fold (Appendix B) and the [m][parity][j][field] layout change that
// the per-m Legendre contraction wants.
//
// A row of I real samples x_i is read as L = I/2 complex values
// z_k = x_{2k} + i x_{2k+1}; an in-place mixed-radix (2/3/4/5) decimation-in-
// frequency FFT of length L runs in shared memory and leaves Z in
// digit-reversed order (rev[k] = position of frequency k).  The real
// spectrum follows from
//   X_m = (Z_m + conj Z_{L-m})/2 + e^{-2 pi i m/I} (Z_m - conj Z_{L-m})/(2i).
// The inverse builds Z_q = (Y_q + conj Y_{L-q}) + i e^{+2 pi i q/I} (Y_q - conj Y_{L-q})
// from the Hermitian spectrum Y (Y_0 real, Y_m = 0 for m > N) and runs the
// same forward FFT on conj(Z): z = conj(FFT(conj Z)), x_{2k} = Re z_k,
// x_{2k+1} = Im z_k.
//
// One CTA owns latitude pair (j, J-1-j) (0-based; the Equator row alone)
// for G consecutive fields: 2G rows of L complex values plus the twiddle
// table in shared memory.
#include "sht_internal.h"

namespace sht {
namespace {

template <typename T> struct C2 {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ V make(T x, T y) { V v; v.x = x; v.y = y; return v; }
    static __device__ __forceinline__ V add(V a, V b) { return make(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V sub(V a, V b) { return make(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ V mul(V a, V b) {
        return make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    static __device__ __forceinline__ V conj(V a) { return make(a.x, -a.y); }
    static __device__ __forceinline__ V scale(V a, T s) { return make(a.x * s, a.y * s); }
    // multiply by -i
    static __device__ __forceinline__ V mul_mi(V a) { return make(a.y, -a.x); }
    // multiply by +i
    static __device__ __forceinline__ V mul_pi(V a) { return make(-a.y, a.x); }
};

template <typename T>
struct FwdArgs {
    using V = typename Vec2<T>::type;
    const T* grid;
    RowSource src;
    V* work;
    const V* tw;
    const V* twpost;
    const int* rev;
    const double* rowscale;
    double mscale0, mscale1;
    int F, J, Jh, L, N, G;
    FftShape shape;
};

template <typename T>
struct InvArgs {
    using V = typename Vec2<T>::type;
    const V* work;
    T* grid;
    const V* tw;
    const V* twpost;
    const int* rev;
    const double* rowscale;
    double mfactor1;
    int F, J, Jh, I, L, N, G;
    FftShape shape;
};

// In-place mixed-radix DIF FFT (forward sign) over `nrows` rows of length L
// held in shared memory.  Pass p: blocks of S = r M, butterfly (blk, n1)
// reads z[blk S + n1 + M t], t < r, applies the radix-r DFT, multiplies
// output k1 by W_S^{n1 k1} = W_L^{n1 k1 L/S}, and writes it to
// z[blk S + n1 + M k1].
template <typename T>
__device__ void fft_rows_inplace(typename Vec2<T>::type* rows, int nrows, int L,
                                 const FftShape& sh,
                                 const typename Vec2<T>::type* tws) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int p = 0; p < sh.npass; ++p) {
        const int r = sh.radix[p];
        const int M = sh.span[p];
        const int S = r * M;
        const int tws_step = L / S;
        const int nb = L / r;
        const int total = nrows * nb;
        for (int idx = tid; idx < total; idx += nthr) {
            const int row = idx / nb;
            const int b = idx - row * nb;
            const int blk = b / M;
            const int n1 = b - blk * M;
            V* z = rows + (size_t)row * L + blk * S + n1;
            const int te = n1 * tws_step;   // twiddle exponent step for k1 = 1
            if (r == 4) {
                V a0 = z[0], a1 = z[M], a2 = z[2 * M], a3 = z[3 * M];
                V s02 = K::add(a0, a2), d02 = K::sub(a0, a2);
                V s13 = K::add(a1, a3), d13 = K::mul_mi(K::sub(a1, a3));
                V y0 = K::add(s02, s13);
                V y2 = K::sub(s02, s13);
                V y1 = K::add(d02, d13);
                V y3 = K::sub(d02, d13);
                z[0] = y0;
                if (te == 0) {
                    z[M] = y1; z[2 * M] = y2; z[3 * M] = y3;
                } else {
                    z[M] = K::mul(y1, tws[te]);
                    z[2 * M] = K::mul(y2, tws[2 * te]);
                    z[3 * M] = K::mul(y3, tws[3 * te]);
                }
            } else if (r == 2) {
                V a0 = z[0], a1 = z[M];
                z[0] = K::add(a0, a1);
                V y1 = K::sub(a0, a1);
                z[M] = te == 0 ? y1 : K::mul(y1, tws[te]);
            } else if (r == 5) {
                // cos/sin of 2 pi/5 and 4 pi/5
                const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
                const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
                V a0 = z[0], a1 = z[M], a2 = z[2 * M], a3 = z[3 * M], a4 = z[4 * M];
                V b1 = K::add(a1, a4), d1 = K::sub(a1, a4);
                V b2 = K::add(a2, a3), d2 = K::sub(a2, a3);
                V y0 = K::add(a0, K::add(b1, b2));
                V p1 = K::make(a0.x + c1 * b1.x + c2 * b2.x, a0.y + c1 * b1.y + c2 * b2.y);
                V p2 = K::make(a0.x + c2 * b1.x + c1 * b2.x, a0.y + c2 * b1.y + c1 * b2.y);
                // q1 = s1 d1 + s2 d2, q2 = s2 d1 - s1 d2; y1 = p1 - i q1, y4 = p1 + i q1,
                // y2 = p2 - i q2, y3 = p2 + i q2
                V q1 = K::make(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
                V q2 = K::make(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
                V y1 = K::add(p1, K::mul_mi(q1));
                V y4 = K::sub(p1, K::mul_mi(q1));
                V y2 = K::add(p2, K::mul_mi(q2));
                V y3 = K::sub(p2, K::mul_mi(q2));
                z[0] = y0;
                if (te == 0) {
                    z[M] = y1; z[2 * M] = y2; z[3 * M] = y3; z[4 * M] = y4;
                } else {
                    z[M] = K::mul(y1, tws[te]);
                    z[2 * M] = K::mul(y2, tws[2 * te]);
                    z[3 * M] = K::mul(y3, tws[3 * te]);
                    z[4 * M] = K::mul(y4, tws[4 * te]);
                }
            } else {   // r == 3
                const T h = (T)0.86602540378443864676;   // sin(2 pi/3)
                V a0 = z[0], a1 = z[M], a2 = z[2 * M];
                V t1 = K::add(a1, a2), t2 = K::sub(a1, a2);
                V y0 = K::add(a0, t1);
                V m0 = K::make(a0.x - (T)0.5 * t1.x, a0.y - (T)0.5 * t1.y);
                V q = K::mul_mi(K::scale(t2, h));
                V y1 = K::add(m0, q);
                V y2 = K::sub(m0, q);
                z[0] = y0;
                if (te == 0) {
                    z[M] = y1; z[2 * M] = y2;
                } else {
                    z[M] = K::mul(y1, tws[te]);
                    z[2 * M] = K::mul(y2, tws[2 * te]);
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, bool STRIDED>
__global__ void __launch_bounds__(256) fft_forward_kernel(FwdArgs<T> A) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = A.L;
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* rows = tws + L;
    const int jh = blockIdx.x;
    const int f0 = blockIdx.y * A.G;
    const int nf = min(A.G, A.F - f0);
    const bool equator = (jh == A.Jh - 1);
    const int nrows = equator ? nf : 2 * nf;
    const int tid = threadIdx.x, nthr = blockDim.x;

    for (int e = tid; e < L; e += nthr) tws[e] = A.tw[e];
    for (int r = 0; r < nrows; ++r) {
        const int f = f0 + (r % nf);
        const int j = (r < nf) ? jh : (A.J - 1 - jh);
        const T* x = A.grid + (long long)f * A.src.field_stride + A.src.row_offset +
                     (long long)j * A.src.row_stride;
        V* z = rows + (size_t)r * L;
        if (!STRIDED) {
            const V* xv = reinterpret_cast<const V*>(x);
            for (int k = tid; k < L; k += nthr) z[k] = xv[k];
        } else {
            const int s = A.src.elem_stride;
            for (int k = tid; k < L; k += nthr)
                z[k] = K::make(x[(long long)(2 * k) * s], x[(long long)(2 * k + 1) * s]);
        }
    }
    __syncthreads();
    fft_rows_inplace<T>(rows, nrows, L, A.shape, tws);

    const int nout = (A.N + 1) * nf;
    const T rs = A.rowscale ? (T)A.rowscale[jh] : (T)1;
    for (int idx = tid; idx < nout; idx += nthr) {
        const int m = idx / nf;
        const int fl = idx - m * nf;
        const int pm = A.rev[m];
        const int pc = A.rev[(L - m) % L];
        const V w = A.twpost[m];
        auto real_spec = [&](const V* z) -> V {
            V zm = z[pm];
            V zc = K::conj(z[pc]);
            V e = K::add(zm, zc);                  // 2 E_m
            V o = K::mul_mi(K::sub(zm, zc));       // 2 O_m
            return K::add(e, K::mul(w, o));        // 2 X_m
        };
        const V xn = real_spec(rows + (size_t)fl * L);
        V S, Asym;
        if (equator) {
            S = xn;
            Asym = K::make((T)0, (T)0);
        } else {
            const V xs = real_spec(rows + (size_t)(nf + fl) * L);
            S = K::add(xn, xs);
            Asym = K::sub(xn, xs);
        }
        const T sc = (T)0.5 * rs * (T)(m == 0 ? A.mscale0 : A.mscale1);
        const size_t base = ((size_t)m * 2 * A.Jh + jh) * A.F + f0 + fl;
        A.work[base] = K::scale(S, sc);
        A.work[base + (size_t)A.Jh * A.F] = K::scale(Asym, sc);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) fft_inverse_kernel(InvArgs<T> A) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = A.L;
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* rows = tws + L;
    const int jh = blockIdx.x;
    const int f0 = blockIdx.y * A.G;
    const int nf = min(A.G, A.F - f0);
    const bool equator = (jh == A.Jh - 1);
    const int nrows = equator ? nf : 2 * nf;
    const int tid = threadIdx.x, nthr = blockDim.x;

    for (int e = tid; e < L; e += nthr) tws[e] = A.tw[e];
    // unfold S/A into the two hemispheres' zonal spectra Y_m, m <= N
    const int nin = (A.N + 1) * nf;
    for (int idx = tid; idx < nin; idx += nthr) {
        const int m = idx / nf;
        const int fl = idx - m * nf;
        const size_t base = ((size_t)m * 2 * A.Jh + jh) * A.F + f0 + fl;
        const V S = A.work[base];
        const T fac = (T)(m == 0 ? 1.0 : A.mfactor1);
        V yn, ys;
        if (equator) {
            yn = K::scale(S, fac);
            ys = yn;
        } else {
            const V Asym = A.work[base + (size_t)A.Jh * A.F];
            yn = K::scale(K::add(S, Asym), fac);
            ys = K::scale(K::sub(S, Asym), fac);
        }
        if (m == 0) {
            yn.y = (T)0;
            ys.y = (T)0;
        }
        rows[(size_t)fl * L + m] = yn;
        if (!equator) rows[(size_t)(nf + fl) * L + m] = ys;
    }
    const int nz = L - (A.N + 1);
    for (int idx = tid; idx < nrows * nz; idx += nthr) {
        const int r = idx / nz;
        const int q = A.N + 1 + (idx - r * nz);
        rows[(size_t)r * L + q] = K::make((T)0, (T)0);
    }
    __syncthreads();
    // Hermitian packing into conj(Z), pairs (q, L-q) owned by one thread
    const int half = L / 2;
    for (int idx = tid; idx < nrows * (half + 1); idx += nthr) {
        const int r = idx / (half + 1);
        const int q = idx - r * (half + 1);
        const int qc = L - q;
        if (q > qc) continue;
        V* z = rows + (size_t)r * L;
        const V yq = z[q];
        const V yc = (q == 0) ? K::make((T)0, (T)0) : z[qc];
        // Z_q = (Y_q + conj Y_{L-q}) + i conj(W_I^q) (Y_q - conj Y_{L-q})
        const V wq = K::conj(A.twpost[q]);
        const V zq = K::add(K::add(yq, K::conj(yc)),
                            K::mul_pi(K::mul(wq, K::sub(yq, K::conj(yc)))));
        if (q != 0 && q != qc) {
            const V wc = K::conj(A.twpost[qc]);
            const V zc = K::add(K::add(yc, K::conj(yq)),
                                K::mul_pi(K::mul(wc, K::sub(yc, K::conj(yq)))));
            z[qc] = K::conj(zc);
        }
        z[q] = K::conj(zq);
    }
    __syncthreads();
    fft_rows_inplace<T>(rows, nrows, L, A.shape, tws);

    const T rs = A.rowscale ? (T)A.rowscale[jh] : (T)1;
    for (int r = 0; r < nrows; ++r) {
        const int f = f0 + (r % nf);
        const int j = (r < nf) ? jh : (A.J - 1 - jh);
        V* xv = reinterpret_cast<V*>(A.grid + ((long long)f * A.J + j) * A.I);
        const V* z = rows + (size_t)r * L;
        for (int k = tid; k < L; k += nthr) {
            const V v = z[A.rev[k]];
            xv[k] = K::make(v.x * rs, -v.y * rs);
        }
    }
}

template <typename K>
void set_smem_attr(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
}

template <typename T>
cudaError_t fwd_impl(const sht_plan_s* p, const void* grid, const RowSource& src,
                     const FwdScale& sc, void* work, cudaStream_t s) {
    using V = typename Vec2<T>::type;
    FwdArgs<T> A;
    A.grid = static_cast<const T*>(grid);
    A.src = src;
    A.work = static_cast<V*>(work);
    A.tw = static_cast<const V*>(p->d_tw);
    A.twpost = static_cast<const V*>(p->d_twpost);
    A.rev = p->d_rev;
    A.rowscale = sc.rowscale;
    A.mscale0 = sc.mscale0;
    A.mscale1 = sc.mscale1;
    A.F = p->F; A.J = p->J; A.Jh = p->Jh; A.L = p->fft.L; A.N = p->N; A.G = p->G;
    A.shape = p->fft;
    dim3 grid_dim(p->Jh, (p->F + p->G - 1) / p->G);
    const size_t smem = p->fft_smem;
    if (src.elem_stride == 1) {
        set_smem_attr(fft_forward_kernel<T, false>, smem);
        fft_forward_kernel<T, false><<<grid_dim, p->fft_threads, smem, s>>>(A);
    } else {
        set_smem_attr(fft_forward_kernel<T, true>, smem);
        fft_forward_kernel<T, true><<<grid_dim, p->fft_threads, smem, s>>>(A);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t inv_impl(const sht_plan_s* p, const void* work, const InvScale& sc,
                     void* grid, cudaStream_t s) {
    using V = typename Vec2<T>::type;
    InvArgs<T> A;
    A.work = static_cast<const V*>(work);
    A.grid = static_cast<T*>(grid);
    A.tw = static_cast<const V*>(p->d_tw);
    A.twpost = static_cast<const V*>(p->d_twpost);
    A.rev = p->d_rev;
    A.rowscale = sc.rowscale;
    A.mfactor1 = sc.mfactor1;
    A.F = p->F; A.J = p->J; A.Jh = p->Jh; A.I = p->I; A.L = p->fft.L; A.N = p->N;
    A.G = p->G;
    A.shape = p->fft;
    dim3 grid_dim(p->Jh, (p->F + p->G - 1) / p->G);
    const size_t smem = p->fft_smem;
    set_smem_attr(fft_inverse_kernel<T>, smem);
    fft_inverse_kernel<T><<<grid_dim, p->fft_threads, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

size_t fft_smem_bytes(int I, int G, bool fp64) {
    const size_t L = (size_t)I / 2;
    const size_t v = fp64 ? sizeof(double2) : sizeof(float2);
    return (L + 2 * (size_t)G * L) * v;
}

cudaError_t launch_fft_forward(const sht_plan_s* p, const void* grid,
                               const RowSource& src, const FwdScale& sc,
                               void* work, cudaStream_t s) {
    if (p->prec == SHT_FP64) return fwd_impl<double>(p, grid, src, sc, work, s);
    return fwd_impl<float>(p, grid, src, sc, work, s);
}

cudaError_t launch_fft_inverse(const sht_plan_s* p, const void* work,
                               const InvScale& sc, void* grid, cudaStream_t s) {
    if (p->prec == SHT_FP64) return inv_impl<double>(p, work, sc, grid, s);
    return inv_impl<float>(p, work, sc, grid, s);
}

}  // namespace sht

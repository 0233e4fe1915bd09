// Batched real FFT along latitude circles, fused with the equatorial
// parity fold (Appendix B) and the [m][parity][j][field] layout change that
// the per-m Legendre contraction wants.
//
// A row of I real samples x_i is read as L = I/2 complex values
// z_k = x_{2k} + i x_{2k+1}; an in-place mixed-radix (2/3/4/5/8) decimation-in-
// frequency FFT of length L runs in shared memory and leaves Z in
// digit-reversed order (rev(k) = position of frequency k).  The real
// spectrum follows from
//   X_m = (Z_m + conj Z_{L-m})/2 + e^{-2 pi i m/I} (Z_m - conj Z_{L-m})/(2i).
// The inverse builds Z_q = (Y_q + conj Y_{L-q}) + i e^{+2 pi i q/I} (Y_q - conj Y_{L-q})
// from the Hermitian spectrum Y (Y_0 real, Y_m = 0 for m > N) and runs the
// same forward FFT on conj(Z): z = conj(FFT(conj Z)), x_{2k} = Re z_k,
// x_{2k+1} = Im z_k.
//
// One CTA owns latitude pair (j, J-1-j) (0-based; the Equator row alone)
// for G consecutive fields: 2G rows of L complex values plus the per-pass
// twiddle tables in shared memory.  Rows use the padded layout of
// PadShift (element pos at pos + (pos >> s), odd row pitch), which keeps the
// passes' power-of-two strides, the digit-reversed accesses and the
// row-to-row distance off a single bank; each pass reads its twiddles from
// a table contiguous in the butterfly index.  Global loads are
// asynchronous element copies (cp.async) straight into the padded layout,
// all in flight before the CTA waits once, except where the FP32 two-pass
// lengths (L = Q x 32, Q >= 8) let the forward's first pass read the grid
// rows into registers and the inverse's last pass write them from
// registers.  The CTAs of all field groups of one latitude are adjacent in
// the launch order, so their partial-sector writes of the same workspace
// rows meet in L2.
//
// The half-lengths of the standard grids (64 ... 1280) have kernels
// specialised at compile time: radices, spans, twiddle offsets and the
// digit reversal are constants, so the index arithmetic needs no integer
// division by a runtime value.  Other lengths use the same code with the
// shape read at run time (radices up to 8: the larger ones only occur in
// the standard lengths).  Grouped launches branch per CTA to the body of
// their plan's length, and a reduced grid launches the compile-time kernel
// once per row length it contains, over a list of latitude pairs.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "sht_internal.h"

namespace sht {
namespace {

constexpr int NT = 256;   // threads per FFT CTA (two CTAs per SM for FP32)

// Paired FP32 arithmetic (add/sub/mul.f32x2): one instruction on both
// components of a complex value.
__device__ __forceinline__ float2 add_f32x2(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t*>(&a)), "l"(*reinterpret_cast<const uint64_t*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}
__device__ __forceinline__ float2 sub_f32x2(float2 a, float2 b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t*>(&a)), "l"(*reinterpret_cast<const uint64_t*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}
__device__ __forceinline__ float2 mul_f32x2(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t*>(&a)), "l"(*reinterpret_cast<const uint64_t*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}

template <typename T> struct C2 {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ V make(T x, T y) { V v; v.x = x; v.y = y; return v; }
    static __device__ __forceinline__ V add(V a, V b) {
        if constexpr (sizeof(T) == 4)
            return add_f32x2(a, b);
        else
            return make(a.x + b.x, a.y + b.y);
    }
    static __device__ __forceinline__ V sub(V a, V b) {
        if constexpr (sizeof(T) == 4)
            return sub_f32x2(a, b);
        else
            return make(a.x - b.x, a.y - b.y);
    }
    static __device__ __forceinline__ V mul(V a, V b) {
        return make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    static __device__ __forceinline__ V conj(V a) { return make(a.x, -a.y); }
    static __device__ __forceinline__ V scale(V a, T s) {
        if constexpr (sizeof(T) == 4)
            return mul_f32x2(a, make(s, s));
        else
            return make(a.x * s, a.y * s);
    }
    // multiply by -i
    static __device__ __forceinline__ V mul_mi(V a) { return make(a.y, -a.x); }
    // multiply by +i
    static __device__ __forceinline__ V mul_pi(V a) { return make(-a.y, a.x); }
};

// The plan's factorisation as a compile-time constant.
template <int L, bool FP64> struct FacOf {
    static constexpr FftShape v = fft_factor(L, FP64);
};

// W_N^e = exp(-2 pi i e/N) for the composite register DFT sizes, written
// once per device by fft_constants_init (offsets per N below).
constexpr int kTw10 = 0, kTw16 = 10, kTw20 = 26, kTw32 = 46, kTw40 = 78, kTwTotal = 118;
__constant__ float2 c_twf[kTwTotal];
__constant__ double2 c_twd[kTwTotal];

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type twc(int idx) {
    if constexpr (sizeof(T) == 4)
        return c_twf[idx];
    else
        return c_twd[idx];
}

// Asynchronous global -> shared copy of one element (cp.async, no register
// staging, so all of a thread's copies are in flight at once).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES)
                     : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ int ph(int pos) {
    return pos + (pos >> PadShift<T>::value);
}

// ---- radix-R DFTs (forward sign) ---------------------------------------
template <typename T, int R> struct Dft;

template <typename T> struct Dft<T, 2> {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return k; }
    static __device__ __forceinline__ void run(V* a) {
        using K = C2<T>;
        const V y0 = K::add(a[0], a[1]);
        a[1] = K::sub(a[0], a[1]);
        a[0] = y0;
    }
};

template <typename T> struct Dft<T, 3> {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return k; }
    static __device__ __forceinline__ void run(V* a) {
        using K = C2<T>;
        const T h = (T)0.86602540378443864676;   // sin(2 pi/3)
        const V t1 = K::add(a[1], a[2]), t2 = K::sub(a[1], a[2]);
        const V y0 = K::add(a[0], t1);
        const V m0 = K::make(a[0].x - (T)0.5 * t1.x, a[0].y - (T)0.5 * t1.y);
        // m0 -+ i h t2, component by component
        a[0] = y0;
        a[1] = K::make(m0.x + h * t2.y, m0.y - h * t2.x);
        a[2] = K::make(m0.x - h * t2.y, m0.y + h * t2.x);
    }
};

template <typename T> struct Dft<T, 4> {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return k; }
    static __device__ __forceinline__ void run(V* a) {
        using K = C2<T>;
        const V s02 = K::add(a[0], a[2]), d02 = K::sub(a[0], a[2]);
        const V s13 = K::add(a[1], a[3]), t = K::sub(a[1], a[3]);
        a[0] = K::add(s02, s13);
        a[2] = K::sub(s02, s13);
        // d02 -+ i t, component by component (no swapped pair)
        a[1] = K::make(d02.x + t.y, d02.y - t.x);
        a[3] = K::make(d02.x - t.y, d02.y + t.x);
    }
};

template <typename T> struct Dft<T, 8> {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return k; }
    static __device__ __forceinline__ void run(V* a) {
        using K = C2<T>;
        const T r = (T)0.70710678118654752440;   // 1/sqrt(2)
        // even and odd halves by radix 4, then y_k = E_k + W8^k O_k,
        // y_{k+4} = E_k - W8^k O_k with W8 = e^{-2 pi i/8}
        V e[4] = {a[0], a[2], a[4], a[6]};
        V o[4] = {a[1], a[3], a[5], a[7]};
        Dft<T, 4>::run(e);
        Dft<T, 4>::run(o);
        const V o1 = K::make(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));   // W8^1 o1
        const V o3 = K::make(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));   // W8^3 o3
        a[0] = K::add(e[0], o[0]);
        a[4] = K::sub(e[0], o[0]);
        a[1] = K::add(e[1], o1);
        a[5] = K::sub(e[1], o1);
        // W8^2 o2 = -i o2, component by component
        a[2] = K::make(e[2].x + o[2].y, e[2].y - o[2].x);
        a[6] = K::make(e[2].x - o[2].y, e[2].y + o[2].x);
        a[3] = K::add(e[3], o3);
        a[7] = K::sub(e[3], o3);
    }
};

template <typename T> struct Dft<T, 5> {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return k; }
    static __device__ __forceinline__ void run(V* a) {
        using K = C2<T>;
        // cos/sin of 2 pi/5 and 4 pi/5
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
        const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
        const V b1 = K::add(a[1], a[4]), d1 = K::sub(a[1], a[4]);
        const V b2 = K::add(a[2], a[3]), d2 = K::sub(a[2], a[3]);
        const V y0 = K::add(a[0], K::add(b1, b2));
        const V p1 = K::make(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
        const V p2 = K::make(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
        // q1 = s1 d1 + s2 d2, q2 = s2 d1 - s1 d2; y1 = p1 - i q1, y4 = p1 + i q1,
        // y2 = p2 - i q2, y3 = p2 + i q2
        const V q1 = K::make(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        const V q2 = K::make(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        a[0] = y0;
        a[1] = K::make(p1.x + q1.y, p1.y - q1.x);
        a[4] = K::make(p1.x - q1.y, p1.y + q1.x);
        a[2] = K::make(p2.x + q2.y, p2.y - q2.x);
        a[3] = K::make(p2.x - q2.y, p2.y + q2.x);
    }
};

// Composite DFT of size N = A B in registers, in place:
//   X[k1 + A k2] = sum_b W_B^{b k2} W_N^{b k1} sum_a x[b + B a] W_A^{a k1},
// i.e. B DFTs of size A over stride-B subsequences (results written back to
// the same registers), the twiddles W_N^{b k1} (constant memory), then A
// DFTs of size B over each contiguous block of B.  X[k] is left in
// register pos(k) = k1 B + k2 (k = k1 + A k2); the butterfly stores with
// this map, so no register array beyond the input is live.
template <typename T, int A, int B, int TWOFF>
struct DftComposite {
    using V = typename Vec2<T>::type;
    static __device__ __forceinline__ constexpr int pos(int k) { return (k % A) * B + k / A; }
    static __device__ __forceinline__ void run(V* x) {
        using K = C2<T>;
        constexpr int N = A * B;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            V t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = x[b + B * a];
            Dft<T, A>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1)
                x[b + B * k1] =
                    (b * k1 == 0) ? t[k1] : K::mul(t[k1], twc<T>(TWOFF + (b * k1) % N));
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            V t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = x[k1 * B + b];
            Dft<T, B>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) x[k1 * B + k2] = t[k2];
        }
    }
};

template <typename T> struct Dft<T, 10> : DftComposite<T, 2, 5, kTw10> {};
template <typename T> struct Dft<T, 16> : DftComposite<T, 4, 4, kTw16> {};
template <typename T> struct Dft<T, 20> : DftComposite<T, 4, 5, kTw20> {};
template <typename T> struct Dft<T, 32> : DftComposite<T, 8, 4, kTw32> {};
template <typename T> struct Dft<T, 40> : DftComposite<T, 8, 5, kTw40> {};

// One DIF butterfly of radix R: reads z[base + t M], t < R, applies the
// radix-R DFT, multiplies output k1 by W_S^{n1 k1} (per-pass table entry
// (k1 - 1) M + n1) and writes it back to z[base + k1 M].
template <typename T, int R>
__device__ __forceinline__ void bfly(typename Vec2<T>::type* z, int base, int M,
                                     const typename Vec2<T>::type* tw, int n1) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    V a[R];
#pragma unroll
    for (int t = 0; t < R; ++t) a[t] = z[ph<T>(base + t * M)];
    Dft<T, R>::run(a);
    // output k1 sits in register pos(k1)
    if (n1 != 0) {
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) {
            a[Dft<T, R>::pos(k1)] = K::mul(a[Dft<T, R>::pos(k1)], tw[(k1 - 1) * M + n1]);
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) z[ph<T>(base + k1 * M)] = a[Dft<T, R>::pos(k1)];
}

// The same with the span M a compile-time constant.  When M is a multiple
// of the padding period P (pad one element per P), or R M divides P, the
// padded positions of the R elements are ph(base) + t STEP with a constant
// STEP, so one padded index serves the whole butterfly.
template <typename T, int R, int M>
__device__ __forceinline__ void bfly_fixed(typename Vec2<T>::type* z, int base,
                                           const typename Vec2<T>::type* tw, int n1) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    constexpr int P = 1 << PadShift<T>::value;
    if constexpr (M % P == 0 || P % (R * M) == 0) {
        constexpr int STEP = (M % P == 0) ? M + M / P : M;
        V* zb = z + ph<T>(base);
        V a[R];
#pragma unroll
        for (int t = 0; t < R; ++t) a[t] = zb[t * STEP];
        Dft<T, R>::run(a);
        if (M > 1 && n1 != 0) {
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1)
                a[Dft<T, R>::pos(k1)] = K::mul(a[Dft<T, R>::pos(k1)], tw[(k1 - 1) * M + n1]);
        }
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) zb[k1 * STEP] = a[Dft<T, R>::pos(k1)];
    } else {
        bfly<T, R>(z, base, M, tw, n1);
    }
}

// In-place mixed-radix DIF FFT over `nrows` padded rows (pitch LP), shape
// known at run time.  BIG = false leaves out the two-pass radices above 8
// (their shapes, L = Q x 32, all have compile-time kernels, so only the
// grouped launches meet them at run time): far fewer registers.
template <typename T, bool BIG = true>
__device__ void passes_runtime(typename Vec2<T>::type* rows, int nrows, int LP,
                               const FftShape& sh, const typename Vec2<T>::type* twp) {
    const int L = sh.L;
    for (int p = 0; p < sh.npass; ++p) {
        const int r = sh.radix[p];
        const int M = sh.span[p];
        const int S = r * M;
        const int nb = L / r;
        const int total = nrows * nb;
        const typename Vec2<T>::type* tw = twp + sh.twoff[p];
        for (int idx = threadIdx.x; idx < total; idx += NT) {
            const int row = idx / nb;
            const int b = idx - row * nb;
            const int blk = b / M;
            const int n1 = b - blk * M;
            auto* z = rows + (size_t)row * LP;
            const int base = blk * S + n1;
            if constexpr (sizeof(T) == 4 && BIG) {   // two-pass shapes (FP32 only)
                if (r > 8) {
                    if (r == 10) bfly<T, 10>(z, base, M, tw, n1);
                    else if (r == 16) bfly<T, 16>(z, base, M, tw, n1);
                    else if (r == 20) bfly<T, 20>(z, base, M, tw, n1);
                    else if (r == 32) bfly<T, 32>(z, base, M, tw, n1);
                    else bfly<T, 40>(z, base, M, tw, n1);
                    continue;
                }
            }
            if (r == 8)
                bfly<T, 8>(z, base, M, tw, n1);
            else if (r == 4)
                bfly<T, 4>(z, base, M, tw, n1);
            else if (r == 2)
                bfly<T, 2>(z, base, M, tw, n1);
            else if (r == 5)
                bfly<T, 5>(z, base, M, tw, n1);
            else
                bfly<T, 3>(z, base, M, tw, n1);
        }
        __syncthreads();
    }
}

// The same with the shape a compile-time constant (passes P .. END-1).
template <typename T, int L, int P, int END = FacOf<L, sizeof(T) == 8>::v.npass>
__device__ __forceinline__ void passes_fixed(typename Vec2<T>::type* rows, int nrows, int LP,
                                             const typename Vec2<T>::type* twp) {
    constexpr FftShape F = FacOf<L, sizeof(T) == 8>::v;
    if constexpr (P < END) {
        constexpr int R = F.radix[P];
        constexpr int M = F.span[P];
        constexpr int S = R * M;
        constexpr int NB = L / R;
        constexpr int OFF = F.twoff[P];
        const int total = nrows * NB;
        for (int idx = threadIdx.x; idx < total; idx += NT) {
            const int row = idx / NB;
            const int b = idx - row * NB;
            const int blk = b / M;
            const int n1 = b - blk * M;
            bfly_fixed<T, R, M>(rows + (size_t)row * LP, blk * S + n1, twp + OFF, n1);
        }
        __syncthreads();
        passes_fixed<T, L, P + 1, END>(rows, nrows, LP, twp);
    }
}

// FP32 two-pass shapes L = Q x 32 with Q >= 8: the forward runs its first
// pass from the grid rows (below), the inverse its last pass into them.
template <typename T, int L>
__host__ __device__ constexpr bool first_pass_from_global() {
    if constexpr (sizeof(T) != 4 || L <= 0) {
        return false;
    } else {
        constexpr FftShape F = FacOf<L, false>::v;
        return F.npass == 2 && F.radix[1] == 32 && F.span[0] == 32 && F.radix[0] >= 8;
    }
}

// FP32 two-pass shapes L = Q x 32 with Q >= 8: the inverse runs its last
// pass (radix 32, span 1) straight into the grid rows.  Butterfly b of a
// row holds frequencies b + Q k1 (k1 < 32) of the digit-reversed output,
// so for each k1 the lanes of a warp store consecutive complex values
// (at least 64 contiguous bytes), and the result needs no shared-memory
// round trip before the store.
template <typename T, int L>
__host__ __device__ constexpr bool inverse_stores_from_last_pass() {
    if constexpr (sizeof(T) != 4 || L <= 0) {
        return false;
    } else {
        constexpr FftShape F = FacOf<L, false>::v;
        return F.npass == 2 && F.radix[1] == 32 && F.radix[0] >= 8;
    }
}

// Digit-reversed position of frequency k.
template <typename T, int L>
__device__ __forceinline__ int rev_fixed(int k) {
    constexpr FftShape F = FacOf<L, sizeof(T) == 8>::v;
    int pos = 0;
#pragma unroll
    for (int q = 0; q < F.npass; ++q) {
        pos += (k % F.radix[q]) * F.span[q];
        k /= F.radix[q];
    }
    return pos;
}

template <typename T>
struct FwdArgs {
    using V = typename Vec2<T>::type;
    const T* grid;
    RowSource src;
    V* work;
    const V* twp;      // per-pass twiddle tables
    const V* twpost;
    const int* rev;
    const double* rowscale;
    double mscale0, mscale1;
    unsigned* colmax;   // FP16 split plans: max |output| per real column (float bits)
    const long long* rowoff;   // reduced grid: first point of each row (null: regular)
    const int* jh_list;        // latitude pair of each CTA row (null: blockIdx.y)
    const V* shiftph;          // rows shifted by half a spacing: e^{-i pi m / I_j} (else null)
    const V* chirp;            // Bluestein rows: e^{-i pi n^2 / L}
    const V* dft;              // Bluestein rows: DFT of the conjugate chirp / L2
    int F, J, Jh, L, LP, N, G;
    FftShape shape;
};

template <typename T>
struct InvArgs {
    using V = typename Vec2<T>::type;
    const V* work;
    T* grid;
    const V* twp;
    const V* twpost;
    const int* rev;
    const double* rowscale;
    double mfactor1;
    const long long* rowoff;   // reduced grid: first point of each row (null: regular)
    long long fstride;         // reduced grid: points per field
    const int* jh_list;        // latitude pair of each CTA row (null: blockIdx.y)
    int accumulate;            // 1: grid += rows (prolongation of a correction);
                               // 2: products (Sec. 4.2): with w the synthesised
                               // value, grid holds u and becomes u v, grid2
                               // holds v and becomes u v w
    T* grid2;                  // second grid of the products (else null)
    const V* shiftph;          // rows shifted by half a spacing: e^{-i pi m / I_j} (else null)
    const V* chirp;            // Bluestein rows: e^{-i pi n^2 / L}
    const V* dft;              // Bluestein rows: DFT of the conjugate chirp / L2
    int F, J, Jh, I, L, LP, N, G;
    FftShape shape;
};

// Copy the per-pass twiddle tables into shared memory asynchronously, so
// that they are in flight together with the CTA's data copies (one wait).
template <typename V>
__device__ __forceinline__ void load_twiddles_async(V* dst, const V* src, int n) {
    for (int e = threadIdx.x; e < n; e += NT) cp_async<sizeof(V)>(dst + e, src + e);
}

// The same by plain loads and stores (measured faster ahead of the inverse
// kernel's gathered copies).
template <typename V>
__device__ __forceinline__ void load_twiddles(V* dst, const V* src, int n) {
    for (int e = threadIdx.x; e < n; e += NT) dst[e] = src[e];
}

// LT > 0: the compile-time shape of that half-length; LT = 0: any shape at
// run time; LT = -1: a run-time shape without the two-pass radices.
template <typename T, int LT>
__device__ __forceinline__ void run_passes(typename Vec2<T>::type* rows, int nrows, int LP,
                                           const FftShape& sh,
                                           const typename Vec2<T>::type* twp) {
    if constexpr (LT > 0)
        passes_fixed<T, LT, 0>(rows, nrows, LP, twp);
    else
        passes_runtime<T, LT == 0>(rows, nrows, LP, sh, twp);
}

template <typename T, int LT>
__device__ __forceinline__ int rev_of(int k, const int* rev) {
    if constexpr (LT > 0)
        return rev_fixed<T, LT>(k);
    else if constexpr (LT == -2)
        return k;   // Bluestein rows end in natural order
    else
        return rev[k];
}

// Bluestein's chirp-z DFT of each of nrows padded rows of half-length L (any
// L; natural order in and out), for the rows of reduced grids whose L has a
// prime factor above 5.  With c_n = e^{-i pi n^2 / L},
//   Z_k = sum_n z_n e^{-2 pi i n k / L} = c_k sum_n (z_n c_n) conj(c_{k-n}),
// a circular convolution of length L2 >= 2L - 1 (sh2.L, 2-3-5-smooth) of
// a_n = z_n c_n (zero-padded) with the conjugate chirp wrapped around L2,
// whose DFT D (divided by L2) is a table.  Per row: the FFT of a, the
// pointwise product with D, conjugated and moved to natural order, a second
// FFT, and Z_k = c_k conj(result at k).  b1, b2: two padded scratch rows of
// length L2; tws: the per-pass twiddles of length L2; rev2: its digit
// reversal.
template <typename T>
__device__ void bluestein_rows(typename Vec2<T>::type* rows, int nrows, int LP, int L,
                               const FftShape& sh2, const typename Vec2<T>::type* tws,
                               const typename Vec2<T>::type* chirp,
                               const typename Vec2<T>::type* dft, const int* rev2,
                               typename Vec2<T>::type* b1, typename Vec2<T>::type* b2) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    const int L2 = sh2.L;
    const int tid = threadIdx.x;
    for (int r = 0; r < nrows; ++r) {
        V* z = rows + (size_t)r * LP;
        for (int n = tid; n < L2; n += NT)
            b1[ph<T>(n)] = n < L ? K::mul(z[ph<T>(n)], chirp[n]) : K::make((T)0, (T)0);
        __syncthreads();
        passes_runtime<T, false>(b1, 1, 0, sh2, tws);
        for (int k = tid; k < L2; k += NT)
            b2[ph<T>(k)] = K::conj(K::mul(b1[ph<T>(rev2[k])], dft[k]));
        __syncthreads();
        passes_runtime<T, false>(b2, 1, 0, sh2, tws);
        for (int k = tid; k < L; k += NT)
            z[ph<T>(k)] = K::mul(chirp[k], K::conj(b2[ph<T>(rev2[k])]));
        __syncthreads();
    }
}

// Padded pitch of a row of n complex values (fft_row_pitch on the device).
template <typename T>
__device__ __forceinline__ int row_pitch(int n) {
    return n + (n >> PadShift<T>::value) + 1;
}

// Iterates idx = tid, tid + NT, ... as (major, minor) = (idx / d, idx % d)
// without dividing inside the loop.
struct Walk2 {
    int major, minor, step_major, step_minor, d;
    __device__ __forceinline__ Walk2(int start, int d_) : d(d_) {
        major = start / d;
        minor = start - major * d;
        step_major = NT / d;
        step_minor = NT - step_major * d;
    }
    __device__ __forceinline__ void next() {
        major += step_major;
        minor += step_minor;
        if (minor >= d) {
            minor -= d;
            ++major;
        }
    }
};

extern __shared__ __align__(16) unsigned char fft_smem_raw[];

template <typename T, int LT, bool STRIDED>
__device__ __forceinline__ void fwd_body(const FwdArgs<T>& A, int fg, int jh) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    const int L = LT > 0 ? LT : A.L;
    const int LP = A.LP;
    V* rows = reinterpret_cast<V*>(fft_smem_raw);
    V* tws = rows + (size_t)2 * A.G * LP;
    const int f0 = fg * A.G;
    const int nf = min(A.G, A.F - f0);
    const bool equator = (jh == A.Jh - 1);
    const int nrows = equator ? nf : 2 * nf;
    const int tid = threadIdx.x;
    auto row_ptr = [&](int r) -> const T* {
        const int f = f0 + (r < nf ? r : r - nf);
        const int j = (r < nf) ? jh : (A.J - 1 - jh);
        if (A.rowoff) return A.grid + (long long)f * A.src.field_stride + A.rowoff[j];
        return A.grid + (long long)f * A.src.field_stride + A.src.row_offset +
               (long long)j * A.src.row_stride;
    };

    if constexpr (!STRIDED && first_pass_from_global<T, LT>()) {
        // The first pass (radix Q, span 32) reads its inputs straight from
        // the grid rows into registers: butterfly n1 of a row takes
        // z[n1 + 32 t], t < Q, so for each t the lanes of a warp load 256
        // contiguous bytes.  Only the twiddle table is copied
        // asynchronously; the first butterfly's loads are in flight while
        // the CTA waits for it.
        constexpr FftShape FS = FacOf<LT, false>::v;
        constexpr int Q = FS.radix[0];
        constexpr int M = FS.span[0];                                  // 32
        constexpr int STEP = M + (M >> PadShift<T>::value);            // padded
        load_twiddles_async(tws, A.twp, FS.twtotal);
        const int total = nrows * M;
        V a[Q];
        auto load = [&](int idx) {
            const int r = idx / M, n1 = idx - r * M;
            const V* x = reinterpret_cast<const V*>(row_ptr(r)) + n1;
#pragma unroll
            for (int t = 0; t < Q; ++t) a[t] = x[t * M];
        };
        auto finish = [&](int idx) {
            const int r = idx / M, n1 = idx - r * M;
            Dft<T, Q>::run(a);
            if (n1 != 0) {
#pragma unroll
                for (int k1 = 1; k1 < Q; ++k1)
                    a[Dft<T, Q>::pos(k1)] =
                        K::mul(a[Dft<T, Q>::pos(k1)], tws[(k1 - 1) * M + n1]);
            }
            V* zb = rows + (size_t)r * LP + n1;
#pragma unroll
            for (int k1 = 0; k1 < Q; ++k1) zb[k1 * STEP] = a[Dft<T, Q>::pos(k1)];
        };
        if (tid < total) load(tid);
        cp_async_wait_all();
        __syncthreads();
        if (tid < total) finish(tid);
        for (int idx = tid + NT; idx < total; idx += NT) {
            load(idx);
            finish(idx);
        }
        __syncthreads();
        passes_fixed<T, LT, 1>(rows, nrows, LP, tws);
    } else {
        {
            // element k of row r goes to rows[r LP + ph(k)], copied
            // asynchronously so that all of the CTA's loads are in flight
            const int s = A.src.elem_stride;
            for (int r = 0; r < nrows; ++r) {
                const T* x = row_ptr(r);
                V* d = rows + (size_t)r * LP;
                for (int k = tid; k < L; k += NT) {
                    if (!STRIDED) {
                        cp_async<sizeof(V)>(d + ph<T>(k), reinterpret_cast<const V*>(x) + k);
                    } else {
                        cp_async<sizeof(T)>(&d[ph<T>(k)].x, x + (long long)(2 * k) * s);
                        cp_async<sizeof(T)>(&d[ph<T>(k)].y, x + (long long)(2 * k + 1) * s);
                    }
                }
            }
            load_twiddles_async(tws, A.twp,
                                LT > 0 ? FacOf<LT, sizeof(T) == 8>::v.twtotal : A.shape.twtotal);
            cp_async_wait_all();
        }
        __syncthreads();
        if constexpr (LT == -2) {
            V* b1 = tws + A.shape.L + (2 * A.G * 4 + sizeof(V) - 1) / sizeof(V);
            V* b2 = b1 + row_pitch<T>(A.shape.L);
            bluestein_rows<T>(rows, nrows, LP, L, A.shape, tws, A.chirp, A.dft, A.rev, b1, b2);
        } else {
            run_passes<T, LT>(rows, nrows, LP, A.shape, tws);
        }
    }

    const int nout = (A.N + 1) * nf;
    const T rs = A.rowscale ? (T)A.rowscale[jh] : (T)1;
    // column maxima of the output (real and imaginary part of each field),
    // gathered per thread while its field stays the same, then per CTA in
    // shared memory, then one global atomic per column and CTA
    const bool track = A.colmax != nullptr;
    unsigned* smax = reinterpret_cast<unsigned*>(
        tws + (LT > 0 ? LT : (LT == -2 ? A.shape.L : A.L)));
    if (track) {
        for (int e = tid; e < 2 * nf; e += NT) smax[e] = 0u;
        __syncthreads();
    }
    float mre = 0.f, mim = 0.f;
    int mcur = -1;
    auto flush = [&]() {
        if (mcur >= 0) {
            atomicMax(&smax[2 * mcur], __float_as_uint(mre));
            atomicMax(&smax[2 * mcur + 1], __float_as_uint(mim));
        }
    };
    auto record = [&](int fl, V os, V oa) {
        if (fl != mcur) {
            flush();
            mcur = fl;
            mre = mim = 0.f;
        }
        mre = fmaxf(mre, fmaxf(fabsf((float)os.x), fabsf((float)oa.x)));
        mim = fmaxf(mim, fmaxf(fabsf((float)os.y), fabsf((float)oa.y)));
    };
    // 2 X_m = (Z_m + conj Z_{L-m}) + W_I^m (-i)(Z_m - conj Z_{L-m})
    auto real_spec = [&](V zm, V zc, V wt) -> V {
        // s = zm + conj zc, d = zm - conj zc; s + wt (-i d), componentwise
        const T sx = zm.x + zc.x, sy = zm.y - zc.y;
        const T dx = zm.x - zc.x, dy = zm.y + zc.y;
        return K::make(sx + wt.x * dy + wt.y * dx, sy - wt.x * dx + wt.y * dy);
    };
    // output scales, converted once (FP64 conversions use the narrow FP64 pipe)
    const T sc0 = (T)0.5 * rs * (T)A.mscale0, sc1 = (T)0.5 * rs * (T)A.mscale1;
    // two outputs (m, fl) per iteration, idx and idx + NT, with all shared-
    // memory reads of both issued before any arithmetic.  A reduced-grid row
    // of half-length L carries the wavenumbers up to min(N, L - 1); those
    // above are written as zeros (computed at the clamped wavenumber, then
    // discarded).  The loop is compiled twice, with and without that clamp.
    const int kmax = A.rowoff ? min(A.N, L - 1) : A.N;
    auto out_loop = [&](auto rag) {
        constexpr bool RAG = decltype(rag)::value;
        auto clampk = [&](int m) -> int {
            if constexpr (RAG)
                return min(m, kmax);
            else
                return m;
        };
        Walk2 wa(tid, nf), wb(tid + NT, nf);
        for (; wa.major * nf + wa.minor < nout; wa.next(), wa.next(), wb.next(), wb.next()) {
            const bool hb = wb.major * nf + wb.minor < nout;
            const int ma = wa.major, fa = wa.minor;
            const int mb = hb ? wb.major : ma, fb = hb ? wb.minor : fa;
            const int ra = clampk(ma), rb = clampk(mb);
            const int pma = ph<T>(rev_of<T, LT>(ra, A.rev));
            const int pca = ph<T>(rev_of<T, LT>(ra == 0 ? 0 : L - ra, A.rev));
            const int pmb = ph<T>(rev_of<T, LT>(rb, A.rev));
            const int pcb = ph<T>(rev_of<T, LT>(rb == 0 ? 0 : L - rb, A.rev));
            const V* na = rows + (size_t)fa * LP;
            const V* nb = rows + (size_t)fb * LP;
            const V a_nm = na[pma], a_nc = na[pca], b_nm = nb[pmb], b_nc = nb[pcb];
            V a_sm = K::make((T)0, (T)0), a_sc = a_sm, b_sm = a_sm, b_sc = a_sm;
            if (!equator) {
                const V* sa = na + (size_t)nf * LP;
                const V* sb = nb + (size_t)nf * LP;
                a_sm = sa[pma];
                a_sc = sa[pca];
                b_sm = sb[pmb];
                b_sc = sb[pcb];
            }
            const V wta = A.twpost[ra], wtb = A.twpost[rb];
            const T sca = ma == 0 ? sc0 : sc1;
            const T scb = mb == 0 ? sc0 : sc1;
            const V xan = real_spec(a_nm, a_nc, wta), xbn = real_spec(b_nm, b_nc, wtb);
            V Sa = xan, Aa = K::make((T)0, (T)0), Sb = xbn, Ab = Aa;
            if (!equator) {
                const V xas = real_spec(a_sm, a_sc, wta), xbs = real_spec(b_sm, b_sc, wtb);
                Sa = K::add(xan, xas);
                Aa = K::sub(xan, xas);
                Sb = K::add(xbn, xbs);
                Ab = K::sub(xbn, xbs);
            }
            V osa = K::scale(Sa, sca), oaa = K::scale(Aa, sca);
            if constexpr (RAG) {
                // rows shifted by half a spacing: X^m e^{-i pi m / I_j}
                if (A.shiftph) {
                    const V pa = A.shiftph[ra];
                    osa = K::mul(osa, pa);
                    oaa = K::mul(oaa, pa);
                }
            }
            if (ra != ma) osa = oaa = K::make((T)0, (T)0);
            const size_t basea = ((size_t)ma * 2 * A.Jh + jh) * A.F + f0 + fa;
            A.work[basea] = osa;
            A.work[basea + (size_t)A.Jh * A.F] = oaa;
            if (track) record(fa, osa, oaa);
            if (hb) {
                V osb = K::scale(Sb, scb), oab = K::scale(Ab, scb);
                if constexpr (RAG) {
                    if (A.shiftph) {
                        const V pb = A.shiftph[rb];
                        osb = K::mul(osb, pb);
                        oab = K::mul(oab, pb);
                    }
                }
                if (rb != mb) osb = oab = K::make((T)0, (T)0);
                const size_t baseb = ((size_t)mb * 2 * A.Jh + jh) * A.F + f0 + fb;
                A.work[baseb] = osb;
                A.work[baseb + (size_t)A.Jh * A.F] = oab;
                if (track) record(fb, osb, oab);
            }
        }
    };
    // The two-pass FP32 lengths L = Q x 32 on regular grids: each thread keeps
    // one field and walks the wavenumbers m = g, g + D, ... (D = NT / nf
    // thread groups), with the digit-reversed positions tracked as the
    // mixed-radix digits of m (m = k1 + Q k2 sits at 32 k1 + k2, padded
    // 33 k1 + k2; L - m at the digits of its complement) and the workspace
    // address advanced by a constant, so the loop needs no division.
    // Consecutive threads write consecutive fields of one m, as above.
    auto out_walk = [&]() {
        constexpr FftShape FS = FacOf<(LT > 0 ? LT : 64), false>::v;
        constexpr int Q = FS.radix[0];
        const int D = NT / nf;
        const int g = tid / nf, fl = tid - g * nf;
        if (g >= D) return;
        const V* zn = rows + (size_t)fl * LP;
        const V* zs = zn + (size_t)nf * LP;
        int k1 = g % Q, k2 = g / Q;
        const int d1 = D % Q, d2 = D / Q;
        V* wp = A.work + ((size_t)g * 2 * A.Jh + jh) * A.F + f0 + fl;
        const size_t wstep = (size_t)D * 2 * A.Jh * A.F;
        const size_t astep = (size_t)A.Jh * A.F;
        for (int m = g; m <= A.N; m += D) {
            const int c1 = k1 == 0 ? 0 : Q - k1;
            const int c2 = k1 == 0 ? ((32 - k2) & 31) : 31 - k2;
            const int pm = 33 * k1 + k2, pc = 33 * c1 + c2;
            const V wt = A.twpost[m];
            const V xn = real_spec(zn[pm], zn[pc], wt);
            V S = xn, Aq = K::make((T)0, (T)0);
            if (!equator) {
                const V xs = real_spec(zs[pm], zs[pc], wt);
                S = K::add(xn, xs);
                Aq = K::sub(xn, xs);
            }
            const T sc = m == 0 ? sc0 : sc1;
            const V os = K::scale(S, sc), oa = K::scale(Aq, sc);
            wp[0] = os;
            wp[astep] = oa;
            if (track) record(fl, os, oa);
            wp += wstep;
            k1 += d1;
            k2 += d2;
            if (k1 >= Q) {
                k1 -= Q;
                ++k2;
            }
        }
    };
    if constexpr (first_pass_from_global<T, LT>()) {
        if (!A.rowoff)
            out_walk();
        else
            out_loop(std::true_type{});
    } else {
        if (LT <= 0 || A.rowoff)
            out_loop(std::true_type{});
        else
            out_loop(std::false_type{});
    }
    if (track) {
        flush();
        __syncthreads();
        for (int e = tid; e < 2 * nf; e += NT) atomicMax(&A.colmax[2 * f0 + e], smax[e]);
    }
}

template <typename T, int LT, bool STRIDED>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_forward_kernel(const __grid_constant__ FwdArgs<T> A) {
    fwd_body<T, LT, STRIDED>(A, blockIdx.x, A.jh_list ? A.jh_list[blockIdx.y] : blockIdx.y);
}

template <typename T, int LT>
__device__ __forceinline__ void inv_body(const InvArgs<T>& A, int fg, int jh) {
    using V = typename Vec2<T>::type;
    using K = C2<T>;
    const int L = LT > 0 ? LT : A.L;
    const int LP = A.LP;
    V* rows = reinterpret_cast<V*>(fft_smem_raw);
    V* tws = rows + (size_t)2 * A.G * LP;
    const int f0 = fg * A.G;
    const int nf = min(A.G, A.F - f0);
    const bool equator = (jh == A.Jh - 1);
    const int nrows = equator ? nf : 2 * nf;
    const int tid = threadIdx.x;
    const int half = L / 2;
    // Loads whose values are needed only after the copies below (the row
    // scale and, for compile-time lengths, the real-spectrum twiddles of the
    // thread's packing frequencies q and L - q), issued first so that their
    // latency hides behind the copies.
    const T rs = A.rowscale ? (T)A.rowscale[jh] : (T)1;
    constexpr int NQ = LT > 0 ? (LT / 2 + NT) / NT : 1;
    V twq[NQ], twc[NQ];
    if constexpr (LT > 0) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int q = tid + i * NT;
            if (q <= half) {
                twq[i] = A.twpost[q];
                twc[i] = A.twpost[q == 0 ? 0 : L - q];
            }
        }
    }

    load_twiddles(tws, A.twp, LT > 0 ? FacOf<LT, sizeof(T) == 8>::v.twtotal : A.shape.twtotal);
    // unfold S/A into the two hemispheres' zonal spectra Y_m, m <= N
    // (S lands in the northern row, A in the southern one, copied
    // asynchronously; then both hemispheres are formed in place)
    // a reduced-grid row of half-length L carries the wavenumbers up to
    // min(N, L - 1) (Y_m = 0 above)
    const int kmax = A.rowoff ? min(A.N, L - 1) : A.N;
    const int nin = (kmax + 1) * nf;
    for (Walk2 w(tid, nf); w.major * nf + w.minor < nin; w.next()) {
        const int m = w.major, fl = w.minor;
        const size_t base = ((size_t)m * 2 * A.Jh + jh) * A.F + f0 + fl;
        cp_async<sizeof(V)>(rows + (size_t)fl * LP + ph<T>(m), A.work + base);
        if (!equator)
            cp_async<sizeof(V)>(rows + (size_t)(nf + fl) * LP + ph<T>(m),
                                A.work + base + (size_t)A.Jh * A.F);
    }
    cp_async_wait_all();
    __syncthreads();
    // One thread owns frequencies (q, L-q) of all fields in both hemispheres
    // Y_m = fac (S_m +- A_m) (Y_0 real, Y_m = 0 for m > kmax; stale slots
    // beyond kmax are never read), then the Hermitian packing
    //   Z_q = (Y_q + conj Y_{L-q}) + i conj(W_I^q) (Y_q - conj Y_{L-q}),
    // stored as conj(Z) in place.
    const T mf1 = (T)A.mfactor1;
    auto pack = [&](V y, V yc, V wv) -> V {
        return K::conj(K::add(K::add(y, K::conj(yc)),
                              K::mul_pi(K::mul(wv, K::sub(y, K::conj(yc))))));
    };
    // frequencies q and L - q with the twiddles W_I^q and W_I^{L-q}
    auto pack_q = [&](int q, V tq, V tc) {
        const int qc = L - q;   // >= q, as q <= L/2
        const int pq = ph<T>(q), pc = ph<T>(qc);
        const bool hq = q <= kmax, hc = q != 0 && qc <= kmax;
        const bool pair = q != 0 && q != qc;
        const T fq = q == 0 ? (T)1 : mf1, fc = mf1;
        const V wq = K::conj(tq);
        const V wc = pair ? K::conj(tc) : wq;
        const V zero = K::make((T)0, (T)0);
        for (int fl = 0; fl < nf; ++fl) {
            V* zn = rows + (size_t)fl * LP;
            V* zs = rows + (size_t)(nf + fl) * LP;
            // S and A at frequencies q and L - q, each read once (zero above
            // kmax; Y_L = 0 for q = 0)
            V Sq = hq ? zn[pq] : zero;
            V Aq = (hq && !equator) ? zs[pq] : zero;
            V Sc = hc ? zn[pc] : zero;
            V Ac = (hc && !equator) ? zs[pc] : zero;
            if (A.shiftph) {
                // rows shifted by half a spacing: Y^m e^{+i pi m / I_j}
                const V cq = K::conj(A.shiftph[q]);
                Sq = K::mul(Sq, cq);
                Aq = K::mul(Aq, cq);
                if (hc) {
                    const V cc = K::conj(A.shiftph[qc]);
                    Sc = K::mul(Sc, cc);
                    Ac = K::mul(Ac, cc);
                }
            }
            V ynq = K::scale(K::add(Sq, Aq), fq), ysq = K::scale(K::sub(Sq, Aq), fq);
            if (q == 0) ynq.y = ysq.y = (T)0;
            const V ync = K::scale(K::add(Sc, Ac), fc), ysc = K::scale(K::sub(Sc, Ac), fc);
            zn[pq] = pack(ynq, ync, wq);
            if (!equator) zs[pq] = pack(ysq, ysc, wq);
            if (pair) {
                zn[pc] = pack(ync, ynq, wc);
                if (!equator) zs[pc] = pack(ysc, ysq, wc);
            }
        }
    };
    // When the spectrum stops below L/2 (kmax < L/2, i.e. I > 4 kmax, true of
    // every grid with I = 4 (N+1)), Y vanishes at L - q for all q <= L/2, so
    // each packed value depends on one Y:
    //   conj Z_q     = conj(Y_q) (1 - i W_I^q),
    //   conj Z_{L-q} = Y_q (1 + i W_I^{L-q}),
    // with the m >= 1 factor folded into the two constants, and both
    // hemispheres' Y = S +- A formed once per field.
    auto pack_q_short = [&](int q, V tq, V tc) {
        const int qc = L - q;
        const int pq = ph<T>(q), pc = ph<T>(qc);
        const bool pair = q != 0 && q != qc;
        const V zero = K::make((T)0, (T)0);
        const T fq = q == 0 ? (T)1 : mf1;
        const V al = K::make(fq * ((T)1 + tq.y), -fq * tq.x);    // f (1 - i W^q)
        const V be = K::make(mf1 * ((T)1 - tc.y), mf1 * tc.x);   // f (1 + i W^{L-q})
        if (q > kmax) {
            for (int fl = 0; fl < nf; ++fl) {
                V* zn = rows + (size_t)fl * LP;
                V* zs = rows + (size_t)(nf + fl) * LP;
                zn[pq] = zero;
                if (!equator) zs[pq] = zero;
                if (pair) {
                    zn[pc] = zero;
                    if (!equator) zs[pc] = zero;
                }
            }
            return;
        }
        const V cs = A.shiftph ? K::conj(A.shiftph[q]) : K::make((T)1, (T)0);
        for (int fl = 0; fl < nf; ++fl) {
            V* zn = rows + (size_t)fl * LP;
            V* zs = rows + (size_t)(nf + fl) * LP;
            V Sq = zn[pq];
            V Aq = equator ? zero : zs[pq];
            if (A.shiftph) {
                Sq = K::mul(Sq, cs);
                Aq = K::mul(Aq, cs);
            }
            V yn = K::add(Sq, Aq), ys = K::sub(Sq, Aq);
            if (q == 0) yn.y = ys.y = (T)0;
            zn[pq] = K::mul(K::conj(yn), al);
            if (!equator) zs[pq] = K::mul(K::conj(ys), al);
            if (pair) {
                zn[pc] = K::mul(yn, be);
                if (!equator) zs[pc] = K::mul(ys, be);
            }
        }
    };
    const bool short_spec = 2 * kmax < L;
    if constexpr (LT > 0) {
        if (short_spec) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int q = tid + i * NT;
                if (q <= half) pack_q_short(q, twq[i], twc[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int q = tid + i * NT;
                if (q <= half) pack_q(q, twq[i], twc[i]);
            }
        }
    } else {
        for (int q = tid; q <= half; q += NT) {
            if (short_spec)
                pack_q_short(q, A.twpost[q], A.twpost[q == 0 ? 0 : L - q]);
            else
                pack_q(q, A.twpost[q], A.twpost[q == 0 ? 0 : L - q]);
        }
    }
    __syncthreads();
    if constexpr (inverse_stores_from_last_pass<T, LT>()) {
        constexpr FftShape FS = FacOf<LT, false>::v;
        constexpr int R = FS.radix[1];   // 32 = the padding period: one padded
        constexpr int Q = FS.radix[0];   // index per butterfly
        passes_fixed<T, LT, 0, 1>(rows, nrows, LP, tws);
        const V sgn = K::make(rs, -rs);   // x = conj(z) rs
        // compiled for the plain store, accumulation into the grid and the
        // products of the aliasing experiment
        auto last_pass = [&](auto mode) {
            constexpr int MODE = decltype(mode)::value;
            for (int idx = tid; idx < nrows * Q; idx += NT) {
                const int r = idx / Q, b = idx - r * Q;
                const int f = f0 + (r < nf ? r : r - nf);
                const int j = (r < nf) ? jh : (A.J - 1 - jh);
                const long long off = A.rowoff ? (long long)f * A.fstride + A.rowoff[j]
                                               : ((long long)f * A.J + j) * A.I;
                V* xv = reinterpret_cast<V*>(A.grid + off) + b;
                const V* zb = rows + (size_t)r * LP + ph<T>(b * R);
                V a[R];
#pragma unroll
                for (int t = 0; t < R; ++t) a[t] = zb[t];
                Dft<T, R>::run(a);
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) {
                    const V y = mul_f32x2(a[Dft<T, R>::pos(k1)], sgn);
                    if constexpr (MODE == 1) {
                        xv[k1 * Q] = K::add(xv[k1 * Q], y);
                    } else if constexpr (MODE == 2) {
                        V* x2 = reinterpret_cast<V*>(A.grid2 + off) + b;
                        const V uv = mul_f32x2(xv[k1 * Q], x2[k1 * Q]);
                        xv[k1 * Q] = uv;
                        x2[k1 * Q] = mul_f32x2(uv, y);
                    } else {
                        xv[k1 * Q] = y;
                    }
                }
            }
        };
        if (A.accumulate == 1)
            last_pass(std::integral_constant<int, 1>{});
        else if (A.accumulate == 2)
            last_pass(std::integral_constant<int, 2>{});
        else
            last_pass(std::integral_constant<int, 0>{});
        return;
    }
    if constexpr (LT == -2) {
        V* b1 = tws + A.shape.L;
        V* b2 = b1 + row_pitch<T>(A.shape.L);
        bluestein_rows<T>(rows, nrows, LP, L, A.shape, tws, A.chirp, A.dft, A.rev, b1, b2);
    } else {
        run_passes<T, LT>(rows, nrows, LP, A.shape, tws);
    }

    // store of one synthesised pair of values y at xv[k] (x2: the second
    // grid of the products)
    auto put = [&](V* xv, V* x2, int k, V y) {
        if (A.accumulate == 1) {
            xv[k] = K::add(xv[k], y);
        } else if (A.accumulate == 2) {
            const V uv = K::make(xv[k].x * x2[k].x, xv[k].y * x2[k].y);
            xv[k] = uv;
            x2[k] = K::make(uv.x * y.x, uv.y * y.y);
        } else {
            xv[k] = y;
        }
    };
    for (int r = 0; r < nrows; ++r) {
        const int f = f0 + (r < nf ? r : r - nf);
        const int j = (r < nf) ? jh : (A.J - 1 - jh);
        const long long off = A.rowoff ? (long long)f * A.fstride + A.rowoff[j]
                                       : ((long long)f * A.J + j) * A.I;
        V* xv = reinterpret_cast<V*>(A.grid + off);
        V* x2 = A.grid2 ? reinterpret_cast<V*>(A.grid2 + off) : nullptr;
        const V* z = rows + (size_t)r * LP;
        if constexpr (LT > 0) {
            // all of the thread's shared-memory reads of the row first
            constexpr int NIT = (LT + NT - 1) / NT;
            V v[NIT];
#pragma unroll
            for (int i = 0; i < NIT; ++i) {
                const int k = tid + i * NT;
                if (LT % NT == 0 || k < LT) v[i] = z[ph<T>(rev_fixed<T, LT>(k))];
            }
#pragma unroll
            for (int i = 0; i < NIT; ++i) {
                const int k = tid + i * NT;
                if (LT % NT == 0 || k < LT) put(xv, x2, k, K::make(v[i].x * rs, -v[i].y * rs));
            }
        } else {
            for (int k = tid; k < L; k += NT) {
                const V v = z[ph<T>(rev_of<T, LT>(k, A.rev))];
                put(xv, x2, k, K::make(v.x * rs, -v.y * rs));
            }
        }
    }
}

template <typename T, int LT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_inverse_kernel(const __grid_constant__ InvArgs<T> A) {
    inv_body<T, LT>(A, blockIdx.x, A.jh_list ? A.jh_list[blockIdx.y] : blockIdx.y);
}

// ---- grouped launches: several plans' rows in one grid ----------------
template <typename T> struct FwdGroup {
    int n;
    int cta_start[kMaxGroup + 1];   // first CTA of each plan
    int nfg[kMaxGroup];             // field groups per latitude of each plan
    FwdArgs<T> a[kMaxGroup];
};

template <typename T> struct InvGroup {
    int n;
    int cta_start[kMaxGroup + 1];
    int nfg[kMaxGroup];
    InvArgs<T> a[kMaxGroup];
};

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_forward_group_kernel(const __grid_constant__ FwdGroup<T> G) {
    const int b = blockIdx.x;
    int p = 0;
    while (p + 1 < G.n && b >= G.cta_start[p + 1]) ++p;
    const int local = b - G.cta_start[p];
    const FwdArgs<T>& A = G.a[p];
    const int fg = local % G.nfg[p], jh = local / G.nfg[p];
    // the plan's half-length picks its compile-time body (one branch per CTA)
    switch (A.L) {
        case 64: fwd_body<T, 64, false>(A, fg, jh); break;
        case 128: fwd_body<T, 128, false>(A, fg, jh); break;
        case 256: fwd_body<T, 256, false>(A, fg, jh); break;
        case 320: fwd_body<T, 320, false>(A, fg, jh); break;
        case 512: fwd_body<T, 512, false>(A, fg, jh); break;
        case 640: fwd_body<T, 640, false>(A, fg, jh); break;
        case 1024: fwd_body<T, 1024, false>(A, fg, jh); break;
        case 1280: fwd_body<T, 1280, false>(A, fg, jh); break;
        default: fwd_body<T, -1, false>(A, fg, jh);
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_inverse_group_kernel(const __grid_constant__ InvGroup<T> G) {
    const int b = blockIdx.x;
    int p = 0;
    while (p + 1 < G.n && b >= G.cta_start[p + 1]) ++p;
    const int local = b - G.cta_start[p];
    const InvArgs<T>& A = G.a[p];
    const int fg = local % G.nfg[p], jh = local / G.nfg[p];
    switch (A.L) {
        case 64: inv_body<T, 64>(A, fg, jh); break;
        case 128: inv_body<T, 128>(A, fg, jh); break;
        case 256: inv_body<T, 256>(A, fg, jh); break;
        case 320: inv_body<T, 320>(A, fg, jh); break;
        case 512: inv_body<T, 512>(A, fg, jh); break;
        case 640: inv_body<T, 640>(A, fg, jh); break;
        case 1024: inv_body<T, 1024>(A, fg, jh); break;
        case 1280: inv_body<T, 1280>(A, fg, jh); break;
        default: inv_body<T, -1>(A, fg, jh);
    }
}

// ---- reduced grids: a half-length per latitude pair -------------------
// Each CTA takes its latitude pair's FFT shape and the offsets of that
// shape's tables; rows, shared memory and the row pitch are sized for the
// longest row of the grid.
template <typename T> struct RaggedFwd {
    FwdArgs<T> a;
    const RShape* shapes;
    const int* shape_of;
    const int* shift_of;                       // per latitude pair (null: none shifted)
    const typename Vec2<T>::type* shiftbase;   // all shapes' shift phases
    const typename Vec2<T>::type* chirpbase;   // all Bluestein shapes' chirps
    const typename Vec2<T>::type* dftbase;     // all Bluestein shapes' chirp spectra
};

template <typename T> struct RaggedInv {
    InvArgs<T> a;
    const RShape* shapes;
    const int* shape_of;
    const int* shift_of;
    const typename Vec2<T>::type* shiftbase;
    const typename Vec2<T>::type* chirpbase;
    const typename Vec2<T>::type* dftbase;
};

// Per-CTA arguments of a reduced-grid row class: the latitude pair's shape,
// its tables, and its shift.
template <typename Args, typename R>
__device__ __forceinline__ void apply_shape(Args& A, const R& Rg, int jh) {
    const RShape& rs = Rg.shapes[Rg.shape_of[jh]];
    A.shape = rs.sh;
    A.L = rs.L;
    A.twp += rs.tw_off;
    A.twpost += rs.post_off;
    A.rev += rs.rev_off;
    A.shiftph = (Rg.shift_of && Rg.shift_of[jh] && rs.shift_off >= 0)
                    ? Rg.shiftbase + rs.shift_off : nullptr;
    if (rs.bluestein) {
        A.chirp = Rg.chirpbase + rs.chirp_off;
        A.dft = Rg.dftbase + rs.dft_off;
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_forward_ragged_kernel(const __grid_constant__ RaggedFwd<T> R) {
    const int jh = R.a.jh_list[blockIdx.y];
    FwdArgs<T> A = R.a;
    apply_shape(A, R, jh);
    fwd_body<T, -1, false>(A, blockIdx.x, jh);
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    fft_inverse_ragged_kernel(const __grid_constant__ RaggedInv<T> R) {
    const int jh = R.a.jh_list[blockIdx.y];
    InvArgs<T> A = R.a;
    apply_shape(A, R, jh);
    inv_body<T, -1>(A, blockIdx.x, jh);
}

// Rows whose half-length has a prime factor above 5: Bluestein's method.
template <typename T>
__global__ void __launch_bounds__(NT, 2)
    fft_forward_bluestein_kernel(const __grid_constant__ RaggedFwd<T> R) {
    const int jh = R.a.jh_list[blockIdx.y];
    FwdArgs<T> A = R.a;
    apply_shape(A, R, jh);
    fwd_body<T, -2, false>(A, blockIdx.x, jh);
}

template <typename T>
__global__ void __launch_bounds__(NT, 2)
    fft_inverse_bluestein_kernel(const __grid_constant__ RaggedInv<T> R) {
    const int jh = R.a.jh_list[blockIdx.y];
    InvArgs<T> A = R.a;
    apply_shape(A, R, jh);
    inv_body<T, -2>(A, blockIdx.x, jh);
}

template <typename T, int LT>
cudaError_t fwd_launch(const FwdArgs<T>& A, bool strided, dim3 grid, size_t smem,
                       cudaStream_t s) {
    cudaError_t e;
    if (!strided) {
        if ((e = ensure_smem((const void*)fft_forward_kernel<T, LT, false>, smem))) return e;
        fft_forward_kernel<T, LT, false><<<grid, NT, smem, s>>>(A);
        note_launch();
    } else {
        if ((e = ensure_smem((const void*)fft_forward_kernel<T, LT, true>, smem))) return e;
        fft_forward_kernel<T, LT, true><<<grid, NT, smem, s>>>(A);
        note_launch();
    }
    return cudaGetLastError();
}

template <typename T, int LT>
cudaError_t inv_launch(const InvArgs<T>& A, dim3 grid, size_t smem, cudaStream_t s) {
    cudaError_t e = ensure_smem((const void*)fft_inverse_kernel<T, LT>, smem);
    if (e) return e;
    fft_inverse_kernel<T, LT><<<grid, NT, smem, s>>>(A);
    note_launch();
    return cudaGetLastError();
}

// Dispatch on the half-length: the standard grids get specialised kernels.
#define SHT_FFT_DISPATCH(L, CALL)          \
    switch (L) {                           \
        case 64: return CALL(64);          \
        case 128: return CALL(128);        \
        case 256: return CALL(256);        \
        case 320: return CALL(320);        \
        case 512: return CALL(512);        \
        case 640: return CALL(640);        \
        case 1024: return CALL(1024);      \
        case 1280: return CALL(1280);      \
        default: return CALL(-1);          \
    }

// The run-time-shape kernels outside grouped launches (LT = -1) carry only
// radices up to 8; every shape with a larger radix has a compile-time kernel.
inline bool small_radices(const FftShape& sh) {
    for (int q = 0; q < sh.npass; ++q)
        if (sh.radix[q] > 8) return false;
    return true;
}

template <typename T>
FwdArgs<T> make_fwd_args(const sht_plan_s* p, const void* grid, const RowSource& src,
                         const FwdScale& sc, void* work) {
    using V = typename Vec2<T>::type;
    FwdArgs<T> A;
    A.grid = static_cast<const T*>(grid);
    A.src = src;
    A.work = static_cast<V*>(work);
    A.twp = static_cast<const V*>(p->d_twpass);
    A.twpost = static_cast<const V*>(p->d_twpost);
    A.rev = p->d_rev;
    A.rowscale = sc.rowscale;
    A.mscale0 = sc.mscale0;
    A.mscale1 = sc.mscale1;
    A.colmax = p->d_colmax;
    A.rowoff = nullptr;
    A.jh_list = nullptr;
    A.shiftph = A.chirp = A.dft = nullptr;
    A.F = p->F; A.J = p->J; A.Jh = p->Jh; A.L = p->fft.L; A.N = p->N; A.G = p->G;
    A.LP = fft_row_pitch(p->fft.L, sizeof(T) == 8);
    A.shape = p->fft;
    return A;
}

template <typename T>
cudaError_t fwd_impl(const sht_plan_s* p, const void* grid, const RowSource& src,
                     const FwdScale& sc, void* work, cudaStream_t s) {
    const FwdArgs<T> A = make_fwd_args<T>(p, grid, src, sc, work);
    if (A.colmax) {
        const cudaError_t e = cudaMemsetAsync(A.colmax, 0, 2 * (size_t)p->F * sizeof(unsigned), s);
        if (e) return e;
    }
    const dim3 g((p->F + p->G - 1) / p->G, p->Jh);
    const bool strided = src.elem_stride != 1;
    if (!fft_has_fixed_kernel(p->fft.L) && !small_radices(p->fft)) return cudaErrorInvalidValue;
#define SHT_FWD(LV) fwd_launch<T, LV>(A, strided, g, p->fft_smem, s)
    SHT_FFT_DISPATCH(p->fft.L, SHT_FWD)
#undef SHT_FWD
}

template <typename T>
InvArgs<T> make_inv_args(const sht_plan_s* p, const void* work, const InvScale& sc,
                         void* grid) {
    using V = typename Vec2<T>::type;
    InvArgs<T> A;
    A.work = static_cast<const V*>(work);
    A.grid = static_cast<T*>(grid);
    A.twp = static_cast<const V*>(p->d_twpass);
    A.twpost = static_cast<const V*>(p->d_twpost);
    A.rev = p->d_rev;
    A.rowscale = sc.rowscale;
    A.mfactor1 = sc.mfactor1;
    A.rowoff = nullptr;
    A.fstride = (long long)p->J * p->I;
    A.jh_list = nullptr;
    A.accumulate = sc.accumulate;
    A.grid2 = static_cast<T*>(sc.grid2);
    A.shiftph = A.chirp = A.dft = nullptr;
    A.F = p->F; A.J = p->J; A.Jh = p->Jh; A.I = p->I; A.L = p->fft.L; A.N = p->N;
    A.G = p->G;
    A.LP = fft_row_pitch(p->fft.L, sizeof(T) == 8);
    A.shape = p->fft;
    return A;
}

template <typename T>
cudaError_t inv_impl(const sht_plan_s* p, const void* work, const InvScale& sc,
                     void* grid, cudaStream_t s) {
    const InvArgs<T> A = make_inv_args<T>(p, work, sc, grid);
    const dim3 g((p->F + p->G - 1) / p->G, p->Jh);
    if (!fft_has_fixed_kernel(p->fft.L) && !small_radices(p->fft)) return cudaErrorInvalidValue;
#define SHT_INV(LV) inv_launch<T, LV>(A, g, p->fft_smem, s)
    SHT_FFT_DISPATCH(p->fft.L, SHT_INV)
#undef SHT_INV
}

// Dispatch of a compile-time length (the lengths of fft_has_fixed_kernel).
#define SHT_FFT_FIXED(L, CALL)                       \
    switch (L) {                                     \
        case 64: return CALL(64);                    \
        case 128: return CALL(128);                  \
        case 256: return CALL(256);                  \
        case 320: return CALL(320);                  \
        case 512: return CALL(512);                  \
        case 640: return CALL(640);                  \
        case 1024: return CALL(1024);                \
        case 1280: return CALL(1280);                \
        default: return cudaErrorInvalidValue;       \
    }

// Arguments of one length class of a reduced grid: that shape's tables and
// row pitch, and the class's latitude-pair list.
template <typename Args>
void set_class(Args& A, const RaggedGrid* rg, const RShape& r, int off, size_t vb) {
    using V = std::remove_cv_t<std::remove_pointer_t<decltype(A.twp)>>;
    A.L = r.sh.L;
    A.shape = r.sh;
    A.LP = fft_row_pitch(r.sh.L, vb == 16);
    A.twp = reinterpret_cast<const V*>(static_cast<const char*>(rg->d_twpass) + r.tw_off * vb);
    A.twpost = reinterpret_cast<const V*>(static_cast<const char*>(rg->d_twpost) + r.post_off * vb);
    A.rev = rg->d_rev + r.rev_off;
    A.jh_list = rg->d_jh + off;
}

template <typename T>
cudaError_t fwd_ragged_class(const FwdArgs<T>& A, dim3 g, size_t smem, cudaStream_t s) {
#define SHT_FWDC(LV) fwd_launch<T, LV>(A, false, g, smem, s)
    SHT_FFT_FIXED(A.L, SHT_FWDC)
#undef SHT_FWDC
}

template <typename T>
cudaError_t inv_ragged_class(const InvArgs<T>& A, dim3 g, size_t smem, cudaStream_t s) {
#define SHT_INVC(LV) inv_launch<T, LV>(A, g, smem, s)
    SHT_FFT_FIXED(A.L, SHT_INVC)
#undef SHT_INVC
}

// Reduced grid: one launch of the compile-time kernel per length class that
// has one, then one launch of the generic kernel (a shape per CTA) over the
// remaining latitude pairs.
template <typename T>
cudaError_t fwd_ragged_impl(const sht_plan_s* p, const void* grid, const FwdScale& sc,
                            void* work, cudaStream_t s) {
    using V = typename Vec2<T>::type;
    const RaggedGrid* rg = p->ragged;
    const size_t vb = sizeof(V);
    RowSource src;
    src.field_stride = rg->npts;
    src.row_stride = 0;
    src.row_offset = 0;
    src.elem_stride = 1;
    FwdArgs<T> base = make_fwd_args<T>(p, grid, src, sc, work);
    base.rowoff = rg->d_rowoff;
    if (base.colmax) {
        const cudaError_t e = cudaMemsetAsync(base.colmax, 0, 2 * (size_t)p->F * sizeof(unsigned), s);
        if (e) return e;
    }
    const unsigned nfg = (p->F + p->G - 1) / p->G;
    for (const auto& c : rg->classes) {
        FwdArgs<T> A = base;
        set_class(A, rg, rg->h_shapes[c.shape], c.off, vb);
        const cudaError_t e = fwd_ragged_class<T>(A, dim3(nfg, c.count),
                                                  fft_smem_bytes(2 * A.L, p->G, vb == 16), s);
        if (e) return e;
    }
    RaggedFwd<T> R;
    R.a = base;
    R.a.twp = static_cast<const V*>(rg->d_twpass);
    R.a.twpost = static_cast<const V*>(rg->d_twpost);
    R.a.rev = rg->d_rev;
    R.shapes = rg->d_shapes;
    R.shape_of = rg->d_shape_of;
    R.shift_of = rg->any_shift ? rg->d_shift_of : nullptr;
    R.shiftbase = static_cast<const V*>(rg->d_shiftph);
    R.chirpbase = static_cast<const V*>(rg->d_chirp);
    R.dftbase = static_cast<const V*>(rg->d_dft);
    cudaError_t e;
    if (rg->generic_count > 0) {
        R.a.jh_list = rg->d_jh + rg->generic_off;
        e = ensure_smem((const void*)fft_forward_ragged_kernel<T>, p->fft_smem);
        if (e) return e;
        fft_forward_ragged_kernel<T><<<dim3(nfg, rg->generic_count), NT, p->fft_smem, s>>>(R);
        note_launch();
        if ((e = cudaGetLastError())) return e;
    }
    if (rg->blue_count > 0) {
        R.a.jh_list = rg->d_jh + rg->blue_off;
        R.a.G = rg->blue_G;
        const unsigned nfb = (p->F + rg->blue_G - 1) / rg->blue_G;
        e = ensure_smem((const void*)fft_forward_bluestein_kernel<T>, rg->blue_smem);
        if (e) return e;
        fft_forward_bluestein_kernel<T><<<dim3(nfb, rg->blue_count), NT, rg->blue_smem, s>>>(R);
        note_launch();
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t inv_ragged_impl(const sht_plan_s* p, const void* work, const InvScale& sc,
                            void* grid, cudaStream_t s) {
    using V = typename Vec2<T>::type;
    const RaggedGrid* rg = p->ragged;
    const size_t vb = sizeof(V);
    InvArgs<T> base = make_inv_args<T>(p, work, sc, grid);
    base.rowoff = rg->d_rowoff;
    base.fstride = rg->npts;
    const unsigned nfg = (p->F + p->G - 1) / p->G;
    for (const auto& c : rg->classes) {
        InvArgs<T> A = base;
        set_class(A, rg, rg->h_shapes[c.shape], c.off, vb);
        const cudaError_t e = inv_ragged_class<T>(A, dim3(nfg, c.count),
                                                  fft_smem_bytes(2 * A.L, p->G, vb == 16), s);
        if (e) return e;
    }
    RaggedInv<T> R;
    R.a = base;
    R.a.twp = static_cast<const V*>(rg->d_twpass);
    R.a.twpost = static_cast<const V*>(rg->d_twpost);
    R.a.rev = rg->d_rev;
    R.shapes = rg->d_shapes;
    R.shape_of = rg->d_shape_of;
    R.shift_of = rg->any_shift ? rg->d_shift_of : nullptr;
    R.shiftbase = static_cast<const V*>(rg->d_shiftph);
    R.chirpbase = static_cast<const V*>(rg->d_chirp);
    R.dftbase = static_cast<const V*>(rg->d_dft);
    cudaError_t e;
    if (rg->generic_count > 0) {
        R.a.jh_list = rg->d_jh + rg->generic_off;
        e = ensure_smem((const void*)fft_inverse_ragged_kernel<T>, p->fft_smem);
        if (e) return e;
        fft_inverse_ragged_kernel<T><<<dim3(nfg, rg->generic_count), NT, p->fft_smem, s>>>(R);
        note_launch();
        if ((e = cudaGetLastError())) return e;
    }
    if (rg->blue_count > 0) {
        R.a.jh_list = rg->d_jh + rg->blue_off;
        R.a.G = rg->blue_G;
        const unsigned nfb = (p->F + rg->blue_G - 1) / rg->blue_G;
        e = ensure_smem((const void*)fft_inverse_bluestein_kernel<T>, rg->blue_smem);
        if (e) return e;
        fft_inverse_bluestein_kernel<T><<<dim3(nfb, rg->blue_count), NT, rg->blue_smem, s>>>(R);
        note_launch();
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t fwd_group_impl(sht_plan_s* const* plans, int n, const void* const* grids,
                           cudaStream_t s) {
    FwdGroup<T> G;
    G.n = n;
    G.cta_start[0] = 0;
    size_t smem = 0;
    for (int q = 0; q < n; ++q) {
        const sht_plan_s* p = plans[q];
        RowSource src;
        src.field_stride = (long long)p->J * p->I;
        src.row_stride = p->I;
        src.row_offset = 0;
        src.elem_stride = 1;
        const FwdScale sc{p->d_w_over_I, 1.0, 1.0};
        G.a[q] = make_fwd_args<T>(p, grids[q], src, sc, p->d_work);
        if (p->d_colmax) {
            const cudaError_t e =
                cudaMemsetAsync(p->d_colmax, 0, 2 * (size_t)p->F * sizeof(unsigned), s);
            if (e) return e;
        }
        G.nfg[q] = (p->F + p->G - 1) / p->G;
        G.cta_start[q + 1] = G.cta_start[q] + G.nfg[q] * p->Jh;
        if (p->fft_smem > smem) smem = p->fft_smem;
    }
    cudaError_t e = ensure_smem((const void*)fft_forward_group_kernel<T>, smem);
    if (e) return e;
    fft_forward_group_kernel<T><<<G.cta_start[n], NT, smem, s>>>(G);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t inv_group_impl(sht_plan_s* const* plans, int n, void* const* grids,
                           cudaStream_t s) {
    InvGroup<T> G;
    G.n = n;
    G.cta_start[0] = 0;
    size_t smem = 0;
    for (int q = 0; q < n; ++q) {
        const sht_plan_s* p = plans[q];
        const InvScale sc{nullptr, 1.0};
        G.a[q] = make_inv_args<T>(p, p->d_work, sc, grids[q]);
        G.nfg[q] = (p->F + p->G - 1) / p->G;
        G.cta_start[q + 1] = G.cta_start[q] + G.nfg[q] * p->Jh;
        if (p->fft_smem > smem) smem = p->fft_smem;
    }
    cudaError_t e = ensure_smem((const void*)fft_inverse_group_kernel<T>, smem);
    if (e) return e;
    fft_inverse_group_kernel<T><<<G.cta_start[n], NT, smem, s>>>(G);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t fft_constants_init() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    float2 hf[kTwTotal];
    double2 hd[kTwTotal];
    const int sizes[5] = {10, 16, 20, 32, 40};
    const int offs[5] = {kTw10, kTw16, kTw20, kTw32, kTw40};
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int q = 0; q < 5; ++q)
        for (int k = 0; k < sizes[q]; ++k) {
            const long double ang = 2.0L * pi * (long double)k / (long double)sizes[q];
            const double c = (double)cosl(ang), sn = -(double)sinl(ang);
            hd[offs[q] + k] = make_double2(c, sn);
            hf[offs[q] + k] = make_float2((float)c, (float)sn);
        }
    e = cudaMemcpyToSymbol(c_twf, hf, sizeof(hf));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_twd, hd, sizeof(hd));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

cudaError_t launch_fft_forward_group(sht_plan_s* const* plans, int n,
                                     const void* const* grids, cudaStream_t s) {
    if (plans[0]->prec == SHT_FP64) return fwd_group_impl<double>(plans, n, grids, s);
    return fwd_group_impl<float>(plans, n, grids, s);
}

cudaError_t launch_fft_inverse_group(sht_plan_s* const* plans, int n,
                                     void* const* grids, cudaStream_t s) {
    if (plans[0]->prec == SHT_FP64) return inv_group_impl<double>(plans, n, grids, s);
    return inv_group_impl<float>(plans, n, grids, s);
}

size_t bluestein_smem_bytes(int Lmax, int L2, int G, bool fp64) {
    const size_t v = fp64 ? sizeof(double2) : sizeof(float2);
    // rows | twiddles of length L2 | column maxima (2 G words, rounded up to
    // whole complex values) | two scratch rows of length L2
    return (2 * (size_t)G * fft_row_pitch(Lmax, fp64) + L2 + (8 * (size_t)G + v - 1) / v +
            2 * (size_t)fft_row_pitch(L2, fp64)) * v;
}

size_t fft_smem_bytes(int I, int G, bool fp64) {
    const size_t L = (size_t)I / 2;
    const size_t v = fp64 ? sizeof(double2) : sizeof(float2);
    // padded rows + per-pass twiddle tables (fewer than L entries) + the
    // column maxima of the forward kernel's output (2 words per field)
    return (2 * (size_t)G * fft_row_pitch((int)L, fp64) + L) * v + 8 * (size_t)G;
}

cudaError_t launch_fft_forward(const sht_plan_s* p, const void* grid,
                               const RowSource& src, const FwdScale& sc,
                               void* work, cudaStream_t s) {
    if (p->ragged) {
        if (p->prec == SHT_FP64) return fwd_ragged_impl<double>(p, grid, sc, work, s);
        return fwd_ragged_impl<float>(p, grid, sc, work, s);
    }
    if (p->prec == SHT_FP64) return fwd_impl<double>(p, grid, src, sc, work, s);
    return fwd_impl<float>(p, grid, src, sc, work, s);
}

cudaError_t launch_fft_inverse(const sht_plan_s* p, const void* work,
                               const InvScale& sc, void* grid, cudaStream_t s) {
    if (p->ragged) {
        if (p->prec == SHT_FP64) return inv_ragged_impl<double>(p, work, sc, grid, s);
        return inv_ragged_impl<float>(p, work, sc, grid, s);
    }
    if (p->prec == SHT_FP64) return inv_impl<double>(p, work, sc, grid, s);
    return inv_impl<float>(p, work, sc, grid, s);
}

}  // namespace sht

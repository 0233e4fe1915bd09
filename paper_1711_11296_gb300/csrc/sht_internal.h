// Internal declarations of the GB300 Clenshaw-Curtis SHT library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sht.h"

namespace sht {

constexpr uint64_t kPlanMagic = 0x53485450'4C414E31ull;   // "SHTPLAN1"
constexpr int kMaxRadixPasses = 16;
constexpr int kMaxI = 8192;
constexpr int kMaxGroup = 8;    // plans per grouped launch

// Raise a kernel's dynamic shared-memory limit on the current device the
// first time a launch needs more than 48 KB (later launches, e.g. under
// stream capture, make no host API call).  Returns the CUDA status.
cudaError_t ensure_smem(const void* kernel, size_t bytes);

// Thread-local error message set by the C entry points (cleared at entry).
void set_error(const char* fmt, ...);
void clear_error();

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// Mixed-radix factorisation of the half-length complex FFT (L = I/2).
struct FftShape {
    int L = 0;
    int npass = 0;
    int radix[kMaxRadixPasses] = {0};
    int span[kMaxRadixPasses] = {0};   // M_p = L / (r_1 ... r_p)
    int twoff[kMaxRadixPasses] = {0};  // offset of pass p's twiddle table
    int twtotal = 0;                   // entries of all per-pass tables
};

// Shared-memory layout of an FFT row: element pos lives at
// pos + (pos >> PAD_SHIFT), rows LP = L + (L >> PAD_SHIFT) + 1 apart, so
// that neither the power-of-two strides of the passes and of the
// digit-reversed reads nor the row-to-row distance map onto one bank.
template <typename T> struct PadShift;
template <> struct PadShift<float> { static constexpr int value = 5; };    // 8-byte complex
template <> struct PadShift<double> { static constexpr int value = 3; };   // 16-byte complex

inline int fft_row_pitch(int L, bool fp64) {
    const int s = fp64 ? PadShift<double>::value : PadShift<float>::value;
    return L + (L >> s) + 1;
}

// Row-source description for the forward FFT (plain or nested/strided).
struct RowSource {
    long long field_stride = 0;   // elements between fields
    long long row_stride = 0;     // elements between consecutive (coarse) rows
    long long row_offset = 0;     // element offset of row 0
    int elem_stride = 1;          // elements between consecutive longitudes
};

// Scaling applied by the forward (analysis-type) FFT kernel.
struct FwdScale {
    const double* rowscale;   // [Jh] per northern row (w_j/I or 1), may be null
    double mscale0;           // factor for m = 0
    double mscale1;           // factor for m >= 1
};

// Scaling applied by the inverse (synthesis-type) FFT kernel.
struct InvScale {
    const double* rowscale;   // [Jh] per northern row (w_j/I or 1), may be null
    double mfactor1;          // factor for m >= 1 before the Hermitian sum
    int accumulate = 0;       // 1: add the rows to the grid instead of writing them;
                              // 2: products of Sec. 4.2 (see grid2)
    void* grid2 = nullptr;    // accumulate = 2: the grid holds u and becomes u v,
                              // grid2 holds v and becomes u v w (w = the rows)
};

struct SplitTables;   // tensor-core operand tables (split plans)

// Reduced grid: latitude j carries its own number I_j of longitudes.  The
// distinct half-lengths L = I_j/2 each have an FFT shape and tables; their
// tables are concatenated in device buffers at the offsets below.
struct RShape {
    FftShape sh;          // the passes: of L, or of L2 for a Bluestein shape
    long long tw_off;     // per-pass twiddle tables (entries)
    long long post_off;   // e^{-2 pi i q / I_j}, q < L (entries)
    long long rev_off;    // digit-reversed positions of the passes' length (entries)
    int L = 0;            // half-length of the rows, L = I_j / 2
    int bluestein = 0;    // 1: L has a prime factor above 5; its DFT is a
                          // chirp-z convolution of length L2 = sh.L >= 2L - 1
    long long chirp_off = 0;   // Bluestein: e^{-pi i n^2 / L}, n < L (entries)
    long long dft_off = 0;     // Bluestein: DFT of the conjugate chirp / L2 (L2 entries)
    long long shift_off = -1;  // e^{-pi i m / I_j}, m < L (entries), or -1: none
};

struct RaggedGrid {
    std::vector<int> Ij;             // [J] longitudes per latitude, j = 0 northernmost
    long long npts = 0;              // grid points per field (sum of I_j)
    long long* d_rowoff = nullptr;   // [J] first point of row j within a field
    int* d_shape_of = nullptr;       // [Jh] shape index of latitude pair jh
    int* d_shift_of = nullptr;       // [Jh] 1: the pair's longitudes are shifted by
                                     // half a spacing (lambda_i = 2 pi (i + 1/2) / I_j)
    RShape* d_shapes = nullptr;      // [nshapes]
    void* d_twpass = nullptr;        // all shapes' per-pass twiddle tables
    void* d_twpost = nullptr;        // all shapes' real-spectrum twiddles
    int* d_rev = nullptr;            // all shapes' digit reversals
    void* d_chirp = nullptr;         // Bluestein shapes' chirps
    void* d_dft = nullptr;           // Bluestein shapes' chirp spectra
    void* d_shiftph = nullptr;       // phase tables of the shifted rows' shapes
    int nshapes = 0;
    bool any_shift = false;
    // Latitude pairs by launch: one launch per half-length that has a
    // compile-time FFT kernel (classes, unshifted rows), one generic launch
    // for the other 2-3-5-smooth rows and one Bluestein launch for the rows
    // whose half-length has a larger prime factor.
    struct Class { int shape; int off; int count; };
    std::vector<Class> classes;
    std::vector<RShape> h_shapes;    // host copy of d_shapes
    int generic_off = 0, generic_count = 0;
    int blue_off = 0, blue_count = 0;
    int blue_G = 1;                  // fields per CTA of the Bluestein launch
    size_t blue_smem = 0;            // its dynamic shared memory
    int* d_jh = nullptr;             // latitude-pair lists of all launches
};

// Shared memory of the Bluestein FFT kernels: the padded rows of G fields
// (pitch of half-length Lmax), the per-pass twiddles of length L2, the
// column maxima and two padded scratch rows of length L2.
size_t bluestein_smem_bytes(int Lmax, int L2, int G, bool fp64);

// Half-lengths with compile-time FFT kernels (the standard grids).
inline bool fft_has_fixed_kernel(int L) {
    return L == 64 || L == 128 || L == 256 || L == 320 || L == 512 || L == 640 || L == 1024 ||
           L == 1280;
}

enum Stage { kStageFftFwd = 0, kStageLegFwd = 1, kStageLegInv = 2,
             kStageFftInv = 3, kStageSplitConv = 4 };

// Optional per-launch event timing.
struct Profiler {
    bool on = false;
    struct Rec { int stage; cudaEvent_t a, b; long long kernels; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get();
};

}  // namespace sht

struct sht_plan_s {
    uint64_t magic;
    int N, J, I, F, prec, exact;
    int Jh;          // (J+1)/2 northern nodes incl. the Equator
    int M;           // N+1 zonal wavenumbers
    int device;
    int num_sms;     // SMs of the device (grid of the persistent kernels)
    size_t ncoef;
    int ldp;         // leading dimension of the P~ table (>= Jh)
    int grid;        // latitude grid: SHT_GRID_CC (Sec. 3) or SHT_GRID_FEJER1 (Sec. 3.3)
    int G;           // fields per FFT CTA
    int fft_threads;
    size_t fft_smem;
    sht::FftShape fft;

    // device tables (FP64)
    double* d_mu;          // [Jh] cos(theta_j)
    double* d_sin;         // [Jh] sin(theta_j)
    double* d_w;           // [Jh] Clenshaw-Curtis weights
    double* d_w_over_I;    // [Jh] w_j / I
    double* d_eps;         // [ncoef] recurrence eps_n^m (host-built)
    double* d_amm;         // [M] sqrt((2m+1)/(2m))
    double* d_pnm;         // [ncoef][ldp] P~_n^m(mu_j), northern nodes
    int* d_rev;            // [L] digit-reversed position of frequency k
    void* d_tw;            // [L] e^{-2 pi i e / L}   (double2 or float2)
    void* d_twpost;        // [L] e^{-2 pi i q / I}   (double2 or float2)
    void* d_twpass;        // per-pass twiddle tables (see FftShape::twoff)
    void* d_work;          // [M][2][Jh][F] complex Fourier workspace
    size_t work_bytes;

    // Legendre tile lists: int4 {m, parity, row0, col0}
    int4* d_tiles_fwd; int ntiles_fwd;
    int4* d_tiles_inv; int ntiles_inv;

    int* d_status;             // device status word: kernels OR in failure bits
                               // (1: tensor-core wait timed out, 2: FFT wait timed out)
    void* d_spec_pad;          // spectrum-sized buffer of sht_prolong_spectral (on first use)
    int* d_jmin;               // FP64 plans with the reduced transform: [2(N+1)]
                               // first node with some |P~| >= 1e-16 (null: off)
    sht::SplitTables* split;   // null for FP64 plans
    unsigned* d_colmax;        // FP16 split plans: [2][2F] column maxima (float bits)
                               // of the forward and inverse GEMMs' FP32 operand
    sht::Profiler* prof;       // per-launch timing, off by default
    sht::RaggedGrid* ragged;   // reduced grid (per-latitude I_j); null: regular J x I
};

namespace sht {

bool plan_is_live(const sht_plan_s* p);

// Bracket a launch with profiling events when the plan's profiler is on.
// Kernels the library has launched on this thread for transforms (every
// per-call launch site calls note_launch); a profiling scope records how
// many fell inside it.
extern thread_local long long g_kernels;
inline void note_launch() { ++g_kernels; }

struct ProfScope {
    const sht_plan_s* p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    long long k0 = 0;
    ProfScope(const sht_plan_s* plan, int st, cudaStream_t stream);
    ~ProfScope();
};

// tables
cudaError_t build_node_tables(sht_plan_s* p, cudaStream_t s);
cudaError_t build_pnm_table(sht_plan_s* p, cudaStream_t s);
cudaError_t build_twiddles(sht_plan_s* p, cudaStream_t s);
cudaError_t launch_twpass(const sht_plan_s* p, cudaStream_t s);
cudaError_t build_fft_tables(const FftShape& sh, bool fp64, void* twpass, void* twpost,
                             int* rev, void* tmp, cudaStream_t s);
// Tables of a Bluestein shape (rows of half-length L, passes sh2 of length
// L2 >= 2L - 1): the passes' twiddles and digit reversal, the row's
// real-spectrum twiddles e^{-2 pi i q / 2L}, the chirp e^{-pi i n^2 / L}
// (n < L) and the DFT of length L2 of the conjugate chirp wrapped around
// L2, divided by L2.  tmp: device scratch of 4 L2 doubles.
cudaError_t build_bluestein_tables(int L, const FftShape& sh2, bool fp64, void* twpass,
                                   void* twpost, int* rev, void* chirp, void* dft, void* tmp,
                                   cudaStream_t s);
// e^{-pi i m / I} for m < n (the zonal phase of a row shifted by half a
// spacing), in the plan's precision.
cudaError_t build_shift_table(int n, int I, bool fp64, void* out, cudaStream_t s);
void ragged_free(RaggedGrid* rg);
int inverse_scaled(sht_plan_s* p, const void* spec, const InvScale& sc, void* grid,
                   cudaStream_t s);

// Register DFT sizes of the two-pass FP32 FFT (L = Q x 32).
__host__ __device__ constexpr bool fft_big_radix(int q) {
    return q == 2 || q == 4 || q == 8 || q == 10 || q == 16 || q == 20 || q == 32 ||
           q == 40;
}

// Mixed-radix factorisation of the half-length FFT, shared by the plans,
// the allocation-free entry point and the compile-time kernels.  FP32
// transforms of L = Q x 32 (Q a register DFT size) use two passes, radix Q
// then radix 32, each butterfly computed in registers; everything else
// uses radices 8 first, then 4, 2, 3, 5.  Spans and per-pass twiddle
// offsets follow.  npass = 0 and L != 1 means "not factorable".
__host__ __device__ constexpr FftShape fft_factor(int L, bool fp64) {
    FftShape sh{};
    sh.L = L;
    int rest = L, np = 0;
    if (!fp64 && L % 32 == 0 && fft_big_radix(L / 32)) {
        sh.radix[np++] = L / 32;
        sh.radix[np++] = 32;
        rest = 1;
    }
    const int cand[5] = {8, 4, 2, 3, 5};
    for (int c = 0; c < 5; ++c)
        while (rest % cand[c] == 0 && np < kMaxRadixPasses) {
            sh.radix[np++] = cand[c];
            rest /= cand[c];
        }
    if (rest != 1) return FftShape{};
    int span = L, off = 0;
    for (int q = 0; q < np; ++q) {
        span /= sh.radix[q];
        sh.span[q] = span;
        sh.twoff[q] = off;
        off += (sh.radix[q] - 1) * span;
    }
    sh.npass = np;
    sh.twtotal = off;
    return sh;
}

__host__ __device__ constexpr bool fft_factorable(int L) {
    return L == 1 || fft_factor(L, true).npass > 0;
}

// Write the constant twiddles of the register DFTs to the current device
// (once per device; safe to call repeatedly).
cudaError_t fft_constants_init();

// FFT launches
cudaError_t launch_fft_forward(const sht_plan_s* p, const void* grid,
                               const RowSource& src, const FwdScale& sc,
                               void* work, cudaStream_t s);
cudaError_t launch_fft_inverse(const sht_plan_s* p, const void* work,
                               const InvScale& sc, void* grid, cudaStream_t s);
// One launch over n plans (same precision): plain analysis / synthesis FFTs.
cudaError_t launch_fft_forward_group(sht_plan_s* const* plans, int n,
                                     const void* const* grids, cudaStream_t s);
cudaError_t launch_fft_inverse_group(sht_plan_s* const* plans, int n,
                                     void* const* grids, cudaStream_t s);
size_t fft_smem_bytes(int I, int G, bool fp64);

// FP64 Legendre launches
cudaError_t launch_legendre_fwd_fp64(const sht_plan_s* p, const double* work,
                                     double* spec, cudaStream_t s);
cudaError_t launch_legendre_inv_fp64(const sht_plan_s* p, const double* spec,
                                     double* work, cudaStream_t s);

__host__ __device__ inline size_t coef_offset(int N, int m) {
    return (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
}

}  // namespace sht

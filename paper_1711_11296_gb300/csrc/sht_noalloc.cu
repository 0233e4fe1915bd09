// Allocation-free FP64 analysis (grid -> spectrum) for small problems.
//
// Some callers cannot allocate device memory at all: a plug-in running
// inside a host application that owns every byte of the GPU through its own
// pool, or code that runs while the application forbids allocations (for
// example during a stream capture or a latency-critical section).  For them
// this file holds one fixed scratch area in a file-scope __device__ array:
// the Clenshaw-Curtis nodes and weights, the P~ table, the FFT tables, the
// Legendre tile list and the Fourier workspace are rebuilt in it by every
// call, with the same kernels the plan-based sht_forward uses.  The caller
// passes only the grid and the spectrum.
//
// The array is SHT_NOALLOC_SCRATCH_BYTES long.  It belongs to this file's
// device module, which the CUDA runtime loads into a context on first use
// (lazily, by default): the first call on a device commits the 32 MiB, and
// every later call in that context finds it there until the process exits.
// A call that is not being captured looks the array's device address up in
// the current context (with the device current) and remembers it per
// context; a call under stream capture uses the remembered address, so the
// first call in a context must come before any capture.  Every call
// overwrites the array, so calls that overlap on the GPU (on different
// streams, or from several threads) race; each call rewrites every entry it
// later reads, so nothing depends on the previous call's contents.
#include <cuda.h>

#include "sht_ctx_cache.h"
#include "sht_internal.h"

namespace sht {

cudaError_t launch_pnm_recurrence(const sht_plan_s* p, cudaStream_t s);
cudaError_t launch_twiddles_fp64(const sht_plan_s* p, cudaStream_t s);
int legendre_fwd_tile_count(int N, int C);
cudaError_t launch_build_fwd_tiles(int N, int C, int4* tiles, cudaStream_t s);

namespace {

constexpr int kMaxContexts = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SHT_NOALLOC_SCRATCH_BYTES];

ContextAddressCache<kMaxContexts> g_scratch_cache;

// The driver's cuCtxGetCurrent, reached through the runtime (no link
// against libcuda): the key of the per-context address memo.
using CtxGetCurrent = CUresult (*)(CUcontext*);

cudaError_t current_context(const void** ctx) {
    static CtxGetCurrent fn = nullptr;
    static cudaError_t init = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000,
                                                         cudaEnableDefault, &q);
        if (e == cudaSuccess && q != cudaDriverEntryPointSuccess) e = cudaErrorNotSupported;
        fn = reinterpret_cast<CtxGetCurrent>(f);
        return e;
    }();
    if (init != cudaSuccess) return init;
    CUcontext c = nullptr;
    if (fn(&c) != CUDA_SUCCESS || !c) return cudaErrorDeviceUninitialized;
    *ctx = c;
    return cudaSuccess;
}

// Device address of the scratch array in the current context; see the file
// comment for when it is looked up and when the remembered one is used.
int scratch_address(cudaStream_t s, unsigned char** out) {
    const void* ctx = nullptr;
    cudaError_t e = current_context(&ctx);
    if (e != cudaSuccess) {
        set_error("no current CUDA context: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
        set_error("cudaStreamIsCapturing: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    cudaError_t lookup_err = cudaSuccess;
    void* addr = nullptr;
    const int rc = scratch_for_context(
        g_scratch_cache, ctx, cs != cudaStreamCaptureStatusNone,
        [&](void** a) {
            lookup_err = cudaGetSymbolAddress(a, g_noalloc_scratch);
            return lookup_err == cudaSuccess ? 0 : 1;
        },
        &addr);
    if (rc == kScratchNeedsSetup) {
        set_error("sht_forward_noalloc under stream capture before any uncaptured call "
                  "in this context: make the first call before capturing");
        return SHT_ERR_ARG;
    }
    if (rc != kScratchOk) {
        set_error("the %u-byte scratch array is not available in this context (%s); it "
                  "is committed when the first call loads it, so make that call at "
                  "start-up, before other code takes the device memory",
                  (unsigned)SHT_NOALLOC_SCRATCH_BYTES, cudaGetErrorString(lookup_err));
        return SHT_ERR_CUDA;
    }
    *out = static_cast<unsigned char*>(addr);
    return SHT_OK;
}

// Recurrence coefficients, the same formulas as plan creation (IEEE sqrt
// and division give the same values on the device): eps_n^m in
// [row0 + n - m], 1/eps_n^m after all eps, a_m = sqrt((2m+1)/(2m)).
// Slot n = m (eps_m^m = 0) is written as zero: the recurrence reads it.
__global__ void eps_kernel(int N, double* eps, double* amm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > N) return;
    const size_t nc = (size_t)(N + 1) * (N + 2) / 2;
    const size_t r0 = coef_offset(N, m);
    amm[m] = m > 0 ? sqrt((2.0 * m + 1.0) / (2.0 * m)) : 0.0;
    eps[r0] = 0.0;
    eps[nc + r0] = 0.0;
    for (int n = m + 1; n <= N; ++n) {
        const double nn = n, mm = m;
        const double e = sqrt((nn * nn - mm * mm) / (4.0 * nn * nn - 1.0));
        eps[r0 + (n - m)] = e;
        eps[nc + r0 + (n - m)] = 1.0 / e;
    }
}

// Digit-reversed output position of frequency k of the in-place FFT.
__global__ void rev_kernel(FftShape sh, int* rev) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sh.L) return;
    int kk = k, pos = 0;
    for (int q = 0; q < sh.npass; ++q) {
        pos += (kk % sh.radix[q]) * sh.span[q];
        kk /= sh.radix[q];
    }
    rev[k] = pos;
}

bool factor(int L, FftShape& sh) {
    if (!fft_factorable(L)) return false;
    sh = fft_factor(L, true);
    return true;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace sht

using namespace sht;

extern "C" int sht_forward_noalloc(int N, int J, int I, int nfields,
                                   const double* grid, double* spec,
                                   void* stream) {
    clear_error();
    if (N < 0 || J < 1 || J % 2 == 0 || I % 2 != 0 || I <= 2 * N || I > kMaxI ||
        nfields < 1) {
        set_error("invalid sizes N=%d J=%d I=%d nfields=%d", N, J, I, nfields);
        return SHT_ERR_ARG;
    }
    if (!grid || !spec) {
        set_error("NULL buffer");
        return SHT_ERR_ARG;
    }
    FftShape shape;
    if (!factor(I / 2, shape)) {
        set_error("I/2 = %d has prime factors other than 2, 3, 5", I / 2);
        return SHT_ERR_ARG;
    }
    sht_plan_s t{};
    t.N = N; t.J = J; t.I = I; t.F = nfields; t.prec = SHT_FP64;
    t.exact = J >= 2 * N + 1;
    t.Jh = (J + 1) / 2;
    t.M = N + 1;
    t.ncoef = (size_t)(N + 1) * (N + 2) / 2;
    t.ldp = (t.Jh + 7) / 8 * 8;
    t.fft = shape;
    const size_t rowbytes = (size_t)fft_row_pitch(shape.L, true) * sizeof(double2);
    const size_t budget = 110 * 1024;
    long g = (long)((budget / rowbytes > 1 ? budget / rowbytes - 1 : 0) / 2);
    g = g < 1 ? 1 : (g > 16 ? 16 : g);
    t.G = (int)(g > nfields ? nfields : g);
    t.fft_threads = 256;
    t.fft_smem = fft_smem_bytes(I, t.G, true);
    if (t.fft_smem > 227 * 1024) {
        set_error("I = %d too large for the shared-memory FFT", I);
        return SHT_ERR_UNSUPPORTED;
    }
    const int C = 2 * nfields;
    t.ntiles_fwd = legendre_fwd_tile_count(N, C);
    t.work_bytes = (size_t)t.M * 2 * t.Jh * nfields * sizeof(double2);

    // layout of the scratch array
    size_t off = 0;
    const size_t o_mu = off; off += up256(t.Jh * sizeof(double));
    const size_t o_sn = off; off += up256(t.Jh * sizeof(double));
    const size_t o_w = off; off += up256(t.Jh * sizeof(double));
    const size_t o_wI = off; off += up256(t.Jh * sizeof(double));
    const size_t o_eps = off; off += up256(2 * t.ncoef * sizeof(double));
    const size_t o_amm = off; off += up256((N + 1) * sizeof(double));
    const size_t o_pnm = off; off += up256(t.ncoef * (size_t)t.ldp * sizeof(double));
    const size_t o_rev = off; off += up256(shape.L * sizeof(int));
    const size_t o_tw = off; off += up256(shape.L * sizeof(double2));
    const size_t o_twp = off; off += up256(shape.L * sizeof(double2));
    const size_t o_tws = off; off += up256((shape.twtotal + 1) * sizeof(double2));
    const size_t o_til = off; off += up256((size_t)t.ntiles_fwd * sizeof(int4));
    const size_t o_wrk = off; off += up256(t.work_bytes);
    if (off > (size_t)SHT_NOALLOC_SCRATCH_BYTES) {
        set_error("N=%d J=%d I=%d nfields=%d needs %zu bytes of scratch; "
                  "sht_forward_noalloc has %zu", N, J, I, nfields, off,
                  (size_t)SHT_NOALLOC_SCRATCH_BYTES);
        return SHT_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    const int arc = scratch_address(s, &base);
    if (arc != SHT_OK) return arc;
    t.device = dev;
    t.d_mu = (double*)(base + o_mu);
    t.d_sin = (double*)(base + o_sn);
    t.d_w = (double*)(base + o_w);
    t.d_w_over_I = (double*)(base + o_wI);
    t.d_eps = (double*)(base + o_eps);
    t.d_amm = (double*)(base + o_amm);
    t.d_pnm = (double*)(base + o_pnm);
    t.d_rev = (int*)(base + o_rev);
    t.d_tw = base + o_tw;
    t.d_twpost = base + o_twp;
    t.d_twpass = base + o_tws;
    t.d_tiles_fwd = (int4*)(base + o_til);
    t.d_work = base + o_wrk;

    const int th = 128;
    e = build_node_tables(&t, s);
    if (e == cudaSuccess) {
        eps_kernel<<<(N + 1 + th - 1) / th, th, 0, s>>>(N, t.d_eps, t.d_amm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_pnm_recurrence(&t, s);
    if (e == cudaSuccess) e = launch_twiddles_fp64(&t, s);
    if (e == cudaSuccess) e = launch_twpass(&t, s);
    if (e == cudaSuccess) {
        rev_kernel<<<(shape.L + th - 1) / th, th, 0, s>>>(shape, t.d_rev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_build_fwd_tiles(N, C, t.d_tiles_fwd, s);
    RowSource src;
    src.field_stride = (long long)J * I;
    src.row_stride = I;
    src.row_offset = 0;
    src.elem_stride = 1;
    FwdScale sc{t.d_w_over_I, 1.0, 1.0};
    if (e == cudaSuccess) e = launch_fft_forward(&t, grid, src, sc, t.d_work, s);
    if (e == cudaSuccess)
        e = launch_legendre_fwd_fp64(&t, (const double*)t.d_work, spec, s);
    if (e != cudaSuccess) {
        set_error("sht_forward_noalloc launch: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    return SHT_OK;
}

// C ABI of the library: plan life cycle and the transform entry points.
// Every transform is a short fixed sequence of kernel launches on the
// caller's stream; no entry point touches host data except plan creation,
// sht_plan_copy_tables and error reporting.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "sht_internal.h"

namespace sht {

void build_legendre_tiles(int N, int Jh, int C, std::vector<int4>& fwd,
                          std::vector<int4>& inv);
cudaError_t split_tables_create(sht_plan_s* p, cudaStream_t s);
void split_tables_destroy(sht_plan_s* p);
cudaError_t launch_legendre_fwd_split(const sht_plan_s* p, const void* work,
                                      void* spec, cudaStream_t s);
cudaError_t launch_legendre_inv_split(const sht_plan_s* p, const void* spec,
                                      void* work, cudaStream_t s);
int split_status_read_and_clear(const sht_plan_s* p);

namespace {
thread_local std::string g_error;
std::mutex g_live_mu;
std::set<const sht_plan_s*> g_live;

struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            switched = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

bool factor_fft(int L, bool fp64, FftShape& sh) {
    if (!fft_factorable(L)) return false;
    sh = fft_factor(L, fp64);
    return true;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SHT_ERR_CUDA;
}

void free_plan_memory(sht_plan_s* p) {
    void* ptrs[] = {p->d_mu, p->d_sin, p->d_w, p->d_w_over_I, p->d_eps, p->d_amm,
                    p->d_pnm, p->d_rev, p->d_tw, p->d_twpost, p->d_twpass, p->d_work,
                    p->d_tiles_fwd, p->d_tiles_inv, p->d_status, p->d_jmin,
                    p->d_spec_pad};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p->split) split_tables_destroy(p);
    if (p->ragged) {
        ragged_free(p->ragged);
        p->ragged = nullptr;
    }
    if (p->prof) {
        for (auto& r : p->prof->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : p->prof->pool) cudaEventDestroy(e);
        delete p->prof;
        p->prof = nullptr;
    }
}

int check_plan(const sht_plan_s* p) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    return SHT_OK;
}

}  // namespace

void clear_error() { g_error.clear(); }

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
}

bool plan_is_live(const sht_plan_s* p) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    return g_live.count(p) != 0 && p->magic == kPlanMagic;
}

cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = done[{dev, kernel}];
    if (bytes <= have) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

thread_local long long g_kernels = 0;

ProfScope::ProfScope(const sht_plan_s* plan, int st, cudaStream_t stream)
    : p(plan), stage(st), s(stream), k0(g_kernels) {
    if (p->prof && p->prof->on) {
        a = p->prof->get();
        if (a) cudaEventRecord(a, s);
    }
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = p->prof->get();
    if (!b) {
        p->prof->pool.push_back(a);
        return;
    }
    cudaEventRecord(b, s);
    p->prof->recs.push_back({stage, a, b, g_kernels - k0});
}

}  // namespace sht

using namespace sht;

extern "C" const char* sht_last_error(void) { return g_error.c_str(); }

extern "C" const char* sht_version(void) { return "cc-sht 0.1 (sm_103a)"; }

extern "C" int sht_plan_create(int N, int J, int I, int nfields, int precision,
                               sht_plan_t* out) {
    return sht_plan_create_grid(N, J, I, nfields, precision, SHT_GRID_CC, out);
}

extern "C" int sht_plan_create_grid(int N, int J, int I, int nfields, int precision,
                                    int grid, sht_plan_t* out) {
    g_error.clear();
    if (!out) { set_error("out is NULL"); return SHT_ERR_ARG; }
    if (grid != SHT_GRID_CC && grid != SHT_GRID_FEJER1) {
        set_error("unknown latitude grid %d", grid);
        return SHT_ERR_ARG;
    }
    if (N < 0) { set_error("N = %d < 0", N); return SHT_ERR_ARG; }
    if (J < 1 || J % 2 == 0) {
        set_error("J = %d must be odd and >= 1 (the Equator node is needed)", J);
        return SHT_ERR_ARG;
    }
    if (I % 2 != 0 || I <= 2 * N || I > kMaxI) {
        set_error("I = %d must be even, > 2N = %d and <= %d", I, 2 * N, kMaxI);
        return SHT_ERR_ARG;
    }
    if (nfields < 1) { set_error("nfields = %d < 1", nfields); return SHT_ERR_ARG; }
    if (precision < SHT_FP64 || precision > SHT_FP16X3) {
        set_error("unknown precision %d", precision);
        return SHT_ERR_ARG;
    }
    FftShape shape;
    if (!factor_fft(I / 2, precision == SHT_FP64, shape)) {
        set_error("I/2 = %d has prime factors other than 2, 3, 5", I / 2);
        return SHT_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
    e = fft_constants_init();
    if (e != cudaSuccess) return cuda_fail(e, "FFT constants");

    sht_plan_s* p = new (std::nothrow) sht_plan_s();
    if (!p) { set_error("host allocation failed"); return SHT_ERR_ALLOC; }
    p->grid = grid;
    p->N = N; p->J = J; p->I = I; p->F = nfields; p->prec = precision;
    p->exact = (J >= 2 * N + 1) ? 1 : 0;
    p->Jh = (J + 1) / 2;
    p->M = N + 1;
    p->device = dev;
    p->num_sms = 148;
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    p->ncoef = (size_t)(N + 1) * (N + 2) / 2;
    p->ldp = (p->Jh + 7) / 8 * 8;
    p->fft = shape;
    const bool fp64 = precision == SHT_FP64;
    const size_t vbytes = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t rowbytes = (size_t)fft_row_pitch(shape.L, fp64) * vbytes;
    const size_t budget = 110 * 1024;
    long g = (long)((budget / rowbytes > 1 ? budget / rowbytes - 1 : 0) / 2);
    if (g < 1) g = 1;
    if (g > 16) g = 16;
    if (g > nfields) g = nfields;
    p->G = (int)g;
    p->fft_threads = 256;
    p->fft_smem = fft_smem_bytes(I, p->G, fp64);
    if (p->fft_smem > 227 * 1024) {
        delete p;
        set_error("I = %d too large for the shared-memory FFT", I);
        return SHT_ERR_UNSUPPORTED;
    }

    cudaStream_t s = nullptr;
    int rc = SHT_OK;
    // failure-detection tests: SHT_INJECT_ALLOC_FAIL=k fails the k-th device
    // allocation of the plan's tables as if the device were out of memory
    int inject_alloc = 0, nalloc = 0;
    if (const char* v = getenv("SHT_INJECT_ALLOC_FAIL")) inject_alloc = atoi(v);
    auto alloc = [&](void** ptr, size_t bytes, const char* what) -> bool {
        e = (++nalloc == inject_alloc) ? cudaErrorMemoryAllocation
                                       : cudaMalloc(ptr, bytes > 0 ? bytes : 16);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            cudaGetLastError();
            set_error("cudaMalloc(%zu) for %s failed: %s", bytes, what,
                      cudaGetErrorString(e));
            rc = SHT_ERR_ALLOC;
            return false;
        }
        return true;
    };
    std::vector<int4> tf, ti;
    build_legendre_tiles(N, p->Jh, 2 * nfields, tf, ti);
    p->ntiles_fwd = (int)tf.size();
    p->ntiles_inv = (int)ti.size();
    p->work_bytes = (size_t)p->M * 2 * p->Jh * nfields * vbytes;
    const int L = shape.L;
    bool ok = alloc((void**)&p->d_mu, p->Jh * sizeof(double), "nodes") &&
              alloc((void**)&p->d_sin, p->Jh * sizeof(double), "nodes") &&
              alloc((void**)&p->d_w, p->Jh * sizeof(double), "weights") &&
              alloc((void**)&p->d_w_over_I, p->Jh * sizeof(double), "weights") &&
              alloc((void**)&p->d_eps, 2 * p->ncoef * sizeof(double), "recurrence") &&
              alloc((void**)&p->d_amm, (N + 1) * sizeof(double), "recurrence") &&
              alloc((void**)&p->d_pnm, p->ncoef * (size_t)p->ldp * sizeof(double), "P table") &&
              alloc((void**)&p->d_rev, L * sizeof(int), "FFT") &&
              alloc(&p->d_tw, L * vbytes, "FFT") &&
              alloc(&p->d_twpost, L * vbytes, "FFT") &&
              alloc(&p->d_twpass, (shape.twtotal + 1) * vbytes, "FFT") &&
              alloc(&p->d_work, p->work_bytes, "workspace") &&
              alloc((void**)&p->d_tiles_fwd, tf.size() * sizeof(int4), "tiles") &&
              alloc((void**)&p->d_tiles_inv, ti.size() * sizeof(int4), "tiles") &&
              alloc((void**)&p->d_status, sizeof(int), "status");
    if (ok) {
        e = cudaMemset(p->d_status, 0, sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_tiles_fwd, tf.data(), tf.size() * sizeof(int4),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_tiles_inv, ti.data(), ti.size() * sizeof(int4),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = build_node_tables(p, s);
        if (e == cudaSuccess) e = build_pnm_table(p, s);
        if (e == cudaSuccess) e = build_twiddles(p, s);
        if (e == cudaSuccess && !fp64) e = split_tables_create(p, s);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            if (e == cudaErrorNotSupported) {
                rc = SHT_ERR_UNSUPPORTED;   // message set by the table builder
            } else {
                rc = e == cudaErrorMemoryAllocation ? SHT_ERR_ALLOC : SHT_ERR_CUDA;
                set_error("plan tables: %s", cudaGetErrorString(e));
            }
            cudaGetLastError();
        }
    }
    if (rc != SHT_OK) {
        free_plan_memory(p);
        delete p;
        return rc;
    }
    p->magic = kPlanMagic;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.insert(p);
    }
    *out = p;
    return p->exact ? SHT_OK : SHT_WARN_INEXACT;
}

extern "C" int sht_plan_destroy(sht_plan_t plan) {
    if (!plan) return SHT_OK;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        if (!g_live.count(plan)) {
            set_error("invalid or destroyed plan handle");
            return SHT_ERR_HANDLE;
        }
        g_live.erase(plan);
    }
    DeviceGuard dg(plan->device);
    cudaDeviceSynchronize();
    free_plan_memory(plan);
    plan->magic = 0;
    delete plan;
    return SHT_OK;
}

extern "C" int sht_plan_query(sht_plan_t p, int* N, int* J, int* I, int* nfields,
                              int* precision, int* exact, size_t* ncoef) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (N) *N = p->N;
    if (J) *J = p->J;
    if (I) *I = p->I;
    if (nfields) *nfields = p->F;
    if (precision) *precision = p->prec;
    if (exact) *exact = p->exact;
    if (ncoef) *ncoef = p->ncoef;
    return SHT_OK;
}

namespace {

int forward_scaled(sht_plan_t p, const void* grid, const RowSource& src,
                   const FwdScale& sc, void* spec, cudaStream_t s) {
    cudaError_t e;
    {
        ProfScope ps(p, kStageFftFwd, s);
        e = launch_fft_forward(p, grid, src, sc, p->d_work, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "forward FFT launch");
    {
        ProfScope ps(p, kStageLegFwd, s);
        if (p->prec == SHT_FP64)
            e = launch_legendre_fwd_fp64(p, (const double*)p->d_work, (double*)spec, s);
        else
            e = launch_legendre_fwd_split(p, p->d_work, spec, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "forward Legendre launch");
    return SHT_OK;
}

int forward_impl(sht_plan_t p, const void* grid, const RowSource& src, void* spec,
                 cudaStream_t s) {
    FwdScale sc{p->d_w_over_I, 1.0, 1.0};
    return forward_scaled(p, grid, src, sc, spec, s);
}

int inverse_impl(sht_plan_t p, const void* spec, const InvScale& sc, void* grid,
                 cudaStream_t s) {
    cudaError_t e;
    {
        ProfScope ps(p, kStageLegInv, s);
        if (p->prec == SHT_FP64)
            e = launch_legendre_inv_fp64(p, (const double*)spec, (double*)p->d_work, s);
        else
            e = launch_legendre_inv_split(p, spec, p->d_work, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "inverse Legendre launch");
    {
        ProfScope ps(p, kStageFftInv, s);
        e = launch_fft_inverse(p, p->d_work, sc, grid, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "inverse FFT launch");
    return SHT_OK;
}

}  // namespace

// The inverse path with the FFT's scaling and store mode given (used by the
// multigrid prolongation, which can add onto the grid).
int sht::inverse_scaled(sht_plan_t p, const void* spec, const InvScale& sc, void* grid,
                        cudaStream_t s) {
    return inverse_impl(p, spec, sc, grid, s);
}

namespace {

RowSource plain_source(const sht_plan_s* p) {
    RowSource src;
    src.field_stride = (long long)p->J * p->I;
    src.row_stride = p->I;
    src.row_offset = 0;
    src.elem_stride = 1;
    return src;
}

}  // namespace

extern "C" int sht_forward(sht_plan_t p, const void* grid, void* spec, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!grid || !spec) { set_error("NULL buffer"); return SHT_ERR_ARG; }
    DeviceGuard dg(p->device);
    return forward_impl(p, grid, plain_source(p), spec, (cudaStream_t)stream);
}

extern "C" int sht_inverse(sht_plan_t p, const void* spec, void* grid, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!grid || !spec) { set_error("NULL buffer"); return SHT_ERR_ARG; }
    DeviceGuard dg(p->device);
    InvScale sc{nullptr, 1.0};
    return inverse_impl(p, spec, sc, grid, (cudaStream_t)stream);
}

extern "C" int sht_adjoint(sht_plan_t p, int which, const void* in, void* out,
                           void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!in || !out) { set_error("NULL buffer"); return SHT_ERR_ARG; }
    if (which != 0 && which != 1) {
        set_error("which = %d must be 0 (adjoint of forward) or 1 (of inverse)", which);
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (which == 0) {
        // spectrum -> grid: P~ contraction, unfold, Hermitian sum with the
        // m >= 1 terms halved, rows scaled by w_j / I.
        InvScale sc{p->d_w_over_I, 0.5};
        return inverse_impl(p, in, sc, out, s);
    }
    // grid -> spectrum: FFT without 1/I, c_m = 1 (m = 0) or 2, fold,
    // P~ contraction without weights.
    FwdScale sc{nullptr, 1.0, 2.0};
    return forward_scaled(p, in, plain_source(p), sc, out, s);
}

extern "C" int sht_alias_products(sht_plan_t p, const void* spec_u, const void* spec_v,
                                  const void* spec_w, void* grid_q, void* grid_c,
                                  void* spec_q, void* spec_c, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!spec_u || !spec_v || !spec_w || !grid_q || !grid_c || !spec_q || !spec_c) {
        set_error("NULL buffer");
        return SHT_ERR_ARG;
    }
    if (grid_q == grid_c || spec_q == spec_c) {
        set_error("the two grids and the two output spectra must be distinct buffers");
        return SHT_ERR_ARG;
    }
    if (p->ragged) {
        set_error("the products are built for full latitude rows only");
        return SHT_ERR_UNSUPPORTED;
    }
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    // U into grid_q, V into grid_c, then W: its inverse FFT forms the
    // products at each point as it stores (grid_q = U V, grid_c = U V W)
    const InvScale plain{nullptr, 1.0};
    rc = inverse_impl(p, spec_u, plain, grid_q, s);
    if (rc) return rc;
    rc = inverse_impl(p, spec_v, plain, grid_c, s);
    if (rc) return rc;
    InvScale prod{nullptr, 1.0, 2, grid_c};
    rc = inverse_impl(p, spec_w, prod, grid_q, s);
    if (rc) return rc;
    rc = forward_impl(p, grid_q, plain_source(p), spec_q, s);
    if (rc) return rc;
    return forward_impl(p, grid_c, plain_source(p), spec_c, s);
}

extern "C" int sht_restrict_nested(sht_plan_t p, const void* fine_grid, int k,
                                   void* coarse_spec, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!fine_grid || !coarse_spec) { set_error("NULL buffer"); return SHT_ERR_ARG; }
    if (p->ragged) {
        set_error("a reduced grid (per-latitude longitudes) does not nest");
        return SHT_ERR_NOT_NESTED;
    }
    if (p->grid != SHT_GRID_CC) {
        set_error("the shifted (Fejer first-rule) grid does not nest (Sec. 3.3)");
        return SHT_ERR_NOT_NESTED;
    }
    if (k < 1 || k > 8) { set_error("k = %d must be in 1..8", k); return SHT_ERR_ARG; }
    const long long s2 = 1LL << k;
    const long long Jf = s2 * (p->J + 1) - 1, If = s2 * p->I;
    if (If > (1LL << 30) || Jf > (1LL << 30)) {
        set_error("fine grid too large");
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    RowSource src;
    src.field_stride = Jf * If;
    src.row_stride = s2 * If;
    src.row_offset = (s2 - 1) * If;
    src.elem_stride = (int)s2;
    return forward_impl(p, fine_grid, src, coarse_spec, (cudaStream_t)stream);
}

extern "C" int sht_plan_copy_tables(sht_plan_t p, double* w, double* mu, double* pnm) {
    int rc = check_plan(p);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    std::vector<double> h(p->Jh);
    cudaError_t e;
    if (w) {
        e = cudaMemcpy(h.data(), p->d_w, p->Jh * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy weights");
        for (int j = 0; j < p->Jh; ++j) w[j] = w[p->J - 1 - j] = h[j];
    }
    if (mu) {
        e = cudaMemcpy(h.data(), p->d_mu, p->Jh * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy nodes");
        for (int j = 0; j < p->Jh; ++j) {
            mu[j] = h[j];
            mu[p->J - 1 - j] = -h[j];
        }
        mu[p->Jh - 1] = h[p->Jh - 1];
    }
    if (pnm) {
        e = cudaMemcpy2D(pnm, p->Jh * sizeof(double), p->d_pnm, p->ldp * sizeof(double),
                         p->Jh * sizeof(double), p->ncoef, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy P table");
    }
    return SHT_OK;
}

extern "C" int sht_profile_enable(sht_plan_t p, int on) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!p->prof) {
        p->prof = new (std::nothrow) Profiler();
        if (!p->prof) { set_error("host allocation failed"); return SHT_ERR_ALLOC; }
    }
    p->prof->on = on != 0;
    return SHT_OK;
}

extern "C" int sht_profile_read_kernels(sht_plan_t p, double* ms, long long* launches,
                                        long long* kernels) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!ms || !launches) { set_error("NULL output"); return SHT_ERR_ARG; }
    for (int k = 0; k < SHT_PROFILE_STAGES; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
        if (kernels) kernels[k] = 0;
    }
    if (!p->prof) return SHT_OK;
    DeviceGuard dg(p->device);
    int status = SHT_OK;
    for (auto& r : p->prof->recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) status = cuda_fail(e, "profile events");
        if (r.stage >= 0 && r.stage < SHT_PROFILE_STAGES) {
            ms[r.stage] += t;
            launches[r.stage] += 1;
            if (kernels) kernels[r.stage] += r.kernels;
        }
        p->prof->pool.push_back(r.a);
        p->prof->pool.push_back(r.b);
    }
    p->prof->recs.clear();
    return status;
}

extern "C" int sht_profile_read(sht_plan_t p, double* ms, long long* launches) {
    return sht_profile_read_kernels(p, ms, launches, nullptr);
}

extern "C" int sht_plan_status(sht_plan_t p) {
    int rc = check_plan(p);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise");
    const int v = split_status_read_and_clear(p);
    if (v < 0) return cuda_fail(cudaGetLastError(), "status read");
    if (v) {
        set_error("a kernel gave up on a bounded wait (status bits %d: 1 tensor-core "
                  "pipeline, 2 FFT copy)", v);
        return SHT_ERR_TIMEOUT;
    }
    return SHT_OK;
}

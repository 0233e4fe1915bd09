// Autotuner for the launch shapes of a plan: the number of fields per FFT
// CTA (the FFT's tile of latitude rows, which sets its shared memory and
// the grid) and the column-tile width of the split tensor-core GEMMs
// (TN = 128: two CTAs per SM; TN = 64: three CTAs per SM, twice the loads
// of the P~ tiles).  Neither changes any result: every output element is
// computed by the same arithmetic in the same order under each choice.
//
// sht_plan_autotune times whole inverse + forward pairs on the plan's own
// workspace and temporary buffers (zero fields: the kernels have no
// data-dependent control flow), first over the fields-per-CTA candidates,
// then over the tile widths with the best of those, and keeps the fastest.
// Choices are remembered per (device, N, J, I, nfields, precision), so
// later plans of the same shape take them without timing.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "sht_internal.h"

namespace sht {

cudaError_t split_set_tile_width(sht_plan_s* p, int tn);
int split_tile_width(const sht_plan_s* p);
cudaError_t split_set_reduced(sht_plan_s* p, int on);
cudaError_t launch_jmin(const sht_plan_s* p, int* d_out, cudaStream_t s);

namespace {

struct Choice {
    int G;
    int tn;
    float ms;
};

using Key = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<Key, Choice> g_tuned;

constexpr size_t kMaxFftSmem = 227 * 1024;

int apply_fields_per_cta(sht_plan_s* p, int G) {
    const bool fp64 = p->prec == SHT_FP64;
    if (G < 1 || G > p->F || G > 64) {
        set_error("fields per FFT CTA must be in 1..min(nfields, 64), got %d", G);
        return SHT_ERR_ARG;
    }
    const size_t smem = fft_smem_bytes(p->I, G, fp64);
    if (smem > kMaxFftSmem) {
        set_error("%d fields per FFT CTA need %zu bytes of shared memory", G, smem);
        return SHT_ERR_ARG;
    }
    p->G = G;
    p->fft_smem = smem;
    return SHT_OK;
}

int apply_tile_width(sht_plan_s* p, int tn) {
    if (p->prec == SHT_FP64) {
        set_error("FP64 plans have no tensor-core tile width");
        return SHT_ERR_UNSUPPORTED;
    }
    if (tn != 64 && tn != 128) {
        set_error("tile width must be 64 or 128, got %d", tn);
        return SHT_ERR_ARG;
    }
    const cudaError_t e = split_set_tile_width(p, tn);
    if (e != cudaSuccess) {
        set_error("tile width %d: %s", tn, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SHT_ERR_ALLOC : SHT_ERR_CUDA;
    }
    return SHT_OK;
}

struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

// Mean milliseconds of one inverse + forward pair (one untimed pair first).
int time_pair(sht_plan_s* p, void* grid, void* spec, int reps, cudaStream_t s, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        set_error("event creation failed");
        return SHT_ERR_CUDA;
    }
    int rc = SHT_OK;
    for (int r = -1; r < reps && rc == SHT_OK; ++r) {
        if (r == 0) cudaEventRecord(a, s);
        rc = sht_inverse(p, spec, grid, s);
        if (rc == SHT_OK) rc = sht_forward(p, grid, spec, s);
    }
    if (rc == SHT_OK) {
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            set_error("tuning run failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = SHT_ERR_CUDA;
        } else {
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            *ms = t / (float)reps;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

}  // namespace
}  // namespace sht

using namespace sht;

extern "C" int sht_plan_set_tuning(sht_plan_t p, int fields_per_cta, int tile_width) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    DeviceGuard dg(p->device);
    int rc = SHT_OK;
    if (fields_per_cta != 0) rc = apply_fields_per_cta(p, fields_per_cta);
    if (rc == SHT_OK && tile_width != 0) rc = apply_tile_width(p, tile_width);
    return rc;
}

extern "C" int sht_plan_get_tuning(sht_plan_t p, int* fields_per_cta, int* tile_width) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    if (fields_per_cta) *fields_per_cta = p->G;
    if (tile_width) *tile_width = split_tile_width(p);
    return SHT_OK;
}

extern "C" int sht_plan_autotune(sht_plan_t p, int reps, void* stream, int* fields_per_cta,
                                 int* tile_width, float* ms_per_pair) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    if (reps < 1 || reps > 1000) {
        set_error("reps must be in 1..1000, got %d", reps);
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp64 = p->prec == SHT_FP64;
    const Key key{p->device, p->N, p->J, p->I, p->F, p->prec};
    Choice best{p->G, split_tile_width(p), -1.f};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            best = it->second;
            cached = true;
        }
    }
    int rc = SHT_OK;
    if (!cached) {
        const size_t gbytes = (size_t)p->F * p->J * p->I * (fp64 ? 8 : 4);
        const size_t sbytes = p->ncoef * p->F * (fp64 ? 16 : 8);
        void* grid = nullptr;
        void* spec = nullptr;
        if (cudaMalloc(&grid, gbytes) != cudaSuccess || cudaMalloc(&spec, sbytes) != cudaSuccess) {
            if (grid) cudaFree(grid);
            cudaGetLastError();
            set_error("tuning buffers (%zu + %zu bytes)", gbytes, sbytes);
            return SHT_ERR_ALLOC;
        }
        cudaMemsetAsync(grid, 0, gbytes, s);
        cudaMemsetAsync(spec, 0, sbytes, s);
        static const int kG[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
        best.ms = -1.f;
        for (int G : kG) {
            if (G > p->F || fft_smem_bytes(p->I, G, fp64) > kMaxFftSmem) continue;
            float ms = 0.f;
            if ((rc = apply_fields_per_cta(p, G)) != SHT_OK) break;
            if ((rc = time_pair(p, grid, spec, reps, s, &ms)) != SHT_OK) break;
            if (best.ms < 0.f || ms < best.ms) best = Choice{G, split_tile_width(p), ms};
        }
        if (rc == SHT_OK) rc = apply_fields_per_cta(p, best.G);
        if (rc == SHT_OK && !fp64) {
            for (int tn : {128, 64}) {
                float ms = 0.f;
                if ((rc = apply_tile_width(p, tn)) != SHT_OK) break;
                if ((rc = time_pair(p, grid, spec, reps, s, &ms)) != SHT_OK) break;
                if (ms < best.ms) best = Choice{best.G, tn, ms};
            }
        }
        cudaStreamSynchronize(s);
        cudaFree(grid);
        cudaFree(spec);
        if (rc != SHT_OK) return rc;
    }
    rc = apply_fields_per_cta(p, best.G);
    if (rc == SHT_OK && !fp64) rc = apply_tile_width(p, best.tn);
    if (rc != SHT_OK) return rc;
    if (!cached) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    if (fields_per_cta) *fields_per_cta = best.G;
    if (tile_width) *tile_width = fp64 ? 0 : best.tn;
    if (ms_per_pair) *ms_per_pair = best.ms;
    return SHT_OK;
}

extern "C" int sht_plan_set_reduced(sht_plan_t p, int on) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    DeviceGuard dg(p->device);
    cudaError_t e = cudaSuccess;
    if (p->prec == SHT_FP64) {
        // the FP64 kernels read the per-problem first node from the device
        if (on && !p->d_jmin) {
            int* d = nullptr;
            e = cudaMalloc(&d, 2 * (size_t)(p->N + 1) * sizeof(int));
            if (e == cudaSuccess) e = launch_jmin(p, d, nullptr);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e == cudaSuccess)
                p->d_jmin = d;
            else if (d)
                cudaFree(d);
        } else if (!on && p->d_jmin) {
            e = cudaDeviceSynchronize();
            cudaFree(p->d_jmin);
            p->d_jmin = nullptr;
        }
    } else {
        e = split_set_reduced(p, on ? 1 : 0);
    }
    if (e != cudaSuccess) {
        set_error("reduced transform: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SHT_ERR_ALLOC : SHT_ERR_CUDA;
    }
    return SHT_OK;
}

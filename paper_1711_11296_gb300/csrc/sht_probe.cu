// Throughput probes of the FP64 and FP32 pipes (instrumentation with no
// counterpart in the paper).  The FP64 Legendre contraction and the FP32
// FFT butterflies are measured against what these kernels reach: chains of
// independent fused multiply-adds kept in registers, one resident wave of
// CTAs per SM, timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "sht_internal.h"

namespace sht {
namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop trip
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int trips, T b, T c, T* sink) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // never true for the values passed (b < 1, c > 0 keep a finite and
    // positive), but the compiler cannot drop the chains
    if (s == (T)-1) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Paired FP32 form: one fma.rn.f32x2 updates two accumulators.
__global__ void __launch_bounds__(kThreads) fma2_probe_kernel(int trips, float b, float c,
                                                              float* sink) {
    uint64_t a[kChains];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    const uint64_t bv = *reinterpret_cast<const uint64_t*>(&bb);
    const uint64_t cv = *reinterpret_cast<const uint64_t*>(&cc);
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float2 v = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
        a[k] = *reinterpret_cast<const uint64_t*>(&v);
    }
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bv), "l"(cv));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float2 v = *reinterpret_cast<const float2*>(&a[k]);
        s += v.x + v.y;
    }
    if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kind 0: DFMA, 1: FFMA, 2: paired FFMA (f32x2).  Returns ms of one launch.
cudaError_t time_probe(int kind, int trips, int blocks, void* sink, cudaStream_t s,
                       float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    cudaEventRecord(e0, s);
    if (kind == 0)
        fma_probe_kernel<double><<<blocks, kThreads, 0, s>>>(trips, 0.999999999, 1e-9,
                                                            (double*)sink);
    else if (kind == 1)
        fma_probe_kernel<float><<<blocks, kThreads, 0, s>>>(trips, 0.9999f, 1e-4f,
                                                           (float*)sink);
    else
        fma2_probe_kernel<<<blocks, kThreads, 0, s>>>(trips, 0.9999f, 1e-4f, (float*)sink);
    e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace sht

using namespace sht;

extern "C" int sht_measure_fma_peak(int kind, int reps, void* stream, double* tflops) {
    if (kind < 0 || kind > 2 || reps < 1 || reps > 100 || !tflops) {
        set_error("kind must be 0 (FP64), 1 (FP32) or 2 (paired FP32), reps 1..100, "
                  "tflops non-NULL");
        return SHT_ERR_ARG;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const void* k = kind == 0 ? (const void*)fma_probe_kernel<double>
                        : kind == 1 ? (const void*)fma_probe_kernel<float>
                                    : (const void*)fma2_probe_kernel;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
    }
    if (e != cudaSuccess) {
        set_error("probe setup: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaStream_t s = (cudaStream_t)stream;
    // the sink is written only if a chain's sum hits an impossible value;
    // the kernels never store, but a pointer must still be passed
    void* sink = nullptr;
    // calibrate the trip count to about 20 ms per launch
    int trips = kind == 0 ? 16 : 256;
    float ms = 0.f;
    for (int it = 0; it < 12; ++it) {
        e = time_probe(kind, trips, blocks, sink, s, &ms);
        if (e != cudaSuccess) break;
        if (ms >= 5.f || trips >= (1 << 24)) break;
        trips *= 4;
    }
    if (e == cudaSuccess && ms > 0.f && ms < 20.f) {
        const double scale = 20.0 / ms;
        trips = (int)(trips * scale > (1 << 26) ? (1 << 26) : trips * scale);
    }
    float best = 0.f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = time_probe(kind, trips, blocks, sink, s, &ms);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    if (e != cudaSuccess || best <= 0.f) {
        set_error("probe launch: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    const double fmas = (double)blocks * kThreads * trips * kUnroll * kChains *
                        (kind == 2 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return SHT_OK;
}

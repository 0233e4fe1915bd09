// Multigrid transfer operators on the nested Clenshaw-Curtis grids
// (Appendix C), beside the nested restriction of a fine grid to a coarse
// spectrum (Sec. 3.2, sht_restrict_nested):
//   * prolongation in spectral space: the lower-resolution spectral space is
//     a subset of the higher one, so a spectrum truncated at Nc <= N is
//     zero-padded to N and synthesised on the fine grid, or added onto it
//     (the V-cycle's correction step, fused into the inverse FFT's store);
//   * restriction in grid space by injection: the coarse grid is every 2^k-th
//     latitude (j_f = 2^k (j_c + 1) - 1, 0-based) and longitude of the fine
//     grid.
#include <cuda_runtime.h>

#include <algorithm>

#include "sht_internal.h"

namespace sht {
namespace {

// Fine spectrum row (m, n), m <= n <= N, from the coarse row when n <= Nc,
// else zero; F complex values per row.  V is double2 or float2.
template <typename V>
__global__ void zero_pad_kernel(const V* __restrict__ coarse, int Nc, V* __restrict__ fine,
                                int N, int F) {
    const int m = blockIdx.y;
    const size_t r0 = coef_offset(N, m);
    const int nrows = N - m + 1;
    const long long total = (long long)nrows * F;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int dn = (int)(e / F), f = (int)(e % F);
        const int n = m + dn;
        V v;
        v.x = 0;
        v.y = 0;
        if (m <= Nc && n <= Nc) v = coarse[(coef_offset(Nc, m) + (size_t)dn) * F + f];
        fine[(r0 + dn) * F + f] = v;
    }
}

// Coarse grid point (f, j, i) = fine grid point (f, 2^k (j+1) - 1, 2^k i).
template <typename T>
__global__ void inject_kernel(const T* __restrict__ fine, int Jf, int If, int k,
                              T* __restrict__ coarse, int J, int I, int F) {
    const long long total = (long long)F * J * I;
    const long long s = 1LL << k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % I);
        const long long fj = e / I;
        const int j = (int)(fj % J), f = (int)(fj / J);
        coarse[e] = fine[((long long)f * Jf + (s * (j + 1) - 1)) * If + s * i];
    }
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

int check(sht_plan_t p) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    return SHT_OK;
}

}  // namespace
}  // namespace sht

using namespace sht;

namespace sht {
namespace {

int prolong(sht_plan_t p, const void* coarse_spec, int Nc, void* fine_grid, void* stream,
            int accumulate) {
    int rc = check(p);
    if (rc) return rc;
    if (!coarse_spec || !fine_grid) {
        set_error("NULL buffer");
        return SHT_ERR_ARG;
    }
    if (Nc < 0 || Nc > p->N) {
        set_error("Nc = %d must be in 0..N = %d", Nc, p->N);
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    const bool fp64 = p->prec == SHT_FP64;
    const size_t vb = fp64 ? sizeof(double2) : sizeof(float2);
    if (!p->d_spec_pad) {
        const cudaError_t e = cudaMalloc(&p->d_spec_pad, p->ncoef * p->F * vb);
        if (e != cudaSuccess) {
            p->d_spec_pad = nullptr;
            cudaGetLastError();
            set_error("prolongation buffer: %s", cudaGetErrorString(e));
            return SHT_ERR_ALLOC;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid((unsigned)std::max(1, std::min(64, (p->N + 1) * p->F / 256 + 1)),
                    (unsigned)(p->N + 1));
    if (fp64)
        zero_pad_kernel<double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(coarse_spec),
                                                      Nc, static_cast<double2*>(p->d_spec_pad),
                                                      p->N, p->F);
    else
        zero_pad_kernel<float2><<<grid, 256, 0, s>>>(static_cast<const float2*>(coarse_spec), Nc,
                                                     static_cast<float2*>(p->d_spec_pad), p->N,
                                                     p->F);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("zero-padding launch: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    InvScale sc{nullptr, 1.0, accumulate};
    return inverse_scaled(p, p->d_spec_pad, sc, fine_grid, s);
}

}  // namespace
}  // namespace sht

extern "C" int sht_prolong_spectral(sht_plan_t p, const void* coarse_spec, int Nc,
                                    void* fine_grid, void* stream) {
    return prolong(p, coarse_spec, Nc, fine_grid, stream, 0);
}

extern "C" int sht_prolong_spectral_add(sht_plan_t p, const void* coarse_spec, int Nc,
                                        void* fine_grid, void* stream) {
    return prolong(p, coarse_spec, Nc, fine_grid, stream, 1);
}

extern "C" int sht_inject_nested(sht_plan_t p, const void* fine_grid, int k, void* coarse_grid,
                                 void* stream) {
    int rc = check(p);
    if (rc) return rc;
    if (!fine_grid || !coarse_grid) {
        set_error("NULL buffer");
        return SHT_ERR_ARG;
    }
    if (p->grid != SHT_GRID_CC || p->ragged) {
        set_error("the shifted (Fejer first-rule) grid and reduced grids do not nest");
        return SHT_ERR_NOT_NESTED;
    }
    if (k < 1 || k > 8) {
        set_error("k = %d must be in 1..8", k);
        return SHT_ERR_ARG;
    }
    const long long Jf = (1LL << k) * (p->J + 1) - 1, If = (1LL << k) * p->I;
    if (Jf > (1LL << 30) || If > (1LL << 30)) {
        set_error("fine grid too large");
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long total = (long long)p->F * p->J * p->I;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    if (p->prec == SHT_FP64)
        inject_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(fine_grid),
                                                     (int)Jf, (int)If, k,
                                                     static_cast<double*>(coarse_grid), p->J,
                                                     p->I, p->F);
    else
        inject_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(fine_grid),
                                                    (int)Jf, (int)If, k,
                                                    static_cast<float*>(coarse_grid), p->J,
                                                    p->I, p->F);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("injection launch: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    return SHT_OK;
}

// FP64 per-m Legendre contractions on the equatorially folded data
// (Eq. cc-quad and Eq. iLT in the parity form of Appendix B).
//
// Forward, per zonal wavenumber m and parity q (n - m = q mod 2):
//   X_n^m[c] = sum_{j < Jh} P~_n^m(mu_j) B_q[j][c]
// where B_0 = (X^m_S) w_j / I and B_1 = (X^m_A) w_j / I were written by the
// forward FFT (weights already folded in) and c runs over the 2F real
// columns (re, im of each field).
// Inverse, per m and q:
//   C_q[j][c] = sum_{n - m = q mod 2} P~_n^m(mu_j) X_n^m[c],
// the symmetric (q = 0) and antisymmetric (q = 1) halves that the inverse
// FFT unfolds into both hemispheres.
//
// One CTA computes a 32 x 64 output tile with 256 threads (4 x 2 outputs
// each) over K chunks of 16 staged in shared memory.  The tile list
// {m, q, row0, col0} is built once per plan.  On GB300 the FP64 pipe, not
// memory, bounds this kernel.
#include "sht_internal.h"

namespace sht {
namespace {

constexpr int BM = 32, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int parity_rows(int N, int m, int q) {
    const int d = N - m - q;
    return d >= 0 ? d / 2 + 1 : 0;
}

__device__ __forceinline__ size_t dcoef_offset(int N, int m) {
    return (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
}

// jmin (may be null): reduced transform (Sec. 4.1), per (m, parity) the
// first node with some |P~| >= 1e-16; the forward K loop starts at its
// K chunk, and inverse row tiles wholly before it are written as zero.
__device__ __forceinline__ void legendre_fwd_body(
    const double* __restrict__ pnm, int ldp, const double* __restrict__ work,
    double* __restrict__ spec, int4 t, int N, int Jh, int C, const int* __restrict__ jmin) {
    __shared__ double Ps[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int m = t.x, q = t.y & 1, r0 = t.z, c0 = t.w;
    const int R = parity_rows(N, m, q);
    const size_t row0 = dcoef_offset(N, m) + q;     // packed row of n = m + q
    const double* B = work + ((size_t)(2 * m + q) * Jh) * C;
    const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
    double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const int kstart = jmin ? (jmin[2 * m + q] / BK) * BK : 0;
    for (int k0 = kstart; k0 < Jh; k0 += BK) {
#pragma unroll
        for (int u = 0; u < (BM * BK) / NT; ++u) {
            const int e = tid + u * NT;
            const int rr = e / BK, kk = e % BK;
            const int r = r0 + rr, k = k0 + kk;
            Ps[kk][rr] = (r < R && k < Jh) ? pnm[(row0 + 2 * (size_t)r) * ldp + k] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < (BK * BN) / NT; ++u) {
            const int e = tid + u * NT;
            const int kk = e / BN, cc = e % BN;
            const int k = k0 + kk, c = c0 + cc;
            Bs[kk][cc] = (k < Jh && c < C) ? B[(size_t)k * C + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ps[kk][ty * 4 + i];
            b[0] = Bs[kk][tx];
            b[1] = Bs[kk][tx + 32];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fma(a[i], b[0], acc[i][0]);
                acc[i][1] = fma(a[i], b[1], acc[i][1]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= R) continue;
        double* out = spec + (row0 + 2 * (size_t)r) * C;
        if (c0 + tx < C) out[c0 + tx] = acc[i][0];
        if (c0 + tx + 32 < C) out[c0 + tx + 32] = acc[i][1];
    }
}

__device__ __forceinline__ void legendre_inv_body(
    const double* __restrict__ pnm, int ldp, const double* __restrict__ spec,
    double* __restrict__ work, int4 t, int N, int Jh, int C, const int* __restrict__ jmin) {
    __shared__ double Ps[BK][BM];
    __shared__ double Bs[BK][BN];
    const int m = t.x, q = t.y & 1, j0 = t.z, c0 = t.w;
    const int R = parity_rows(N, m, q);
    const size_t row0 = dcoef_offset(N, m) + q;
    const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
    double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    // (block-uniform: the loop holds barriers)
    const int kend = (jmin && j0 + BM <= jmin[2 * m + q]) ? 0 : R;
    for (int k0 = 0; k0 < kend; k0 += BK) {
#pragma unroll
        for (int u = 0; u < (BM * BK) / NT; ++u) {
            const int e = tid + u * NT;
            const int kk = e / BM, jj = e % BM;
            const int r = k0 + kk, j = j0 + jj;
            Ps[kk][jj] = (r < R && j < Jh) ? pnm[(row0 + 2 * (size_t)r) * ldp + j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < (BK * BN) / NT; ++u) {
            const int e = tid + u * NT;
            const int kk = e / BN, cc = e % BN;
            const int r = k0 + kk, c = c0 + cc;
            Bs[kk][cc] = (r < R && c < C) ? spec[(row0 + 2 * (size_t)r) * C + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ps[kk][ty * 4 + i];
            b[0] = Bs[kk][tx];
            b[1] = Bs[kk][tx + 32];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fma(a[i], b[0], acc[i][0]);
                acc[i][1] = fma(a[i], b[1], acc[i][1]);
            }
        }
        __syncthreads();
    }
    double* W = work + ((size_t)(2 * m + q) * Jh) * C;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int j = j0 + ty * 4 + i;
        if (j >= Jh) continue;
        if (c0 + tx < C) W[(size_t)j * C + c0 + tx] = acc[i][0];
        if (c0 + tx + 32 < C) W[(size_t)j * C + c0 + tx + 32] = acc[i][1];
    }
}

__global__ void __launch_bounds__(NT) legendre_fwd_fp64_kernel(
    const double* __restrict__ pnm, int ldp, const double* __restrict__ work,
    double* __restrict__ spec, const int4* __restrict__ tiles, int N, int Jh, int C,
    const int* __restrict__ jmin) {
    legendre_fwd_body(pnm, ldp, work, spec, tiles[blockIdx.x], N, Jh, C, jmin);
}

__global__ void __launch_bounds__(NT) legendre_inv_fp64_kernel(
    const double* __restrict__ pnm, int ldp, const double* __restrict__ spec,
    double* __restrict__ work, const int4* __restrict__ tiles, int N, int Jh, int C,
    const int* __restrict__ jmin) {
    legendre_inv_body(pnm, ldp, spec, work, tiles[blockIdx.x], N, Jh, C, jmin);
}

// Grouped launches: tile.y = parity + 2 * (plan index in the group).
struct LegGroup {
    int n;
    const double* pnm[kMaxGroup];
    const double* in[kMaxGroup];
    double* out[kMaxGroup];
    int ldp[kMaxGroup], N[kMaxGroup], Jh[kMaxGroup], C[kMaxGroup];
    const int* jmin[kMaxGroup];
};

__global__ void __launch_bounds__(NT) legendre_fwd_fp64_group_kernel(
    const __grid_constant__ LegGroup G, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const int p = t.y >> 1;
    legendre_fwd_body(G.pnm[p], G.ldp[p], G.in[p], G.out[p], t, G.N[p], G.Jh[p], G.C[p],
                      G.jmin[p]);
}

__global__ void __launch_bounds__(NT) legendre_inv_fp64_group_kernel(
    const __grid_constant__ LegGroup G, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const int p = t.y >> 1;
    legendre_inv_body(G.pnm[p], G.ldp[p], G.in[p], G.out[p], t, G.N[p], G.Jh[p], G.C[p],
                      G.jmin[p]);
}

}  // namespace

cudaError_t launch_legendre_fp64_group(sht_plan_s* const* plans, int n, bool inverse,
                                       const void* const* in, void* const* out,
                                       const int4* tiles, int ntiles, cudaStream_t s) {
    LegGroup G;
    G.n = n;
    for (int q = 0; q < n; ++q) {
        G.pnm[q] = plans[q]->d_pnm;
        G.ldp[q] = plans[q]->ldp;
        G.N[q] = plans[q]->N;
        G.Jh[q] = plans[q]->Jh;
        G.C[q] = 2 * plans[q]->F;
        G.in[q] = static_cast<const double*>(in[q]);
        G.out[q] = static_cast<double*>(out[q]);
        G.jmin[q] = plans[q]->d_jmin;
    }
    if (ntiles == 0) return cudaSuccess;
    if (inverse)
        legendre_inv_fp64_group_kernel<<<ntiles, NT, 0, s>>>(G, tiles);
    else
        legendre_fwd_fp64_group_kernel<<<ntiles, NT, 0, s>>>(G, tiles);
    note_launch();
    return cudaGetLastError();
}

// Tile lists (host): forward tiles cover the parity rows of each (m, q);
// inverse tiles cover the Jh northern rows of each (m, q), including the
// empty parity (m = N, q = 1), whose output must still be written as zero.
void build_legendre_tiles(int N, int Jh, int C, std::vector<int4>& fwd,
                          std::vector<int4>& inv) {
    fwd.clear();
    inv.clear();
    for (int m = 0; m <= N; ++m) {
        for (int q = 0; q < 2; ++q) {
            const int d = N - m - q;
            const int R = d >= 0 ? d / 2 + 1 : 0;
            for (int r0 = 0; r0 < R; r0 += BM)
                for (int c0 = 0; c0 < C; c0 += BN) fwd.push_back(make_int4(m, q, r0, c0));
            for (int j0 = 0; j0 < Jh; j0 += BM)
                for (int c0 = 0; c0 < C; c0 += BN) inv.push_back(make_int4(m, q, j0, c0));
        }
    }
}

cudaError_t launch_legendre_fwd_fp64(const sht_plan_s* p, const double* work,
                                     double* spec, cudaStream_t s) {
    if (p->ntiles_fwd == 0) return cudaSuccess;
    legendre_fwd_fp64_kernel<<<p->ntiles_fwd, NT, 0, s>>>(
        p->d_pnm, p->ldp, work, spec, p->d_tiles_fwd, p->N, p->Jh, 2 * p->F, p->d_jmin);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_legendre_inv_fp64(const sht_plan_s* p, const double* spec,
                                     double* work, cudaStream_t s) {
    if (p->ntiles_inv == 0) return cudaSuccess;
    legendre_inv_fp64_kernel<<<p->ntiles_inv, NT, 0, s>>>(
        p->d_pnm, p->ldp, spec, work, p->d_tiles_inv, p->N, p->Jh, 2 * p->F, p->d_jmin);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sht

namespace sht {
namespace {

// One thread per zonal wavenumber m: its tiles start after those of all
// m' < m (same order and geometry as build_legendre_tiles).
__global__ void fwd_tiles_kernel(int N, int C, int4* tiles) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > N) return;
    const int nct = (C + BN - 1) / BN;
    auto rows = [&](int mm, int q) {
        const int d = N - mm - q;
        return d >= 0 ? d / 2 + 1 : 0;
    };
    long long off = 0;
    for (int mm = 0; mm < m; ++mm)
        off += (long long)((rows(mm, 0) + BM - 1) / BM + (rows(mm, 1) + BM - 1) / BM) * nct;
    for (int q = 0; q < 2; ++q) {
        const int R = rows(m, q);
        for (int r0 = 0; r0 < R; r0 += BM)
            for (int c0 = 0; c0 < C; c0 += BN) tiles[off++] = make_int4(m, q, r0, c0);
    }
}

}  // namespace

// Number of forward Legendre tiles for truncation N and C real columns.
int legendre_fwd_tile_count(int N, int C) {
    long long n = 0;
    const int nct = (C + BN - 1) / BN;
    for (int m = 0; m <= N; ++m)
        for (int q = 0; q < 2; ++q) {
            const int d = N - m - q;
            const int R = d >= 0 ? d / 2 + 1 : 0;
            n += (long long)((R + BM - 1) / BM) * nct;
        }
    return (int)n;
}

// Build the forward tile list on the device (no host memory involved).
cudaError_t launch_build_fwd_tiles(int N, int C, int4* tiles, cudaStream_t s) {
    const int threads = 128;
    fwd_tiles_kernel<<<(N + 1 + threads - 1) / threads, threads, 0, s>>>(N, C, tiles);
    return cudaGetLastError();
}

}  // namespace sht

// Reduced Clenshaw-Curtis grids: the Clenshaw-Curtis latitudes with a
// longitude count I_j of their own on each latitude, as in the reduced and
// octahedral grids Sec. 6 proposes for the Clenshaw-Curtis nodes.
//
// Sec. 6 quotes the reduction rule of the JMA model: latitude j needs at
// least 4 M_j + 1 longitudes, M_j being the zonal wavenumber beyond which
// every |P~_n^m(mu_j)| is below 1e-16.  sht_reduced_grid_sizes applies it
// to a plan's P~ table: M_j = the largest m with some |P~_n^m(mu_j)| >=
// 1e-16, and I_j = the smallest even count >= 4 M_j + 1 whose half has no
// prime factor above 5 (SHT_REDUCED_SMOOTH), or whose half is one of the
// lengths with a compile-time FFT kernel (SHT_REDUCED_FAST: fewer distinct
// lengths, a few more points), capped at the plan's I.
//
// Octahedral and icositetrahedral counts (sht_octahedral_grid_sizes,
// sht_icositetrahedral_grid_sizes) have half-lengths with prime factors
// above 5; their rows are transformed by Bluestein's chirp-z method (the
// DFT of length L as a circular convolution of length L2 >= 2L - 1 with
// 2-3-5-smooth L2, evaluated by two FFTs of length L2).  The tropical rows
// of the icositetrahedral grid sit half a spacing east of the meridian,
// lambda_i = 2 pi (i + 1/2) / I_j: their zonal transforms carry the phase
// e^{-i m pi / I_j} (forward) and its conjugate (inverse).
//
// A reduced plan is a Clenshaw-Curtis plan of I >= max I_j whose FFT kernels
// take, per latitude pair, the half-length L_j = I_j/2 and its tables.  Row
// j of a field holds I_j points, rows packed one after another.  The
// forward FFT of row j keeps the wavenumbers m <= min(N, L_j - 1) (the
// Nyquist wavenumber L_j is not a mode of a real row) and writes zeros
// above; the inverse synthesises the same range.  The weights of the
// forward quadrature become w_j / I_j.  The Legendre contractions are those
// of the full grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "sht_internal.h"

namespace sht {
namespace {

// M_j for every northern node: thread per node, block row per m; a node
// takes m if some n of that m is significant there.
__global__ void latitude_mmax_kernel(const double* __restrict__ pnm, int ldp, int N, int Jh,
                                     double thr, int* __restrict__ mmax) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (j >= Jh) return;
    const size_t row0 = coef_offset(N, m);
    bool sig = false;
    for (int n = m; n <= N && !sig; ++n) sig = fabs(pnm[(row0 + (n - m)) * (size_t)ldp + j]) >= thr;
    if (sig) atomicMax(&mmax[j], m);
}

bool smooth_half(int n) {
    if (n < 2 || n % 2 != 0) return false;
    int h = n / 2;
    for (int p : {2, 3, 5})
        while (h % p == 0) h /= p;
    return h == 1;
}

int even_smooth_ceil(int x) {
    int n = std::max(2, x);
    while (!smooth_half(n)) ++n;
    return n;
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

}  // namespace

void ragged_free(RaggedGrid* rg) {
    if (!rg) return;
    void* ptrs[] = {rg->d_rowoff, rg->d_shape_of, rg->d_shift_of, rg->d_shapes,
                    rg->d_twpass,  rg->d_twpost,   rg->d_rev,      rg->d_chirp,
                    rg->d_dft,     rg->d_shiftph,  rg->d_jh};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete rg;
}

namespace {

// The smallest length >= n whose FFT factors into radices 2, 3, 4, 5 and 8
// (the run-time kernels' radices): the Bluestein convolution length.
int small_radix_ceil(int n) {
    for (int m = std::max(n, 1);; ++m)
        if (fft_factorable(m)) return m;
}

// How a latitude pair's rows are transformed.
enum Route { kRouteClass = 0, kRouteGeneric = 1, kRouteBluestein = 2 };

// Per-latitude tables of a reduced plan (I_lat and shift already checked;
// shift may be null).
int attach_ragged(sht_plan_s* p, const int* I_lat, const int* shift) {
    const bool fp64 = p->prec == SHT_FP64;
    const size_t vb = fp64 ? sizeof(double2) : sizeof(float2);
    RaggedGrid* rg = new (std::nothrow) RaggedGrid();
    if (!rg) {
        set_error("host allocation failed");
        return SHT_ERR_ALLOC;
    }
    rg->Ij.assign(I_lat, I_lat + p->J);
    std::vector<long long> rowoff(p->J);
    long long acc = 0;
    for (int j = 0; j < p->J; ++j) {
        rowoff[j] = acc;
        acc += rg->Ij[j];
    }
    rg->npts = acc;
    // Distinct (half-length, route) pairs, in order of first appearance from
    // the pole.  Unshifted rows whose half-length has a compile-time kernel
    // go to that kernel; other 2-3-5-smooth rows to the generic kernel with
    // radices up to 8; the rest to the Bluestein kernel.
    std::map<std::pair<int, int>, int> id;
    std::vector<RShape> shapes;
    std::vector<int> shape_of(p->Jh), shift_of(p->Jh), route_of;
    long long tw_total = 0, post_total = 0, rev_total = 0, chirp_total = 0, dft_total = 0,
              shift_total = 0;
    int Lmax = 1, L2max = 1;
    for (int jh = 0; jh < p->Jh; ++jh) {
        const int L = rg->Ij[jh] / 2;
        const int sh = shift ? shift[jh] : 0;
        shift_of[jh] = sh;
        const int route = !fft_factorable(L) ? kRouteBluestein
                          : (fft_has_fixed_kernel(L) && !sh) ? kRouteClass
                                                               : kRouteGeneric;
        auto it = id.find({L, route});
        if (it == id.end()) {
            RShape r;
            r.L = L;
            if (route == kRouteBluestein) {
                r.bluestein = 1;
                r.sh = fft_factor(small_radix_ceil(2 * L - 1), true);
                r.chirp_off = chirp_total;
                r.dft_off = dft_total;
                chirp_total += L;
                dft_total += r.sh.L;
                L2max = std::max(L2max, r.sh.L);
            } else {
                r.sh = fft_factor(L, route == kRouteClass ? fp64 : true);
            }
            r.tw_off = tw_total;
            r.post_off = post_total;
            r.rev_off = rev_total;
            tw_total += std::max(r.sh.twtotal, 1);
            post_total += L;
            rev_total += r.sh.L;
            it = id.emplace(std::make_pair(L, route), (int)shapes.size()).first;
            shapes.push_back(r);
            route_of.push_back(route);
            Lmax = std::max(Lmax, L);
        }
        shape_of[jh] = it->second;
        if (sh && shapes[it->second].shift_off < 0) {
            shapes[it->second].shift_off = shift_total;
            shift_total += L;
        }
        rg->any_shift = rg->any_shift || sh;
    }
    rg->nshapes = (int)shapes.size();
    rg->h_shapes = shapes;
    // launch lists: latitude pairs of each compile-time length, then the
    // generic ones, then the Bluestein ones
    std::vector<int> jh_all;
    for (int k = 0; k < rg->nshapes; ++k) {
        if (route_of[k] != kRouteClass) continue;
        RaggedGrid::Class c{k, (int)jh_all.size(), 0};
        for (int jh = 0; jh < p->Jh; ++jh)
            if (shape_of[jh] == k) jh_all.push_back(jh);
        c.count = (int)jh_all.size() - c.off;
        rg->classes.push_back(c);
    }
    rg->generic_off = (int)jh_all.size();
    for (int jh = 0; jh < p->Jh; ++jh)
        if (route_of[shape_of[jh]] == kRouteGeneric) jh_all.push_back(jh);
    rg->generic_count = (int)jh_all.size() - rg->generic_off;
    rg->blue_off = (int)jh_all.size();
    for (int jh = 0; jh < p->Jh; ++jh)
        if (route_of[shape_of[jh]] == kRouteBluestein) jh_all.push_back(jh);
    rg->blue_count = (int)jh_all.size() - rg->blue_off;
    if (rg->blue_count > 0) {
        // fields per CTA of the Bluestein launch: as many as fit (rows at
        // the pitch of the plan's own half-length, which the kernels use)
        const int Lrow = std::max(Lmax, p->fft.L);
        int G = std::min(1, p->F);
        while (G > 1 && bluestein_smem_bytes(Lrow, L2max, G, fp64) > 227 * 1024) --G;
        rg->blue_G = G;
        rg->blue_smem = bluestein_smem_bytes(Lrow, L2max, G, fp64);
        if (rg->blue_smem > 227 * 1024) {
            delete rg;
            set_error("rows of %d longitudes are too long for the Bluestein FFT", 2 * Lmax);
            return SHT_ERR_UNSUPPORTED;
        }
    }
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(q, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) *q = nullptr;
    };
    alloc((void**)&rg->d_rowoff, p->J * sizeof(long long));
    alloc((void**)&rg->d_shape_of, p->Jh * sizeof(int));
    alloc((void**)&rg->d_shift_of, p->Jh * sizeof(int));
    alloc((void**)&rg->d_shapes, shapes.size() * sizeof(RShape));
    alloc(&rg->d_twpass, tw_total * vb);
    alloc(&rg->d_twpost, post_total * vb);
    alloc((void**)&rg->d_rev, rev_total * sizeof(int));
    alloc(&rg->d_chirp, chirp_total * vb);
    alloc(&rg->d_dft, dft_total * vb);
    alloc(&rg->d_shiftph, shift_total * vb);
    alloc((void**)&rg->d_jh, jh_all.size() * sizeof(int));
    alloc(&tmp, 64 * (size_t)std::max(Lmax, L2max));
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (size_t k = 0; k < shapes.size() && e == cudaSuccess; ++k) {
        const RShape& r = shapes[k];
        char* tw = static_cast<char*>(rg->d_twpass) + r.tw_off * vb;
        char* post = static_cast<char*>(rg->d_twpost) + r.post_off * vb;
        if (r.bluestein)
            e = build_bluestein_tables(r.L, r.sh, fp64, tw, post, rg->d_rev + r.rev_off,
                                       static_cast<char*>(rg->d_chirp) + r.chirp_off * vb,
                                       static_cast<char*>(rg->d_dft) + r.dft_off * vb, tmp, s);
        else
            e = build_fft_tables(r.sh, fp64, tw, post, rg->d_rev + r.rev_off, tmp, s);
        if (e == cudaSuccess && r.shift_off >= 0)
            e = build_shift_table(r.L, 2 * r.L, fp64,
                                  static_cast<char*>(rg->d_shiftph) + r.shift_off * vb, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rg->d_rowoff, rowoff.data(), p->J * sizeof(long long),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rg->d_shape_of, shape_of.data(), p->Jh * sizeof(int),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rg->d_shift_of, shift_of.data(), p->Jh * sizeof(int),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rg->d_shapes, shapes.data(), shapes.size() * sizeof(RShape),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rg->d_jh, jh_all.data(), jh_all.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s);
    // forward weights w_j / I_j (the discretised Eq. dFT of row j carries 1/I_j)
    std::vector<double> w(p->Jh);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.data(), p->d_w, p->Jh * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        for (int jh = 0; jh < p->Jh; ++jh) w[jh] /= (double)rg->Ij[jh];
        e = cudaMemcpyAsync(p->d_w_over_I, w.data(), p->Jh * sizeof(double),
                            cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        ragged_free(rg);
        cudaGetLastError();
        set_error("reduced-grid tables: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SHT_ERR_ALLOC : SHT_ERR_CUDA;
    }
    p->ragged = rg;
    return SHT_OK;
}

int create_reduced(int N, int J, const int* I_lat, const int* shift, int nfields,
                   int precision, sht_plan_t* out) {
    if (!out) {
        set_error("out is NULL");
        return SHT_ERR_ARG;
    }
    *out = nullptr;
    if (!I_lat) {
        set_error("I_lat is NULL");
        return SHT_ERR_ARG;
    }
    if (J < 1 || J % 2 == 0) {
        set_error("J = %d must be odd and >= 1 (the Equator node is needed)", J);
        return SHT_ERR_ARG;
    }
    int Imax = 0;
    for (int j = 0; j < J; ++j) {
        const int n = I_lat[j];
        if (n < 2 || n > kMaxI || n % 2 != 0) {
            set_error("I_lat[%d] = %d must be even and in 2..%d", j, n, kMaxI);
            return SHT_ERR_ARG;
        }
        if (n != I_lat[J - 1 - j]) {
            set_error("I_lat must be symmetric about the Equator (I_lat[%d] = %d, I_lat[%d] = %d)",
                      j, n, J - 1 - j, I_lat[J - 1 - j]);
            return SHT_ERR_ARG;
        }
        if (shift && ((shift[j] != 0 && shift[j] != 1) || shift[j] != shift[J - 1 - j])) {
            set_error("half_shift[%d] = %d must be 0 or 1 and symmetric about the Equator",
                      j, shift[j]);
            return SHT_ERR_ARG;
        }
        Imax = std::max(Imax, n);
    }
    if (Imax <= 2 * N) {
        set_error("the longest row (%d longitudes) must exceed 2N = %d", Imax, 2 * N);
        return SHT_ERR_ARG;
    }
    // the plan's own grid: the smallest 2-3-5-smooth count >= the longest
    // row (its tables size the shared memory of the per-row kernels)
    const int Ibase = even_smooth_ceil(Imax);
    if (Ibase > kMaxI) {
        set_error("rows of %d longitudes exceed the FFT limit", Imax);
        return SHT_ERR_ARG;
    }
    sht_plan_t p = nullptr;
    const int rc = sht_plan_create_grid(N, J, Ibase, nfields, precision, SHT_GRID_CC, &p);
    if (rc < 0) return rc;
    int rc2;
    {
        DeviceGuard dg(p->device);
        rc2 = attach_ragged(p, I_lat, shift);
    }
    if (rc2 != SHT_OK) {
        sht_plan_destroy(p);
        return rc2;
    }
    *out = p;
    return rc;
}

}  // namespace
}  // namespace sht

using namespace sht;

extern "C" int sht_reduced_grid_sizes(sht_plan_t p, int rule, int* I_lat) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    if (!I_lat) {
        set_error("I_lat is NULL");
        return SHT_ERR_ARG;
    }
    if (rule != SHT_REDUCED_SMOOTH && rule != SHT_REDUCED_FAST) {
        set_error("unknown reduction rule %d", rule);
        return SHT_ERR_ARG;
    }
    DeviceGuard dg(p->device);
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, p->Jh * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, p->Jh * sizeof(int));
    if (e == cudaSuccess) {
        const dim3 grid((p->Jh + 127) / 128, p->N + 1);
        latitude_mmax_kernel<<<grid, 128>>>(p->d_pnm, p->ldp, p->N, p->Jh, 1e-16, d);
        e = cudaGetLastError();
    }
    std::vector<int> mmax(p->Jh, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(mmax.data(), d, p->Jh * sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("reduced-grid sizes: %s", cudaGetErrorString(e));
        return SHT_ERR_CUDA;
    }
    for (int jh = 0; jh < p->Jh; ++jh) {
        const int need = 4 * mmax[jh] + 1;
        int n = even_smooth_ceil(need);
        if (rule == SHT_REDUCED_FAST) {
            n = p->I;
            for (int L : {64, 128, 256, 320, 512, 640, 1024, 1280})
                if (2 * L >= need) {
                    n = 2 * L;
                    break;
                }
        }
        n = std::min(p->I, n);
        I_lat[jh] = n;
        I_lat[p->J - 1 - jh] = n;
    }
    return SHT_OK;
}

extern "C" int sht_plan_create_reduced(int N, int J, const int* I_lat, int nfields,
                                       int precision, sht_plan_t* out) {
    clear_error();
    return create_reduced(N, J, I_lat, nullptr, nfields, precision, out);
}

extern "C" int sht_plan_create_reduced_shifted(int N, int J, const int* I_lat,
                                               const int* half_shift, int nfields,
                                               int precision, sht_plan_t* out) {
    clear_error();
    if (!half_shift) {
        set_error("half_shift is NULL");
        return SHT_ERR_ARG;
    }
    return create_reduced(N, J, I_lat, half_shift, nfields, precision, out);
}

extern "C" int sht_octahedral_grid_sizes(int J, int first, int step, int* I_lat) {
    clear_error();
    if (J < 1 || J % 2 == 0 || !I_lat || first < 2 || first % 2 != 0 || step < 0 ||
        step % 2 != 0) {
        set_error("J odd >= 1, first even >= 2, step even >= 0 and a non-NULL I_lat");
        return SHT_ERR_ARG;
    }
    const int Jh = (J + 1) / 2;
    if ((long long)first + (long long)step * (Jh - 1) > kMaxI) {
        set_error("the Equator row would exceed %d longitudes", kMaxI);
        return SHT_ERR_ARG;
    }
    for (int j = 0; j < Jh; ++j) {
        I_lat[j] = first + step * j;
        I_lat[J - 1 - j] = I_lat[j];
    }
    return SHT_OK;
}

extern "C" int sht_icositetrahedral_grid_sizes(int J, int* I_lat, int* half_shift) {
    clear_error();
    if (J < 1 || J % 2 == 0 || !I_lat || !half_shift) {
        set_error("J odd >= 1 and non-NULL I_lat and half_shift");
        return SHT_ERR_ARG;
    }
    const int Jh = (J + 1) / 2;
    const int j30 = std::max(1, (int)((J + 1) / 3.0 + 0.5));
    if (6LL * std::min(j30, Jh) > kMaxI) {
        set_error("the tropical rows would exceed %d longitudes", kMaxI);
        return SHT_ERR_ARG;
    }
    for (int j = 1; j <= Jh; ++j) {
        I_lat[j - 1] = 6 * std::min(j, j30);
        half_shift[j - 1] = j > j30 ? (j - j30) % 2 : 0;
        I_lat[J - j] = I_lat[j - 1];
        half_shift[J - j] = half_shift[j - 1];
    }
    return SHT_OK;
}

extern "C" int sht_plan_grid_points(sht_plan_t p, long long* npts) {
    if (!p || !plan_is_live(p)) {
        set_error("invalid or destroyed plan handle");
        return SHT_ERR_HANDLE;
    }
    if (!npts) {
        set_error("npts is NULL");
        return SHT_ERR_ARG;
    }
    *npts = p->ragged ? p->ragged->npts : (long long)p->J * p->I;
    return SHT_OK;
}

// Grouped execution of several plans: one launch per kernel stage covers
// every plan of the group (uneven truncations, ensemble members, levels),
// so a whole batch costs four launches per transform pair and can be
// captured in one CUDA graph.  The per-plan kernel bodies are the ones the
// single-plan entry points use; the group kernels only map their block
// index to (plan, tile) through per-plan argument blocks.  Legendre tiles
// of all plans are sorted by their K-loop length, longest first, so the
// uneven per-m row counts balance over the SMs.
#include <algorithm>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "sht_internal.h"

namespace sht {

void build_legendre_tiles(int N, int Jh, int C, std::vector<int4>& fwd,
                          std::vector<int4>& inv);
cudaError_t launch_legendre_fp64_group(sht_plan_s* const* plans, int n, bool inverse,
                                       const void* const* in, void* const* out,
                                       const int4* tiles, int ntiles, cudaStream_t s);
void split_group_tiles(sht_plan_s* const* plans, int n, bool inverse, std::vector<int4>& out);
cudaError_t launch_split_group(sht_plan_s* const* plans, int n, bool inverse,
                               const void* const* in, void* const* out, const int4* tiles,
                               int ntiles, cudaStream_t s);

int split_tile_width(const sht_plan_s* p);

constexpr uint64_t kGroupMagic = 0x53485447'524F5550ull;   // "SHTGROUP"

}  // namespace sht

struct sht_group_s {
    uint64_t magic;
    int n;
    int prec;
    int device;
    sht_plan_s* plans[sht::kMaxGroup];
    int tile_width;   // split plans: the GEMM tile width the tile lists were built for
    int4* d_tiles_fwd;
    int ntiles_fwd;
    int4* d_tiles_inv;
    int ntiles_inv;
};

namespace sht {
namespace {

std::mutex g_group_mu;
std::set<const sht_group_s*> g_groups;

bool group_live(const sht_group_s* g) {
    std::lock_guard<std::mutex> lk(g_group_mu);
    return g && g_groups.count(g) && g->magic == kGroupMagic;
}

int fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SHT_ERR_CUDA;
}

// FP64 tiles of all plans; tile.y = parity + 2 * plan.  Forward tiles run
// over the plan's Jh nodes, inverse tiles over the parity's row count.
void fp64_group_tiles(sht_plan_s* const* plans, int n, bool inverse, std::vector<int4>& out) {
    std::vector<std::pair<int, int4>> all;
    for (int q = 0; q < n; ++q) {
        const sht_plan_s* p = plans[q];
        std::vector<int4> tf, ti;
        build_legendre_tiles(p->N, p->Jh, 2 * p->F, tf, ti);
        for (int4 t : inverse ? ti : tf) {
            const int d = p->N - t.x - t.y;
            const int R = d >= 0 ? d / 2 + 1 : 0;
            const int cost = inverse ? R : p->Jh;
            t.y += 2 * q;
            all.push_back({cost, t});
        }
    }
    std::stable_sort(all.begin(), all.end(),
                     [](const std::pair<int, int4>& a, const std::pair<int, int4>& b) {
                         return a.first > b.first;
                     });
    out.clear();
    for (auto& e : all) out.push_back(e.second);
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
}  // namespace sht

using namespace sht;

extern "C" int sht_group_create(const sht_plan_t* plans, int nplans, sht_group_t* out) {
    if (!plans || !out || nplans < 1 || nplans > kMaxGroup) {
        set_error("need 1..%d plans and an output handle", kMaxGroup);
        return SHT_ERR_ARG;
    }
    for (int q = 0; q < nplans; ++q) {
        if (!plans[q] || !plan_is_live(plans[q])) {
            set_error("plan %d is invalid or destroyed", q);
            return SHT_ERR_HANDLE;
        }
        if (plans[q]->ragged) {
            set_error("plan %d has a reduced grid; grouped launches take regular grids", q);
            return SHT_ERR_UNSUPPORTED;
        }
        if (plans[q]->prec != plans[0]->prec || plans[q]->device != plans[0]->device) {
            set_error("plans of a group must share precision and device");
            return SHT_ERR_ARG;
        }
        for (int r = 0; r < q; ++r)
            if (plans[r] == plans[q]) {
                set_error("plan %d appears twice (its workspace cannot be shared)", q);
                return SHT_ERR_ARG;
            }
        if (split_tile_width(plans[q]) != split_tile_width(plans[0])) {
            set_error("plans of a group must share the GEMM tile width");
            return SHT_ERR_ARG;
        }
    }
    sht_group_s* g = new (std::nothrow) sht_group_s();
    if (!g) {
        set_error("host allocation failed");
        return SHT_ERR_ALLOC;
    }
    g->n = nplans;
    g->prec = plans[0]->prec;
    g->device = plans[0]->device;
    g->tile_width = split_tile_width(plans[0]);
    for (int q = 0; q < nplans; ++q) g->plans[q] = plans[q];
    std::vector<int4> tf, ti;
    if (g->prec == SHT_FP64) {
        fp64_group_tiles(g->plans, nplans, false, tf);
        fp64_group_tiles(g->plans, nplans, true, ti);
    } else {
        split_group_tiles(g->plans, nplans, false, tf);
        split_group_tiles(g->plans, nplans, true, ti);
    }
    g->ntiles_fwd = (int)tf.size();
    g->ntiles_inv = (int)ti.size();
    DeviceGuard dg(g->device);
    cudaError_t e = cudaMalloc(&g->d_tiles_fwd, (tf.size() + 1) * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_tiles_inv, (ti.size() + 1) * sizeof(int4));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_tiles_fwd, tf.data(), tf.size() * sizeof(int4),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_tiles_inv, ti.data(), ti.size() * sizeof(int4),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (g->d_tiles_fwd) cudaFree(g->d_tiles_fwd);
        if (g->d_tiles_inv) cudaFree(g->d_tiles_inv);
        delete g;
        set_error("group tiles: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SHT_ERR_ALLOC : SHT_ERR_CUDA;
    }
    g->magic = kGroupMagic;
    {
        std::lock_guard<std::mutex> lk(g_group_mu);
        g_groups.insert(g);
    }
    *out = g;
    return SHT_OK;
}

extern "C" int sht_group_destroy(sht_group_t g) {
    if (!g) return SHT_OK;
    {
        std::lock_guard<std::mutex> lk(g_group_mu);
        if (!g_groups.count(g)) {
            set_error("invalid or destroyed group handle");
            return SHT_ERR_HANDLE;
        }
        g_groups.erase(g);
    }
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->d_tiles_fwd);
    cudaFree(g->d_tiles_inv);
    g->magic = 0;
    delete g;
    return SHT_OK;
}

namespace {

int check_group(sht_group_t g, const void* const* a, const void* const* b) {
    if (!group_live(g)) {
        set_error("invalid or destroyed group handle");
        return SHT_ERR_HANDLE;
    }
    for (int q = 0; q < g->n; ++q) {
        if (!plan_is_live(g->plans[q])) {
            set_error("plan %d of the group was destroyed", q);
            return SHT_ERR_HANDLE;
        }
        if (split_tile_width(g->plans[q]) != g->tile_width) {
            set_error("plan %d changed its GEMM tile width after the group was created", q);
            return SHT_ERR_ARG;
        }
    }
    if (!a || !b) {
        set_error("NULL buffer array");
        return SHT_ERR_ARG;
    }
    for (int q = 0; q < g->n; ++q)
        if (!a[q] || !b[q]) {
            set_error("NULL buffer for plan %d", q);
            return SHT_ERR_ARG;
        }
    return SHT_OK;
}

}  // namespace

extern "C" int sht_group_forward(sht_group_t g, const void* const* grids, void* const* specs,
                                 void* stream) {
    int rc = check_group(g, grids, (const void* const*)specs);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    {
        ProfScope ps(g->plans[0], kStageFftFwd, s);
        e = launch_fft_forward_group(g->plans, g->n, grids, s);
    }
    if (e != cudaSuccess) return fail(e, "grouped forward FFT launch");
    const void* works[kMaxGroup];
    for (int q = 0; q < g->n; ++q) works[q] = g->plans[q]->d_work;
    {
        ProfScope ps(g->plans[0], kStageLegFwd, s);
        if (g->prec == SHT_FP64)
            e = launch_legendre_fp64_group(g->plans, g->n, false, works, specs,
                                           g->d_tiles_fwd, g->ntiles_fwd, s);
        else
            e = launch_split_group(g->plans, g->n, false, works, specs, g->d_tiles_fwd,
                                   g->ntiles_fwd, s);
    }
    if (e != cudaSuccess) return fail(e, "grouped forward Legendre launch");
    return SHT_OK;
}

extern "C" int sht_group_inverse(sht_group_t g, const void* const* specs, void* const* grids,
                                 void* stream) {
    int rc = check_group(g, specs, (const void* const*)grids);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    void* works[kMaxGroup];
    for (int q = 0; q < g->n; ++q) works[q] = g->plans[q]->d_work;
    cudaError_t e;
    {
        ProfScope ps(g->plans[0], kStageLegInv, s);
        if (g->prec == SHT_FP64)
            e = launch_legendre_fp64_group(g->plans, g->n, true, specs, works, g->d_tiles_inv,
                                           g->ntiles_inv, s);
        else
            e = launch_split_group(g->plans, g->n, true, specs, works, g->d_tiles_inv,
                                   g->ntiles_inv, s);
    }
    if (e != cudaSuccess) return fail(e, "grouped inverse Legendre launch");
    {
        ProfScope ps(g->plans[0], kStageFftInv, s);
        e = launch_fft_inverse_group(g->plans, g->n, grids, s);
    }
    if (e != cudaSuccess) return fail(e, "grouped inverse FFT launch");
    return SHT_OK;
}

// Split-precision Legendre contractions on the 5th-generation tensor cores
// (tcgen05 + TMEM), for split plans (FP32 grid and spectrum).
//
// Both directions are per-(m, parity) products D = A . B over K, with the
// same shape as the FP64 path (Eq. cc-quad and Eq. iLT in the parity form
// of Appendix B):
//   forward  D[r][c] = sum_{j}  P~_{n_r}^m(mu_j)  Bw[j][c]     A: rows n_r, K = j
//   inverse  D[j][c] = sum_{r}  P~_{n_r}^m(mu_j)  X_{n_r}[c]    A: rows j,  K = r
// where c runs over the 2F real columns.  Operands are split into T = 2 or
// 3 BF16 terms, x = x_1 + x_2 (+ x_3), x_{t+1} = bf16(x - x_1 - .. - x_t),
// and the products x_a y_b with a + b <= T - 1 (0-based) are accumulated in
// FP32 in tensor memory (3 products for T = 2, 6 for T = 3): the leading
// product x_1 y_1 in one accumulator, the corrections in a second.
//
// A (the P~ table) is split once at plan time and stored pre-tiled in the
// canonical no-swizzle K-major layout of the tensor-core shared-memory
// descriptor: 8 x 8 core matrices of 128 contiguous bytes, core (i8, k8)
// at ((i8 * TK/8) + k8) * 128 within a K-slab of TK = 16.  A 128-row tile
// of a slab is therefore one contiguous block that one bulk asynchronous
// copy (TMA engine, cp.async.bulk) moves into shared memory.
// B (the FP32 Fourier data or spectrum) stays FP32 in HBM.  The TK x TN
// block of a tile arrives as one tiled tensor copy (cp.async.bulk.tensor
// over the whole Fourier workspace viewed as a row-major matrix of 2F
// columns) when the rows are 16-byte aligned (even field counts), else the
// converters load it directly.  (Sixteen
// 512-byte row copies per stage kept the copy warp issuing for most of a
// stage; one tiled copy does not.)  The converter warps split B into BF16
// terms, stored in the same K-major core-matrix layout, reading the next
// stage's values before they split this stage's.
//
// A CTA computes 128 x TN output tiles through rings of mbarrier stages
// (the A tiles, the FP32 B rows and the converted B terms each in a ring of
// its own; two CTAs share an SM, so one's prologue and epilogue overlap the
// other's main loop): the forward launches one CTA per tile, the inverse
// persistent CTAs that stride over the tile list.  Warps 0-7 convert B and
// run the epilogue (tcgen05.ld of the 32 TMEM lanes a warp may access, for
// half of the columns each), warp 8 issues the bulk copies of A (and of the
// pre-split inverse B), warp 10 those of the forward's FP32 B, one thread
// of warp 9 issues tcgen05.mma (M = 128, N = TN or, transposed, N = the
// tile's rows; K = 16) and commits to mbarriers.  Every wait is bounded by a clock limit;
// a CTA that gives up records SHT_ERR_TIMEOUT in the plan's status word,
// waits (bounded) for its MMAs and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "sht_internal.h"

namespace sht {

struct SplitProb {
    long long a_off;   // byte offset of this problem's A block in each term plane
    long long b_off;   // float offset of B row 0
    long long o_off;   // float offset of output row 0
    int R8;            // A rows padded to 8 (K-slab height)
    int Mrows;         // valid output rows
    int K;             // valid K (rows of B)
    int nkt;           // K tiles of TK
    int b_stride;      // floats between B rows
    int o_stride;      // floats between output rows
    long long rs_off;  // first row of this problem in the row-scale array
    long long bt_off;  // pre-split B: byte offset of this problem's tiles in each plane
    int kt0;           // reduced transform, forward: first K tile with |P~| >= 1e-16
    int mt0;           // reduced transform, inverse: row tiles below mt0 are all < 1e-16
};

struct SplitTables {
    int terms = 3;
    int tn = 128;                 // column-tile width of the GEMMs (64 or 128)
    bool fp16 = false;
    float* rs_fwd = nullptr;      // FP16 plans: 1 / row scale of each A row
    float* rs_inv = nullptr;
    unsigned char* fwd_planes = nullptr;   // terms planes of fwd_plane_bytes
    size_t fwd_plane_bytes = 0;
    unsigned char* inv_planes = nullptr;
    size_t inv_plane_bytes = 0;
    unsigned char* inv_bplanes = nullptr;   // the spectrum split per call (inverse B)
    size_t inv_bplane_bytes = 0;
    int inv_max_nkt = 0;
    int inject_stall = 0;         // SHT_INJECT_STALL at plan creation (tests only)
    std::vector<int> jmin;        // reduced transform: per problem, the first node
                                  // (from the pole) with some |P~| >= 1e-16; empty: off
    SplitProb* d_probs_fwd = nullptr;
    SplitProb* d_probs_inv = nullptr;
    int4* d_tiles_fwd = nullptr;
    int4* d_tiles_inv = nullptr;
    int ntiles_fwd = 0, ntiles_inv = 0;
};

namespace {

constexpr int TM = 128, TK = 16, UK = 16;
constexpr int TN_MAX = 128;                // column tiles are TN = 64 or 128 wide
constexpr int NCONV = 256;                 // converter / epilogue threads (8 warps)
constexpr int NTHREADS = NCONV + 96;       // + bulk-copy warp + MMA warp + B-row copy warp
constexpr int WARP_PRODUCER = NCONV / 32, WARP_MMA = NCONV / 32 + 1, WARP_RAW = NCONV / 32 + 2;
constexpr int A_TILE_BYTES = TM * TK * 2;   // one term
constexpr uint32_t kSBO = (TK / 8) * 128;   // stride between 8-row core groups
constexpr long long kWaitCycles = 4LL << 30;   // ~2 s at 2 GHz

// Per column-tile width TN: one 16-bit B tile (TK x TN), the FP32 staging of
// B (TK rows of TN) and the tensor memory of the two TN-column accumulators.
template <int TN> struct Wid {
    static constexpr int B_TILE_BYTES = TN * TK * 2;
    static constexpr int RAW_BYTES = TK * TN * 4;
    static constexpr int TMEM_COLS = 2 * TN;
    static constexpr int CTAS_PER_SM = TN == 64 ? 3 : 2;
};

// Shared-memory rings.  Pre-split B (BPRE): NA slots of T A tiles followed
// by T 16-bit B tiles, all loaded by the copy warp.  B converted in the
// kernel: three rings, each as deep as its latency needs -- NA slots of T A
// tiles (bulk copies from L2 / HBM, the longest wait), NR slots of FP32 B
// rows (TK rows of TN, their own copy warp, freed as soon as the converters
// have read them) and NB slots of the converted 16-bit B terms (written
// just before the MMAs read them, so two or three suffice).  Counts keep
// TN = 128 under 113 KB (two CTAs per SM, 2 x 256 TMEM columns) and TN = 64
// under 75 KB (three CTAs per SM, 3 x 128 columns).
template <int T, bool BPRE, int TN> struct Cfg {
    static constexpr int NA = BPRE ? (T == 3 ? 4 : 6)
                                   : (TN == 128 ? (T == 3 ? 5 : 6) : (T == 3 ? 4 : 5));
    static constexpr int NB = BPRE ? 0 : (TN == 128 && T == 2 ? 3 : 2);
    static constexpr int NR = BPRE ? 0 : (T == 3 ? 3 : 4);
    static constexpr int A_SLOT = T * A_TILE_BYTES + (BPRE ? T * Wid<TN>::B_TILE_BYTES : 0);
    static constexpr int BPRE_OFF = T * A_TILE_BYTES;   // pre-split B tiles within an A slot
    static constexpr int B_SLOT = T * Wid<TN>::B_TILE_BYTES;
    static constexpr int B_OFF = NA * A_SLOT;           // B-term slot b at B_OFF + b B_SLOT
    static constexpr int RAW_OFF = B_OFF + NB * B_SLOT;   // raw slot r at RAW_OFF + r RAW_BYTES
    static constexpr int BAR_OFF = RAW_OFF + NR * Wid<TN>::RAW_BYTES;
    static constexpr int NBAR = 2 * NA + 2 * NB + 2 * NR + 3;
    static constexpr int SMEM = BAR_OFF + 256;
    static_assert(8 * NBAR + 12 <= 256, "barriers, TMEM address and abort flag fit 256 bytes");
};
static_assert(Cfg<3, false, 128>::SMEM <= 113 * 1024 && Cfg<2, false, 128>::SMEM <= 113 * 1024 &&
                  Cfg<3, true, 128>::SMEM <= 113 * 1024 && Cfg<2, true, 128>::SMEM <= 113 * 1024,
              "two CTAs per SM at TN = 128");
static_assert(Cfg<3, false, 64>::SMEM <= 75 * 1024 && Cfg<2, false, 64>::SMEM <= 75 * 1024 &&
                  Cfg<3, true, 64>::SMEM <= 75 * 1024 && Cfg<2, true, 64>::SMEM <= 75 * 1024,
              "three CTAs per SM at TN = 64");

struct GemmArgs {
    const unsigned char* planes;   // term t plane at planes + t * plane_bytes
    long long plane_bytes;
    const SplitProb* probs;
    const int4* tiles;
    int ntiles;                     // tiles in the list (persistent CTAs stride over them)
    const float* B;
    float* O;
    int C;                          // valid columns (2F)
    int raw_bulk;                   // 1: B's rows arrive as one tiled tensor copy per
                                    // stage (bmap); 0: the converters load them
    int* status;
    const float* rs_inv;            // FP16: 1 / row scale per A row (pr.rs_off + row)
    const unsigned* colmax;         // FP16: max |B| per column (float bits)
    const unsigned char* bplanes;   // pre-split B: term t plane at bplanes + t * bplane_bytes
    long long bplane_bytes;
    int nct;                        // column tiles (pre-split B tile index = it * nct + ct)
    int stall;                      // fault injection for tests: CTA 0 never arms stage 0
    // raw_bulk: B as a row-major matrix [rows][C] of floats (problem
    // rows at b_off / b_stride), box TN columns x TK rows; out-of-range
    // columns and rows read as zero
    CUtensorMap bmap;
};

// FP16 operands are scaled by powers of two into [-1, 1): column c of B by
// 2^-(E+1) where 2^E <= max|B[., c]| < 2^(E+1), i.e. by the float whose
// biased exponent is 253 - (E + 127); the product is scaled back by 2^(E+1).
// Exponents are clamped so that both stay normal floats.
__device__ __forceinline__ float col_scale(unsigned maxbits) {
    const unsigned eb = min(maxbits >> 23, 252u);
    return __uint_as_float((253u - eb) << 23);
}
__device__ __forceinline__ float col_unscale(unsigned maxbits) {
    const unsigned eb = min(maxbits >> 23, 252u);
    return __uint_as_float((eb + 1u) << 23);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// One TK x TN box of the tensor map at column x, row y (x * 4 bytes is a
// multiple of 16: x is a multiple of TN).
__device__ __forceinline__ void tensor_g2s_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The same box fetched into L2 only (no shared memory, no barrier).
__device__ __forceinline__ void tensor_prefetch_l2_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction core stride) and stride (M/N-direction 8-row-group stride)
// byte offsets, descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bit 4), A and B
// BF16 (format 1 at bits 7 and 10) or FP16 (format 0), both K-major,
// N = TN (N/8 at bit 17), M = 128 (M/16 at bit 24).
template <bool F16, int TN>
constexpr uint32_t idesc_f16() {
    return (1u << 4) | (F16 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)(TM >> 4) << 24);
}

// The same MMA with the instruction descriptor in a register (N chosen per tile).
__device__ __forceinline__ void mma_f16_rt(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

template <bool F16, int TN>
__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b,
                                        uint32_t accum) {
    constexpr uint32_t idesc = idesc_f16<F16, TN>();
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Terms of 16-bit floats.  BF16: x_1 = bf16(x), x_{t+1} = bf16(x - x_1 -
// .. - x_t).  FP16 (x scaled into [-1, 1) first): x_1 = fp16(x), and the
// remainder scaled by 2^11 so that it keeps FP16's precision:
// x_2 = fp16(2^11 (x - x_1)), x_3 = fp16(2^11 (x - x_1) - x_2), so that
// x = x_1 + 2^-11 (x_2 + x_3) + O(2^-35).
// One term of 8 values: x[e] rounded to 16 bits, packed in pairs (one
// packed conversion per pair); unless it is the last term, x keeps the
// remainder x - term (exact, as the term is x rounded), formed from the
// packed bits without a second conversion.
template <bool F16, bool LAST>
__device__ __forceinline__ uint4 split_term8(float (&x)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if constexpr (F16) {
            const __half2 h = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&h);
            if (!LAST) {
                const float2 f = __half22float2(h);
                x[2 * i] -= f.x;
                x[2 * i + 1] -= f.y;
            }
        } else {
            const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&b);
            if (!LAST) {
                x[2 * i] -= __uint_as_float(w[i] << 16);
                x[2 * i + 1] -= __uint_as_float(w[i] & 0xffff0000u);
            }
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

extern __shared__ __align__(1024) unsigned char split_smem[];

// Per-tile arguments of a launch: one plan's for every tile, or, for a
// grouped launch, those of plan tile.w.
struct OnePlanArgs {
    const GemmArgs& g;
    __device__ __forceinline__ const GemmArgs& operator()(const int4&) const { return g; }
    __device__ __forceinline__ void mark_timeout() const {
        if (g.status) atomicOr(g.status, 1);
    }
};
struct GroupPlanArgs {
    const GemmArgs* a;
    int n;
    __device__ __forceinline__ const GemmArgs& operator()(const int4& t) const { return a[t.w]; }
    __device__ __forceinline__ void mark_timeout() const {
        for (int q = 0; q < n; ++q)
            if (a[q].status) atomicOr(a[q].status, 1);
    }
};

// CTA b computes tiles b, b + gridDim.x, ... of the list (one tile when the
// grid has a CTA per tile; many for the persistent inverse grid).  The
// rings and their phases run on across tiles (every role walks the
// same tiles and stages, so its running stage count names the slot and
// phase), the copy warps prefetch the next tile's operands while the
// converter warps drain the accumulator of the last one, and the MMA warp
// starts a tile once that drain is done (acc_empty).
template <int T, bool F16, bool BPRE, int TN, class Args>
__device__ __forceinline__ void split_gemm_body(const Args& args, const int4* __restrict__ tiles,
                                                int ntiles) {
    using CF = Cfg<T, BPRE, TN>;
    constexpr int B_TILE_BYTES = Wid<TN>::B_TILE_BYTES;
    constexpr int TMEM_COLS = Wid<TN>::TMEM_COLS;
    constexpr int NA = CF::NA;
    constexpr int NBS = CF::NB;
    constexpr int NR = CF::NR;
    constexpr int NBB = NBS > 0 ? NBS : 1;
    constexpr int NRS = NR > 0 ? NR : 1;
    // With 128-wide column tiles the product is formed transposed,
    // D^T = B^T A^T, with the 128 columns of B on the MMA's M side and the
    // tile's A rows (at most 128, rounded up to 16) on its N side, so a
    // partial row tile issues only the MMA work of its rows.  TMEM lanes are
    // then columns and TMEM columns rows, and the epilogue stores each output
    // row as 32 adjacent columns per warp instruction (coalesced; with the
    // rows on the lanes, every lane would write its own row).
    constexpr bool SWAP = TN == 128;
    constexpr int NB = CF::NBAR;   // barriers
    unsigned char* smem = split_smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + CF::BAR_OFF);
    // bars: full_a[NA], empty_a[NA], full_b[NBS], empty_b[NBS], full_r[NR],
    // empty_r[NR], done, acc_empty, fin
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + CF::BAR_OFF + 8 * NB);
    volatile int* abort_flag =
        reinterpret_cast<volatile int*>(smem + CF::BAR_OFF + 8 * NB + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_a = [&](int s) { return bar0 + 8u * s; };
    auto empty_a = [&](int s) { return bar0 + 8u * (NA + s); };
    auto full_b = [&](int b) { return bar0 + 8u * (2 * NA + b); };
    auto empty_b = [&](int b) { return bar0 + 8u * (2 * NA + NBS + b); };
    auto full_r = [&](int r) { return bar0 + 8u * (2 * NA + 2 * NBS + r); };
    auto empty_r = [&](int r) { return bar0 + 8u * (2 * NA + 2 * NBS + NR + r); };
    const uint32_t done = bar0 + 8u * (2 * NA + 2 * NBS + 2 * NR);   // accumulator full
    const uint32_t acc_empty = done + 8u;   // accumulator read out by the epilogue
    const uint32_t fin = done + 16u;        // every MMA of the CTA completed

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(full_a(s), 1);
            mbar_init(empty_a(s), 1);
        }
        for (int b = 0; b < NBS; ++b) {
            mbar_init(full_b(b), NCONV);
            mbar_init(empty_b(b), 1);
        }
        for (int r = 0; r < NR; ++r) {
            mbar_init(full_r(r), 1);
            mbar_init(empty_r(r), NCONV);
        }
        mbar_init(done, 1);
        mbar_init(acc_empty, NCONV);
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // stages it = kb .. kb + nst - 1 of a tile (the reduced transform skips
    // the K tiles of negligible P~ in the forward direction and whole row
    // tiles in the inverse one, whose outputs are then written as zero)
    auto stages = [](const SplitProb& pr, int mt) { return (mt < pr.mt0) ? 0 : pr.nkt - pr.kt0; };
    // warp-uniform view of the abort flag
    auto aborted = [&]() { return __any_sync(0xffffffffu, *abort_flag != 0) != 0; };

    if (warp == WARP_PRODUCER) {
        // ---- producer: A tiles (and pre-split B tiles), lane 0 ----
        uint32_t q = 0, issued = 0;   // stages passed / issued in this CTA
        bool stalled = false;         // injected: the CTA's first stage never armed
        bool ok = true;
        for (int tt = blockIdx.x; tt < ntiles && ok && !aborted(); tt += gridDim.x) {
            const int4 tile = tiles[tt];
            const GemmArgs& g = args(tile);
            const SplitProb pr = g.probs[tile.x];
            const int mt = tile.y, ct = tile.z, kb = pr.kt0, nst = stages(pr, mt);
            const int h = min(TM, pr.R8 - TM * mt);   // A rows present in this tile
            const uint32_t abytes = (uint32_t)h * TK * 2;
            for (int li = 0; li < nst; ++li, ++q) {
                const int it = kb + li;
                const int s = q % NA;
                const uint32_t ph = (q / NA) & 1u;
                if (lane == 0) ok = mbar_wait(empty_a(s), ph ^ 1u, abort_flag);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                issued = q + 1;
                if (q == 0 && g.stall && blockIdx.x == 0) {
                    stalled = true;
                    continue;
                }
                unsigned char* st = smem + s * CF::A_SLOT;
                if (lane == 0) {
                    mbar_expect_tx(full_a(s),
                                   abytes * T + (BPRE ? (uint32_t)(T * B_TILE_BYTES) : 0u));
                    const long long src_off = pr.a_off + (long long)it * pr.R8 * TK * 2 +
                                              (long long)mt * TM * TK * 2;
                    for (int t = 0; t < T; ++t)
                        bulk_g2s(smem_u32(st + t * A_TILE_BYTES),
                                 g.planes + (long long)t * g.plane_bytes + src_off, abytes,
                                 full_a(s));
                    if (BPRE) {
                        const long long b_src =
                            pr.bt_off + ((long long)it * g.nct + ct) * B_TILE_BYTES;
                        for (int t = 0; t < T; ++t)
                            bulk_g2s(smem_u32(st + CF::BPRE_OFF + t * B_TILE_BYTES),
                                     g.bplanes + (long long)t * g.bplane_bytes + b_src,
                                     B_TILE_BYTES, full_a(s));
                    }
                }
                __syncwarp();
            }
        }
        // after an abort, let the copies already issued land before the CTA
        // releases its shared memory (bounded; a stage never armed is skipped)
        if (lane == 0 && *abort_flag) {
            for (uint32_t j = issued > (uint32_t)NA ? issued - NA : 0u; j < issued; ++j) {
                if (stalled && j == 0) continue;
                const long long t0 = clock64();
                while (!mbar_try(full_a(j % NA), (j / NA) & 1u) &&
                       clock64() - t0 < kWaitCycles) {
                }
            }
        }
    } else if (warp == WARP_RAW) {
        // ---- the FP32 rows of B into the raw ring, NR stages ahead of the
        // converters: one tiled tensor copy per stage ----
        constexpr int PF_L2 = 4;   // L2 prefetch distance beyond the copy, in stages
        uint32_t q = 0, issued = 0;   // raw stages passed / issued in this CTA
        bool ok = true;
        for (int tt = blockIdx.x; !BPRE && tt < ntiles && ok && !aborted(); tt += gridDim.x) {
            const int4 tile = tiles[tt];
            const GemmArgs& g = args(tile);
            if (!g.raw_bulk) continue;
            const SplitProb pr = g.probs[tile.x];
            const int mt = tile.y, ct = tile.z, kb = pr.kt0, nst = stages(pr, mt);
            const int cbase = ct * TN;
            const int y0 = (int)(pr.b_off / pr.b_stride);   // matrix row of k = 0
            for (int li = 0; li < nst; ++li, ++q) {
                const int it = kb + li;
                const int r = q % NRS;
                const uint32_t ph = (q / NRS) & 1u;
                if (lane == 0) ok = mbar_wait(empty_r(r), ph ^ 1u, abort_flag);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                issued = q + 1;
                const int k0 = it * TK;
                const uint32_t dst = smem_u32(smem + CF::RAW_OFF + r * Wid<TN>::RAW_BYTES);
                // the whole box lands (rows past K belong to the next problem
                // or read as zero; the converters skip them)
                if (lane == 0) {
                    mbar_expect_tx(full_r(r), (uint32_t)(TK * TN * 4));
                    tensor_g2s_2d(dst, &g.bmap, cbase, y0 + k0, full_r(r));
                    // the rows of a later stage into L2, so that its copy
                    // into the ring comes from L2 rather than HBM
                    if (li + PF_L2 < nst)
                        tensor_prefetch_l2_2d(&g.bmap, cbase, y0 + k0 + PF_L2 * TK);
                }
                __syncwarp();
            }
        }
        // after an abort, let the copies already issued land (bounded)
        if (lane == 0 && *abort_flag) {
            for (uint32_t j = issued > (uint32_t)NRS ? issued - NRS : 0u; j < issued; ++j) {
                const long long t0 = clock64();
                while (!mbar_try(full_r(j % NRS), (j / NRS) & 1u) &&
                       clock64() - t0 < kWaitCycles) {
                }
            }
        }
    } else if (warp == WARP_MMA) {
        // ---- MMA issuer ----
        if (lane == 0) {
            uint32_t q = 0, qb = 0;   // stages of the A ring / B-term ring passed
            uint32_t nacc = 0;        // tiles accumulated so far
            bool ok = true;
            for (int tt = blockIdx.x; tt < ntiles && ok && !*abort_flag; tt += gridDim.x) {
                const int4 tile = tiles[tt];
                const SplitProb pr = args(tile).probs[tile.x];
                const int mt = tile.y, nst = stages(pr, mt);
                if (nst == 0) continue;
                // SWAP: M = 128 (the column tile), N = the tile's A rows rounded to 16
                const int nrows = ((min(TM, pr.R8 - TM * mt) + 15) / 16) * 16;
                const uint32_t idesc_swap = (1u << 4) | (F16 ? 0u : ((1u << 7) | (1u << 10))) |
                                            ((uint32_t)(nrows >> 3) << 17) |
                                            ((uint32_t)(TM >> 4) << 24);
                (void)idesc_swap;
                // the epilogue has read the previous tile's accumulator
                if (nacc > 0 && !(ok = mbar_wait(acc_empty, (nacc - 1) & 1u, abort_flag))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int li = 0; li < nst; ++li, ++q) {
                    const int s = q % NA;
                    const int sb = qb % NBB;
                    ok = mbar_wait(full_a(s), (q / NA) & 1u, abort_flag) &&
                         (BPRE || mbar_wait(full_b(sb), (qb / NBB) & 1u, abort_flag));
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = smem_u32(smem + s * CF::A_SLOT);
                    const uint32_t bst = BPRE ? st + CF::BPRE_OFF
                                              : smem_u32(smem + CF::B_OFF + sb * CF::B_SLOT);
#pragma unroll
                    for (int ks = 0; ks < TK / UK; ++ks) {
#pragma unroll
                        for (int a = 0; a < T; ++a) {
#pragma unroll
                            for (int b = 0; b < T - a; ++b) {
                                // FP16: x_2 y_2 has weight 2^-22 (below 2^-24
                                // of the scaled operands) and is dropped
                                if (F16 && a == 1 && b == 1) continue;
                                const uint64_t ad =
                                    sdesc(st + a * A_TILE_BYTES + ks * 256, 128, kSBO);
                                const uint64_t bd =
                                    sdesc(bst + b * B_TILE_BYTES + ks * 256, 128, kSBO);
                                // (0,0) -> leading accumulator; the first of
                                // the others, (0,1), opens the correction one
                                const bool lead = (a == 0 && b == 0);
                                const uint32_t acc =
                                    (li > 0 || ks > 0 || !(lead || (a == 0 && b == 1))) ? 1u
                                                                                         : 0u;
                                if constexpr (SWAP)
                                    mma_f16_rt(lead ? tmem : tmem + TN, bd, ad, idesc_swap, acc);
                                else
                                    mma_f16<F16, TN>(lead ? tmem : tmem + TN, ad, bd, acc);
                            }
                        }
                    }
                    mma_commit(empty_a(s));
                    if (!BPRE) {
                        mma_commit(empty_b(sb));
                        ++qb;
                    }
                }
                if (!ok) break;
                // done fires once every MMA of the tile has completed
                mma_commit(done);
                ++nacc;
            }
            // fin fires once every MMA this CTA issued has completed
            mma_commit(fin);
        }
    } else {
        // ---- converters: B (FP32, rows k, columns c) -> T BF16 K-major tiles
        // from the staged rows in shared memory (raw_bulk) or straight from
        // global memory (rows not 16-byte aligned: odd field counts); then
        // the tile's epilogue ----
        const int tid = threadIdx.x;   // 0..NCONV-1
        static_assert(NCONV % TN == 0, "a converter thread keeps one column");
        uint32_t qb = 0, qr = 0;   // B-term / raw ring stages passed
        uint32_t nacc = 0;         // tiles accumulated so far
        bool ok = true;
        for (int tt = blockIdx.x; tt < ntiles && ok && !aborted(); tt += gridDim.x) {
            const int4 tile = tiles[tt];
            const GemmArgs& g = args(tile);
            const SplitProb pr = g.probs[tile.x];
            const int mt = tile.y, ct = tile.z, kb = pr.kt0, nst = stages(pr, mt);
            const int cbase = ct * TN;
            float cs = 1.f;
            if (F16) {
                const int cg = cbase + tid % TN;
                if (cg < g.C) cs = col_scale(g.colmax[cg]);
            }
            // Thread tid converts column c, K rows k8 * 8 .. + 7 of each
            // stage (threads past TN * TK / 8 only take part in the
            // barriers).  Software-pipelined over two register buffers: the
            // next stage's values are read (and their raw slot released)
            // before this stage's terms are formed and stored.
            static_assert(TN * TK / 8 <= NCONV, "one 8-value unit per thread and stage");
            const bool unit = tid < TN * TK / 8;
            const int c = tid % TN, k8 = tid / TN, cg = cbase + c;
            const bool cin = unit && cg < g.C;
            const int off = ((c >> 3) * (TK / 8) + k8) * 128 + (c & 7) * 16;
            // the 8 values of stage li into x (false: the wait gave up)
            auto fetch = [&](int li, float (&x)[8]) -> bool {
                const int k = (kb + li) * TK + k8 * 8;
                if (g.raw_bulk) {
                    const uint32_t q = qr + (uint32_t)li;
                    const int r = q % NRS;
                    if (!mbar_wait(full_r(r), (q / NRS) & 1u, abort_flag)) return false;
                    const float* raw = reinterpret_cast<const float*>(
                        smem + CF::RAW_OFF + r * Wid<TN>::RAW_BYTES);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        x[e] = (cin && k + e < pr.K) ? raw[(k8 * 8 + e) * TN + c] : 0.f;
                    mbar_arrive(empty_r(r));
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        x[e] = (cin && k + e < pr.K)
                                   ? __ldg(g.B + pr.b_off + (long long)(k + e) * pr.b_stride + cg)
                                   : 0.f;
                }
                return true;
            };
            // B-term slot of stage li free (the MMAs of its previous use are
            // done), then the T terms of x stored into it
            auto convert = [&](int li, float (&x)[8]) -> bool {
                const uint32_t qq = qb + (uint32_t)li;
                const int sb = qq % NBB;
                if (!mbar_wait(empty_b(sb), ((qq / NBB) & 1u) ^ 1u, abort_flag)) return false;
                unsigned char* bst = smem + CF::B_OFF + sb * CF::B_SLOT;
                if (unit) {
                    if (F16) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] *= cs;
                    }
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const uint4 pk = t == T - 1 ? split_term8<F16, true>(x)
                                                    : split_term8<F16, false>(x);
                        if (F16 && t == 0) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) x[e] *= 2048.f;   // x_2, x_3: weight 2^-11
                        }
                        *reinterpret_cast<uint4*>(bst + t * B_TILE_BYTES + off) = pk;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(full_b(sb));
                return true;
            };
            // (a lane that gives up leaves alone; the warp agrees on ok
            // again before the epilogue's collective operations)
            const int ncv = BPRE ? 0 : nst;
            float xa[8];
            if constexpr (TN == 128) {
                float xb[8];
                if (ncv > 0) ok = fetch(0, xa);
                for (int li = 0; li < ncv && ok; li += 2) {
                    if (li + 1 < ncv && !(ok = fetch(li + 1, xb))) break;
                    if (!(ok = convert(li, xa))) break;
                    if (li + 1 >= ncv) break;
                    if (li + 2 < ncv && !(ok = fetch(li + 2, xa))) break;
                    if (!(ok = convert(li + 1, xb))) break;
                }
            } else {
                // three CTAs per SM leave 56 registers a thread: one buffer
                for (int li = 0; li < ncv && ok; ++li)
                    ok = fetch(li, xa) && convert(li, xa);
            }
            if (!BPRE) {
                qb += (uint32_t)ncv;
                if (g.raw_bulk) qr += (uint32_t)ncv;
            }
            // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (the
            // tile rows it may access) for column half w / 4 ----
            const bool have = nst > 0;
            if (have && ok) ok = mbar_wait(done, nacc & 1u, abort_flag);
            // the TMEM loads and shuffles below are warp-collective: agree on ok
            ok = __all_sync(0xffffffffu, ok) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int lq = warp & 3, half = warp >> 2;
            if constexpr (SWAP) {
                // TMEM lane 32 lq + lane = column c of the tile; TMEM columns =
                // rows n.  For each row the 32 lanes store 32 adjacent columns.
                const int c = cbase + 32 * lq + lane;
                const bool col_ok = c < g.C && ok && !*abort_flag;
                const float csi = (F16 && c < g.C) ? col_unscale(g.colmax[c]) : 0.f;
                constexpr int NCH = TN / 16 / (NCONV / 128);
                for (int cc = 0; cc < NCH; ++cc) {
                    const int ch = half * NCH + cc;
                    const int n0 = TM * mt + ch * 16;
                    if (n0 >= pr.Mrows) break;   // uniform over the warp
                    uint32_t r[16];
                    if (have && ok) {
                        uint32_t r2[16];
                        const uint32_t ta =
                            tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(ch * 16);
                        tmem_ld16(ta, r);
                        tmem_ld16(ta + TN, r2);
                        // FP16: lane k < 16 fetches the row scale of row n0 + k
                        const int nl = n0 + (lane & 15);
                        const float my_rsi =
                            (F16 && nl < pr.Mrows) ? g.rs_inv[pr.rs_off + nl] : 0.f;
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            float v;
                            if (F16) {
                                const float rsi = __shfl_sync(0xffffffffu, my_rsi, k);
                                v = (__uint_as_float(r[k]) +
                                     __uint_as_float(r2[k]) * (1.f / 2048.f)) *
                                    rsi * csi;
                            } else {
                                v = __uint_as_float(r[k]) + __uint_as_float(r2[k]);
                            }
                            r[k] = __float_as_uint(v);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k) r[k] = 0u;
                    }
                    if (!col_ok) continue;
                    float* ocol = g.O + pr.o_off + c;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (n0 + k < pr.Mrows)
                            ocol[(long long)(n0 + k) * pr.o_stride] = __uint_as_float(r[k]);
                }
            } else {
                const int row = TM * mt + 32 * lq + lane;
                const bool row_ok = row < pr.Mrows && ok && !*abort_flag;
                float* orow = g.O + pr.o_off + (long long)row * pr.o_stride;
                const bool vec = ((pr.o_stride & 3) == 0) && ((pr.o_off & 3) == 0) &&
                                 ((g.C & 3) == 0);
                constexpr int NCH = TN / 16 / (NCONV / 128);
                for (int cc = 0; cc < NCH; ++cc) {
                    const int ch = half * NCH + cc;
                    const int c0 = cbase + ch * 16;
                    uint32_t r[16];
                    if (have && ok) {
                        uint32_t r2[16];
                        const uint32_t ta =
                            tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(ch * 16);
                        tmem_ld16(ta, r);
                        tmem_ld16(ta + TN, r2);
                        if (F16) {
                            // lead + 2^-11 corrections, then undo the row and
                            // column scales
                            const float rsi = row_ok ? g.rs_inv[pr.rs_off + row] : 0.f;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float csi =
                                    c0 + i < g.C ? col_unscale(g.colmax[c0 + i]) : 0.f;
                                r[i] = __float_as_uint((__uint_as_float(r[i]) +
                                                        __uint_as_float(r2[i]) * (1.f / 2048.f)) *
                                                       rsi * csi);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                r[i] = __float_as_uint(__uint_as_float(r[i]) +
                                                       __uint_as_float(r2[i]));
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) r[i] = 0u;
                    }
                    if (!row_ok || c0 >= g.C) continue;
                    if (vec && c0 + 16 <= g.C) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float4 f;
                            f.x = __uint_as_float(r[4 * i + 0]);
                            f.y = __uint_as_float(r[4 * i + 1]);
                            f.z = __uint_as_float(r[4 * i + 2]);
                            f.w = __uint_as_float(r[4 * i + 3]);
                            *reinterpret_cast<float4*>(orow + c0 + 4 * i) = f;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < g.C) orow[c0 + i] = __uint_as_float(r[i]);
                    }
                }
            }
            if (have && ok) {
                // the accumulator is free for the next tile's MMAs
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(acc_empty);
                ++nacc;
            }
        }
    }
    if (*abort_flag && threadIdx.x == 0) args.mark_timeout();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        // every MMA has completed before the accumulator is released
        // (bounded as well)
        const long long t0 = clock64();
        while (!mbar_try(fin, 0) && clock64() - t0 < kWaitCycles) {
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

template <int T, bool F16, bool BPRE, int TN>
__global__ void __launch_bounds__(NTHREADS, Wid<TN>::CTAS_PER_SM)
    split_gemm_kernel(const __grid_constant__ GemmArgs g) {
    split_gemm_body<T, F16, BPRE, TN>(OnePlanArgs{g}, g.tiles, g.ntiles);
}

// Grouped launch: tile.w is the plan's index in the group.
struct GemmGroup {
    int n;
    int ntiles;
    GemmArgs a[kMaxGroup];
    const int4* tiles;
};
// passed by value as a kernel parameter (each GemmArgs holds a tensor map)
static_assert(sizeof(GemmGroup) <= 4096, "grouped GEMM arguments fit the 4 KB parameter space");

template <int T, bool F16, bool BPRE, int TN>
__global__ void __launch_bounds__(NTHREADS, Wid<TN>::CTAS_PER_SM)
    split_gemm_group_kernel(const __grid_constant__ GemmGroup G) {
    split_gemm_body<T, F16, BPRE, TN>(GroupPlanArgs{G.a, G.n}, G.tiles, G.ntiles);
}

// Split the FP32 operand B of every inverse problem (the spectrum rows of
// one (m, parity)) into T 16-bit terms, stored as pre-tiled K-major B tiles
// (the layout the converters build in shared memory): tile (problem,
// k-tile it, column tile ct) at bt_off + (it nct + ct) * B_TILE_BYTES of
// each term plane.  Block (problem, 128 columns); warp w keeps 32 columns
// (lane = column of group w % 4) and takes the groups of 8 K rows
// g = w / 4, w / 4 + 2, ... (reads coalesced over the columns, 16 bytes
// written per term and group).  FP16 scales each column as the GEMM's
// converters do.
// The same pass computes the Equator row of the problem's output,
// sum_r P~_{n_r}^m(0) X_{n_r}[c] (Eq. iLT at mu = 0), which the GEMM tiles
// leave out: a compensated FP32 dot product (P~ as a float pair hi + lo,
// exact products by FMA, two-sum accumulation) of the unscaled FP32
// inputs, the two warps' partial sums of a column combined in a fixed
// order.  For the odd parity (n - m odd) P~(0) vanishes and the Equator
// value is 0.
__device__ __forceinline__ void two_sum_acc(float& h, float& l, float a, float al) {
    const float sum = __fadd_rn(h, a);
    const float bp = __fsub_rn(sum, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bp)), __fsub_rn(a, bp));
    h = sum;
    l = __fadd_rn(l, __fadd_rn(err, al));
}

template <int T, bool F16, int TN>
__global__ void __launch_bounds__(256)
    split_b_kernel(const float* __restrict__ B, const SplitProb* __restrict__ probs, int C,
                   int nct, const unsigned* __restrict__ colmax, unsigned char* planes,
                   long long plane_bytes, const double* __restrict__ pnm, int ldp, int N,
                   int Jh, float* __restrict__ O) {
    constexpr int B_TILE_BYTES = Wid<TN>::B_TILE_BYTES;
    extern __shared__ float2 peq[];   // [K] P~(0) of the problem's rows, (hi, lo)
    __shared__ float2 red[8][32];
    const int p = blockIdx.x;
    const SplitProb pr = probs[p];
    const bool even = (p & 1) == 0;
    const size_t row0 = coef_offset(N, p >> 1) + (p & 1);
    if (even) {
        for (int k = threadIdx.x; k < pr.K; k += blockDim.x) {
            const double v = pnm[(row0 + 2 * (size_t)k) * ldp + (Jh - 1)];
            const float hi = (float)v;
            peq[k] = make_float2(hi, (float)(v - (double)hi));
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.y * 128 + (w & 3) * 32 + lane;
    const bool cin = c < C;
    const float cs = (F16 && cin) ? col_scale(colmax[c]) : 1.f;
    const int ct = c / TN, cc = c % TN;
    float eh = 0.f, el = 0.f;
    for (int g = w >> 2; g < pr.nkt * (TK / 8); g += 2) {
        const int it = g / (TK / 8), k8 = g % (TK / 8);
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = g * 8 + e;
            x[e] = (k < pr.K && cin) ? __ldg(B + pr.b_off + (long long)k * pr.b_stride + c)
                                     : 0.f;
        }
        if (even) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = g * 8 + e;
                if (k < pr.K) {
                    const float2 pe = peq[k];
                    const float ph = __fmul_rn(pe.x, x[e]);
                    two_sum_acc(eh, el, ph, fmaf(pe.y, x[e], fmaf(pe.x, x[e], -ph)));
                }
            }
        }
        if (F16) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] *= cs;
        }
        const long long off = pr.bt_off + ((long long)it * nct + ct) * B_TILE_BYTES +
                              ((cc >> 3) * (TK / 8) + k8) * 128 + (cc & 7) * 16;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint4 pk = t == T - 1 ? split_term8<F16, true>(x) : split_term8<F16, false>(x);
            if (F16 && t == 0) {
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] *= 2048.f;
            }
            // columns past C inside the last tile are written as zero;
            // those past the tiles (64-wide tiles) are not stored
            if (ct < nct) *reinterpret_cast<uint4*>(planes + (long long)t * plane_bytes + off) = pk;
        }
    }
    red[w][lane] = make_float2(eh, el);
    __syncthreads();
    if (w < 4) {
        const float2 r = red[w + 4][lane];
        two_sum_acc(eh, el, r.x, r.y);
        if (cin) O[pr.o_off + (long long)pr.Mrows * pr.o_stride + c] = __fadd_rn(eh, el);
    }
}

// Split the FP64 P~ table into T BF16 planes, pre-tiled (see top of file).
// One block per (m, parity) problem.  fwd: A rows are the parity rows n_r,
// K the northern nodes; inv: A rows are the nodes, K the parity rows.
__global__ void split_table_kernel(const double* __restrict__ pnm, int ldp, int N, int Jh,
                                   const SplitProb* __restrict__ probs, int inverse, int T,
                                   unsigned char* planes, long long plane_bytes) {
    const int p = blockIdx.x;
    const int m = p >> 1, q = p & 1;
    const SplitProb pr = probs[p];
    const size_t row0 = coef_offset(N, m) + q;
    const long long K32 = (long long)pr.nkt * TK;
    const long long n_el = (long long)pr.R8 * K32;
    for (long long e = threadIdx.x; e < n_el; e += blockDim.x) {
        const int r = (int)(e / K32);
        const int k = (int)(e % K32);
        double v = 0.0;
        if (!inverse) {
            if (r < pr.Mrows && k < Jh) v = pnm[(row0 + 2 * (size_t)r) * ldp + k];
        } else {
            if (r < pr.Mrows && k < pr.K) v = pnm[(row0 + 2 * (size_t)k) * ldp + r];
        }
        const int kt = k / TK, kk = k % TK;
        const long long off = pr.a_off + (long long)kt * pr.R8 * TK * 2 +
                              (long long)(((r >> 3) * (TK / 8) + (kk >> 3)) * 128 +
                                          (r & 7) * 16 + (kk & 7) * 2);
        for (int t = 0; t < T; ++t) {
            const __nv_bfloat16 hb = __float2bfloat16_rn((float)v);
            *reinterpret_cast<__nv_bfloat16*>(planes + t * plane_bytes + off) = hb;
            v -= (double)__bfloat162float(hb);
        }
    }
}

// The same for FP16 terms, with one power-of-two scale per A row: row r is
// scaled by 2^-e, where 2^(e-1) <= max_k |A[r][k]| < 2^e (e clamped to
// [-100, 100]), so that its entries lie in [-1, 1); rs_inv[rs_off + r] = 2^e
// undoes it in the epilogue.  One warp per row finds the row maximum.
__global__ void split_table_f16_kernel(const double* __restrict__ pnm, int ldp, int N, int Jh,
                                       const SplitProb* __restrict__ probs, int inverse, int T,
                                       unsigned char* planes, long long plane_bytes,
                                       float* rs_inv) {
    const int p = blockIdx.x;
    const int m = p >> 1, q = p & 1;
    const SplitProb pr = probs[p];
    const size_t row0 = coef_offset(N, m) + q;
    const long long K32 = (long long)pr.nkt * TK;
    auto aval = [&](int r, int k) -> double {
        if (!inverse) return (r < pr.Mrows && k < Jh) ? pnm[(row0 + 2 * (size_t)r) * ldp + k] : 0.0;
        return (r < pr.Mrows && k < pr.K) ? pnm[(row0 + 2 * (size_t)k) * ldp + r] : 0.0;
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < pr.R8; r += nw) {
        double mx = 0.0;
        for (long long k = lane; k < K32; k += 32) mx = fmax(mx, fabs(aval(r, (int)k)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int e = 0;
            if (mx > 0.0) frexp(mx, &e);
            e = max(-100, min(100, e));
            rs_inv[pr.rs_off + r] = ldexpf(1.f, e);
        }
    }
    __syncthreads();
    const long long n_el = (long long)pr.R8 * K32;
    for (long long e = threadIdx.x; e < n_el; e += blockDim.x) {
        const int r = (int)(e / K32);
        const int k = (int)(e % K32);
        double v = aval(r, k) / (double)rs_inv[pr.rs_off + r];   // exact: a power of two
        const int kt = k / TK, kk = k % TK;
        const long long off = pr.a_off + (long long)kt * pr.R8 * TK * 2 +
                              (long long)(((r >> 3) * (TK / 8) + (kk >> 3)) * 128 +
                                          (r & 7) * 16 + (kk & 7) * 2);
        for (int t = 0; t < T; ++t) {
            const __half h = __double2half(v);
            *reinterpret_cast<__half*>(planes + t * plane_bytes + off) = h;
            v -= (double)__half2float(h);
            if (t == 0) v *= 2048.0;
        }
    }
}

// Column maxima of a row-major FP32 operand of nrows x C (the spectrum of
// an inverse GEMM); the imaginary column of each field is skipped in the
// first skip_odd rows (the m = 0 coefficients, whose imaginary parts are
// not inputs).  Block (x, y) covers columns 32x .. 32x+31 of a contiguous
// range of rows; its 8 warps stride that range with 8 independent loads in
// flight per thread, then reduce through shared memory to one atomic per
// column.  colmax must be zero on entry.
__global__ void __launch_bounds__(256) colmax_kernel(const float* __restrict__ B,
                                                     long long nrows, int C, int skip_odd,
                                                     unsigned* colmax) {
    __shared__ float red[8][32];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const long long per = (nrows + gridDim.y - 1) / gridDim.y;
    const long long r0 = (long long)blockIdx.y * per;
    const long long r1 = min(nrows, r0 + per);
    float mx = 0.f;
    if (c < C) {
        const long long rs = ((c & 1) ? max(r0, (long long)skip_odd) : r0) + threadIdx.y;
        long long r = rs;
        for (; r + 56 < r1; r += 64) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(B + (r + 8 * u) * C + c);
#pragma unroll
            for (int u = 0; u < 8; ++u) mx = fmaxf(mx, fabsf(v[u]));
        }
        for (; r < r1; r += 8) mx = fmaxf(mx, fabsf(__ldg(B + r * C + c)));
    }
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && c < C) {
#pragma unroll
        for (int y = 1; y < 8; ++y) mx = fmaxf(mx, red[y][threadIdx.x]);
        atomicMax(&colmax[c], __float_as_uint(mx));
    }
}

cudaError_t launch_colmax_inverse(const sht_plan_s* p, const void* spec, cudaStream_t s) {
    const int C = 2 * p->F;
    unsigned* cm = p->d_colmax + C;
    cudaError_t e = cudaMemsetAsync(cm, 0, (size_t)C * sizeof(unsigned), s);
    if (e) return e;
    const long long nrows = (long long)p->ncoef;
    const int cx = (C + 31) / 32;
    // about 16 blocks per SM in all, each over at least 64 rows
    long long ry = std::max<long long>(1, (16LL * p->num_sms + cx - 1) / cx);
    ry = std::min<long long>(ry, std::max<long long>(1, nrows / 64));
    colmax_kernel<<<dim3(cx, (unsigned)ry), dim3(32, 8), 0, s>>>(
        static_cast<const float*>(spec), nrows, C, p->N + 1, cm);
    note_launch();
    return cudaGetLastError();
}

int terms_of(int prec) { return (prec == SHT_BF16X2 || prec == SHT_FP16X2) ? 2 : 3; }

// Problems (one per (m, parity)) and tiles of both directions for
// truncation N, Jh northern nodes and C real columns; tile.w = plan.
void build_split_lists(int N, int Jh, int C, int tn, int plan, const std::vector<int>& jmin,
                       std::vector<SplitProb>& pf, std::vector<SplitProb>& pi,
                       std::vector<int4>& tf, std::vector<int4>& ti, long long& fwd_bytes,
                       long long& inv_bytes) {
    const int nprob = 2 * (N + 1);
    pf.assign(nprob, SplitProb{});
    pi.assign(nprob, SplitProb{});
    tf.clear();
    ti.clear();
    fwd_bytes = inv_bytes = 0;
    long long fwd_rows = 0, inv_rows = 0, inv_bt = 0;
    const int nct = (C + tn - 1) / tn;
    for (int m = 0; m <= N; ++m) {
        for (int q = 0; q < 2; ++q) {
            const int d = N - m - q;
            const int R = d >= 0 ? d / 2 + 1 : 0;
            const long long row0 = (long long)coef_offset(N, m) + q;
            SplitProb& f = pf[2 * m + q];
            f.a_off = fwd_bytes;
            f.R8 = (R + 7) / 8 * 8;
            f.Mrows = R;
            f.K = Jh;
            f.nkt = (Jh + TK - 1) / TK;
            // reduced transform: K tiles entirely nearer the pole than the
            // first significant node are skipped; inverse row tiles entirely
            // there are written as zero
            const int j0 = jmin.empty() ? 0 : jmin[2 * m + q];
            f.kt0 = std::min(j0 / TK, f.nkt);
            f.mt0 = 0;
            f.b_off = (long long)(2 * m + q) * Jh * C;
            f.b_stride = C;
            f.o_off = row0 * C;
            f.o_stride = 2 * C;
            fwd_bytes += (long long)f.R8 * f.nkt * TK * 2;
            f.rs_off = fwd_rows;
            fwd_rows += f.R8;
            for (int mt = 0; mt * TM < R; ++mt)
                for (int c = 0; c < nct; ++c) tf.push_back(make_int4(2 * m + q, mt, c, plan));
            // inverse rows: the nodes north of the Equator; the Equator row
            // (node Jh - 1) is computed by split_b_kernel
            SplitProb& v = pi[2 * m + q];
            v.a_off = inv_bytes;
            v.R8 = (Jh - 1 + 7) / 8 * 8;
            v.Mrows = Jh - 1;
            v.K = R;
            v.nkt = (R + TK - 1) / TK;
            v.kt0 = 0;
            v.mt0 = j0 / TM;
            v.b_off = row0 * C;
            v.b_stride = 2 * C;
            v.o_off = (long long)(2 * m + q) * Jh * C;
            v.o_stride = C;
            inv_bytes += (long long)v.R8 * v.nkt * TK * 2;
            v.rs_off = inv_rows;
            inv_rows += v.R8;
            v.bt_off = inv_bt;
            inv_bt += (long long)v.nkt * nct * tn * TK * 2;
            f.bt_off = 0;
            for (int mt = 0; mt * TM < Jh - 1; ++mt)
                for (int c = 0; c < nct; ++c) ti.push_back(make_int4(2 * m + q, mt, c, plan));
        }
    }
}

// The driver's cuTensorMapEncodeTiled, reached through the runtime (no link
// against libcuda); nullptr if the driver does not offer it.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiled) nullptr;
        }
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}

// Tensor map of the forward operand B: rows x C floats, row pitch C (the
// rows are 16-byte aligned), box tn columns x TK rows.  False if it cannot
// be made (the row copies are used instead).
bool encode_b_map(CUtensorMap* map, const void* B, int C, long long rows, int tn) {
    const EncodeTiled enc = encode_tiled();
    if (!enc || rows <= 0 || rows > (1LL << 31)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)C * 4};
    const cuuint32_t box[2] = {(cuuint32_t)tn, (cuuint32_t)TK};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(B), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

GemmArgs make_gemm_args(const sht_plan_s* p, bool inverse, const void* B, void* O) {
    const SplitTables* st = p->split;
    GemmArgs g;
    g.planes = inverse ? st->inv_planes : st->fwd_planes;
    g.plane_bytes = (long long)(inverse ? st->inv_plane_bytes : st->fwd_plane_bytes);
    g.probs = inverse ? st->d_probs_inv : st->d_probs_fwd;
    g.tiles = inverse ? st->d_tiles_inv : st->d_tiles_fwd;
    g.ntiles = inverse ? st->ntiles_inv : st->ntiles_fwd;
    g.B = static_cast<const float*>(B);
    g.O = static_cast<float*>(O);
    g.C = 2 * p->F;
    g.raw_bulk = 0;
    g.status = p->d_status;
    g.rs_inv = inverse ? st->rs_inv : st->rs_fwd;
    g.colmax = p->d_colmax ? p->d_colmax + (inverse ? g.C : 0) : nullptr;
    g.nct = (g.C + st->tn - 1) / st->tn;
    g.bplanes = inverse ? st->inv_bplanes : nullptr;
    g.stall = (!inverse && st->inject_stall) ? 1 : 0;
    g.bplane_bytes = inverse ? (long long)st->inv_bplane_bytes : 0;
    // forward B: the Fourier workspace, problem (m, parity) at rows
    // (2 m + parity) Jh .. + Jh - 1 of a [2 (N + 1) Jh][C] matrix; tiled
    // copies need 16-byte aligned rows (C a multiple of 4 floats)
    if (!inverse && (g.C & 3) == 0 && ((uintptr_t)B & 15) == 0 &&
        encode_b_map(&g.bmap, B, g.C, 2LL * (p->N + 1) * p->Jh, st->tn))
        g.raw_bulk = 1;
    return g;
}

// Persistent grid: as many CTAs as are resident on the device at once (the
// per-SM count the shared memory and tensor memory are sized for), at most
// one per tile.
int persistent_ctas(int per_sm, int ntiles) {
    static std::mutex mu;
    static std::map<int, int> sms_of;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = sms_of.find(dev);
        if (it != sms_of.end()) sms = it->second;
    }
    if (sms == 0) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
        std::lock_guard<std::mutex> lk(mu);
        sms_of[dev] = sms;
    }
    return std::max(1, std::min(ntiles, sms * per_sm));
}

template <int T, bool F16, bool BPRE, int TN>
cudaError_t gemm_launch(const GemmArgs& g, int ntiles, cudaStream_t s) {
    constexpr int smem = Cfg<T, BPRE, TN>::SMEM;
    const void* fn = (const void*)split_gemm_kernel<T, F16, BPRE, TN>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e) return e;
    // inverse (short tiles, K <= N / 2 + 1): persistent CTAs, so that the
    // next tile's operands load during the last one's epilogue; forward (41
    // K steps per tile at T639): one CTA per tile, which the hardware
    // schedules in list order, so that the column tiles sharing a P~ tile
    // run together and that tile comes from L2 after its first read
    const int nctas = BPRE ? persistent_ctas(Wid<TN>::CTAS_PER_SM, ntiles) : ntiles;
    split_gemm_kernel<T, F16, BPRE, TN><<<nctas, NTHREADS, smem, s>>>(g);
    note_launch();
    return cudaGetLastError();
}

// Variant index: bit 0 three terms, bit 1 FP16, bit 2 pre-split B, bit 3 TN = 64.
int variant(int terms, bool f16, bool bpre, int tn) {
    return (terms == 3 ? 1 : 0) | (f16 ? 2 : 0) | (bpre ? 4 : 0) | (tn == 64 ? 8 : 0);
}

#define SHT_VARIANTS(F)                                                                       \
    {F<2, false, false, 128>, F<3, false, false, 128>, F<2, true, false, 128>,                \
     F<3, true, false, 128>,  F<2, false, true, 128>,  F<3, false, true, 128>,                \
     F<2, true, true, 128>,   F<3, true, true, 128>,   F<2, false, false, 64>,                \
     F<3, false, false, 64>,  F<2, true, false, 64>,   F<3, true, false, 64>,                 \
     F<2, false, true, 64>,   F<3, false, true, 64>,   F<2, true, true, 64>,                  \
     F<3, true, true, 64>}

cudaError_t launch_gemm_variant(int v, const GemmArgs& g, int ntiles, cudaStream_t s) {
    using Fn = cudaError_t (*)(const GemmArgs&, int, cudaStream_t);
    static const Fn tab[16] = SHT_VARIANTS(gemm_launch);
    return tab[v](g, ntiles, s);
}

// Inverse B (the spectrum): column maxima for FP16, then the term planes.
cudaError_t launch_split_b_inverse(const sht_plan_s* p, const void* spec, void* work,
                                   cudaStream_t s) {
    const SplitTables* st = p->split;
    const int C = 2 * p->F, nct = (C + st->tn - 1) / st->tn;
    cudaError_t e;
    if (st->fp16 && (e = launch_colmax_inverse(p, spec, s))) return e;
    const dim3 grid(2 * (p->N + 1), (C + 127) / 128);
    const size_t smem = (size_t)std::max(st->inv_max_nkt, 1) * TK * sizeof(float2);
    const float* B = static_cast<const float*>(spec);
    float* O = static_cast<float*>(work);
    const unsigned* cm = p->d_colmax ? p->d_colmax + C : nullptr;
    const long long pb = (long long)st->inv_bplane_bytes;
    using Fn = void (*)(const float*, const SplitProb*, int, int, const unsigned*,
                        unsigned char*, long long, const double*, int, int, int, float*);
    static const Fn tab[8] = {split_b_kernel<2, false, 128>, split_b_kernel<3, false, 128>,
                              split_b_kernel<2, true, 128>,  split_b_kernel<3, true, 128>,
                              split_b_kernel<2, false, 64>,  split_b_kernel<3, false, 64>,
                              split_b_kernel<2, true, 64>,   split_b_kernel<3, true, 64>};
    const Fn k = tab[(variant(st->terms, st->fp16, false, st->tn) & 3) | (st->tn == 64 ? 4 : 0)];
    k<<<grid, 256, smem, s>>>(B, st->d_probs_inv, C, nct, cm, st->inv_bplanes, pb, p->d_pnm,
                              p->ldp, p->N, p->Jh, O);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gemm(const sht_plan_s* p, bool inverse, const void* B, void* O,
                        cudaStream_t s) {
    const SplitTables* st = p->split;
    const GemmArgs g = make_gemm_args(p, inverse, B, O);
    const int ntiles = inverse ? st->ntiles_inv : st->ntiles_fwd;
    if (inverse) {
        // the spectrum is split once per call, then every row tile loads it
        // (this pass also writes the Equator row, which no tile covers)
        const cudaError_t e = launch_split_b_inverse(p, B, O, s);
        if (e || ntiles == 0) return e;
        return launch_gemm_variant(variant(st->terms, st->fp16, true, st->tn), g, ntiles, s);
    }
    // forward: the FFT kernel gathered the column maxima of its output (FP16)
    if (ntiles == 0) return cudaSuccess;
    return launch_gemm_variant(variant(st->terms, st->fp16, false, st->tn), g, ntiles, s);
}

}  // namespace

cudaError_t split_tables_create(sht_plan_s* p, cudaStream_t s) {
    SplitTables* st = new (std::nothrow) SplitTables();
    if (!st) return cudaErrorMemoryAllocation;
    p->split = st;
    st->terms = terms_of(p->prec);
    st->fp16 = p->prec == SHT_FP16X2 || p->prec == SHT_FP16X3;
    // failure-detection tests: the forward GEMM's first CTA never arms its
    // first stage, so its bounded waits run out and the plan's status word
    // records SHT_ERR_TIMEOUT (no fault, no hang)
    {
        const char* v = getenv("SHT_INJECT_STALL");
        st->inject_stall = (v && v[0] == '1') ? 1 : 0;
    }
    const int N = p->N, Jh = p->Jh, C = 2 * p->F;
    const int nprob = 2 * (N + 1);
    std::vector<SplitProb> pf, pi;
    std::vector<int4> tf, ti;
    long long fwd_bytes = 0, inv_bytes = 0;
    build_split_lists(N, Jh, C, TN_MAX, 0, st->jmin, pf, pi, tf, ti, fwd_bytes, inv_bytes);
    st->fwd_plane_bytes = (size_t)(fwd_bytes + 255) / 256 * 256;
    st->inv_plane_bytes = (size_t)(inv_bytes + 255) / 256 * 256;
    st->ntiles_fwd = (int)tf.size();
    st->ntiles_inv = (int)ti.size();
    cudaError_t e;
    if ((e = cudaMalloc(&st->fwd_planes, st->fwd_plane_bytes * st->terms + 256)) != cudaSuccess ||
        (e = cudaMalloc(&st->inv_planes, st->inv_plane_bytes * st->terms + 256)) != cudaSuccess ||
        (e = cudaMalloc(&st->d_probs_fwd, nprob * sizeof(SplitProb))) != cudaSuccess ||
        (e = cudaMalloc(&st->d_probs_inv, nprob * sizeof(SplitProb))) != cudaSuccess ||
        (e = cudaMalloc(&st->d_tiles_fwd, (tf.size() + 1) * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&st->d_tiles_inv, (ti.size() + 1) * sizeof(int4))) != cudaSuccess) {
        set_error("split tables: %s", cudaGetErrorString(e));
        return e;
    }
    if (st->fp16) {
        const size_t rf = (size_t)(pf.back().rs_off + pf.back().R8);
        const size_t ri = (size_t)(pi.back().rs_off + pi.back().R8);
        if ((e = cudaMalloc(&st->rs_fwd, (rf + 1) * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&st->rs_inv, (ri + 1) * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_colmax, 2 * (size_t)C * sizeof(unsigned))) != cudaSuccess) {
            set_error("split scales: %s", cudaGetErrorString(e));
            return e;
        }
    }
    {
        // laid out for the widest tiles: the 64-wide layout needs no more
        const int nct = (C + TN_MAX - 1) / TN_MAX;
        const SplitProb& last = pi.back();
        st->inv_bplane_bytes = (size_t)((last.bt_off +
                                         (long long)last.nkt * nct * Wid<TN_MAX>::B_TILE_BYTES +
                                         255) / 256 * 256);
        for (const SplitProb& v : pi) st->inv_max_nkt = std::max(st->inv_max_nkt, v.nkt);
        if ((e = cudaMalloc(&st->inv_bplanes, st->inv_bplane_bytes * st->terms + 256)) !=
            cudaSuccess) {
            set_error("split spectrum planes: %s", cudaGetErrorString(e));
            return e;
        }
    }
    // rows of A beyond R8 inside a 128-row tile are never copied; zero the
    // planes so K padding and row padding read as zero
    if ((e = cudaMemsetAsync(st->fwd_planes, 0, st->fwd_plane_bytes * st->terms, s)) ||
        (e = cudaMemsetAsync(st->inv_planes, 0, st->inv_plane_bytes * st->terms, s)) ||
        (e = cudaMemcpyAsync(st->d_probs_fwd, pf.data(), nprob * sizeof(SplitProb),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(st->d_probs_inv, pi.data(), nprob * sizeof(SplitProb),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(st->d_tiles_fwd, tf.data(), tf.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(st->d_tiles_inv, ti.data(), ti.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, s)))
        return e;
    if (st->fp16) {
        split_table_f16_kernel<<<nprob, 256, 0, s>>>(p->d_pnm, p->ldp, N, Jh, st->d_probs_fwd, 0,
                                                    st->terms, st->fwd_planes,
                                                    (long long)st->fwd_plane_bytes, st->rs_fwd);
        split_table_f16_kernel<<<nprob, 256, 0, s>>>(p->d_pnm, p->ldp, N, Jh, st->d_probs_inv, 1,
                                                    st->terms, st->inv_planes,
                                                    (long long)st->inv_plane_bytes, st->rs_inv);
    } else {
        split_table_kernel<<<nprob, 256, 0, s>>>(p->d_pnm, p->ldp, N, Jh, st->d_probs_fwd, 0,
                                                st->terms, st->fwd_planes,
                                                (long long)st->fwd_plane_bytes);
        split_table_kernel<<<nprob, 256, 0, s>>>(p->d_pnm, p->ldp, N, Jh, st->d_probs_inv, 1,
                                                st->terms, st->inv_planes,
                                                (long long)st->inv_plane_bytes);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // host vectors above must outlive the copies
}

void split_tables_destroy(sht_plan_s* p) {
    SplitTables* st = p->split;
    if (!st) return;
    void* ptrs[] = {st->fwd_planes, st->inv_planes, st->d_probs_fwd, st->d_probs_inv,
                    st->d_tiles_fwd, st->d_tiles_inv, st->rs_fwd, st->rs_inv, p->d_colmax,
                    st->inv_bplanes};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete st;
    p->split = nullptr;
    p->d_colmax = nullptr;
}

// Rebuild the problem and tile lists of a split plan for column tiles
// TN = tn (64 or 128) and the reduced-transform ranges st->jmin.  The term
// planes and row scales depend on neither; the pre-split spectrum planes
// were sized for the widest tiles.  Synchronises the device: kernels in
// flight may still read the old lists.
cudaError_t split_rebuild_lists(sht_plan_s* p, int tn) {
    SplitTables* st = p->split;
    std::vector<SplitProb> pf, pi;
    std::vector<int4> tf, ti;
    long long fb = 0, ib = 0;
    build_split_lists(p->N, p->Jh, 2 * p->F, tn, 0, st->jmin, pf, pi, tf, ti, fb, ib);
    int4 *dtf = nullptr, *dti = nullptr;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc(&dtf, (tf.size() + 1) * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&dti, (ti.size() + 1) * sizeof(int4));
    if (e == cudaSuccess)
        e = cudaMemcpy(dtf, tf.data(), tf.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dti, ti.data(), ti.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(st->d_probs_fwd, pf.data(), pf.size() * sizeof(SplitProb),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(st->d_probs_inv, pi.data(), pi.size() * sizeof(SplitProb),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (dtf) cudaFree(dtf);
        if (dti) cudaFree(dti);
        return e;
    }
    cudaFree(st->d_tiles_fwd);
    cudaFree(st->d_tiles_inv);
    st->d_tiles_fwd = dtf;
    st->d_tiles_inv = dti;
    st->ntiles_fwd = (int)tf.size();
    st->ntiles_inv = (int)ti.size();
    st->tn = tn;
    return cudaSuccess;
}

cudaError_t split_set_tile_width(sht_plan_s* p, int tn) {
    SplitTables* st = p->split;
    if (!st || (tn != 64 && tn != 128)) return cudaErrorInvalidValue;
    if (st->tn == tn) return cudaSuccess;
    return split_rebuild_lists(p, tn);
}

namespace {
// First northern node (0 = nearest the pole) at which some P~_n^m of the
// problem's parity reaches thr in magnitude; Jh if none.  One block per
// (m, parity) problem, threads over the nodes.
__global__ void jmin_kernel(const double* __restrict__ pnm, int ldp, int N, int Jh, double thr,
                            int* out) {
    __shared__ int first;
    const int p = blockIdx.x, m = p >> 1, q = p & 1;
    if (threadIdx.x == 0) first = Jh;
    __syncthreads();
    const size_t row0 = coef_offset(N, m) + q;
    const int d = N - m - q;
    const int R = d >= 0 ? d / 2 + 1 : 0;
    for (int j = threadIdx.x; j < Jh; j += blockDim.x) {
        bool sig = false;
        for (int r = 0; r < R && !sig; ++r) sig = fabs(pnm[(row0 + 2 * (size_t)r) * ldp + j]) >= thr;
        if (sig) atomicMin(&first, j);
    }
    __syncthreads();
    if (threadIdx.x == 0) out[p] = first;
}
}  // namespace

// jmin for every (m, parity) problem of the plan into d_out[2(N+1)].
cudaError_t launch_jmin(const sht_plan_s* p, int* d_out, cudaStream_t s) {
    jmin_kernel<<<2 * (p->N + 1), 256, 0, s>>>(p->d_pnm, p->ldp, p->N, p->Jh, 1e-16, d_out);
    return cudaGetLastError();
}

// Reduced transform (Sec. 4.1: terms with |P~| < 1e-16 neglected, as in the
// paper's own runs), for split plans: on = 1 finds the per-problem ranges
// and rebuilds the lists, on = 0 restores the full transform.
cudaError_t split_set_reduced(sht_plan_s* p, int on) {
    SplitTables* st = p->split;
    if (!st) return cudaErrorInvalidValue;
    if ((on != 0) == !st->jmin.empty()) return cudaSuccess;
    const int nprob = 2 * (p->N + 1);
    if (on) {
        int* d = nullptr;
        cudaError_t e = cudaMalloc(&d, nprob * sizeof(int));
        if (e != cudaSuccess) return e;
        e = launch_jmin(p, d, nullptr);
        std::vector<int> h(nprob);
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), d, nprob * sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(d);
        if (e != cudaSuccess) return e;
        st->jmin = h;
    } else {
        st->jmin.clear();
    }
    return split_rebuild_lists(p, st->tn);
}

int split_tile_width(const sht_plan_s* p) { return p->split ? p->split->tn : 0; }

// Tiles of a group of split plans (same term count), heaviest first: every
// tile's K loop has nkt steps.  Returns the host list.
void split_group_tiles(sht_plan_s* const* plans, int n, bool inverse, std::vector<int4>& out) {
    std::vector<std::pair<int, int4>> all;
    for (int q = 0; q < n; ++q) {
        const sht_plan_s* p = plans[q];
        std::vector<SplitProb> pf, pi;
        std::vector<int4> tf, ti;
        long long fb, ib;
        build_split_lists(p->N, p->Jh, 2 * p->F, p->split->tn, q, p->split->jmin, pf, pi, tf,
                          ti, fb, ib);
        const std::vector<SplitProb>& pr = inverse ? pi : pf;
        for (const int4& t : inverse ? ti : tf) {
            const SplitProb& v = pr[t.x];
            all.push_back({t.y < v.mt0 ? 0 : v.nkt - v.kt0, t});
        }
    }
    std::stable_sort(all.begin(), all.end(),
                     [](const std::pair<int, int4>& a, const std::pair<int, int4>& b) {
                         return a.first > b.first;
                     });
    out.clear();
    for (auto& e : all) out.push_back(e.second);
}

template <int T, bool F16, bool BPRE, int TN>
cudaError_t group_launch(const GemmGroup& G, int ntiles, cudaStream_t s) {
    constexpr int smem = Cfg<T, BPRE, TN>::SMEM;
    const void* fn = (const void*)split_gemm_group_kernel<T, F16, BPRE, TN>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e) return e;
    // inverse (short tiles, K <= N / 2 + 1): persistent CTAs, so that the
    // next tile's operands load during the last one's epilogue; forward (41
    // K steps per tile at T639): one CTA per tile, which the hardware
    // schedules in list order, so that the column tiles sharing a P~ tile
    // run together and that tile comes from L2 after its first read
    const int nctas = BPRE ? persistent_ctas(Wid<TN>::CTAS_PER_SM, ntiles) : ntiles;
    split_gemm_group_kernel<T, F16, BPRE, TN><<<nctas, NTHREADS, smem, s>>>(G);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_split_group(sht_plan_s* const* plans, int n, bool inverse,
                               const void* const* in, void* const* out, const int4* tiles,
                               int ntiles, cudaStream_t s) {
    GemmGroup G;
    G.n = n;
    G.ntiles = ntiles;
    G.tiles = tiles;
    for (int q = 0; q < n; ++q) G.a[q] = make_gemm_args(plans[q], inverse, in[q], out[q]);
    const SplitTables* st = plans[0]->split;
    if (inverse)
        for (int q = 0; q < n; ++q) {
            const cudaError_t e = launch_split_b_inverse(plans[q], in[q], out[q], s);
            if (e) return e;
        }
    if (ntiles == 0) return cudaSuccess;
    using Fn = cudaError_t (*)(const GemmGroup&, int, cudaStream_t);
    static const Fn tab[16] = SHT_VARIANTS(group_launch);
    return tab[variant(st->terms, st->fp16, inverse, st->tn)](G, ntiles, s);
}

cudaError_t launch_legendre_fwd_split(const sht_plan_s* p, const void* work, void* spec,
                                      cudaStream_t s) {
    return launch_gemm(p, false, work, spec, s);
}

cudaError_t launch_legendre_inv_split(const sht_plan_s* p, const void* spec, void* work,
                                      cudaStream_t s) {
    return launch_gemm(p, true, spec, work, s);
}

int split_status_read_and_clear(const sht_plan_s* p) {
    if (!p->d_status) return 0;
    int v = 0;
    if (cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    if (v) cudaMemset(p->d_status, 0, sizeof(int));
    return v;
}

}  // namespace sht

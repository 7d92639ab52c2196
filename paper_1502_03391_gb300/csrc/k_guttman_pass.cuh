// K1: the fused all-pairs pass of one Guttman transform (Eq. B, Eq. update,
// Remark faststress), upper triangle of every Delta_l only.
//
// For every unordered pair {i, j} (i < j) of modality l the pass forms
//     d_ij = ||x_i - x_j||,  b_ij = Delta_ij / d_ij  (0 when d_ij = 0, Eq. B),
// and adds   b_ij (x_i - x_j)  to row i and  b_ij (x_j - x_i)  to row j of B'_l X_l
// (B'_l = B_l / w_ll; since B_l's diagonal is minus its off-diagonal row sum,
// (B_l X_l)_i = w_ll sum_j b_ij (x_i - x_j)), plus w_ll (s_l Delta_ij - d_ij)^2 to the
// fidelity.  Reading the symmetric Delta once per unordered pair is the half of
// Remark faststress's 1/2 ||Delta_i - d(X^(i))||_F^2.
//
// Work layout (GB300): a persistent grid of G CTAs, CTA b owning the contiguous range
// [b*T/G, (b+1)*T/G) of RB x CW sub-tiles in walk order (row block I visits column
// sub-tiles from its diagonal to n).  Each sub-tile is staged HBM -> shared memory by
// one 2-D TMA (cp.async.bulk.tensor) into a STAGES-deep ring completed on mbarriers;
// the last warp to finish reading a stage (shared-memory counter) issues its refill.
// Warp w owns R consecutive rows of the row block (x_i and the row accumulators stay in
// registers for the whole walk segment; the next walk's x_i are fetched one sub-tile
// ahead); lane owns C consecutive columns of every sub-tile.  Column accumulators go
// through a small ring of shared-memory slots; each warp reduces its share of the
// previous sub-tile's columns in a fixed order and writes one partial per (sub-tile,
// column).  Row accumulators are reduced across the warp (reduce-scatter butterfly) at
// walk-segment ends.  Warps never meet at a CTA-wide barrier inside the loop; they
// synchronise only through mbarriers and the stage counters, with one sub-tile of
// slack.  K2 sums every partial in a fixed order, so results are bitwise reproducible
// run to run.  Every wait is bounded.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"

namespace fjofc {

template <int D> struct K1Cfg;
// Largest embedding dimension that uses the column-strip layout of the sub-tile (every
// warp owns a strip of columns, so column partials are reduced inside the warp); larger
// d use the row-band layout (every warp owns a band of rows, column partials reduced
// across the warps through shared memory).
#ifndef FJOFC_K1_STRIP_MAX_D
#define FJOFC_K1_STRIP_MAX_D 4
#endif
// rows/thread, cols/lane, compute warps, pipeline stages (float32)
#define FJOFC_K1CFG(D_, R_, C_, W_, S_)                                                     \
    template <> struct K1Cfg<D_> {                                                          \
        static constexpr int R = R_, C = C_, CWARPS = W_, STAGES = S_;                      \
        static constexpr bool STRIP = (D_ <= FJOFC_K1_STRIP_MAX_D);                         \
    };
// The d <= 4 tile can be overridden at build time (tuning sweeps).
#ifndef FJOFC_K1_SMALLD_R
#define FJOFC_K1_SMALLD_R 16
#endif
#ifndef FJOFC_K1_SMALLD_C
#define FJOFC_K1_SMALLD_C 4
#endif
#ifndef FJOFC_K1_SMALLD_WARPS
#define FJOFC_K1_SMALLD_WARPS 8
#endif
#ifndef FJOFC_K1_SMALLD_STAGES
#define FJOFC_K1_SMALLD_STAGES 3
#endif
// smallest embedding dimension whose x_j are staged in shared memory per sub-tile
// (below it every warp loads its columns' x_j from L2 one sub-tile ahead)
#ifndef FJOFC_K1_XSTAGE_MIN_D
#define FJOFC_K1_XSTAGE_MIN_D 1
#endif
// resident CTAs per SM the all-pairs kernels are compiled for (register budget)
#ifndef FJOFC_K1_MINB
#define FJOFC_K1_MINB 1
#endif
#define FJOFC_SMALLD FJOFC_K1_SMALLD_R, FJOFC_K1_SMALLD_C, FJOFC_K1_SMALLD_WARPS, FJOFC_K1_SMALLD_STAGES
#define FJOFC_K1CFG_X(...) FJOFC_K1CFG(__VA_ARGS__)
FJOFC_K1CFG_X(1, FJOFC_SMALLD)    // default: 128 x 128 sub-tile, 64 KB at float32
FJOFC_K1CFG_X(2, FJOFC_SMALLD)
FJOFC_K1CFG_X(3, FJOFC_SMALLD)
FJOFC_K1CFG(4, 16, 4, 8, 2)       // two stages: three and the staged rows exceed 227 KB
FJOFC_K1CFG(5, 8, 4, 8, 3)        // 64 x 128, 32 KB
FJOFC_K1CFG(6, 8, 4, 8, 3)
FJOFC_K1CFG(7, 8, 2, 8, 5)        // 64 x 64, 16 KB
FJOFC_K1CFG(8, 8, 2, 8, 5)
FJOFC_K1CFG(9, 4, 2, 8, 6)        // 32 x 64, 8 KB
FJOFC_K1CFG(10, 4, 2, 8, 6)
FJOFC_K1CFG(11, 4, 2, 8, 6)
FJOFC_K1CFG(12, 4, 2, 8, 6)
FJOFC_K1CFG(13, 4, 2, 8, 6)
FJOFC_K1CFG(14, 2, 2, 8, 8)       // 16 x 64, 4 KB
FJOFC_K1CFG(15, 2, 2, 8, 8)
FJOFC_K1CFG(16, 2, 2, 8, 8)
#undef FJOFC_K1CFG_X
#undef FJOFC_K1CFG

// Rows of the walk in shared memory, per warp: row r's coordinates as (x_k, x_k) pairs,
// XB = ceil(D/2) float4 per row ((x_0, x_0, x_1, x_1), (x_2, x_2, x_3, x_3), ...), so that a
// packed (two-column) operation can take x_i as one operand; all lanes of the warp read
// the same address (a broadcast).
template <int D>
struct XiBcast {
    static constexpr int XB = (D + 1) / 2;
};

// Dynamic shared memory a CTA of the all-pairs kernels may use: the 227 KB per-CTA limit
// less 2 KB for the kernels' static shared variables.
constexpr size_t kK1SmemBudget = 232448 - 2048;

template <int D, typename TD>
struct K1Shape {
    static constexpr int R = K1Cfg<D>::R, C = K1Cfg<D>::C, CWARPS = K1Cfg<D>::CWARPS;
    static constexpr bool STRIP = K1Cfg<D>::STRIP;
    static constexpr int SLOTS = 2;                    // column-partial ring (row-band layout)
    static constexpr int NT = CWARPS * 32;
    static constexpr int RB = CWARPS * R;
    static constexpr int CW = 32 * C;
    static constexpr int STAGE_ELEMS = RB * CW;
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(TD);
    // column-strip layout: a stage is BOXES TMA boxes of RB rows x 128 bytes, each stored
    // with the 128-byte swizzle (16-byte chunk j of row r at chunk j ^ (r & 7)), so that the
    // eight rows a warp reads at once fall on different banks
    static constexpr int BOX_ELEMS = 128 / int(sizeof(TD));
    static constexpr int BOXES = STRIP ? (CW * int(sizeof(TD))) / 128 : 1;
    static constexpr int SW = CW / CWARPS;             // columns of a warp's strip
    static_assert(!STRIP || (CWARPS == 8 && SW == 4 * C && BOXES >= 1 && (CW * sizeof(TD)) % 128 == 0),
                  "column-strip layout: 8 warps, 4 column groups of C per warp, whole 128-byte boxes");
    static constexpr size_t PHB_FLOATS = size_t(2) * FJOFC_MAX_M * 32;   // phase B's staging of one unit
    static constexpr size_t RED_FLOATS =
        STRIP ? (size_t(CWARPS) * RB * D > PHB_FLOATS ? size_t(CWARPS) * RB * D : PHB_FLOATS)   // row hand-off
              : size_t(SLOTS) * CWARPS * D * CW;
    static constexpr size_t ALIGN = STRIP ? 1024 : 128;
    // x_i of the walk as broadcast pairs (column-strip layout: one shared copy per walk
    // segment, two buffers)
    static constexpr int XROW_FLOATS = (STRIP ? 2 : 1) * CWARPS * R * XiBcast<D>::XB * 4;
    // every sub-tile's x_j (CW columns x d, a 16-byte aligned window) staged in shared
    // memory by the issuing warp (cp.async), STAGES uses ahead like Delta
    static constexpr bool XSTAGE = D >= FJOFC_K1_XSTAGE_MIN_D;
    static constexpr int XS_FLOATS = XSTAGE ? CW * D + 8 : 0;
    static constexpr size_t smem_for(int stages) {
        return size_t(stages) * STAGE_BYTES + RED_FLOATS * sizeof(float) + size_t(XROW_FLOATS) * sizeof(float) +
               size_t(stages) * XS_FLOATS * sizeof(float) + size_t(2 * stages + 2 * SLOTS) * 8 +
               size_t((stages + 1) & ~1) * 4 + 64 + ALIGN;
    }
    // 16-bit Delta halves the stage: keep about the same bytes in flight, as many stages
    // as fit in the budget
    static constexpr int STAGES_WANTED = sizeof(TD) == 4 ? K1Cfg<D>::STAGES : 2 * K1Cfg<D>::STAGES;
    static constexpr int fit_stages(int st) { return (st > 2 && smem_for(st) > kK1SmemBudget) ? fit_stages(st - 1) : st; }
    static constexpr int STAGES = fit_stages(STAGES_WANTED);
    static constexpr size_t SMEM = smem_for(STAGES);
    static_assert(SMEM <= kK1SmemBudget, "all-pairs tile does not fit in shared memory");
};

// Position of a sub-tile: modality l, walk position wp visiting row block I, sub-tile s
// of that walk (walk length L).
struct Cursor {
    int64_t t;
    int l, wp, I, s, L;
};

__device__ __forceinline__ void cursor_init(Cursor& c, int64_t t, const K1Params& p) {
    c.t = t;
    c.l = static_cast<int>(t / p.Tm);
    const int64_t r = t - int64_t(c.l) * p.Tm;
    int lo = 0, hi = p.nRB - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(p.walk_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    c.wp = lo;
    c.I = walk_row(lo, p.nRB);
    c.s = static_cast<int>(r - __ldg(p.walk_off + lo));
    c.L = static_cast<int>(__ldg(p.walk_off + lo + 1) - __ldg(p.walk_off + lo));
}

__device__ __forceinline__ void cursor_next(Cursor& c, const K1Params& p) {
    ++c.t;
    if (++c.s == c.L) {
        c.s = 0;
        if (++c.wp == p.nRB) { c.wp = 0; ++c.l; }
        c.I = walk_row(c.wp, p.nRB);
        if (c.l < p.m) c.L = static_cast<int>(__ldg(p.walk_off + c.wp + 1) - __ldg(p.walk_off + c.wp));
    }
}

// The pairs of one RB x CW sub-tile owned by this thread: rows r0 + warp*R + r (x_i from
// the warp's broadcast rows at shared address xib), columns c0 + lane*C + c (x_j, negated,
// in nxj: column pair cp holds columns 2cp and 2cp+1 as the two halves of a float2); the
// sub-tile's Delta at shared address tile.  Coordinates come in pre-divided by the
// modality's Delta scale s (x' = x / s, so d' = d / s and b = Delta'/d' = Delta/d).  Two
// columns are processed per instruction with Blackwell's packed float32 operations
// (add/mul/fma .f32x2: same rounding per element as the scalar operation, half the issue
// slots); the reciprocal square root stays scalar.  With q = -b_ij and e' = d'_ij -
// Delta'_ij (the packed forms take no negated operand, so the signs are arranged to need
// one negation of Delta per column pair): adds q (x'_i - x'_j) = -b_ij (x'_i - x'_j) to
// racc[r] (scalar, columns in order; the row flush negates it), q (x'_i - x'_j), the
// contribution to column j, to
// the column accumulators (two interleaved chains by row parity) and e'^2 to sf0/sf1 (per
// column parity halves).  The squared distance starts from FLT_MIN instead of 0: this
// changes no d^2 above 2^-102 and keeps rsqrt finite when x_i = x_j (then
// b (x_i - x_j) = 0, the d_ij = 0 rule of Eq. B, and the fidelity term is Delta'^2).
// MASKED: only pairs with i < j < n count (diagonal and ragged sub-tiles); otherwise
// every pair of the sub-tile is valid.
// Rows processed together by subtile_pairs: each step of the computation is written for
// RI rows side by side, so that the independent rows' dependency chains are interleaved.
#ifndef FJOFC_ROW_INTERLEAVE
#define FJOFC_ROW_INTERLEAVE 2
#endif

template <int D, typename TD, int R, int C, int CW, bool MASKED>
__device__ __forceinline__ void subtile_pairs(uint32_t tile, int warp, int lane, int r0, int c0, int n,
                                              uint32_t xib, const float2 (&nxj)[C / 2][D],
                                              float (&racc)[R][D], float2 (&cacc0)[C / 2][D],
                                              float2 (&cacc1)[C / 2][D], float2& sf0, float2& sf1) {
    static_assert(C % 2 == 0, "columns are processed in pairs");
    constexpr int CP = C / 2, XB = XiBcast<D>::XB;
    constexpr int RI = (R % FJOFC_ROW_INTERLEAVE == 0) ? FJOFC_ROW_INTERLEAVE : 1;
    const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int cp = 0; cp < CP; ++cp)
#pragma unroll
        for (int k = 0; k < D; ++k) { cacc0[cp][k] = make_float2(0.f, 0.f); cacc1[cp][k] = make_float2(0.f, 0.f); }
    sf0 = make_float2(0.f, 0.f);
    sf1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int rb = 0; rb < R; rb += RI) {
        float2 xb[RI][2 * XB];
        float dl[RI][C];
#pragma unroll
        for (int h = 0; h < RI; ++h) {
            const int r = rb + h;
#pragma unroll
            for (int x = 0; x < XB; ++x) {
                const float4 v = lds_f4(xib + 16 * (r * XB + x));
                xb[h][2 * x] = make_float2(v.x, v.y);
                xb[h][2 * x + 1] = make_float2(v.z, v.w);
            }
            lds_delta_row<TD, C>(tile + uint32_t(((warp * R + r) * CW + lane * C) * sizeof(TD)), dl[h]);
        }
#pragma unroll
        for (int cp = 0; cp < CP; ++cp) {
            float2 ndel[RI], diff[RI][D], d2[RI], rinv[RI], q[RI], e[RI];
#pragma unroll
            for (int h = 0; h < RI; ++h) {
                ndel[h] = __fmul2_rn(make_float2(dl[h][2 * cp], dl[h][2 * cp + 1]), neg1);
                d2[h] = make_float2(FLT_MIN, FLT_MIN);
            }
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int h = 0; h < RI; ++h) {
                    diff[h][k] = __fadd2_rn(xb[h][k], nxj[cp][k]);
                    d2[h] = __ffma2_rn(diff[h][k], diff[h][k], d2[h]);
                }
#pragma unroll
            for (int h = 0; h < RI; ++h) rinv[h] = make_float2(rsqrt_approx(d2[h].x), rsqrt_approx(d2[h].y));
#pragma unroll
            for (int h = 0; h < RI; ++h) {
                q[h] = __fmul2_rn(ndel[h], rinv[h]);             // -b
                e[h] = __ffma2_rn(d2[h], rinv[h], ndel[h]);      // d - Delta
                if (MASKED) {
                    const int i = r0 + warp * R + rb + h;
                    const int j = c0 + lane * C + 2 * cp;
                    const bool v0 = (j > i) && (j < n), v1 = (j + 1 > i) && (j + 1 < n);
                    q[h].x = v0 ? q[h].x : 0.f;
                    e[h].x = v0 ? e[h].x : 0.f;
                    q[h].y = v1 ? q[h].y : 0.f;
                    e[h].y = v1 ? e[h].y : 0.f;
                }
            }
#pragma unroll
            for (int h = 0; h < RI; ++h) {
                if ((rb + h) & 1) sf1 = __ffma2_rn(e[h], e[h], sf1); else sf0 = __ffma2_rn(e[h], e[h], sf0);
            }
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int h = 0; h < RI; ++h) {
                    const int r = rb + h;
                    racc[r][k] = fmaf(q[h].x, diff[h][k].x, racc[r][k]);
                    racc[r][k] = fmaf(q[h].y, diff[h][k].y, racc[r][k]);
                    if (r & 1) cacc1[cp][k] = __ffma2_rn(q[h], diff[h][k], cacc1[cp][k]);
                    else cacc0[cp][k] = __ffma2_rn(q[h], diff[h][k], cacc0[cp][k]);
                }
        }
    }
}

// Sum of v[0..V-1] over the 32 lanes as a reduce-scatter butterfly: at each level a lane
// keeps half of its values (or all of them when the count is odd) and adds its partner's.
// On return v[0..F-1] holds the totals of indices base .. base+F-1, and exactly one lane
// per index has writer == true.  Every total is formed by the same pairing tree as
// warp_sum_f32 (partners xor 16, 8, 4, 2, 1), with V/2 + V/4 + ... shuffles instead of 5V.
template <int V, int OFF>
struct WarpScatter {
    static __device__ __forceinline__ void run(float* v, int lane, int& base, bool& writer) {
        if constexpr (OFF > 0) {
            if constexpr (V % 2 == 0) {
                constexpr int H = V / 2;
                const bool up = (lane & OFF) != 0;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float send = up ? v[h] : v[h + H];
                    const float keep = up ? v[h + H] : v[h];
                    v[h] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
                }
                if (up) base += H;
                WarpScatter<H, OFF / 2>::run(v, lane, base, writer);
            } else {
#pragma unroll
                for (int h = 0; h < V; ++h) v[h] += __shfl_xor_sync(0xffffffffu, v[h], OFF);
                if (lane & OFF) writer = false;
                WarpScatter<V, OFF / 2>::run(v, lane, base, writer);
            }
        }
    }
};
template <int V, int OFF>
struct WarpScatterCount {
    static constexpr int value = OFF == 0 ? V : (V % 2 == 0 ? WarpScatterCount<V / 2, OFF / 2>::value
                                                            : WarpScatterCount<V, OFF / 2>::value);
};
template <int V>
struct WarpScatterCount<V, 0> {
    static constexpr int value = V;
};

// Staging of the next walk's x_i: plain L2 loads (ld.global.cg; the iterate may have been
// written earlier in the same launch) issued one sub-tile ahead into PER_LANE registers,
// stored to this warp's shared-memory rows when the walk changes.
template <int R, int D>
struct RowStage {
    static constexpr int PER_LANE = (R * D + 31) / 32;
    float v[PER_LANE];
};

// Shared-memory carve-up and TMA ring state of one CTA of the all-pairs pass.  The ring
// runs over a global sequence qg = 0, 1, ... of sub-tile uses; use qg is sub-tile
// t_begin + (qg mod nq) of the CTA's range (the range repeats every pass).  The warp that
// releases a stage last issues the use STAGES ahead, which at the end of a pass is one of
// the next pass's first sub-tiles (Delta does not change between passes).
template <int D, typename TD>
struct K1Ring {
    using S = K1Shape<D, TD>;
    TD* stages;
    float* red;            // [SLOTS][CWARPS][D][CW] column accumulators
    float* xrow;           // [CWARPS][R][XB] float4 x_i of the current walk as (x_k, x_k) pairs
    float* xs;             // [STAGES][XS_FLOATS]    staged x_j (XSTAGE)
    uint64_t* full;        // [STAGES]
    uint64_t* xfull;       // [STAGES] x_j landed (XSTAGE)
    uint64_t* rfull;       // [SLOTS]
    uint64_t* rempty;      // [SLOTS]
    int* released;         // [STAGES] releases so far (monotone)
    Cursor* pc_start;      // cursor of the range's first sub-tile (read when the ring wraps)
    int* xissued;          // uses whose x_j have been issued (monotone)
    int* red_cnt;          // arrivals at segment ends summed inside a pass (column-strip layout)
    uint64_t* red_full;    // those arrivals (count CWARPS)
    uint64_t* red_empty;   // the row buffer summed (count 1)
    int nred;              // segments summed inside a pass so far (the same in every thread)
    int* issued;           // ring uses issued so far
    int* abort_flag;       // set by a warp whose bounded wait gave up
    Cursor pc;             // cursor of the next use to issue (every thread keeps a copy)
    int pc_local;
    int packed;            // Delta in the packed band layout
    int64_t n;
    int64_t t_begin;
    int nq;
    int64_t total_q;

    int nflush;            // row hand-offs done so far (column-strip layout; the same in every thread)

    __device__ __forceinline__ void carve(unsigned char* smem_raw) {
        // generic -> shared offsets: align the shared-window address (the 128-byte swizzle
        // pattern repeats every 1024 bytes of shared address)
        const uint32_t a0 = smem_u32(smem_raw);
        const uint32_t a1 = (a0 + uint32_t(S::ALIGN) - 1) & ~uint32_t(S::ALIGN - 1);
        unsigned char* smem = smem_raw + (a1 - a0);
        stages = reinterpret_cast<TD*>(smem);
        red = reinterpret_cast<float*>(smem + size_t(S::STAGES) * S::STAGE_BYTES);
        xrow = red + S::RED_FLOATS;
        xs = xrow + S::XROW_FLOATS;
        full = reinterpret_cast<uint64_t*>(xs + size_t(S::STAGES) * S::XS_FLOATS);
        xfull = full + S::STAGES;
        rfull = xfull + S::STAGES;
        rempty = rfull + S::SLOTS;
        released = reinterpret_cast<int*>(rempty + S::SLOTS);
        pc_start = reinterpret_cast<Cursor*>(released + ((S::STAGES + 1) & ~1));
        xissued = reinterpret_cast<int*>(pc_start + 1);
        red_cnt = xissued + 1;
        red_full = reinterpret_cast<uint64_t*>(xissued + 2);
        red_empty = red_full + 1;
    }

    __device__ __forceinline__ void issue(const TMaps& tm, int64_t qg) { issue_at(tm, qg, pc); }

    // Delta of use qg, the sub-tile at cursor c, into its stage (one thread).
    __device__ __forceinline__ void issue_at(const TMaps& tm, int64_t qg, const Cursor& c) {
        const int stage = int(qg % S::STAGES);
        atomicMax(issued, int(qg + 1));
        const uint32_t bar = smem_u32(&full[stage]);
        mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
        const uint32_t dst = smem_u32(stages + size_t(stage) * S::STAGE_ELEMS);
        // the sub-tile's first element: Delta[I RB][I RB + s CW], or its packed position
        int64_t x0 = int64_t(c.I) * S::RB + int64_t(c.s) * S::CW, y0 = int64_t(c.I) * S::RB;
        if (packed) pack_pos(n, int(sizeof(TD)), y0, x0, x0, y0);
        if constexpr (S::STRIP) {
            // BOXES boxes of 128 bytes x RB rows; x is a multiple of 16 bytes
#pragma unroll
            for (int bx = 0; bx < S::BOXES; ++bx)
                tma_load_2d(dst + uint32_t(bx) * S::RB * 128u, &tm.map[c.l], int(x0) + bx * S::BOX_ELEMS, int(y0), bar);
        } else {
            tma_load_2d(dst, &tm.map[c.l], int(x0), int(y0), bar);
        }
    }

    // x_j of use u (cursor c) into its stage, by all 32 lanes of one warp: the 16-byte
    // aligned window of X (16-byte aligned) that holds the CW columns' coordinates.  Inside
    // X: one bulk copy completing on xfull (lane 0 arrives with its byte count, the other
    // lanes plainly); at the end of X: 16-byte cp.async copies cut there (zero-filled
    // beyond), each lane arriving on xfull once its copies have landed.  32 arrivals
    // either way.
    __device__ __forceinline__ void issue_x(const K1Params& p, const float* X, int64_t u, const Cursor& c) {
        const int lane = threadIdx.x & 31;
        const int stage = int(u % S::STAGES);
        const int64_t total = int64_t(p.m) * p.n * D;
        const int64_t start = (int64_t(c.l) * p.n + c.I * S::RB + c.s * S::CW) * D;
        const int64_t base = start & ~int64_t(3);
        const int nch = (int(start - base) + S::CW * D + 3) / 4;
        float* dst = xs + size_t(stage) * S::XS_FLOATS;
        if (lane == 0) atomicMax(xissued, int(u + 1));
        if (base + 4 * int64_t(nch) <= total) {
            const uint32_t bar = smem_u32(&xfull[stage]);
            if (lane == 0) {
                mbar_arrive_expect_tx(bar, uint32_t(nch) * 16u);
                bulk_load(smem_u32(dst), X + base, uint32_t(nch) * 16u, bar);
            } else {
                mbar_arrive(bar);
            }
            return;
        }
        for (int k = lane; k < nch; k += 32) {
            const int64_t f = base + 4 * int64_t(k);
            const int64_t left = total - f;
            const int bytes = left >= 4 ? 16 : (left > 0 ? int(left) * 4 : 0);
            cp_async_16(smem_u32(dst + 4 * k), bytes ? static_cast<const void*>(X + f) : static_cast<const void*>(X),
                        bytes);
        }
        cp_async_arrive_noinc(smem_u32(&xfull[stage]));
    }

    __device__ __forceinline__ void advance(const K1Params& p) {
        if (++pc_local == nq) {
            pc_local = 0;
            pc = *pc_start;
        } else {
            cursor_next(pc, p);
        }
    }

    // Barrier set-up and the first STAGES uses (thread 0 issues; every thread advances its
    // cursor copy).  Ends with __syncthreads.
    __device__ __forceinline__ void start(const TMaps& tm, const K1Params& p, int64_t t_begin_, int nq_,
                                          int64_t total_q_, int* issued_, int* abort_) {
        issued = issued_;
        abort_flag = abort_;
        t_begin = t_begin_;
        nq = nq_;
        total_q = total_q_;
        pc_local = 0;
        nflush = 0;
        nred = 0;
        packed = p.packed;
        n = p.n;
        cursor_init(pc, t_begin, p);
        if (threadIdx.x == 0) {
            for (int s = 0; s < S::STAGES; ++s) {
                mbar_init(smem_u32(&full[s]), 1);
                if (S::XSTAGE) mbar_init(smem_u32(&xfull[s]), 32);
                released[s] = 0;
            }
            for (int s = 0; s < S::SLOTS; ++s) {
                mbar_init(smem_u32(&rfull[s]), S::CWARPS);
                mbar_init(smem_u32(&rempty[s]), S::CWARPS);
            }
            mbar_init(smem_u32(red_full), S::CWARPS);
            mbar_init(smem_u32(red_empty), 1);
            *red_cnt = 0;
            *abort_flag = 0;
            *issued = 0;
            *xissued = 0;
            *pc_start = pc;
            fence_barrier_init();
            for (int l = 0; l < p.m; ++l) tma_prefetch_desc(&tm.map[l]);
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int64_t q = 0; q < S::STAGES && q < total_q; ++q) {
                issue(tm, q);
                advance(p);
            }
        else
            for (int64_t q = 0; q < S::STAGES && q < total_q; ++q) advance(p);
        __syncthreads();
    }

    // Invalidate the ring's barriers once every copy has landed and every thread is past
    // its last wait (the caller's __syncthreads), so that start() may initialise them
    // again.  Thread 0 only.
    __device__ __forceinline__ void invalidate() {
        for (int s = 0; s < S::STAGES; ++s) {
            mbar_inval(smem_u32(&full[s]));
            if (S::XSTAGE) mbar_inval(smem_u32(&xfull[s]));
        }
        for (int s = 0; s < S::SLOTS; ++s) {
            mbar_inval(smem_u32(&rfull[s]));
            mbar_inval(smem_u32(&rempty[s]));
        }
        mbar_inval(smem_u32(red_full));
        mbar_inval(smem_u32(red_empty));
    }

    // After an abort: wait (bounded) for the copies that may still be in flight, the most
    // recent use of every stage.  Thread 0 only.
    __device__ __forceinline__ void drain() {
        const int hi = *issued;
        for (int qq = (hi > S::STAGES ? hi - S::STAGES : 0); qq < hi; ++qq)
            (void)mbar_wait_bounded(smem_u32(&full[qq % S::STAGES]), uint32_t((qq / S::STAGES) & 1));
        // the x_j windows in flight (bulk copies are not covered by cp.async.wait_all)
        if (S::XSTAGE) {
            const int xh = *xissued;
            for (int qq = (xh > S::STAGES ? xh - S::STAGES : 0); qq < xh; ++qq)
                (void)mbar_wait_bounded(smem_u32(&xfull[qq % S::STAGES]), uint32_t((qq / S::STAGES) & 1));
        }
    }
};

// Instrumented builds (-DFJOFC_STAMPS): clock cycles warp 0 of every CTA spends in the
// ring's waits (rfull, full, xfull, rempty) and the number of passes, summed over every
// launch of the process.
#ifdef FJOFC_STAMPS
static __device__ unsigned long long g_waitcyc[1024][5];
#define FJ_WAIT_T0() const long long fj_w0 = clock64()
#define FJ_WAIT_ADD(which_) \
    do { if (threadIdx.x == 0 && blockIdx.x < 1024) fj_wait[which_] += (unsigned long long)(clock64() - fj_w0); } while (0)
#else
#define FJ_WAIT_T0() do { } while (0)
#define FJ_WAIT_ADD(which_) do { } while (0)
#endif
// Instrumented builds (-DFJOFC_SECTIONS): clock cycles thread 0 of every CTA spends in each
// section of the column-strip loop, summed over every launch of the process.
#ifdef FJOFC_SECTIONS
static __device__ unsigned long long g_seccyc[1024][8];
#define FJ_SEC(i_)                                                                  \
    do {                                                                            \
        const long long now_ = clock64();                                           \
        if (threadIdx.x == 0) s_sec[i_] += (unsigned long long)(now_ - fj_last);    \
        fj_last = now_;                                                             \
    } while (0)
#else
#define FJ_SEC(i_) do { } while (0)
#endif

// One all-pairs pass over the CTA's range (ring uses qbase .. qbase + nq - 1) against the
// iterate X.  Writes the column partials of every sub-tile, the row partials of every
// walk segment and returns this thread's weighted fidelity in fid_total.  Returns false
// if a bounded wait gave up (the caller raises the error and drains the ring).
template <int D, typename TD>
__device__ __forceinline__ bool phase_a(K1Ring<D, TD>& rg, const TMaps& tm, const K1Params& p, const float* X,
                                        int64_t qbase, int b, FF& fid_total) {
    using S = K1Shape<D, TD>;
    constexpr int R = S::R, C = S::C, CWARPS = S::CWARPS, STAGES = S::STAGES, SLOTS = S::SLOTS;
    constexpr int RB = S::RB, CW = S::CW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n, nq = rg.nq;
    const volatile int* abort_flag = rg.abort_flag;
    fid_total = FF{0.f, 0.f};

    Cursor cc, cn;
    cc = *rg.pc_start;                                 // the range's first cursor (set by start())
    cn = cc;
    bool seg_head = (cc.s == 0);
    constexpr int XB = XiBcast<D>::XB;
    float racc[R][D], xjn[S::XSTAGE ? 1 : C][D];
    float* xrow = rg.xrow + warp * (R * XB * 4);
    // this warp's R rows of a walk (row block I of modality l) into its broadcast rows;
    // element e = r*D + k of the R x D block comes from lane e % 32
    auto put_rows = [&](const float (&v)[RowStage<R, D>::PER_LANE], float xs) {
#pragma unroll
        for (int u = 0; u < RowStage<R, D>::PER_LANE; ++u) {
            const int e = u * 32 + lane;
            if (e < R * D) {
                const int r = e / D, k = e - r * D;
                const float x = v[u] * xs;
                *reinterpret_cast<float2*>(xrow + r * XB * 4 + 2 * k) = make_float2(x, x);
            }
        }
        __syncwarp();
    };
    {
        RowStage<R, D> rs0;
        const float* src = X + (int64_t(cc.l) * n + int64_t(cc.I) * RB + warp * R) * D;
        const int lim = (n - (cc.I * RB + warp * R)) * D;
#pragma unroll
        for (int u = 0; u < RowStage<R, D>::PER_LANE; ++u) {
            const int e = u * 32 + lane;
            rs0.v[u] = (e < R * D && e < lim) ? __ldcg(src + e) : 0.f;
        }
        __syncwarp();          // the previous pass's readers of xrow are done
        put_rows(rs0.v, p.xscale[cc.l]);
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < D; ++k) racc[r][k] = 0.f;
    }
    auto load_cols = [&](const Cursor& c) {
        if constexpr (!S::XSTAGE) {
            const float* Xl = X + int64_t(c.l) * n * D;
            const float nxs = -p.xscale[c.l];      // -x_j in Delta's units
            const int c0 = c.I * RB + c.s * CW + lane * C;
#pragma unroll
            for (int ci = 0; ci < C; ++ci)
#pragma unroll
                for (int k = 0; k < D; ++k)
                    xjn[ci][k] = (c0 + ci < n) ? __ldcg(Xl + int64_t(c0 + ci) * D + k) * nxs : 0.f;
        }
    };
    load_cols(cn);
    if constexpr (S::XSTAGE) {
        // the iterate was written with ordinary stores; x_j windows are bulk copies
        fence_proxy_async_global();
        // x_j of this pass's first uses (their Delta may have been issued during the
        // previous pass, before this iterate existed)
        if (warp == 0) {
            Cursor c = cc;
            const int k0 = nq < STAGES ? nq : STAGES;
            for (int j = 0; j < k0; ++j) {
                rg.issue_x(p, X, qbase + j, c);
                if (j + 1 < k0) cursor_next(c, p);
            }
        }
    }
    FF fid{0.f, 0.f};
    int cur_l = cc.l;
#ifdef FJOFC_STAMPS
    unsigned long long fj_wait[4] = {0, 0, 0, 0};
#endif

    // reduce this warp's share of the columns of ring use qg (deferred by one sub-tile)
    auto reduce_share = [&](int64_t qg, int64_t tglob) -> bool {
        const int slot = int(qg % SLOTS);
        FJ_WAIT_T0();
        if (!mbar_wait_or_abort(smem_u32(&rg.rfull[slot]), uint32_t((qg / SLOTS) & 1), abort_flag)) return false;
        FJ_WAIT_ADD(0);
        const float* rb = rg.red + size_t(slot) * CWARPS * D * CW;
        float* cp = p.colpart + tglob * int64_t(D * CW);
        constexpr int SHARE = (D * CW + CWARPS - 1) / CWARPS;
        for (int e = warp * SHARE + lane; e < (warp + 1) * SHARE && e < D * CW; e += 32) {
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < CWARPS; ++w) v += rb[w * D * CW + e];
            cp[e] = v;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&rg.rempty[slot]));
        return true;
    };

    // ring position of use qbase: stage and use count of that stage, advanced incrementally
    int stage = int(qbase % STAGES);
    uint32_t kuse = uint32_t(qbase / STAGES);
    for (int q = 0; q < nq; ++q) {
        const int64_t qg = qbase + q;
        const int slot = int(qg & (SLOTS - 1));
        static_assert((SLOTS & (SLOTS - 1)) == 0, "SLOTS must be a power of two");
        const int r0 = cc.I * RB;
        const int c0 = r0 + cc.s * CW;
        const bool walk_ends = (cc.s + 1 == cc.L);
        const bool last = (q + 1 == nq);
        float2 nxj[C / 2][D];      // -x_j, column pairs
        if constexpr (!S::XSTAGE) {
#pragma unroll
            for (int c = 0; c < C; c += 2)
#pragma unroll
                for (int k = 0; k < D; ++k) nxj[c / 2][k] = make_float2(xjn[c][k], xjn[c + 1][k]);
        }
        if (!last) {                // prefetch the next sub-tile's columns
            cursor_next(cn, p);
            load_cols(cn);
        }
        RowStage<R, D> rs;          // the next walk's rows, in flight during this sub-tile
        if (walk_ends && !last) {
            const float* src = X + (int64_t(cn.l) * n + int64_t(cn.I) * RB + warp * R) * D;
            const int lim = (n - (cn.I * RB + warp * R)) * D;    // elements inside the modality
#pragma unroll
            for (int u = 0; u < RowStage<R, D>::PER_LANE; ++u) {
                const int e = u * 32 + lane;
                rs.v[u] = (e < R * D && e < lim) ? __ldcg(src + e) : 0.f;
            }
        }
        if (cc.l != cur_l) {        // modality changed inside this CTA's range
            fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
            fid = FF{0.f, 0.f};
            cur_l = cc.l;
        }

        {
            FJ_WAIT_T0();
            if (!mbar_wait_or_abort(smem_u32(&rg.full[stage]), kuse & 1u, abort_flag)) return false;
            FJ_WAIT_ADD(1);
        }
        if constexpr (S::XSTAGE) {
            FJ_WAIT_T0();
            if (!mbar_wait_or_abort(smem_u32(&rg.xfull[stage]), kuse & 1u, abort_flag))
                return false;
            FJ_WAIT_ADD(2);
            const int64_t start = (int64_t(cc.l) * n + c0) * D;
            const uint32_t xsrc = smem_u32(rg.xs + size_t(stage) * S::XS_FLOATS + int(start & 3) + lane * C * D);
            const float nxsc = -p.xscale[cc.l];
            if (c0 + CW <= n) {
#pragma unroll
                for (int c = 0; c < C; c += 2)
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        nxj[c / 2][k] = make_float2(lds_f1(xsrc + 4 * (c * D + k)) * nxsc,
                                                    lds_f1(xsrc + 4 * ((c + 1) * D + k)) * nxsc);
            } else {                // ragged sub-tile: columns past n hold other data
#pragma unroll
                for (int c = 0; c < C; c += 2)
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        nxj[c / 2][k] =
                            make_float2((c0 + lane * C + c < n) ? lds_f1(xsrc + 4 * (c * D + k)) * nxsc : 0.f,
                                        (c0 + lane * C + c + 1 < n) ? lds_f1(xsrc + 4 * ((c + 1) * D + k)) * nxsc : 0.f);
            }
        }
        const uint32_t tile = smem_u32(rg.stages + size_t(stage) * S::STAGE_ELEMS);
        const bool masked = (cc.s * CW < RB) || (c0 + CW > n);
        float2 cacc0[C / 2][D], cacc1[C / 2][D];
        float2 sf0, sf1;
        const uint32_t xib = smem_u32(xrow);
        if (!masked)
            subtile_pairs<D, TD, R, C, CW, false>(tile, warp, lane, r0, c0, n, xib, nxj, racc, cacc0, cacc1, sf0, sf1);
        else
            subtile_pairs<D, TD, R, C, CW, true>(tile, warp, lane, r0, c0, n, xib, nxj, racc, cacc0, cacc1, sf0, sf1);
        // release the stage; the last warp to do so refills it with use qg + STAGES
        const bool refill = qg + STAGES < rg.total_q;
        __syncwarp();
        int is_last = 0;
        if (lane == 0) {
            __threadfence_block();
            // use k = qg / STAGES of this stage is fully released at count (k+1)*CWARPS
            if (atomicAdd(&rg.released[stage], 1) == int(kuse + 1) * CWARPS - 1) {
                __threadfence_block();
                is_last = 1;
                if (refill) rg.issue(tm, qg + STAGES);
            }
        }
        if constexpr (S::XSTAGE) {
            // x_j of the refilled use, if it belongs to this pass (this iterate)
            is_last = __shfl_sync(0xffffffffu, is_last, 0);
            if (is_last && refill && q + STAGES < nq) rg.issue_x(p, X, qg + STAGES, rg.pc);
        }
        if (refill) rg.advance(p);
        fid = ff_add(fid, (sf0.x + sf0.y) + (sf1.x + sf1.y));

        // column partials of this sub-tile into its ring slot
        {
            FJ_WAIT_T0();
            if (qg >= SLOTS &&
                !mbar_wait_or_abort(smem_u32(&rg.rempty[slot]), uint32_t(((qg / SLOTS) - 1) & 1), abort_flag))
                return false;
            FJ_WAIT_ADD(3);
        }
        float* rbuf = rg.red + (size_t(slot) * CWARPS + warp) * D * CW;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if constexpr (C % 4 == 0) {
#pragma unroll
                for (int c = 0; c < C; c += 4)
                    *reinterpret_cast<float4*>(rbuf + k * CW + lane * C + c) =
                        make_float4(cacc0[c / 2][k].x + cacc1[c / 2][k].x, cacc0[c / 2][k].y + cacc1[c / 2][k].y,
                                    cacc0[c / 2 + 1][k].x + cacc1[c / 2 + 1][k].x,
                                    cacc0[c / 2 + 1][k].y + cacc1[c / 2 + 1][k].y);
            } else {
#pragma unroll
                for (int c = 0; c < C; c += 2)
                    *reinterpret_cast<float2*>(rbuf + k * CW + lane * C + c) =
                        make_float2(cacc0[c / 2][k].x + cacc1[c / 2][k].x, cacc0[c / 2][k].y + cacc1[c / 2][k].y);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&rg.rfull[slot]));
        if (q >= 1 && !reduce_share(qg - 1, cc.t - 1)) return false;

        if (walk_ends || last) {
            // row partials of this walk segment: reduce-scatter over the warp
            float* dst = seg_head ? p.rowhead + (int64_t(cc.l) * p.nRB + cc.I) * (D * RB)
                                  : p.rowcont + int64_t(b) * (D * RB);
            float v[R * D];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < D; ++k) v[r * D + k] = -racc[r][k];   // racc holds -sum b (x_i - x_j)
            int base = 0;
            bool writer = true;
            WarpScatter<R * D, 16>::run(v, lane, base, writer);
            constexpr int F = WarpScatterCount<R * D, 16>::value;
            if (writer)
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const int e = base + f, r = e / D, k = e - r * D;
                    dst[k * RB + warp * R + r] = v[f];
                }
        }
        cursor_next(cc, p);
        if (++stage == STAGES) {
            stage = 0;
            ++kuse;
        }
        if (walk_ends && !last) {
            seg_head = true;
            __syncwarp();          // every lane is done reading the old rows
            put_rows(rs.v, p.xscale[cc.l]);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < D; ++k) racc[r][k] = 0.f;
        }
    }
    if (!reduce_share(qbase + nq - 1, rg.t_begin + nq - 1)) return false;
    fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
#ifdef FJOFC_STAMPS
    if (threadIdx.x == 0 && blockIdx.x < 1024) {
        for (int x = 0; x < 4; ++x) atomicAdd(&g_waitcyc[blockIdx.x][x], fj_wait[x]);
        atomicAdd(&g_waitcyc[blockIdx.x][4], 1ull);
    }
#endif
    return true;
}

// ---------------------------------------------------------------------------------------
// Column-strip layout of a sub-tile (S::STRIP): warp w owns the SW = CW / 8 columns
// [w SW, (w + 1) SW); lane (rg, cl) = (lane >> 2, lane & 3) owns the C columns
// w SW + cl C + (0 .. C-1) and the R rows rg + 8 u (u = 0 .. R-1) of the row block.  Row
// accumulators stay in registers for the whole walk segment (as in the row-band layout);
// a sub-tile's column sums are complete inside the warp: a reduce-scatter over the eight
// row groups (lane bits 2..4) leaves every (column, coordinate) total in one lane, which
// writes it.  Warps meet only at the TMA ring (stage release) and, at the end of a walk
// segment, to add their row partials (mbarrier hand-off through shared memory, bounded).
// Sign convention here: q = +b (no negation of Delta), so the row accumulators hold
// sum_j b (x_i - x_j) and the column accumulators its negation for the columns.
// ---------------------------------------------------------------------------------------

// Sum of v[0..V-1] over the lanes that differ in lane bits OFF, OFF/2, .., LOW (a
// reduce-scatter, pairing as an xor butterfly): on return v[0..F-1] holds totals of
// indices base .. base+F-1 and exactly one lane of each group has writer == true.
template <int V, int OFF, int LOW>
struct LaneScatter {
    static constexpr int F = OFF < LOW ? V : (V % 2 == 0 ? LaneScatter<V / 2, OFF / 2, LOW>::F
                                                        : LaneScatter<V, OFF / 2, LOW>::F);
    static __device__ __forceinline__ void run(float* v, int lane, int& base, bool& writer) {
        if constexpr (OFF >= LOW) {
            if constexpr (V % 2 == 0) {
                constexpr int H = V / 2;
                const bool up = (lane & OFF) != 0;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float send = up ? v[h] : v[h + H];
                    const float keep = up ? v[h + H] : v[h];
                    v[h] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
                }
                if (up) base += H;
                LaneScatter<H, OFF / 2, LOW>::run(v, lane, base, writer);
            } else {
#pragma unroll
                for (int h = 0; h < V; ++h) v[h] += __shfl_xor_sync(0xffffffffu, v[h], OFF);
                if (lane & OFF) writer = false;
                LaneScatter<V, OFF / 2, LOW>::run(v, lane, base, writer);
            }
        }
    }
};

// The pairs of one sub-tile owned by lane (rg, cl) of warp w in the column-strip layout.
// tile: shared address of the stage (BOXES swizzled boxes); xib: the walk rows as
// broadcast pairs, layout [XB][R][8] float4 (row rg + 8u at (x R + u) 8 + rg); nxj: -x_j
// of the lane's columns as column pairs.  MASKED: only pairs with i < j < n count.
template <int D, typename TD, int R, int C, int RB, int SW, bool MASKED>
__device__ __forceinline__ void strip_pairs(uint32_t tile, int warp, int rg, int cl, int r0, int c0, int n,
                                            uint32_t xib, const float2 (&nxj)[C / 2][D], float (&racc)[R][D],
                                            float2 (&cacc)[C / 2][D], float2& sf) {
    static_assert(C % 2 == 0, "columns are processed in pairs");
    constexpr int CP = C / 2, XB = XiBcast<D>::XB;
    constexpr int RI = (R % 2 == 0) ? 2 : 1;
    // byte offset of the lane's columns inside a 128-column row, split into box, 16-byte
    // chunk and offset inside the chunk
    const int cbyte = (warp * SW + cl * C) * int(sizeof(TD));
    const uint32_t box_off = uint32_t(cbyte >> 7) * RB * 128u;
    const int chunk = (cbyte & 127) >> 4, sub = cbyte & 15;
#pragma unroll
    for (int cp = 0; cp < CP; ++cp)
#pragma unroll
        for (int k = 0; k < D; ++k) cacc[cp][k] = make_float2(0.f, 0.f);
    sf = make_float2(0.f, 0.f);
#pragma unroll
    for (int ub = 0; ub < R; ub += RI) {
        float2 xb[RI][2 * XB];
        float dl[RI][C];
#pragma unroll
        for (int h = 0; h < RI; ++h) {
            const int u = ub + h, lr = rg + 8 * u;            // row of the block
#pragma unroll
            for (int x = 0; x < XB; ++x) {
                const float4 v = lds_f4(xib + 16 * ((x * R + u) * 8 + rg));
                xb[h][2 * x] = make_float2(v.x, v.y);
                xb[h][2 * x + 1] = make_float2(v.z, v.w);
            }
            lds_delta_row<TD, C>(tile + box_off + uint32_t(lr) * 128u + uint32_t(((chunk ^ (lr & 7)) << 4) + sub),
                                 dl[h]);
        }
#pragma unroll
        for (int cp = 0; cp < CP; ++cp) {
            float2 diff[RI][D], d2[RI], rinv[RI], q[RI], e[RI];
#pragma unroll
            for (int h = 0; h < RI; ++h) d2[h] = make_float2(FLT_MIN, FLT_MIN);
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int h = 0; h < RI; ++h) {
                    diff[h][k] = __fadd2_rn(xb[h][k], nxj[cp][k]);
                    d2[h] = __ffma2_rn(diff[h][k], diff[h][k], d2[h]);
                }
#pragma unroll
            for (int h = 0; h < RI; ++h) rinv[h] = make_float2(rsqrt_approx(d2[h].x), rsqrt_approx(d2[h].y));
#pragma unroll
            for (int h = 0; h < RI; ++h) {
                q[h] = __fmul2_rn(make_float2(dl[h][2 * cp], dl[h][2 * cp + 1]), rinv[h]);   // b
                e[h].x = fmaf(d2[h].x, rinv[h].x, -dl[h][2 * cp]);                           // d - Delta
                e[h].y = fmaf(d2[h].y, rinv[h].y, -dl[h][2 * cp + 1]);
                if (MASKED) {
                    const int i = r0 + rg + 8 * (ub + h);
                    const int j = c0 + warp * SW + cl * C + 2 * cp;
                    const bool v0 = (j > i) && (j < n), v1 = (j + 1 > i) && (j + 1 < n);
                    q[h].x = v0 ? q[h].x : 0.f;
                    e[h].x = v0 ? e[h].x : 0.f;
                    q[h].y = v1 ? q[h].y : 0.f;
                    e[h].y = v1 ? e[h].y : 0.f;
                }
                sf = __ffma2_rn(e[h], e[h], sf);
            }
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int h = 0; h < RI; ++h) {
                    const int u = ub + h;
                    racc[u][k] = fmaf(q[h].x, diff[h][k].x, racc[u][k]);
                    racc[u][k] = fmaf(q[h].y, diff[h][k].y, racc[u][k]);
                    cacc[cp][k] = __ffma2_rn(q[h], diff[h][k], cacc[cp][k]);
                }
        }
    }
}

// One all-pairs pass over the CTA's range in the column-strip layout (same inputs,
// outputs and ring as phase_a).  Walk rows: one shared copy per walk segment, double
// buffered (segment g uses buffer g & 1); every warp loads 1/8 of the next segment's rows
// one sub-tile ahead and writes them during the row hand-off that ends the segment, which
// every warp passes before it reads them.  The hand-off (rfull: partials and rows written,
// rempty: partials read, count 8 each) is bounded like every other wait.
template <int D, typename TD>
__device__ __forceinline__ bool phase_a_strip(K1Ring<D, TD>& rg, const TMaps& tm, const K1Params& p, const float* X,
                                              int64_t qbase, int b, FF& fid_total) {
    using S = K1Shape<D, TD>;
    constexpr int R = S::R, C = S::C, CWARPS = S::CWARPS, STAGES = S::STAGES, SW = S::SW;
    constexpr int RB = S::RB, CW = S::CW, XB = XiBcast<D>::XB;
    constexpr int XBUF = RB * XB * 4;                 // floats of one walk-rows buffer
    constexpr int RSH = (RB * D + CWARPS * 32 - 1) / (CWARPS * 32);   // next rows per lane
    static_assert(S::XSTAGE, "the column-strip layout stages x_j in shared memory");
    static_assert(S::XROW_FLOATS == 2 * XBUF, "two walk-row buffers");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int rgp = lane >> 2, cl = lane & 3;
    const int n = p.n, nq = rg.nq;
    const volatile int* abort_flag = rg.abort_flag;
    fid_total = FF{0.f, 0.f};
    // A wait that gives up ends this warp's loop and raises the CTA's abort flag, so that
    // every other warp's next wait gives up too; every warp then reaches the barriers after
    // the loop.
    bool failed = false;
    auto fail = [&]() {
        failed = true;
        *reinterpret_cast<volatile int*>(rg.abort_flag) = 1;
    };
#ifdef FJOFC_SECTIONS
    __shared__ unsigned long long s_sec[8];
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) s_sec[i] = 0ull;
    long long fj_last = clock64();
#endif

    Cursor cc, cn;
    cc = *rg.pc_start;                                 // the range's first cursor (set by start())
    cn = cc;
    bool seg_head = (cc.s == 0);
    float racc[R][D];
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) racc[u][k] = 0.f;

    // element e = lr*D + k of a walk's RB x D rows, loaded by thread e % NT (round e / NT)
    auto load_rows = [&](const Cursor& c, float (&v)[RSH]) {
        const float* src = X + (int64_t(c.l) * n + int64_t(c.I) * RB) * D;
        const int lim = (n - c.I * RB) * D;            // elements inside the modality
#pragma unroll
        for (int t = 0; t < RSH; ++t) {
            const int e = t * CWARPS * 32 + tid;
            v[t] = (e < RB * D && e < lim) ? __ldcg(src + e) : 0.f;
        }
    };
    auto put_rows = [&](const float (&v)[RSH], float* buf, float xs) {
#pragma unroll
        for (int t = 0; t < RSH; ++t) {
            const int e = t * CWARPS * 32 + tid;
            if (e < RB * D) {
                const int lr = e / D, k = e - lr * D;
                const int u = lr >> 3, g = lr & 7;
                const float x = v[t] * xs;
                *reinterpret_cast<float2*>(buf + ((k / 2 * R + u) * 8 + g) * 4 + 2 * (k & 1)) = make_float2(x, x);
            }
        }
    };
    // the first segment's rows: their loads go out first, so that their latency overlaps
    // the fence and the x_j copies below
    float v0[RSH];
    load_rows(cc, v0);
    // the iterate was written with ordinary stores (by the previous per-object phase);
    // any thread of the CTA may copy parts of it with bulk copies during this pass
    fence_proxy_async_global();
    if (warp == 0) {
        // x_j of this pass's first uses (their Delta may have been issued during the
        // previous pass, before this iterate existed), in flight while the rows load
        Cursor c = cc;
        const int k0 = nq < STAGES ? nq : STAGES;
        for (int j = 0; j < k0; ++j) {
            rg.issue_x(p, X, qbase + j, c);
            if (j + 1 < k0) cursor_next(c, p);
        }
    }
#ifdef FJOFC_STAMPS
    unsigned long long fj_wait[4] = {0, 0, 0, 0};
#endif
    // Walk rows of segment s (counted over the ring's life, rg.nflush) sit in buffer s & 1:
    // every warp writes its share once segment s - 2 is done by every warp (rempty[s & 1])
    // and arrives on rfull[s & 1]; a warp reads them once all eight have (rfull).
    auto rows_write = [&](int sg, const float (&v)[RSH], int l) -> bool {
        if (sg >= 2) {
            FJ_WAIT_T0();
            if (!mbar_wait_or_abort(smem_u32(&rg.rempty[sg & 1]), uint32_t(((sg >> 1) - 1) & 1), abort_flag))
                return false;
            FJ_WAIT_ADD(3);
        }
        put_rows(v, rg.xrow + (sg & 1) * XBUF, p.xscale[l]);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&rg.rfull[sg & 1]));
        return true;
    };
    // the first segment's rows into their buffer
    {
        if (!rows_write(rg.nflush, v0, cc.l)) fail();
    }
    bool rows_pending = true;                          // the segment's rows are not yet waited for
    int mid_done = 0;                                  // segments of this pass summed inside the loop
    float* end_dst = nullptr;                          // destination of the pass's last segment

    FF fid{0.f, 0.f};
    int cur_l = cc.l;
    int stage = int(qbase % STAGES);
    uint32_t kuse = uint32_t(qbase / STAGES);
    // -x_j of the lane's columns of the sub-tile at cursor c (ring stage stg, use count
    // ku of that stage) as column pairs, once its staged x_j have landed; columns at or
    // beyond n read as 0
    const int cbase = warp * SW + cl * C;              // first column of the lane in a sub-tile
    auto load_nxj = [&](const Cursor& c, int stg, uint32_t ku, float2 (&o)[C / 2][D]) -> bool {
        FJ_WAIT_T0();
        if (!mbar_wait_or_abort(smem_u32(&rg.xfull[stg]), ku & 1u, abort_flag)) return false;
        FJ_WAIT_ADD(2);
        const int cc0 = c.I * RB + c.s * CW;
        const int64_t start = (int64_t(c.l) * n + cc0) * D;
        const uint32_t xsrc = smem_u32(rg.xs + size_t(stg) * S::XS_FLOATS + int(start & 3) + cbase * D);
        const float nxsc = -p.xscale[c.l];
#pragma unroll
        for (int cx = 0; cx < C; cx += 2)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const bool in0 = cc0 + cbase + cx < n, in1 = cc0 + cbase + cx + 1 < n;
                o[cx / 2][k] = make_float2(in0 ? lds_f1(xsrc + 4 * (cx * D + k)) * nxsc : 0.f,
                                           in1 ? lds_f1(xsrc + 4 * ((cx + 1) * D + k)) * nxsc : 0.f);
            }
        return true;
    };
    FJ_SEC(7);
    for (int q = 0; q < nq && !failed; ++q) {
        const int64_t qg = qbase + q;
        const int r0 = cc.I * RB;
        const int c0 = r0 + cc.s * CW;
        const bool walk_ends = (cc.s + 1 == cc.L);
        const bool last = (q + 1 == nq);
        if (!last) cursor_next(cn, p);
        float rs[RSH];                                 // the next segment's rows, in flight
        if (walk_ends && !last) load_rows(cn, rs);
        if (cc.l != cur_l) {                           // modality changed inside this CTA's range
            fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
            fid = FF{0.f, 0.f};
            cur_l = cc.l;
        }
        FJ_SEC(0);
        {
            FJ_WAIT_T0();
            if (!mbar_wait_or_abort(smem_u32(&rg.full[stage]), kuse & 1u, abort_flag)) { fail(); break; }
            FJ_WAIT_ADD(1);
        }
        FJ_SEC(1);
        float2 nxj[C / 2][D];
        if (!load_nxj(cc, stage, kuse, nxj)) { fail(); break; }
        const uint32_t tile = smem_u32(rg.stages + size_t(stage) * S::STAGE_ELEMS);
        const bool masked = (cc.s * CW < RB) || (c0 + CW > n);
        float2 cacc[C / 2][D];
        float2 sf;
        if (rows_pending) {
            FJ_WAIT_T0();
            if (!mbar_wait_or_abort(smem_u32(&rg.rfull[rg.nflush & 1]), uint32_t((rg.nflush >> 1) & 1), abort_flag)) {
                fail();
                break;
            }
            FJ_WAIT_ADD(0);
            rows_pending = false;
        }
        const uint32_t xib = smem_u32(rg.xrow + (rg.nflush & 1) * XBUF);
        FJ_SEC(2);
        if (!masked)
            strip_pairs<D, TD, R, C, RB, SW, false>(tile, warp, rgp, cl, r0, c0, n, xib, nxj, racc, cacc, sf);
        else
            strip_pairs<D, TD, R, C, RB, SW, true>(tile, warp, rgp, cl, r0, c0, n, xib, nxj, racc, cacc, sf);
        FJ_SEC(3);
        // release the stage; the last warp to do so refills it with use qg + STAGES
        const bool refill = qg + STAGES < rg.total_q;
        // (every lane's reads of the stage have returned: their values were consumed
        // above, so no fence is needed before the count)
        __syncwarp();
        int is_last = 0;
        if (lane == 0) {
            if (atomicAdd(&rg.released[stage], 1) == int(kuse + 1) * CWARPS - 1) {
                is_last = 1;
                if (refill) rg.issue(tm, qg + STAGES);
            }
        }
        is_last = __shfl_sync(0xffffffffu, is_last, 0);
        if (is_last && refill && q + STAGES < nq) rg.issue_x(p, X, qg + STAGES, rg.pc);
        if (refill) rg.advance(p);
        fid = ff_add(fid, sf.x + sf.y);
        FJ_SEC(4);

        // this sub-tile's column sums: reduce-scatter over the eight row groups (lane bits
        // 2..4); the writer lane of each (column, coordinate) stores its total, negated
        // (the accumulators hold the rows' sign)
        {
            float v[C * D];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int k = 0; k < D; ++k) v[c * D + k] = (c & 1) ? cacc[c / 2][k].y : cacc[c / 2][k].x;
            int base = 0;
            bool writer = true;
            LaneScatter<C * D, 16, 4>::run(v, lane, base, writer);
            constexpr int F = LaneScatter<C * D, 16, 4>::F;
            float* cpart = p.colpart + cc.t * int64_t(D * CW);
            if (writer)
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const int e = base + f, c = e / D, k = e - c * D;
                    cpart[k * CW + warp * SW + cl * C + c] = -v[f];
                }
        }
        FJ_SEC(5);

        if (walk_ends || last) {
            // row partials of this walk segment: the sum over the four column groups in the
            // warp (lane bits 0, 1) into the warp's part of the shared buffer, then the sum
            // over the eight warps in warp order: for a segment that ends inside the pass by
            // the last warp to get there (the others go on), for the pass's last segment by
            // every warp after the loop
            float* dst = seg_head ? p.rowhead + (int64_t(cc.l) * p.nRB + cc.I) * (D * RB)
                                  : p.rowcont + int64_t(b) * (D * RB);
            if (mid_done > 0) {                        // the buffer's previous segment is summed
                FJ_WAIT_T0();
                if (!mbar_wait_or_abort(smem_u32(rg.red_empty), uint32_t((rg.nred - 1) & 1), abort_flag)) {
                    fail();
                    break;
                }
                FJ_WAIT_ADD(3);
            }
            {
                float v[R * D];
#pragma unroll
                for (int u = 0; u < R; ++u)
#pragma unroll
                    for (int k = 0; k < D; ++k) v[u * D + k] = racc[u][k];
                int base = 0;
                bool writer = true;
                LaneScatter<R * D, 2, 1>::run(v, lane, base, writer);
                constexpr int F = LaneScatter<R * D, 2, 1>::F;
                if (writer)
#pragma unroll
                    for (int f = 0; f < F; ++f) {
                        const int e = base + f, u = e / D, k = e - u * D;
                        rg.red[(warp * D + k) * RB + rgp + 8 * u] = v[f];
                    }
            }
            if (!last) {
                // the next segment's rows first: the other warps wait for every share of
                // them, not for this warp's sum below
                if (!rows_write(rg.nflush + 1, rs, cn.l)) {
                    fail();
                    break;
                }
                __syncwarp();
                int lastw = 0;
                if (lane == 0) {
                    mbar_arrive(smem_u32(rg.red_full));
                    lastw = (atomicAdd(rg.red_cnt, 1) & (CWARPS - 1)) == CWARPS - 1;
                }
                lastw = __shfl_sync(0xffffffffu, lastw, 0);
                if (lastw) {
                    FJ_WAIT_T0();
                    if (!mbar_wait_or_abort(smem_u32(rg.red_full), uint32_t(rg.nred & 1), abort_flag)) { fail(); break; }
                    FJ_WAIT_ADD(0);
                    for (int e = lane; e < RB * D; e += 32) {
                        const int k = e / RB, row = e - k * RB;
                        float sv = 0.f;
#pragma unroll
                        for (int w = 0; w < CWARPS; ++w) sv += rg.red[(w * D + k) * RB + row];
                        dst[e] = sv;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(rg.red_empty));
                }
                ++rg.nred;
                ++mid_done;
            } else {
                end_dst = dst;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&rg.rempty[rg.nflush & 1]));   // done with this segment's rows
            ++rg.nflush;
            rows_pending = true;
            seg_head = true;
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int k = 0; k < D; ++k) racc[u][k] = 0.f;
        }
        cc = cn;                                       // cn is one sub-tile ahead (unused after the last)
        if (++stage == STAGES) {
            stage = 0;
            ++kuse;
        }
        FJ_SEC(6);
    }
    fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
    // the pass's last segment: every warp has written its part (a warp whose wait gave up
    // gets here too, and the abort flag ends every other warp's loop at its next wait); each
    // warp sums a share over the eight warps, and the buffer is free after the second barrier
    __syncthreads();
    if (!failed) {
        constexpr int SHARE = (RB * D + CWARPS - 1) / CWARPS;
        for (int e = warp * SHARE + lane; e < (warp + 1) * SHARE && e < RB * D; e += 32) {
            const int k = e / RB, row = e - k * RB;
            float sv = 0.f;
#pragma unroll
            for (int w = 0; w < CWARPS; ++w) sv += rg.red[(w * D + k) * RB + row];
            end_dst[e] = sv;
        }
    }
    __syncthreads();
#ifdef FJOFC_STAMPS
    if (threadIdx.x == 0 && blockIdx.x < 1024) {
        for (int x = 0; x < 4; ++x) atomicAdd(&g_waitcyc[blockIdx.x][x], fj_wait[x]);
        atomicAdd(&g_waitcyc[blockIdx.x][4], 1ull);
    }
#endif
#ifdef FJOFC_SECTIONS
    if (threadIdx.x == 0 && blockIdx.x < 1024)
        for (int x = 0; x < 8; ++x) atomicAdd(&g_seccyc[blockIdx.x][x], s_sec[x]);
#endif
    return !failed;
}

// Standalone pass (one launch per Guttman transform, used when the persistent kernel is
// not: per-kernel timing).  Same ring, tiles and partials as the persistent kernel.
template <int D, typename TD>
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, FJOFC_K1_MINB)
k_guttman_pass(const __grid_constant__ TMaps tm, const __grid_constant__ K1Params p) {
    using S = K1Shape<D, TD>;
    constexpr int CWARPS = S::CWARPS;
    extern __shared__ unsigned char smem_raw[];
    __shared__ FF s_redff[CWARPS];
    __shared__ int s_abort, s_issued;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x;

    if (ld_volatile(&p.st->done)) return;   // the loop has stopped: nothing to compute

    K1Ring<D, TD> rg;
    rg.carve(smem_raw);
    const int64_t t_begin = p.cta_start[b];
    const int nq = static_cast<int>(p.cta_start[b + 1] - t_begin);   // >= 1 because G <= T
    rg.start(tm, p, t_begin, nq, nq, &s_issued, &s_abort);

    FF fid_total{0.f, 0.f};
    bool ok_a;
    if constexpr (S::STRIP) ok_a = phase_a_strip<D, TD>(rg, tm, p, p.X, 0, b, fid_total);
    else ok_a = phase_a<D, TD>(rg, tm, p, p.X, 0, b, fid_total);
    if (!ok_a) {
        atomicExch(&s_abort, 1);
        if (lane == 0) raise_error(p.st, FJOFC_ERR_TIMEOUT, 2);
    }
    cp_async_wait_all();
    __syncthreads();
    if (s_abort && tid == 0) rg.drain();

    // fidelity partial of this CTA (fixed-order float-float reduction)
    const FF ws = warp_sum_ff(fid_total);
    if (lane == 0) s_redff[warp] = ws;
    __syncthreads();
    if (tid == 0) {
        FF tot{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < CWARPS; ++w) tot = ff_add(tot, s_redff[w]);
        p.fid[b] = make_float2(tot.hi, tot.lo);
    }
}

template <int D, typename TD>
cudaError_t k1_launch_impl(int grid, const TMaps& tm, const K1Params& p, cudaStream_t s) {
    using S = K1Shape<D, TD>;
    int dev = 0;
    cudaGetDevice(&dev);
    static bool configured[64] = {};
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_guttman_pass<D, TD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    k_guttman_pass<D, TD><<<grid, S::NT, S::SMEM, s>>>(tm, p);
    return cudaGetLastError();
}

template <int D, typename TD>
int k1_bps_impl() {
    using S = K1Shape<D, TD>;
    cudaFuncSetAttribute(k_guttman_pass<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_guttman_pass<D, TD>, S::NT, S::SMEM) != cudaSuccess)
        return 0;
    return nb;
}

template <int D, typename TD>
K1Geom k1_geom_impl() {
    using S = K1Shape<D, TD>;
    return K1Geom{S::R, S::C, S::CWARPS, S::STAGES, S::RB, S::CW, S::NT, S::SMEM, S::STRIP ? S::BOX_ELEMS : 0};
}

#define FJOFC_INSTANTIATE_K1(D)                                                                   \
    template cudaError_t k1_launch_impl<D, float>(int, const TMaps&, const K1Params&, cudaStream_t); \
    template cudaError_t k1_launch_impl<D, __half>(int, const TMaps&, const K1Params&, cudaStream_t); \
    template cudaError_t k1_launch_impl<D, __nv_bfloat16>(int, const TMaps&, const K1Params&, cudaStream_t); \
    template int k1_bps_impl<D, float>();                                                         \
    template int k1_bps_impl<D, __half>();                                                        \
    template int k1_bps_impl<D, __nv_bfloat16>();                                                 \
    template K1Geom k1_geom_impl<D, float>();                                                     \
    template K1Geom k1_geom_impl<D, __half>();                                                    \
    template K1Geom k1_geom_impl<D, __nv_bfloat16>();

}  // namespace fjofc

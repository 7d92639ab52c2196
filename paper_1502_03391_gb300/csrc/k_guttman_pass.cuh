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
// registers for the whole walk segment); lane owns C consecutive columns of every
// sub-tile.  Column accumulators go through a small ring of shared-memory slots; each
// warp reduces its share of the previous sub-tile's columns in a fixed order and writes
// one partial per (sub-tile, column).  Row accumulators are reduced across the warp at
// walk-segment ends.  Warps never meet at a CTA-wide barrier inside the loop; they
// synchronise only through mbarriers and the stage counters, with one sub-tile of
// slack.  K2 sums every partial in a fixed order, so results are bitwise reproducible
// run to run.  Every wait is bounded.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"

namespace fjofc {

template <int D> struct K1Cfg;
// rows/thread, cols/lane, compute warps, pipeline stages (float32)
#define FJOFC_K1CFG(D_, R_, C_, W_, S_)                                                     \
    template <> struct K1Cfg<D_> { static constexpr int R = R_, C = C_, CWARPS = W_, STAGES = S_; };
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
#define FJOFC_SMALLD FJOFC_K1_SMALLD_R, FJOFC_K1_SMALLD_C, FJOFC_K1_SMALLD_WARPS, FJOFC_K1_SMALLD_STAGES
#define FJOFC_K1CFG_X(...) FJOFC_K1CFG(__VA_ARGS__)
FJOFC_K1CFG_X(1, FJOFC_SMALLD)    // default: 128 x 128 sub-tile, 64 KB at float32
FJOFC_K1CFG_X(2, FJOFC_SMALLD)
FJOFC_K1CFG_X(3, FJOFC_SMALLD)
FJOFC_K1CFG_X(4, FJOFC_SMALLD)
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

template <int D, typename TD>
struct K1Shape {
    static constexpr int R = K1Cfg<D>::R, C = K1Cfg<D>::C, CWARPS = K1Cfg<D>::CWARPS;
    // 16-bit Delta halves the stage: keep about the same bytes in flight
    static constexpr int STAGES = sizeof(TD) == 4 ? K1Cfg<D>::STAGES : 2 * K1Cfg<D>::STAGES;
    static constexpr int SLOTS = 2;                    // column-partial ring
    static constexpr int NT = CWARPS * 32;
    static constexpr int RB = CWARPS * R;
    static constexpr int CW = 32 * C;
    static constexpr int STAGE_ELEMS = RB * CW;
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(TD);
    static constexpr size_t RED_FLOATS = size_t(SLOTS) * CWARPS * D * CW;
    static constexpr size_t SMEM = size_t(STAGES) * STAGE_BYTES + RED_FLOATS * sizeof(float) +
                                   size_t(STAGES + 2 * SLOTS) * 8 + size_t(STAGES) * 4 + 128;
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


// The pairs of one RB x CW sub-tile owned by this thread: rows r0 + warp*R + r (x_i in
// xi[r]), columns c0 + lane*C + c (x_j in xj[c]).  Adds b_ij (x_i - x_j) to racc[r], its
// negative to the column accumulators (two interleaved chains by row parity) and
// (s Delta_ij - d_ij)^2 to sf0/sf1.  MASKED: only pairs with i < j < n count (diagonal and
// ragged sub-tiles); otherwise every pair of the sub-tile is valid.
template <int D, typename TD, int R, int C, int CW, bool MASKED>
__device__ __forceinline__ void subtile_pairs(const TD* tile, int warp, int lane, int r0, int c0, int n, float sc,
                                              const float (&xi)[R][D], const float (&xj)[C][D],
                                              float (&racc)[R][D], float (&cacc0)[C][D], float (&cacc1)[C][D],
                                              float& sf0, float& sf1) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < D; ++k) { cacc0[c][k] = 0.f; cacc1[c][k] = 0.f; }
    sf0 = 0.f;
    sf1 = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = r0 + warp * R + r;
        float dl[C];
        load_delta_row<TD, C>(tile + (warp * R + r) * CW + lane * C, dl);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float diff[D];
            float d2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                diff[k] = xi[r][k] - xj[c][k];
                d2 = fmaf(diff[k], diff[k], d2);
            }
            const float rinv = rsqrt_approx(fmaxf(d2, FLT_MIN));
            float bb = dl[c] * rinv;
            float e = fmaf(sc, dl[c], -(d2 * rinv));
            if (MASKED) {
                const int j = c0 + lane * C + c;
                const bool valid = (j > i) && (j < n);
                bb = valid ? bb : 0.f;
                e = valid ? e : 0.f;
            }
            if (r & 1) sf1 = fmaf(e, e, sf1); else sf0 = fmaf(e, e, sf0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                racc[r][k] = fmaf(bb, diff[k], racc[r][k]);
                if (r & 1) cacc1[c][k] = fmaf(-bb, diff[k], cacc1[c][k]);
                else cacc0[c][k] = fmaf(-bb, diff[k], cacc0[c][k]);
            }
        }
    }
}

template <int D, typename TD>
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, 1)
k_guttman_pass(const __grid_constant__ TMaps tm, const K1Params p) {
    using S = K1Shape<D, TD>;
    constexpr int R = S::R, C = S::C, CWARPS = S::CWARPS, STAGES = S::STAGES, SLOTS = S::SLOTS;
    constexpr int RB = S::RB, CW = S::CW;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    TD* stages = reinterpret_cast<TD*>(smem);
    float* red = reinterpret_cast<float*>(smem + size_t(STAGES) * S::STAGE_BYTES);   // [SLOTS][CWARPS][D][CW]
    uint64_t* full = reinterpret_cast<uint64_t*>(red + S::RED_FLOATS);
    uint64_t* rfull = full + STAGES;
    uint64_t* rempty = rfull + SLOTS;
    int* released = reinterpret_cast<int*>(rempty + SLOTS);       // [STAGES] releases so far (monotone)
    __shared__ FF s_redff[CWARPS];
    __shared__ int s_abort;
    __shared__ int s_issued;                                       // sub-tiles issued so far

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x;

    if (ld_volatile(&p.st->done)) return;   // the loop has stopped: nothing to compute

    const int64_t t_begin = int64_t(b) * p.T / p.G;
    const int64_t t_end = int64_t(b + 1) * p.T / p.G;
    const int nq = static_cast<int>(t_end - t_begin);   // >= 1 because G <= T

    auto issue = [&](int q, const Cursor& c) {
        const int stage = q % STAGES;
        atomicMax(&s_issued, q + 1);
        const uint32_t bar = smem_u32(&full[stage]);
        mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
        tma_load_2d(smem_u32(stages + size_t(stage) * S::STAGE_ELEMS), &tm.map[c.l], c.I * RB + c.s * CW,
                    c.I * RB, bar);
    };

    Cursor pc;   // cursor of the sub-tile STAGES ahead (every warp keeps its own copy)
    cursor_init(pc, t_begin, p);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            released[s] = 0;
        }
        for (int s = 0; s < SLOTS; ++s) {
            mbar_init(smem_u32(&rfull[s]), CWARPS);
            mbar_init(smem_u32(&rempty[s]), CWARPS);
        }
        s_abort = 0;
        s_issued = 0;
        fence_barrier_init();
        for (int l = 0; l < p.m; ++l) tma_prefetch_desc(&tm.map[l]);
        Cursor c0 = pc;
        for (int q = 0; q < STAGES && q < nq; ++q) {
            issue(q, c0);
            cursor_next(c0, p);
        }
    }
    for (int q = 0; q < STAGES && q < nq; ++q) cursor_next(pc, p);
    __syncthreads();
    const volatile int* abort_flag = &s_abort;
    FF fid_total{0.f, 0.f};

    {
        // ------------------------------------------------------------ compute
        const int n = p.n;
        Cursor cc, cn;
        cursor_init(cc, t_begin, p);
        cn = cc;
        bool seg_head = (cc.s == 0);
        float xi[R][D], racc[R][D];
        auto load_rows = [&](const Cursor& c) {
            const float* Xl = p.X + int64_t(c.l) * n * D;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = c.I * RB + warp * R + r;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    xi[r][k] = (i < n) ? __ldg(Xl + int64_t(i) * D + k) : 0.f;
                    racc[r][k] = 0.f;
                }
            }
        };
        float xjn[C][D];
        auto load_cols = [&](const Cursor& c) {
            const float* Xl = p.X + int64_t(c.l) * n * D;
            const int c0 = c.I * RB + c.s * CW + lane * C;
#pragma unroll
            for (int cidx = 0; cidx < C; ++cidx)
#pragma unroll
                for (int k = 0; k < D; ++k)
                    xjn[cidx][k] = (c0 + cidx < n) ? __ldg(Xl + int64_t(c0 + cidx) * D + k) : 0.f;
        };
        load_rows(cc);
        load_cols(cn);
        FF fid{0.f, 0.f};          // fidelity of the current modality (float-float)
        int cur_l = cc.l;

        // reduce this warp's share of the columns of sub-tile qq (deferred by one)
        auto reduce_share = [&](int qq) -> bool {
            const int slot = qq % SLOTS;
            if (!mbar_wait_or_abort(smem_u32(&rfull[slot]), uint32_t((qq / SLOTS) & 1), abort_flag)) return false;
            const float* rb = red + size_t(slot) * CWARPS * D * CW;
            float* cp = p.colpart + (t_begin + qq) * int64_t(D * CW);
            constexpr int SHARE = (D * CW + CWARPS - 1) / CWARPS;
            for (int e = warp * SHARE + lane; e < (warp + 1) * SHARE && e < D * CW; e += 32) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < CWARPS; ++w) v += rb[w * D * CW + e];
                cp[e] = v;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&rempty[slot]));
            return true;
        };

        bool ok = true;
        for (int q = 0; q < nq && ok; ++q) {
            const int stage = q % STAGES;
            const int slot = q % SLOTS;
            const int r0 = cc.I * RB;
            const int c0 = r0 + cc.s * CW;
            float xj[C][D];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int k = 0; k < D; ++k) xj[c][k] = xjn[c][k];
            if (q + 1 < nq) {           // prefetch the next sub-tile's columns
                cursor_next(cn, p);
                load_cols(cn);
            }
            if (cc.l != cur_l) {        // modality changed inside this CTA's range
                fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
                fid = FF{0.f, 0.f};
                cur_l = cc.l;
            }
            const float sc = p.dscale[cc.l];

            if (!mbar_wait_or_abort(smem_u32(&full[stage]), uint32_t((q / STAGES) & 1), abort_flag)) {
                ok = false;
                break;
            }
            const TD* tile = stages + size_t(stage) * S::STAGE_ELEMS;
            const bool masked = (cc.s * CW < RB) || (c0 + CW > n);
            float cacc0[C][D], cacc1[C][D];
            float sf0, sf1;
            if (!masked)
                subtile_pairs<D, TD, R, C, CW, false>(tile, warp, lane, r0, c0, n, sc, xi, xj, racc, cacc0, cacc1, sf0, sf1);
            else
                subtile_pairs<D, TD, R, C, CW, true>(tile, warp, lane, r0, c0, n, sc, xi, xj, racc, cacc0, cacc1, sf0, sf1);
            // release the stage; the last warp to do so refills it with sub-tile q + STAGES
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                // use k = q / STAGES of this stage is fully released at count (k+1)*CWARPS
                if (atomicAdd(&released[stage], 1) == (q / STAGES + 1) * CWARPS - 1) {
                    __threadfence_block();
                    if (q + STAGES < nq) issue(q + STAGES, pc);
                }
            }
            if (q + STAGES < nq) cursor_next(pc, p);
            fid = ff_add(fid, sf0 + sf1);

            // column partials of this sub-tile into its ring slot
            if (q >= SLOTS &&
                !mbar_wait_or_abort(smem_u32(&rempty[slot]), uint32_t(((q / SLOTS) - 1) & 1), abort_flag)) {
                ok = false;
                break;
            }
            float* rb = red + (size_t(slot) * CWARPS + warp) * D * CW;
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int c = 0; c < C; ++c) rb[k * CW + lane * C + c] = cacc0[c][k] + cacc1[c][k];
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&rfull[slot]));

            if (q >= 1 && !reduce_share(q - 1)) {
                ok = false;
                break;
            }

            const bool walk_ends = (cc.s + 1 == cc.L);
            const bool last = (q + 1 == nq);
            if (walk_ends || last) {
                // row partials of this walk segment: full-warp sum of each accumulator
                float* dst = seg_head
                    ? p.rowhead + (int64_t(cc.l) * p.nRB + cc.I) * (D * RB)
                    : p.rowcont + int64_t(b) * (D * RB);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float v = warp_sum_f32(racc[r][k]);
                        if (lane == ((r * D + k) & 31)) dst[k * RB + warp * R + r] = v;
                    }
            }
            cursor_next(cc, p);
            if (walk_ends && !last) {
                seg_head = true;
                load_rows(cc);
            }
        }
        if (ok) ok = reduce_share(nq - 1);
        if (!ok) {
            atomicExch(&s_abort, 1);
            if (lane == 0) raise_error(p.st, FJOFC_ERR_TIMEOUT, 2);
        }
        fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {
        // wait (bounded) for the copies this CTA may still have in flight: the most
        // recent use of every stage
        const int hi = s_issued;
        for (int qq = (hi > STAGES ? hi - STAGES : 0); qq < hi; ++qq)
            (void)mbar_wait_bounded(smem_u32(&full[qq % STAGES]), uint32_t((qq / STAGES) & 1));
    }

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
    return K1Geom{S::R, S::C, S::CWARPS, S::STAGES, S::RB, S::CW, S::NT, S::SMEM};
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

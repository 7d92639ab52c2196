// K1: the fused all-pairs pass of one Guttman transform (Eq. B, Eq. update,
// Remark faststress), upper triangle of every Delta_l only.
//
// For every unordered pair {i, j} (i < j) of modality l the pass forms
//     d_ij = ||x_i - x_j||,  b_ij = Delta_ij / d_ij  (0 when d_ij = 0, Eq. B),
// and adds   b_ij (x_i - x_j)  to row i and  b_ij (x_j - x_i)  to row j of B'_l X_l
// (B'_l = B_l / w_ll; since B_l's diagonal is minus its off-diagonal row sum,
// (B_l X_l)_i = sum_j b_ij (x_i - x_j) w_ll), plus w_ll (s_l Delta_ij - d_ij)^2 to the
// fidelity.  Reading the symmetric Delta once per unordered pair is the half of
// Remark faststress's 1/2 ||Delta_i - d(X^(i))||_F^2.
//
// Work layout (GB300): a persistent grid of G CTAs, CTA b owning the contiguous range
// [b*T/G, (b+1)*T/G) of RB x CW sub-tiles in walk order.  Each sub-tile is staged
// HBM -> shared memory by one TMA (cp.async.bulk.tensor) into a STAGES-deep ring
// completed on mbarriers; thread 0 refills a stage right after the CTA-wide barrier
// that ends its use.  Warp w owns R consecutive rows of the row block (x_i and the
// row accumulators live in registers for the whole walk segment); lane owns C
// consecutive columns of every sub-tile.  Column accumulators are reduced across
// warps through shared memory once per sub-tile and written as one partial per
// (sub-tile, column); row accumulators are reduced across the warp once per walk
// segment.  K2 sums all partials in a fixed order, so results are bitwise
// reproducible run to run.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"

namespace fjofc {

template <int D> struct K1Cfg;
// rows/thread, cols/lane, warps, pipeline stages (stage bytes at float32 in comments)
#define FJOFC_K1CFG(DMIN, DMAX, R_, C_, W_, S_)                                  \
    template <> struct K1Cfg<DMIN> { static constexpr int R = R_, C = C_, WARPS = W_, STAGES = S_; };
FJOFC_K1CFG(1, 1, 16, 2, 8, 5)    // 128 x 64, 32 KB
FJOFC_K1CFG(2, 2, 16, 2, 8, 5)
FJOFC_K1CFG(3, 3, 16, 2, 8, 5)
FJOFC_K1CFG(4, 4, 16, 2, 8, 5)
FJOFC_K1CFG(5, 5, 8, 2, 8, 6)     // 64 x 64, 16 KB
FJOFC_K1CFG(6, 6, 8, 2, 8, 6)
FJOFC_K1CFG(7, 7, 8, 2, 8, 6)
FJOFC_K1CFG(8, 8, 8, 2, 8, 6)
FJOFC_K1CFG(9, 9, 4, 2, 8, 8)     // 32 x 64, 8 KB
FJOFC_K1CFG(10, 10, 4, 2, 8, 8)
FJOFC_K1CFG(11, 11, 4, 2, 8, 8)
FJOFC_K1CFG(12, 12, 4, 2, 8, 8)
FJOFC_K1CFG(13, 13, 4, 2, 8, 8)
FJOFC_K1CFG(14, 14, 4, 2, 8, 8)
FJOFC_K1CFG(15, 15, 4, 2, 8, 8)
FJOFC_K1CFG(16, 16, 4, 2, 8, 8)
#undef FJOFC_K1CFG

template <int D, typename TD>
struct K1Shape {
    static constexpr int R = K1Cfg<D>::R, C = K1Cfg<D>::C, WARPS = K1Cfg<D>::WARPS,
                         STAGES = K1Cfg<D>::STAGES;
    static constexpr int NT = WARPS * 32;
    static constexpr int RB = WARPS * R;
    static constexpr int CW = 32 * C;
    static constexpr int STAGE_ELEMS = RB * CW;
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(TD);
    static constexpr size_t RED_BYTES = size_t(2) * WARPS * D * CW * sizeof(float);
    static constexpr size_t SMEM = size_t(STAGES) * STAGE_BYTES + RED_BYTES + STAGES * 8 + 128;
};

// Position of a sub-tile: modality l, row block I, walk position s (walk length L).
struct Cursor {
    int64_t t;
    int l, I, s, L;
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
    c.I = lo;
    c.s = static_cast<int>(r - __ldg(p.walk_off + lo));
    c.L = static_cast<int>(__ldg(p.walk_off + lo + 1) - __ldg(p.walk_off + lo));
}

__device__ __forceinline__ void cursor_next(Cursor& c, const K1Params& p) {
    ++c.t;
    if (++c.s == c.L) {
        c.s = 0;
        if (++c.I == p.nRB) { c.I = 0; ++c.l; }
        if (c.l < p.m) c.L = static_cast<int>(__ldg(p.walk_off + c.I + 1) - __ldg(p.walk_off + c.I));
    }
}

template <int D, typename TD>
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, 1)
k_guttman_pass(const __grid_constant__ TMaps tm, const K1Params p) {
    using S = K1Shape<D, TD>;
    constexpr int R = S::R, C = S::C, WARPS = S::WARPS, STAGES = S::STAGES, NT = S::NT;
    constexpr int RB = S::RB, CW = S::CW;

    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base for the TMA destinations
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    TD* stages = reinterpret_cast<TD*>(smem);
    float* red = reinterpret_cast<float*>(smem + size_t(STAGES) * S::STAGE_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(red + 2 * WARPS * D * CW);
    __shared__ double s_red64[WARPS];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x;

    if (ld_volatile(&p.st->done)) return;   // the loop has stopped: nothing to compute

    const int64_t t_begin = int64_t(b) * p.T / p.G;
    const int64_t t_end = int64_t(b + 1) * p.T / p.G;
    const int64_t nq = t_end - t_begin;      // >= 1 because G <= T

    Cursor pc;   // producer cursor (thread 0 only)
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&full[s]), 1);
        fence_barrier_init();
        for (int l = 0; l < p.m; ++l) tma_prefetch_desc(&tm.map[l]);
    }
    __syncthreads();
    if (tid == 0) {
        cursor_init(pc, t_begin, p);
        for (int64_t q = 0; q < STAGES && q < nq; ++q) {
            const uint32_t bar = smem_u32(&full[q]);
            mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
            tma_load_2d(smem_u32(stages + q * S::STAGE_ELEMS), &tm.map[pc.l],
                        pc.I * RB + pc.s * CW, pc.I * RB, bar);
            cursor_next(pc, p);
        }
    }

    Cursor cc;
    cursor_init(cc, t_begin, p);
    bool seg_head = (cc.s == 0);

    const int n = p.n;
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
    load_rows(cc);

    double sfid = 0.0;
    bool failed = false;

    for (int64_t q = 0; q < nq; ++q) {
        const int stage = static_cast<int>(q % STAGES);
        const uint32_t parity = static_cast<uint32_t>((q / STAGES) & 1);
        const int r0 = cc.I * RB;
        const int c0 = r0 + cc.s * CW;
        const float* Xl = p.X + int64_t(cc.l) * n * D;

        float xj[C][D], cacc[C][D];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int j = c0 + lane * C + c;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                xj[c][k] = (j < n) ? __ldg(Xl + int64_t(j) * D + k) : 0.f;
                cacc[c][k] = 0.f;
            }
        }
        const float sc = p.dscale[cc.l];

        failed |= !mbar_wait_bounded(smem_u32(&full[stage]), parity);

        const TD* tile = stages + size_t(stage) * S::STAGE_ELEMS;
        const bool masked = (cc.s * CW < RB) || (c0 + CW > n);
        float sf = 0.f;
        if (!masked) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
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
                    const float bb = dl[c] * rinv;
                    const float e = fmaf(sc, dl[c], -(d2 * rinv));
                    sf = fmaf(e, e, sf);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        racc[r][k] = fmaf(bb, diff[k], racc[r][k]);
                        cacc[c][k] = fmaf(-bb, diff[k], cacc[c][k]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = r0 + warp * R + r;
                float dl[C];
                load_delta_row<TD, C>(tile + (warp * R + r) * CW + lane * C, dl);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int j = c0 + lane * C + c;
                    const bool valid = (j > i) && (j < n);
                    float diff[D];
                    float d2 = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        diff[k] = xi[r][k] - xj[c][k];
                        d2 = fmaf(diff[k], diff[k], d2);
                    }
                    const float rinv = rsqrt_approx(fmaxf(d2, FLT_MIN));
                    const float bb = valid ? dl[c] * rinv : 0.f;
                    const float e = valid ? fmaf(sc, dl[c], -(d2 * rinv)) : 0.f;
                    sf = fmaf(e, e, sf);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        racc[r][k] = fmaf(bb, diff[k], racc[r][k]);
                        cacc[c][k] = fmaf(-bb, diff[k], cacc[c][k]);
                    }
                }
            }
        }
        sfid += double(p.wfid[cc.l]) * double(sf);

        float* rbuf = red + (q & 1) * (WARPS * D * CW);
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
            for (int c = 0; c < C; ++c) rbuf[(warp * D + k) * CW + lane * C + c] = cacc[c][k];

        if (__syncthreads_or(failed)) {
            // A stage never arrived within the wait limit: record it, wait (bounded)
            // for the copies this CTA still has in flight, and leave.
            if (tid == 0) {
                raise_error(p.st, FJOFC_ERR_TIMEOUT, 1);
                for (int64_t qq = q; qq < q + STAGES && qq < nq; ++qq)
                    (void)mbar_wait_bounded(smem_u32(&full[qq % STAGES]), uint32_t((qq / STAGES) & 1));
            }
            return;
        }

        // refill the stage everyone has just finished reading
        if (tid == 0 && q + STAGES < nq) {
            const uint32_t bar = smem_u32(&full[stage]);
            mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
            tma_load_2d(smem_u32(stages + size_t(stage) * S::STAGE_ELEMS), &tm.map[pc.l],
                        pc.I * RB + pc.s * CW, pc.I * RB, bar);
            cursor_next(pc, p);
        }

        // column partials of this sub-tile: fixed-order sum over the warps
        float* cp = p.colpart + cc.t * int64_t(D * CW);
        for (int e = tid; e < D * CW; e += NT) {
            const int k = e / CW, c = e - k * CW;
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) v += rbuf[(w * D + k) * CW + c];
            cp[e] = v;
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

    // fidelity partial of this CTA (fixed-order float64 reduction)
    const double ws = warp_sum_f64(sfid);
    if (lane == 0) s_red64[warp] = ws;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) tot += s_red64[w];
        p.fid[b] = tot;
    }
}

template <int D, typename TD>
cudaError_t k1_launch_impl(int grid, const TMaps& tm, const K1Params& p, cudaStream_t s) {
    using S = K1Shape<D, TD>;
    static bool configured = false;   // attribute set once per process and device family
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_guttman_pass<D, TD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
        if (e != cudaSuccess) return e;
        configured = true;
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
    return K1Geom{S::R, S::C, S::WARPS, S::STAGES, S::RB, S::CW, S::NT, S::SMEM};
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

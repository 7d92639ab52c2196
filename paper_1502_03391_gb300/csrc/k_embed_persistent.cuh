// The whole in-sample loop (Algorithm 2's while-loop from X_0) as one persistent,
// cooperatively launched kernel: one CTA per SM, resident for every pass.
//
// Pass t (reads X_{t-1}, writes X_t):
//   A. the fused all-pairs sub-tiles of this CTA's fixed range (same work, layout and
//      partials as k_guttman_pass; see k_guttman_pass.cuh), fidelity partial -> fid[t&1][b];
//   -- grid barrier --
//   B. for object groups g = b, b+G, ... (32 objects each): sum the partials, centre
//      X_{t-1} in place with the previous pass's means, its commensurability, the Wmod^-1
//      mix into X_t (Eq. update / Cor. 1) and per-group float-float sums -> bpart[g];
//   -- grid barrier --
//   C. every CTA reduces bpart and fid in the same fixed order, so all CTAs obtain the
//      same means of X_t, sigma(X_{t-1}) and stopping decision (Algorithm 1 with the
//      decrease reading); CTA 0 records the history.
// Data written by other CTAs earlier in the same launch (iterates, partials) is read with
// ld.global.cg (L2, never a possibly stale L1 line); the grid barrier orders the phases.
// Delta does not change between passes, so the TMA ring keeps prefetching the next
// pass's first sub-tiles while phases B and C run.  Grid barriers and every other wait
// are bounded (FJOFC_ERR_TIMEOUT instead of a hang).
#pragma once

#include "k_guttman_pass.cuh"
#include "k_apply_common.cuh"

namespace fjofc {


__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over a monotone counter: arrival k of every CTA waits for G*k
// arrivals.  Bounded: returns false after kWaitLimitNs (or when *abort_flag is set).
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* s_flag,
                                             const volatile int* abort_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        bool ok = true;
        if (ld_acquire_gpu(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1;; ++it) {
                if (ld_acquire_gpu(ctr) >= target) break;
                if ((it & 63u) == 0u && (*abort_flag || globaltimer_ns() - t0 > kWaitLimitNs)) {
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        *s_flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

template <int D, typename TD>
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, 1)
k_embed_persistent(const __grid_constant__ TMaps tm, const PersistParams P) {
    using S = K1Shape<D, TD>;
    constexpr int R = S::R, C = S::C, CWARPS = S::CWARPS, STAGES = S::STAGES, SLOTS = S::SLOTS;
    constexpr int RB = S::RB, CW = S::CW, NT = S::NT;
    constexpr int GOBJ = 32;
    const K1Params& p = P.k1;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    TD* stages = reinterpret_cast<TD*>(smem);
    float* red = reinterpret_cast<float*>(smem + size_t(STAGES) * S::STAGE_BYTES);   // [SLOTS][CWARPS][D][CW]
    uint64_t* full = reinterpret_cast<uint64_t*>(red + S::RED_FLOATS);
    uint64_t* rfull = full + STAGES;
    uint64_t* rempty = rfull + SLOTS;
    int* released = reinterpret_cast<int*>(rempty + SLOTS);
    float* s_bx = red;                          // phase B overlay: [m*d][32] floats
    static_assert(S::RED_FLOATS >= FJOFC_MAX_M * D * GOBJ, "phase-B overlay does not fit");
    __shared__ FF s_ff[CWARPS];
    __shared__ FF s_part[FJOFC_MAX_M * FJOFC_MAX_D];
    __shared__ float s_mu[FJOFC_MAX_M * FJOFC_MAX_D];
    __shared__ int s_abort, s_issued, s_flag, s_stop, s_final;
    __shared__ double s_prev;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, G = p.G;
    const int m = p.m, n = p.n;
    const int passes = P.max_iter + 1;
    const int64_t t_begin = P.cta_start[b];
    const int nq = static_cast<int>(P.cta_start[b + 1] - t_begin);
    const int64_t total_q = int64_t(passes) * nq;     // sub-tiles this CTA may ever issue

    // issue the sub-tile with global index qg (pass-major; the range wraps every pass)
    Cursor pc;
    cursor_init(pc, t_begin, p);
    int pc_local = 0;                                  // position of pc within the range
    auto issue = [&](int64_t qg) {
        const int stage = int(qg % STAGES);
        atomicMax(&s_issued, int(qg + 1));
        const uint32_t bar = smem_u32(&full[stage]);
        mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
        tma_load_2d(smem_u32(stages + size_t(stage) * S::STAGE_ELEMS), &tm.map[pc.l], pc.I * RB + pc.s * CW,
                    pc.I * RB, bar);
    };
    auto advance_pc = [&]() {
        if (++pc_local == nq) {
            pc_local = 0;
            cursor_init(pc, t_begin, p);
        } else {
            cursor_next(pc, p);
        }
    };

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
        s_stop = 0;
        s_final = 0;
        s_prev = 0.0;
        fence_barrier_init();
        for (int l = 0; l < m; ++l) tma_prefetch_desc(&tm.map[l]);
    }
    for (int e = tid; e < FJOFC_MAX_M * FJOFC_MAX_D; e += NT) s_mu[e] = 0.f;
    __syncthreads();
    if (tid == 0) {
        for (int64_t q = 0; q < STAGES && q < total_q; ++q) {
            issue(q);
            advance_pc();
        }
    }
    // every thread keeps its own copy of the prefetch cursor STAGES ahead
    if (tid != 0)
        for (int64_t q = 0; q < STAGES && q < total_q; ++q) advance_pc();
    __syncthreads();
    const volatile int* abort_flag = &s_abort;
    unsigned bar_target = 0;
    bool ok = true;
    int last_finite = 0;          // newest iterate whose stress was finite
    int t = 1;

    for (; t <= passes && ok; ++t) {
        const bool final_pass = (t == passes);
        const float* X = P.buf[(t - 1) % 3];
        const int64_t qbase = int64_t(t - 1) * nq;

        // ================================================================ phase A
        FF fid_total{0.f, 0.f};
        {
            Cursor cc, cn;
            cursor_init(cc, t_begin, p);
            cn = cc;
            bool seg_head = (cc.s == 0);
            float xi[R][D], racc[R][D], xjn[C][D];
            auto load_rows = [&](const Cursor& c) {
                const float* Xl = X + int64_t(c.l) * n * D;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = c.I * RB + warp * R + r;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        xi[r][k] = (i < n) ? __ldcg(Xl + int64_t(i) * D + k) : 0.f;
                        racc[r][k] = 0.f;
                    }
                }
            };
            auto load_cols = [&](const Cursor& c) {
                const float* Xl = X + int64_t(c.l) * n * D;
                const int c0 = c.I * RB + c.s * CW + lane * C;
#pragma unroll
                for (int ci = 0; ci < C; ++ci)
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        xjn[ci][k] = (c0 + ci < n) ? __ldcg(Xl + int64_t(c0 + ci) * D + k) : 0.f;
            };
            load_rows(cc);
            load_cols(cn);
            FF fid{0.f, 0.f};
            int cur_l = cc.l;

            auto reduce_share = [&](int64_t qg, int64_t tglob) -> bool {
                const int slot = int(qg % SLOTS);
                if (!mbar_wait_or_abort(smem_u32(&rfull[slot]), uint32_t((qg / SLOTS) & 1), abort_flag)) return false;
                const float* rb = red + size_t(slot) * CWARPS * D * CW;
                float* cp = p.colpart + tglob * int64_t(D * CW);
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

            for (int q = 0; q < nq && ok; ++q) {
                const int64_t qg = qbase + q;
                const int stage = int(qg % STAGES);
                const int slot = int(qg % SLOTS);
                const int r0 = cc.I * RB;
                const int c0 = r0 + cc.s * CW;
                float xj[C][D];
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int k = 0; k < D; ++k) xj[c][k] = xjn[c][k];
                if (q + 1 < nq) {
                    cursor_next(cn, p);
                    load_cols(cn);
                }
                if (cc.l != cur_l) {
                    fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
                    fid = FF{0.f, 0.f};
                    cur_l = cc.l;
                }
                const float sc = p.dscale[cc.l];
                if (!mbar_wait_or_abort(smem_u32(&full[stage]), uint32_t((qg / STAGES) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                const TD* tile = stages + size_t(stage) * S::STAGE_ELEMS;
                const bool masked = (cc.s * CW < RB) || (c0 + CW > n);
                float cacc0[C][D], cacc1[C][D];
                float sf0, sf1;
                if (!masked)
                    subtile_pairs<D, TD, R, C, CW, false>(tile, warp, lane, r0, c0, n, sc, xi, xj, racc, cacc0, cacc1,
                                                          sf0, sf1);
                else
                    subtile_pairs<D, TD, R, C, CW, true>(tile, warp, lane, r0, c0, n, sc, xi, xj, racc, cacc0, cacc1,
                                                         sf0, sf1);
                // release the stage; the last warp to do so refills it (next pass wraps)
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();
                    if (atomicAdd(&released[stage], 1) == int(qg / STAGES + 1) * CWARPS - 1) {
                        __threadfence_block();
                        if (qg + STAGES < total_q) issue(qg + STAGES);
                    }
                }
                if (qg + STAGES < total_q) advance_pc();
                fid = ff_add(fid, sf0 + sf1);

                if (qg >= SLOTS &&
                    !mbar_wait_or_abort(smem_u32(&rempty[slot]), uint32_t(((qg / SLOTS) - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                float* rbuf = red + (size_t(slot) * CWARPS + warp) * D * CW;
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int c = 0; c < C; ++c) rbuf[k * CW + lane * C + c] = cacc0[c][k] + cacc1[c][k];
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&rfull[slot]));
                if (q >= 1 && !reduce_share(qg - 1, cc.t - 1)) {
                    ok = false;
                    break;
                }
                const bool walk_ends = (cc.s + 1 == cc.L);
                const bool last = (q + 1 == nq);
                if (walk_ends || last) {
                    float* dst = seg_head ? p.rowhead + (int64_t(cc.l) * p.nRB + cc.I) * (D * RB)
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
            if (ok) ok = reduce_share(qbase + nq - 1, t_begin + nq - 1);
            fid_total = ff_add(fid_total, ff_mul(fid, p.wfid[cur_l]));
        }
        if (!ok) atomicExch(&s_abort, 1);
        {
            const FF ws = warp_sum_ff(fid_total);
            __syncthreads();
            if (lane == 0) s_ff[warp] = ws;
            __syncthreads();
            if (tid == 0) {
                FF tot{0.f, 0.f};
#pragma unroll
                for (int w = 0; w < CWARPS; ++w) tot = ff_add(tot, s_ff[w]);
                P.fid2[(t & 1) * G + b] = make_float2(tot.hi, tot.lo);
            }
        }
        bar_target += unsigned(G);
        if (!grid_barrier(P.bar, bar_target, &s_flag, abort_flag) || *abort_flag) {
            ok = false;
            break;
        }

        // ================================================================ phase B
        float* Xprev = P.buf[(t - 1) % 3];
        float* Xnext = P.buf[t % 3];
        for (int g = b; g < P.ngroups; g += G) {
            const int i = g * GOBJ + lane;
            if (!final_pass)
                for (int lk = warp; lk < m * D; lk += CWARPS) {
                    const int l = lk / D, k = lk - l * D;
                    s_bx[lk * GOBJ + lane] = (i < n) ? bx_partials(P.tb, l, k, i) : 0.f;
                }
            __syncthreads();
            FF comm{0.f, 0.f};
            for (int k = warp; k < D; k += CWARPS) {
                float cm, xn[FJOFC_MAX_M];
                mix_and_centre(Xprev, Xnext, m, n, D, i, k, t, final_pass, s_mu, P.coef, P.wcomm,
                               s_bx + k * GOBJ + lane, D * GOBJ, &cm, xn);
                comm = ff_add(comm, cm);
                if (!final_pass)
                    for (int j = 0; j < m; ++j) {
                        const FF cs = warp_sum_ff(FF{xn[j], 0.f});
                        if (lane == 0) s_part[j * D + k] = cs;
                    }
            }
            const FF cw = warp_sum_ff(comm);
            __syncthreads();
            if (lane == 0) s_ff[warp] = cw;
            __syncthreads();
            if (tid == 0) {
                FF tot{0.f, 0.f};
                for (int w = 0; w < CWARPS; ++w) tot = ff_add(tot, s_ff[w]);
                const int npart = m * D + 1;
                for (int e = 0; e < m * D; ++e)
                    P.bpart[int64_t(g) * npart + e] =
                        final_pass ? make_float2(0.f, 0.f) : make_float2(s_part[e].hi, s_part[e].lo);
                P.bpart[int64_t(g) * npart + m * D] = make_float2(tot.hi, tot.lo);
            }
            __syncthreads();
        }
        bar_target += unsigned(G);
        if (!grid_barrier(P.bar, bar_target, &s_flag, abort_flag)) {
            ok = false;
            break;
        }

        // ================================================================ phase C
        {
            // one warp per total: m*D column sums, commensurability, fidelity (all loads
            // of a lane in one round); the same order in every CTA
            const int npart = m * D + 1;
            __shared__ FF s_tot[FJOFC_MAX_M * FJOFC_MAX_D + 2];
            for (int e = warp; e < npart + 1; e += CWARPS)
                s_tot[e] = (e < npart) ? totals_ff(P.bpart + e, npart, P.ngroups)
                                       : totals_ff(P.fid2 + (t & 1) * G, 1, G);
            __syncthreads();
            if (tid == 0) {
                for (int e = 0; e < m * D; ++e)
                    s_mu[(e / D) * FJOFC_MAX_D + (e % D)] =
                        final_pass ? 0.f : (s_tot[e].hi + s_tot[e].lo) / float(n);
                const FF ct = s_tot[npart - 1], ft = s_tot[npart];
                const double sigma = (double(ft.hi) + double(ft.lo)) + (double(ct.hi) + double(ct.lo));
                const int tp = t - 1;
                int stop = final_pass ? 1 : 0;
                if (b == 0) P.hist[tp] = sigma;
                if (!isfinite(sigma)) {
                    stop = 2;                         // non-finite: keep the last finite iterate
                } else {
                    last_finite = tp;
                    if (!stop && tp >= 1 && P.tol >= 0.0) {
                        const double dec = s_prev - sigma;
                        const bool cont = (P.tol_mode == FJOFC_TOL_RELATIVE) ? (dec > P.tol * s_prev)
                                                                             : (dec / P.npairs > P.tol);
                        if (!cont) stop = 1;
                    }
                    s_prev = sigma;
                }
                s_stop = stop;
                s_final = last_finite;
                if (b == 0) {
                    DevStatus* st = p.st;
                    if (stop == 2) st->error = FJOFC_ERR_NONFINITE;
                    else {
                        st->final_iter = tp;
                        st->stress = sigma;
                    }
                    if (stop) st->done = 1;
                }
            }
            __syncthreads();
            if (s_stop) break;
        }
    }

    if (!ok && tid == 0) {
        atomicExch(&s_abort, 1);
        raise_error(p.st, FJOFC_ERR_TIMEOUT, 3);
    }
    __syncthreads();
    // wait (bounded) for the sub-tiles prefetched for passes that did not run
    if (tid == 0) {
        const int hi = s_issued;
        for (int qq = (hi > STAGES ? hi - STAGES : 0); qq < hi; ++qq)
            (void)mbar_wait_bounded(smem_u32(&full[qq % STAGES]), uint32_t((qq / STAGES) & 1));
    }
    // the returned iterate (centred in place by the pass that computed its stress) goes
    // to the caller's buffer
    if (ok) {
        const int f = s_final;
        if (f % 3 != 0) {
            const float* src = P.buf[f % 3];
            float* dst = P.buf[0];
            const int64_t count = int64_t(m) * n * D;
            for (int64_t e = int64_t(b) * NT + tid; e < count; e += int64_t(G) * NT) dst[e] = __ldcg(src + e);
        }
    }
}

template <int D, typename TD>
cudaError_t persist_launch_impl(int grid, const TMaps& tm, const PersistParams& P, cudaStream_t s) {
    using S = K1Shape<D, TD>;
    cudaError_t e = cudaFuncSetAttribute(k_embed_persistent<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(S::SMEM));
    if (e != cudaSuccess) return e;
    void* args[2] = {const_cast<TMaps*>(&tm), const_cast<PersistParams*>(&P)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_embed_persistent<D, TD>), dim3(grid),
                                       dim3(S::NT), args, S::SMEM, s);
}

template <int D, typename TD>
int persist_bps_impl() {
    using S = K1Shape<D, TD>;
    cudaFuncSetAttribute(k_embed_persistent<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_embed_persistent<D, TD>, S::NT, S::SMEM) != cudaSuccess)
        return 0;
    return nb;
}

#define FJOFC_INSTANTIATE_PERSIST(D)                                                                  \
    template cudaError_t persist_launch_impl<D, float>(int, const TMaps&, const PersistParams&, cudaStream_t); \
    template cudaError_t persist_launch_impl<D, __half>(int, const TMaps&, const PersistParams&, cudaStream_t); \
    template cudaError_t persist_launch_impl<D, __nv_bfloat16>(int, const TMaps&, const PersistParams&,     \
                                                               cudaStream_t);                            \
    template int persist_bps_impl<D, float>();                                                           \
    template int persist_bps_impl<D, __half>();                                                          \
    template int persist_bps_impl<D, __nv_bfloat16>();

}  // namespace fjofc

// The whole in-sample loop (Algorithm 2's while-loop from X_0) as one persistent,
// cooperatively launched kernel: one CTA per SM, resident for every pass.
//
// Pass t (reads X_{t-1}, writes X_t):
//   A. the fused all-pairs sub-tiles of this CTA's fixed range (phase_a, the same code as
//      the standalone pass k_guttman_pass), fidelity partial -> fid2[t&1][b];
//   C. one CTA with the fewest sub-tiles reduces the fidelity partials of pass t-1 and
//      phase B's per-group parts of pass t-1 in a fixed order and publishes the totals;
//   -- grid barrier --
//      every CTA reads the totals and takes the same means of X_{t-1}, sigma(X_{t-2}) and
//      stopping decision about X_{t-2} (Algorithm 1 with the decrease reading); the totals
//      CTA records the history;
//   B. for the (group, coordinate) units of this CTA (phase_b, the same code as K2): sum
//      the partials, centre X_{t-1} in place with its means, its commensurability, the
//      Wmod^-1 mix into X_t (Eq. update / Cor. 1) and per-group float-float sums;
//   -- grid barrier --
// The decision about an iterate is taken one pass after its stress is complete (the
// all-pairs pass computed meanwhile is discarded at a stop).
// Data written by other CTAs earlier in the same launch (iterates, partials) is read with
// ld.global.cg (L2, never a possibly stale L1 line); the grid barrier orders the phases.
// Delta does not change between passes, so the TMA ring keeps prefetching the next
// pass's first sub-tiles while phases C and B run.  Grid barriers and every other wait
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
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Arrival on a grid barrier counter: a reduction with release semantics at GPU scope (the
// CTA's earlier writes, ordered before this thread by the preceding CTA barrier, are
// visible to any thread that acquires the counter's new value; no separate fence, no
// returned value).  The waiting side's ld.acquire.gpu orders the CTA's later reads.
__device__ __forceinline__ void grid_count_arrive(unsigned* ctr) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(ctr) : "memory");
}

// Barrier of the G CTAs of one problem over a monotone counter: arrival k of every CTA
// waits for G*k arrivals (G == 1: a CTA barrier).  Bounded: returns false after
// limit_ns (or when *abort_flag is set).
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* s_flag,
                                             const volatile int* abort_flag, int G, uint64_t limit_ns) {
    if (G == 1) {
        __threadfence();
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        grid_count_arrive(ctr);
        bool ok = true;
        if (ld_acquire_gpu(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1;; ++it) {
                if (ld_acquire_gpu(ctr) >= target) break;
                if ((it & 63u) == 0u && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) {
                    ok = false;
                    break;
                }
            }
        }
        *s_flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

// The same barrier in two halves, so that a CTA can work between its arrival and the
// completion: grid_arrive (every thread; the CTA's earlier writes are published before
// the arrival) and grid_wait (every thread; bounded like grid_barrier).
__device__ __forceinline__ void grid_arrive(unsigned* ctr, int G) {
    __syncthreads();
    if (G > 1 && threadIdx.x == 0) grid_count_arrive(ctr);
}
// grid_wait that, while it spins, also copies the pass totals the totals CTA published
// (npub float2 at pub, valid once *seq == t) into out; *s_have tells whether it did.
__device__ __forceinline__ bool grid_wait_pub(unsigned* ctr, unsigned target, int* s_flag,
                                              const volatile int* abort_flag, int G, uint64_t limit_ns,
                                              const unsigned* seq, unsigned t, const float2* pub, int npub, FF* out,
                                              int* s_have) {
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true, have = false;
        const uint64_t t0 = globaltimer_ns();
        for (uint32_t it = 1;; ++it) {
            if (!have && ld_acquire_gpu(seq) == t) {
                for (int e = 0; e < npub; ++e) {
                    const float2 v = __ldcg(pub + e);
                    out[e] = FF{v.x, v.y};
                }
                have = true;
            }
            if (ld_acquire_gpu(ctr) >= target) break;
            if ((it & 63u) == 0u && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) {
                ok = false;
                break;
            }
        }
        *s_flag = ok ? 1 : 0;
        *s_have = have ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ bool grid_wait(unsigned* ctr, unsigned target, int* s_flag, const volatile int* abort_flag,
                                          int G, uint64_t limit_ns) {
    if (G == 1) {
        __threadfence();
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        if (ld_acquire_gpu(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1;; ++it) {
                if (ld_acquire_gpu(ctr) >= target) break;
                if ((it & 63u) == 0u && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) {
                    ok = false;
                    break;
                }
            }
        }
        *s_flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Per-phase clock stamps of passes 2..17 (instrumented builds, -DFJOFC_STAMPS): thread 0 of
// every CTA records clock64 at the start of phase A, before and after the first grid
// barrier, after phase C, after phase B and after phase C's totals.
#ifdef FJOFC_STAMPS
constexpr int kStampPasses = 16, kStampCtas = 1024, kStampPoints = 7;
static __device__ long long g_stamps[kStampPasses * kStampCtas * kStampPoints];
#define FJ_STAMP(t, j)                                                                                   \
    do {                                                                                                 \
        if (threadIdx.x == 0 && (t) >= 2 && (t) < 2 + kStampPasses && b < kStampCtas)                   \
            g_stamps[((int64_t((t) - 2) * kStampCtas + b) * kStampPoints) + (j)] = clock64();             \
    } while (0)
#else
#define FJ_STAMP(t, j) do { } while (0)
#endif

// Column partials a lane of phase B keeps in flight (one round covers up to BATCH walks).
#ifndef FJOFC_PHASEB_BATCH_SMALLD
#define FJOFC_PHASEB_BATCH_SMALLD 16
#endif
template <int D>
struct PhaseBBatch {
    static constexpr int value = D >= 5 ? 64 : FJOFC_PHASEB_BATCH_SMALLD;
};

// The whole loop of one problem on the CTA of rank b among its P.k1.G CTAs.
template <int D, typename TD>
__device__ __forceinline__ void persist_problem(const TMaps& tm, const PersistParams& P, const int b,
                                                unsigned char* smem_raw) {
    using S = K1Shape<D, TD>;
    constexpr int CWARPS = S::CWARPS, NT = S::NT;
    const K1Params& p = P.k1;

    __shared__ FF s_ff[CWARPS];
    __shared__ int s_abort, s_issued, s_flag, s_stop, s_final, s_have;
    __shared__ double s_prev;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = p.G;
    const int m = p.m, n = p.n;
    const int passes = P.max_iter + 1;
    const int64_t t_begin = P.cta_start[b];
    const int nq = static_cast<int>(P.cta_start[b + 1] - t_begin);
    const int npart = phase_b_parts(m, D);
    const int tcb = *P.tc;                         // the totals CTA (written by the set-up kernel)
    // phase-B units (group, coordinate) of this CTA
    const int64_t nunits = int64_t(P.ngroups) * D;
    const int u0 = int(int64_t(b) * nunits / G), u1 = int(int64_t(b + 1) * nunits / G);

    K1Ring<D, TD> rg;
    rg.carve(smem_raw);
    // phases C and B reuse the column-partial ring (free between passes), and the means of
    // X_{t-1} ([m][D], from phase C to phase B) sit in the walk rows of phase A
    float* s_phb = rg.red;
    FF* s_tot = reinterpret_cast<FF*>(rg.red);     // [m*D + D + 1], phase C only
    float* s_mu = rg.xrow;
    static_assert(S::RED_FLOATS * sizeof(float) >= (FJOFC_MAX_M * D + D + 1) * sizeof(FF),
                  "phase-C totals do not fit");
    static_assert(S::XROW_FLOATS >= FJOFC_MAX_M * D, "the means do not fit in the walk rows");
    const int bcap = int(S::RED_FLOATS / size_t(phase_b_floats_per_unit(m)));
    static_assert(S::RED_FLOATS >= size_t(phase_b_floats_per_unit(FJOFC_MAX_M)), "phase-B overlay does not fit");

    // a failed input check stopped the loop before it started: every CTA of the problem
    // reads the same value (written by an earlier kernel) and leaves X as given
    if (ld_volatile(&p.st->done)) return;
    if (tid == 0) {
        s_stop = 0;
        s_final = 0;
        s_prev = 0.0;
    }
    // ring over every pass's sub-tiles; Delta does not change, so it prefetches the next
    // pass's first sub-tiles while phase B runs
    rg.start(tm, p, t_begin, nq, int64_t(passes) * nq, &s_issued, &s_abort);
    const volatile int* abort_flag = &s_abort;
    unsigned bar_target = 0;
    bool ok = true;
    int fail_site = 0;            // 31: all-pairs pass wait, 32: barrier after A, 33: barrier after B
    int last_finite = 0;          // newest iterate whose stress was finite

    // Pass t (t = 1 .. passes) reads X_{t-1}; a last round t = passes + 1 only decides.
    //   A(t): all pairs of X_{t-1} -> partials, fidelity of X_{t-1} -> fid2[t & 1]
    //   -- grid barrier, arrival --
    //   C(t): totals of fid2[(t-1) & 1] and of B(t-1)'s parts -> means of X_{t-1},
    //         sigma(X_{t-2}) and the stopping decision about X_{t-2}
    //   -- grid barrier, wait --
    //   B(t): centre X_{t-1}, its commensurability, X_t (none in the final pass)
    //   -- grid barrier --
    // The decision comes one pass after the iterate it concerns (a stop discards the
    // all-pairs pass computed meanwhile), so that the totals are formed while the CTA
    // waits for the slowest one to finish phase A.
    for (int t = 1; ok; ++t) {
        const bool do_a = t <= passes;
        float* Xprev = P.buf[(t - 1) % 3];
        float* Xnext = P.buf[t % 3];

        // ================================================================ phase A
        FJ_STAMP(t, 0);
        if (do_a) {
            FF fid_total{0.f, 0.f};
            bool ok_a;
            if constexpr (S::STRIP) ok_a = phase_a_strip<D, TD>(rg, tm, p, Xprev, int64_t(t - 1) * nq, b, fid_total);
            else ok_a = phase_a<D, TD>(rg, tm, p, Xprev, int64_t(t - 1) * nq, b, fid_total);
            if (!ok_a) {
                ok = false;
                fail_site = 31;
            }
            if (!ok) atomicExch(&s_abort, 1);
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
        FJ_STAMP(t, 1);
        bar_target += unsigned(G);
        // ================================================================ phase C
        // The totals of pass t-1 (phase B's parts and the fidelity partials of A(t-1),
        // complete since the previous barriers) -> means of X_{t-1}, sigma(X_{t-2}) and the
        // stopping decision about X_{t-2}.  One CTA with the least work (*P.tc) forms
        // them before it arrives at the barrier and publishes them; every other CTA reads
        // them after the barrier, so the slowest CTA does not compute them on the critical
        // path.  Every CTA then takes the same decision from the same values.
        const bool tc = (b == tcb);
        if (tc) {
            pass_totals(P.bpart + int64_t((t - 1) & 1) * P.ngroups * npart, npart, t >= 2 ? P.ngroups : 0,
                        P.fid2 + ((t - 1) & 1) * G, t >= 2 ? G : 0, s_tot);
            __syncthreads();
            if (G > 1) {
                for (int e = tid; e <= npart; e += NT) P.pub[e] = make_float2(s_tot[e].hi, s_tot[e].lo);
                __syncthreads();
                if (tid == 0) st_release_gpu(P.pub_seq, unsigned(t));   // after the totals
            }
        }
        FJ_STAMP(t, 5);
        grid_arrive(P.bar, G);
        // every CTA has finished phase A (its partial tables are complete) and no CTA still
        // reads X_{t-1} for phase A; the waiting thread of a CTA other than the totals CTA
        // copies the published totals as soon as they are out (few of them only)
        const bool prefetch = !tc && G > 1 && npart + 1 <= 64;
        const unsigned wtarget = bar_target + (t == 1 ? P.bar_skew : 0u);
        s_have = 0;
        if (!(prefetch ? grid_wait_pub(P.bar, wtarget, &s_flag, abort_flag, G, P.wait_ns, P.pub_seq, unsigned(t),
                                       P.pub, npart + 1, s_tot, &s_have)
                       : grid_wait(P.bar, wtarget, &s_flag, abort_flag, G, P.wait_ns)) ||
            *abort_flag) {
            if (ok) fail_site = 32;
            ok = false;
            break;
        }
        FJ_STAMP(t, 2);
        if (!tc && !s_have) {
            for (int e = tid; e <= npart; e += NT) {
                const float2 v = __ldcg(P.pub + e);
                s_tot[e] = FF{v.x, v.y};
            }
            __syncthreads();
        }
        for (int e = tid; e < m * D; e += NT)
            s_mu[e] = (t >= 2 && t - 1 < passes) ? (s_tot[e].hi + s_tot[e].lo) * P.inv_n : 0.f;
        if (tid == 0) {
            int stop = 0;
            if (t >= 2) {
                const int tp = t - 2;                        // the iterate decided about
                const double sigma = stress_from_totals(s_tot, s_tot[npart], m, D);
                stop = (tp == P.max_iter) ? 1 : 0;
                if (tc) P.hist[tp] = sigma;
                if (!isfinite(sigma)) {
                    stop = 2;                                // non-finite: keep the last finite iterate
                } else {
                    last_finite = tp;
                    if (!stop && tp >= 1 && P.tol >= 0.0) {
                        const double dec = s_prev - sigma;
                        const bool cont = (P.tol_mode == FJOFC_TOL_RELATIVE) ? (dec > P.tol * s_prev)
                                                                             : (dec > P.tol * P.npairs);
                        if (!cont) stop = 1;
                    }
                    s_prev = sigma;
                }
                if (tc) {
                    DevStatus* st = p.st;
                    if (stop == 2) st->error = FJOFC_ERR_NONFINITE;
                    else {
                        st->final_iter = tp;
                        st->stress = sigma;
                    }
                    if (stop) st->done = 1;
                }
            }
            s_stop = stop;
            s_final = last_finite;
        }
        __syncthreads();
        FJ_STAMP(t, 3);
        if (s_stop || !do_a) break;

        // ================================================================ phase B
        {
            PhaseBArgs a;
            a.tb = P.tb;
            a.Xprev = Xprev;
            a.Xnext = Xnext;
            a.bpart = P.bpart + int64_t(t & 1) * P.ngroups * npart;
            a.mu_prev = s_mu;
            a.mu_stride = D;
            a.coef_g = P.coef_g;
            a.wcomm_g = P.wcomm_g;
            a.m = m; a.n = n; a.d = D; a.t = t; a.ngroups = P.ngroups;
            a.centre = P.centre != 0;
            a.relax = P.relax;
            a.final_pass = (t == passes);
#ifdef FJOFC_STAMPS
            if (t >= 2 && t < 2 + kStampPasses && b < kStampCtas)
                a.stamp = &g_stamps[((int64_t(t - 2) * kStampCtas + b) * kStampPoints) + 6];
#endif
            phase_b<PhaseBBatch<D>::value>(a, u0, u1, bcap, s_phb);
        }
        FJ_STAMP(t, 4);
        // X_t is complete, and every CTA is done with pass t's partial tables, before any
        // CTA starts pass t+1
        bar_target += unsigned(G);
        if (!grid_barrier(P.bar, bar_target, &s_flag, abort_flag, G, P.wait_ns)) {
            fail_site = 33;
            ok = false;
            break;
        }
    }

    if (!ok && tid == 0) {
        atomicExch(&s_abort, 1);
        raise_error(p.st, FJOFC_ERR_TIMEOUT, fail_site);
    }
    __syncthreads();
    // wait (bounded) for the sub-tiles prefetched for passes that did not run, then retire
    // the ring's barriers (the CTA may run another problem next)
    if (tid == 0) rg.drain();
    cp_async_wait_all();
    __syncthreads();
    if (tid == 0) rg.invalidate();
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
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, FJOFC_K1_MINB)
k_embed_persistent(const __grid_constant__ TMaps tm, const __grid_constant__ PersistParams P) {
    extern __shared__ unsigned char smem_raw[];
    persist_problem<D, TD>(tm, P, blockIdx.x, smem_raw);
}

// Many independent problems of one embedding dimension in one cooperative launch: CTA b
// runs the problems of its list bl.assign[bl.cta_off[b] .. bl.cta_off[b+1]) one after the
// other, each as rank `y` of that problem's CTA group.  A problem with a group of several
// CTAs is first in all of their lists, so its ranks start together.  The problem's
// parameters are copied to shared memory; its tensor maps stay in global memory.
template <int D, typename TD>
__global__ void __launch_bounds__(K1Shape<D, TD>::NT, FJOFC_K1_MINB)
k_embed_batched(const __grid_constant__ BatchLaunch bl) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(16) PersistParams s_P;
    static_assert(sizeof(PersistParams) % 4 == 0, "PersistParams copy");
    const int b = blockIdx.x;
    for (int a = bl.cta_off[b]; a < bl.cta_off[b + 1]; ++a) {
        const int2 as = bl.assign[a];
        const unsigned* src = reinterpret_cast<const unsigned*>(bl.probs + as.x);
        unsigned* dst = reinterpret_cast<unsigned*>(&s_P);
        for (int e = threadIdx.x; e < int(sizeof(PersistParams) / 4); e += blockDim.x) dst[e] = src[e];
        __syncthreads();
        persist_problem<D, TD>(bl.maps[as.x], s_P, as.y, smem_raw);
        __syncthreads();
    }
}

template <int D, typename TD>
cudaError_t batched_launch_impl(int grid, const BatchLaunch& bl, cudaStream_t s) {
    using S = K1Shape<D, TD>;
    cudaError_t e = cudaFuncSetAttribute(k_embed_batched<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(S::SMEM));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(S::NT);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_embed_batched<D, TD>, bl);
}

template <int D, typename TD>
int batched_bps_impl() {
    using S = K1Shape<D, TD>;
    cudaFuncSetAttribute(k_embed_batched<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_embed_batched<D, TD>, S::NT, S::SMEM) != cudaSuccess)
        return 0;
    return nb;
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
    template int persist_bps_impl<D, __nv_bfloat16>();                                                   \
    template cudaError_t batched_launch_impl<D, float>(int, const BatchLaunch&, cudaStream_t);             \
    template cudaError_t batched_launch_impl<D, __half>(int, const BatchLaunch&, cudaStream_t);            \
    template cudaError_t batched_launch_impl<D, __nv_bfloat16>(int, const BatchLaunch&, cudaStream_t);     \
    template int batched_bps_impl<D, float>();                                                             \
    template int batched_bps_impl<D, __half>();                                                            \
    template int batched_bps_impl<D, __nv_bfloat16>();

}  // namespace fjofc

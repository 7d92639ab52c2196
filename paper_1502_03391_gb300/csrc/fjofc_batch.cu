// Batched in-sample embedding: many independent fJOFC problems of uneven size in one
// plan.  Problems are grouped by (embedding dimension, Delta type), the kernel
// instantiation they need; each class runs as one cooperative launch of the persistent
// loop kernel over all SMs (k_embed_batched), and the whole plan (per-problem set-up,
// the class launches, the result gather) is captured once into a CUDA graph.
//
// Scheduling (host, once per plan): the cost of a problem is its sub-tiles per pass plus
// a fixed per-pass cost (the per-object phase and totals, about kPassCost sub-tiles)
// times its number of passes; a problem split over a group pays kBarrierCost per pass
// on every rank for the group barriers.  A binary search finds the smallest per-CTA load
// M such that every problem costing more than M gets a group of its own (ceil(cost /
// (M - barrier cost)) CTAs, first in those CTAs' lists so that all ranks start
// together) and the others fit, largest first, into the remaining capacity (first fit).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "fjofc.h"
#include "fjofc_internal.h"
#include "k1_decl.h"

namespace {

using fjofc::InsampleSetup;

constexpr double kPassCost = 4.0;      // default per-pass fixed cost, in sub-tiles
constexpr double kBarrierCost = 1.0;   // default per pass and group barrier pair, in sub-tiles

template <typename TD>
cudaError_t batched_launch_dt(int d, int grid, const fjofc::BatchLaunch& bl, cudaStream_t s) {
    switch (d) {
#define C_(D) case D: return fjofc::batched_launch_impl<D, TD>(grid, bl, s);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return cudaErrorInvalidValue;
}
template <typename TD>
int batched_bps_dt(int d) {
    switch (d) {
#define C_(D) case D: return fjofc::batched_bps_impl<D, TD>();
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return 0;
}
cudaError_t batched_launch(int d, int dtype, int grid, const fjofc::BatchLaunch& bl, cudaStream_t s) {
    return dtype == FJOFC_F32 ? batched_launch_dt<float>(d, grid, bl, s)
         : dtype == FJOFC_F16 ? batched_launch_dt<__half>(d, grid, bl, s)
                              : batched_launch_dt<__nv_bfloat16>(d, grid, bl, s);
}
int batched_bps(int d, int dtype) {
    return dtype == FJOFC_F32 ? batched_bps_dt<float>(d)
         : dtype == FJOFC_F16 ? batched_bps_dt<__half>(d)
                              : batched_bps_dt<__nv_bfloat16>(d);
}

int fail(int code, const char* msg) {
    fjofc::set_message(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    fjofc::set_message(msg);
    return e == cudaErrorMemoryAllocation ? FJOFC_ERR_NOMEM : FJOFC_ERR_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Class {
    int d, dtype, grid;
    std::vector<int> cta_off;          // [grid + 1]
    std::vector<int2> assign;          // (problem, rank)
    size_t o_off = 0, o_assign = 0;    // device offsets
};

}  // namespace

struct fjofc_plan {
    int device = 0;
    int nprob = 0;
    std::vector<int> groups;           // CTAs per problem
    std::vector<Class> classes;
    char* mem = nullptr;               // one device allocation for everything
    char* delta16 = nullptr;           // float16 copies of Delta chosen by the tuner (or NULL)
    size_t o_maps = 0, o_probs = 0, o_init = 0, o_stp = 0, o_res = 0, o_stress = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    int enqueue(cudaStream_t s) const {
        cudaError_t e = fjofc::launch_init_batched(reinterpret_cast<const fjofc::InitParams*>(mem + o_init), nprob, s);
        if (e != cudaSuccess) return cuda_fail(e, "batched init");
        for (const Class& c : classes) {
            fjofc::BatchLaunch bl{};
            bl.maps = reinterpret_cast<const fjofc::TMaps*>(mem + o_maps);
            bl.probs = reinterpret_cast<const fjofc::PersistParams*>(mem + o_probs);
            bl.cta_off = reinterpret_cast<const int*>(mem + c.o_off);
            bl.assign = reinterpret_cast<const int2*>(mem + c.o_assign);
            if ((e = batched_launch(c.d, c.dtype, c.grid, bl, s)) != cudaSuccess) return cuda_fail(e, "batched launch");
        }
        e = fjofc::launch_batch_results(reinterpret_cast<const fjofc::DevStatus* const*>(mem + o_stp), nprob,
                                        reinterpret_cast<int*>(mem + o_res), reinterpret_cast<double*>(mem + o_stress),
                                        s);
        if (e != cudaSuccess) return cuda_fail(e, "batch results");
        return FJOFC_OK;
    }

    ~fjofc_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (mem) cudaFree(mem);
        if (delta16) cudaFree(delta16);
    }
};

namespace {

int create_plan(const fjofc_problem* probs, int32_t nprob, const fjofc_opts* opts, double pass_cost,
                double barrier_cost, fjofc_plan** out) {
    if (!out) return fail(FJOFC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!probs || nprob < 1) return fail(FJOFC_ERR_ARG, "need at least one problem");
    if (!opts) return fail(FJOFC_ERR_ARG, "opts is NULL");
    fjofc_opts o = *opts;
    if (o.max_iter < 0) return fail(FJOFC_ERR_ARG, "max_iter must be >= 0");
    if (o.tol_mode != FJOFC_TOL_ABS_NORMALIZED && o.tol_mode != FJOFC_TOL_RELATIVE)
        return fail(FJOFC_ERR_ARG, "unknown tol_mode");
    if (std::isnan(o.tol)) return fail(FJOFC_ERR_ARG, "tol is NaN");
    if (o.profile != 0) return fail(FJOFC_ERR_ARG, "profile must be 0 for a plan");
    if (!(o.relax >= 0.f && o.relax <= 2.f)) return fail(FJOFC_ERR_ARG, "relax must be in [0, 2]");
    for (int r = 0; r < 2; ++r)
        if (o.reserved[r] != 0) return fail(FJOFC_ERR_ARG, "opts.reserved must be zero");
    if (o.delta_layout != FJOFC_LAYOUT_FULL && o.delta_layout != FJOFC_LAYOUT_PACKED)
        return fail(FJOFC_ERR_ARG, "unknown delta_layout");
    if (o.deterministic != 0 && o.deterministic != 1) return fail(FJOFC_ERR_ARG, "deterministic must be 0 or 1");
    if (o.wait_limit_us < 0) return fail(FJOFC_ERR_ARG, "wait_limit_us must be >= 0");
    if (o.check_inputs != 0)
        return fail(FJOFC_ERR_UNSUPPORTED, "check_inputs is not available for plans (check each problem with "
                                           "fjofc_embed and max_iter = 0)");
    int rc;
    if ((rc = fjofc::tensor_map_encoder())) return rc;
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop || sms < 1) return fail(FJOFC_ERR_UNSUPPORTED, "cooperative launch is not available");

    // ---- validate, cost and classify
    std::vector<InsampleSetup> S(nprob);
    std::vector<std::vector<double>> winv(nprob, std::vector<double>(FJOFC_MAX_M * FJOFC_MAX_M));
    std::vector<double> cost(nprob);
    std::vector<int> cls(nprob);
    std::vector<Class> classes;
    for (int p = 0; p < nprob; ++p) {
        const fjofc_problem& q = probs[p];
        if (q.m < 1 || q.m > FJOFC_MAX_M || q.d < 1 || q.d > FJOFC_MAX_D || q.n < 2 || q.n > (int64_t(1) << 30))
            return fail(FJOFC_ERR_ARG, "problem sizes out of range (1 <= m <= 8, 1 <= d <= 16, n >= 2)");
        if (!q.delta || !q.X || !q.weights) return fail(FJOFC_ERR_ARG, "problem with a NULL pointer");
        if (q.delta_dtype != FJOFC_F32 && q.delta_dtype != FJOFC_F16 && q.delta_dtype != FJOFC_BF16)
            return fail(FJOFC_ERR_ARG, "unknown delta_dtype");
        if ((rc = fjofc::validate_problem(q.m, q.n, q.d, q.delta, q.ld, q.delta_dtype, q.delta_scale, q.X))) return rc;
        if ((rc = fjofc::modified_weights_inverse(q.m, q.n, q.weights, winv[p].data()))) return rc;
        if ((rc = S[p].plan(q.m, q.n, q.d, q.delta_dtype, o, true, 1))) return rc;
        cost[p] = double(o.max_iter + 1) * (double(S[p].P.T) + pass_cost);
        int c = 0;
        while (c < int(classes.size()) && !(classes[c].d == q.d && classes[c].dtype == q.delta_dtype)) ++c;
        if (c == int(classes.size())) {
            Class k;
            k.d = q.d;
            k.dtype = q.delta_dtype;
            k.grid = std::max(1, batched_bps(q.d, q.delta_dtype)) * sms;
            classes.push_back(k);
        }
        cls[p] = c;
    }

    // ---- schedule every class onto its grid: the smallest per-CTA load M (binary search)
    // for which every problem costing more than M fits on a group of its own and the others
    // fit, first-fit decreasing, into what is left
    const double passes = double(o.max_iter + 1);
    std::vector<int> groups(nprob, 1);
    for (int c = 0; c < int(classes.size()); ++c) {
        Class& k = classes[c];
        std::vector<int> mine;
        double total = 0.0, lo = 0.0;
        for (int p = 0; p < nprob; ++p)
            if (cls[p] == c) {
                mine.push_back(p);
                total += cost[p];
                lo = std::max(lo, cost[p] / double(S[p].P.T) + passes * barrier_cost);
            }
        std::stable_sort(mine.begin(), mine.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        lo = std::max(lo, total / k.grid);
        std::vector<std::vector<int2>> lists;
        std::vector<int> G(nprob, 1);
        auto fits = [&](double M) {
            lists.assign(k.grid, {});
            std::vector<double> load(k.grid, 0.0);
            int used = 0;
            for (int p : mine) {
                if (cost[p] <= M) continue;
                const double room = M - passes * barrier_cost;
                if (room <= 0.0) return false;
                const int64_t g = int64_t(std::ceil(cost[p] / room));
                if (g < 2 || g > S[p].P.T || used + g > k.grid) return false;
                for (int r = 0; r < int(g); ++r) {
                    lists[used + r].push_back(make_int2(p, r));
                    load[used + r] = cost[p] / double(g) + passes * barrier_cost;
                }
                G[p] = int(g);
                used += int(g);
            }
            for (int p : mine) {
                if (cost[p] > M) continue;
                int b = 0;
                while (b < k.grid && load[b] + cost[p] > M) ++b;
                if (b == k.grid) return false;
                lists[b].push_back(make_int2(p, 0));
                load[b] += cost[p];
                G[p] = 1;
            }
            return true;
        };
        double hi = std::max(lo, total) * 1.0001 + 1.0;
        for (int it = 0; it < 60 && hi - lo > 1e-4 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (fits(mid)) hi = mid; else lo = mid;
        }
        if (!fits(hi)) return fail(FJOFC_ERR_UNSUPPORTED, "internal: no schedule");
        for (int p : mine) groups[p] = G[p];
        k.cta_off.assign(k.grid + 1, 0);
        for (int b = 0; b < k.grid; ++b) {
            k.cta_off[b + 1] = k.cta_off[b] + int(lists[b].size());
            for (const int2& a : lists[b]) k.assign.push_back(a);
        }
    }
    for (int p = 0; p < nprob; ++p)
        if (groups[p] != 1 && (rc = S[p].plan(probs[p].m, probs[p].n, probs[p].d, probs[p].delta_dtype, o, true,
                                               groups[p])))
            return rc;
    for (int p = 0; p < nprob; ++p)
        if (S[p].P.G != groups[p]) return fail(FJOFC_ERR_UNSUPPORTED, "internal: group size was clamped");

    // ---- one device allocation: problem scratch, then the plan's tables
    std::vector<size_t> o_prob(nprob);
    size_t off = 0;
    for (int p = 0; p < nprob; ++p) {
        o_prob[p] = off;
        off = align256(off + S[p].bytes);
    }
    fjofc_plan* plan = new fjofc_plan();
    plan->device = dev;
    plan->nprob = nprob;
    plan->groups = groups;
    plan->o_maps = off;
    off = align256(off + sizeof(fjofc::TMaps) * nprob);
    plan->o_probs = off;
    off = align256(off + sizeof(fjofc::PersistParams) * nprob);
    plan->o_init = off;
    off = align256(off + sizeof(fjofc::InitParams) * nprob);
    plan->o_stp = off;
    off = align256(off + sizeof(void*) * nprob);
    plan->o_res = off;
    off = align256(off + sizeof(int) * 3 * nprob);
    plan->o_stress = off;
    off = align256(off + sizeof(double) * nprob);
    for (Class& k : classes) {
        k.o_off = off;
        off = align256(off + sizeof(int) * k.cta_off.size());
        k.o_assign = off;
        off = align256(off + sizeof(int2) * std::max<size_t>(1, k.assign.size()));
    }
    plan->classes = classes;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&plan->mem), off);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "plan allocation");
    }

    // ---- bind every problem and upload the tables
    std::vector<fjofc::TMaps> maps(nprob);
    std::vector<fjofc::PersistParams> pps(nprob);
    std::vector<fjofc::InitParams> ips(nprob);
    std::vector<const fjofc::DevStatus*> stp(nprob);
    for (int p = 0; p < nprob; ++p) {
        const fjofc_problem& q = probs[p];
        if ((rc = S[p].bind(plan->mem + o_prob[p], q.delta, q.ld, q.delta_scale, q.weights, winv[p].data(), q.X))) {
            delete plan;
            return rc;
        }
        maps[p] = S[p].tm;
        pps[p] = S[p].pp;
        ips[p] = S[p].ip;
        stp[p] = S[p].k1.st;
    }
    auto up = [&](size_t o_dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpy(plan->mem + o_dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    if ((e = up(plan->o_maps, maps.data(), sizeof(fjofc::TMaps) * nprob)) != cudaSuccess ||
        (e = up(plan->o_probs, pps.data(), sizeof(fjofc::PersistParams) * nprob)) != cudaSuccess ||
        (e = up(plan->o_init, ips.data(), sizeof(fjofc::InitParams) * nprob)) != cudaSuccess ||
        (e = up(plan->o_stp, stp.data(), sizeof(void*) * nprob)) != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "plan upload");
    }
    for (const Class& k : plan->classes)
        if ((e = up(k.o_off, k.cta_off.data(), sizeof(int) * k.cta_off.size())) != cudaSuccess ||
            (e = up(k.o_assign, k.assign.data(), sizeof(int2) * k.assign.size())) != cudaSuccess) {
            delete plan;
            return cuda_fail(e, "plan upload");
        }

    // ---- capture the whole plan once; without graph support it runs as plain launches
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) ok = plan->enqueue(cs) == FJOFC_OK;
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &g);
        ok = ok && ee == cudaSuccess && g;
        if (ok && cudaGraphInstantiate(&plan->exec, g, 0) == cudaSuccess) {
            plan->graph = g;
        } else {
            if (g) cudaGraphDestroy(g);
            plan->exec = nullptr;
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
    }
    *out = plan;
    return FJOFC_OK;
}

}  // namespace

extern "C" int fjofc_plan_create(const fjofc_problem* probs, int32_t nprob, const fjofc_opts* opts,
                                 fjofc_plan** out) {
    return create_plan(probs, nprob, opts, kPassCost, kBarrierCost, out);
}

extern "C" int fjofc_plan_run(fjofc_plan* plan, void* cuda_stream) {
    if (!plan) return fail(FJOFC_ERR_ARG, "plan is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (plan->exec) {
        const cudaError_t e = cudaGraphLaunch(plan->exec, s);
        return e == cudaSuccess ? FJOFC_OK : cuda_fail(e, "cudaGraphLaunch");
    }
    return plan->enqueue(s);
}

extern "C" int fjofc_plan_results(const fjofc_plan* plan, int32_t* status, int32_t* iters, double* stress,
                                  void* cuda_stream) {
    if (!plan) return fail(FJOFC_ERR_ARG, "plan is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int> res(3 * size_t(plan->nprob));
    std::vector<double> st(plan->nprob);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(res.data(), plan->mem + plan->o_res, res.size() * sizeof(int), cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(st.data(), plan->mem + plan->o_stress, st.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "plan results");
    int worst = FJOFC_OK;
    for (int p = 0; p < plan->nprob; ++p) {
        if (status) status[p] = res[3 * p];
        if (iters) iters[p] = res[3 * p + 1];
        if (stress) stress[p] = st[p];
        if (res[3 * p] != FJOFC_OK && worst == FJOFC_OK) {
            worst = res[3 * p];
            char msg[160];
            snprintf(msg, sizeof(msg), "problem %d (SMs %d): status %d, wait site %d", p, plan->groups[p],
                     res[3 * p], res[3 * p + 2]);
            fjofc::set_message(msg);
        }
    }
    return worst;
}

extern "C" int fjofc_plan_info(const fjofc_plan* plan, int32_t* groups, int32_t* graphed, int32_t* launches) {
    if (!plan) return fail(FJOFC_ERR_ARG, "plan is NULL");
    if (groups)
        for (int p = 0; p < plan->nprob; ++p) groups[p] = plan->groups[p];
    if (graphed) *graphed = plan->exec ? 1 : 0;
    if (launches) *launches = int(plan->classes.size()) + 2;
    return FJOFC_OK;
}

extern "C" void fjofc_plan_destroy(fjofc_plan* plan) { delete plan; }

// ------------------------------------------------------------------ autotuner
// Times a short run (probe_iters transforms, fixed count) of every candidate plan and
// builds the plan of the fastest one with the caller's options.  Candidates: the
// schedule's cost constants (how problems are cut into per-SM (problem, sub-tile range)
// work) and, if the caller allows it, float16 storage of the float32 Delta (converted
// into plan-owned buffers, scale max|Delta|/2^10 per matrix).  Every X is saved before
// the probes and restored after each one.
extern "C" int fjofc_plan_autotune(const fjofc_problem* probs, int32_t nprob, const fjofc_opts* opts,
                                   const fjofc_tune_opts* topts, fjofc_plan** out, fjofc_tune_result* result,
                                   void* cuda_stream) {
    if (!out) return fail(FJOFC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!probs || nprob < 1 || !opts) return fail(FJOFC_ERR_ARG, "need problems and opts");
    const int probe = (topts && topts->probe_iters > 0) ? topts->probe_iters : 8;
    // float16 copies are made of whole n x n matrices: not for the packed layout
    const bool allow16 = topts && topts->allow_f16 && !(opts && opts->delta_layout == FJOFC_LAYOUT_PACKED);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;

    // save every X
    std::vector<size_t> xoff(nprob + 1, 0);
    for (int p = 0; p < nprob; ++p) xoff[p + 1] = xoff[p] + size_t(probs[p].m) * probs[p].n * probs[p].d;
    float* xsave = nullptr;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&xsave), std::max<size_t>(1, xoff[nprob]) * 4)) != cudaSuccess)
        return cuda_fail(e, "tuner X backup");
    struct Free {
        void* p;
        ~Free() { if (p) cudaFree(p); }
    } fx{xsave};
    auto copy_x = [&](bool save) -> cudaError_t {
        for (int p = 0; p < nprob; ++p) {
            const size_t bytes = (xoff[p + 1] - xoff[p]) * 4;
            cudaError_t ee = save ? cudaMemcpyAsync(xsave + xoff[p], probs[p].X, bytes, cudaMemcpyDeviceToDevice, s)
                                  : cudaMemcpyAsync(probs[p].X, xsave + xoff[p], bytes, cudaMemcpyDeviceToDevice, s);
            if (ee != cudaSuccess) return ee;
        }
        return cudaSuccess;
    };
    if ((e = copy_x(true)) != cudaSuccess) return cuda_fail(e, "tuner X backup");

    // float16 copies of the float32 Delta (only if allowed and useful)
    std::vector<fjofc_problem> p16(probs, probs + nprob);
    std::vector<std::vector<const void*>> ptr16(nprob);
    std::vector<std::vector<float>> scale16(nprob);
    char* d16 = nullptr;
    bool have16 = false;
    if (allow16) {
        size_t bytes = 0;
        std::vector<size_t> off16(nprob);
        for (int p = 0; p < nprob; ++p) {
            off16[p] = bytes;
            if (probs[p].delta_dtype != FJOFC_F32) continue;
            const int64_t ld16 = (probs[p].n + 7) / 8 * 8;
            bytes = align256(bytes + size_t(probs[p].m) * probs[p].n * ld16 * 2);
            have16 = true;
        }
        const size_t maxbytes = align256(bytes) + sizeof(unsigned) * 8 * size_t(nprob);
        if (have16 && (e = cudaMalloc(reinterpret_cast<void**>(&d16), maxbytes)) != cudaSuccess)
            return cuda_fail(e, "tuner float16 Delta");
        if (have16) {
            unsigned* mx = reinterpret_cast<unsigned*>(d16 + align256(bytes));
            cudaMemsetAsync(mx, 0, sizeof(unsigned) * 8 * size_t(nprob), s);
            for (int p = 0; p < nprob; ++p)
                if (probs[p].delta_dtype == FJOFC_F32)
                    for (int l = 0; l < probs[p].m; ++l)
                        if ((e = fjofc::launch_absmax(static_cast<const float*>(probs[p].delta[l]), probs[p].n,
                                                      probs[p].ld, mx + 8 * p + l, s)) != cudaSuccess) {
                            cudaFree(d16);
                            return cuda_fail(e, "tuner max");
                        }
            std::vector<unsigned> hm(8 * size_t(nprob));
            cudaMemcpyAsync(hm.data(), mx, hm.size() * 4, cudaMemcpyDeviceToHost, s);
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
                cudaFree(d16);
                return cuda_fail(e, "tuner max");
            }
            for (int p = 0; p < nprob; ++p) {
                if (probs[p].delta_dtype != FJOFC_F32) continue;
                const int64_t n = probs[p].n, ld16 = (n + 7) / 8 * 8;
                ptr16[p].resize(probs[p].m);
                scale16[p].resize(probs[p].m);
                for (int l = 0; l < probs[p].m; ++l) {
                    float mxv;
                    std::memcpy(&mxv, &hm[8 * p + l], 4);
                    const float sc = (mxv > 0.f && std::isfinite(mxv)) ? mxv / 1024.f : 1.f;
                    const float base = probs[p].delta_scale ? probs[p].delta_scale[l] : 1.f;
                    char* dst = d16 + off16[p] + size_t(l) * n * ld16 * 2;
                    if ((e = fjofc::launch_to_half(static_cast<const float*>(probs[p].delta[l]), n, probs[p].ld,
                                                   1.f / sc, dst, ld16, s)) != cudaSuccess) {
                        cudaFree(d16);
                        return cuda_fail(e, "tuner convert");
                    }
                    ptr16[p][l] = dst;
                    scale16[p][l] = sc * base;
                }
                p16[p].delta = ptr16[p].data();
                p16[p].ld = ld16;
                p16[p].delta_dtype = FJOFC_F16;
                p16[p].delta_scale = scale16[p].data();
            }
        }
    }

    struct Cand {
        double pc, bc;
        bool f16;
    };
    std::vector<Cand> cands;
    const double pcs[4][2] = {{2.0, 0.5}, {4.0, 1.0}, {8.0, 2.0}, {4.0, 3.0}};
    for (int f = 0; f < (have16 ? 2 : 1); ++f)
        for (const auto& c : pcs) cands.push_back(Cand{c[0], c[1], f == 1});
    fjofc_opts po = *opts;
    po.max_iter = probe;
    po.tol = -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    float best_ms = 0.f;
    int rc = FJOFC_OK;
    for (int ci = 0; ci < int(cands.size()); ++ci) {
        fjofc_plan* cand = nullptr;
        rc = create_plan(cands[ci].f16 ? p16.data() : probs, nprob, &po, cands[ci].pc, cands[ci].bc, &cand);
        if (rc) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == FJOFC_OK; ++rep) {        // the first run warms up
            cudaEventRecord(e0, s);
            rc = fjofc_plan_run(cand, s);
            cudaEventRecord(e1, s);
            if (rc == FJOFC_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "tuner probe");
            if (rc == FJOFC_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (rc == FJOFC_OK && (e = copy_x(false)) != cudaSuccess) rc = cuda_fail(e, "tuner X restore");
        }
        if (rc == FJOFC_OK) rc = fjofc_plan_results(cand, nullptr, nullptr, nullptr, s);
        delete cand;
        if (rc) break;
        if (best < 0 || ms < best_ms) {
            best = ci;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == FJOFC_OK && (e = copy_x(false)) != cudaSuccess) rc = cuda_fail(e, "tuner X restore");
    if (rc == FJOFC_OK) rc = create_plan(cands[best].f16 ? p16.data() : probs, nprob, opts, cands[best].pc,
                                         cands[best].bc, out);
    if (rc != FJOFC_OK) {
        if (d16) cudaFree(d16);
        return rc;
    }
    if (cands[best].f16) (*out)->delta16 = d16;      // the plan owns the float16 copies
    else if (d16) cudaFree(d16);
    if (result) {
        std::memset(result, 0, sizeof(*result));
        result->pass_cost = float(cands[best].pc);
        result->barrier_cost = float(cands[best].bc);
        result->delta_dtype = cands[best].f16 ? FJOFC_F16 : -1;
        result->probe_ms = best_ms;
        result->candidates = int(cands.size());
    }
    return FJOFC_OK;
}

// Batched in-sample embedding: many independent fJOFC problems of uneven size in one
// plan.  Problems are grouped by (embedding dimension, Delta type), the kernel
// instantiation they need; each class runs as one cooperative launch of the persistent
// loop kernel over all SMs (k_embed_batched), and the whole plan (per-problem set-up,
// the class launches, the result gather) is captured once into a CUDA graph.
//
// Scheduling (host, once per plan): the cost of a problem is its sub-tiles per pass plus
// a fixed per-pass cost (the per-object phase, totals and barriers, about kPassCost
// sub-tiles; one more per pass for each group barrier) times its number of passes.
// Problems costing more than the per-CTA average get a group of G >= 2 CTAs of their
// own, placed first in those CTAs' lists so that all ranks start together; the others
// go, largest first, to the least-loaded CTA (longest-processing-time rule).
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

constexpr double kPassCost = 4.0;      // per-pass fixed cost, in sub-tiles
constexpr double kBarrierCost = 1.0;   // per pass and group barrier pair, in sub-tiles

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
    }
};

extern "C" int fjofc_plan_create(const fjofc_problem* probs, int32_t nprob, const fjofc_opts* opts,
                                 fjofc_plan** out) {
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
    for (int r = 0; r < 4; ++r)
        if (o.reserved[r] != 0) return fail(FJOFC_ERR_ARG, "opts.reserved must be zero");
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
        if ((rc = fjofc::modified_weights_inverse(q.m, q.n, q.weights, winv[p].data()))) return rc;
        if ((rc = S[p].plan(q.m, q.n, q.d, q.delta_dtype, o, true, 1))) return rc;
        cost[p] = double(o.max_iter + 1) * (double(S[p].P.T) + kPassCost);
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

    // ---- schedule every class onto its grid
    std::vector<int> groups(nprob, 1);
    for (int c = 0; c < int(classes.size()); ++c) {
        Class& k = classes[c];
        std::vector<int> mine;
        double total = 0.0;
        for (int p = 0; p < nprob; ++p)
            if (cls[p] == c) { mine.push_back(p); total += cost[p]; }
        std::stable_sort(mine.begin(), mine.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        const double target = total / k.grid;
        std::vector<std::vector<int2>> lists(k.grid);
        std::vector<double> load(k.grid, 0.0);
        int fresh = 0;                                     // CTAs [fresh, grid) hold nothing yet
        for (int p : mine) {
            int G = 1;
            if (cost[p] > 1.5 * target) {
                G = int(std::ceil(cost[p] / target));
                G = int(std::min<int64_t>(G, S[p].P.T));
                G = std::min(G, k.grid - fresh);
                if (G < 2) G = 1;
            }
            if (G >= 2) {
                for (int r = 0; r < G; ++r) {
                    lists[fresh + r].push_back(make_int2(p, r));
                    load[fresh + r] = (cost[p] + double(o.max_iter + 1) * kBarrierCost * G) / G;
                }
                fresh += G;
            } else {
                const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
                lists[b].push_back(make_int2(p, 0));
                load[b] += cost[p];
                fresh = std::max(fresh, b + 1);
            }
            groups[p] = G;
        }
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

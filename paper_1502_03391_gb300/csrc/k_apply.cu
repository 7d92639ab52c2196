// K2 and the small per-call kernels of the in-sample loop.
//
// K2 (one launch per Guttman transform) finishes iteration t:
//   * (B'_l X_l)_i = sum of the K1 partials of object i in modality l, in a fixed order
//     (its row-walk head, the continuation segments, then the column partials of the
//     walks of row blocks 0..I(i));
//   * X_t^(j)_i = sum_l [Wmod^-1]_{jl} w_ll s_l (B'_l X_l)_i      (Eq. update / Cor. 1:
//     L^+ = Wmod^-1 (x) I_n + Z (x) J_n, and the J_n part vanishes on B(X) X because the
//     rows and columns of every B_l sum to zero, Sec. 2.1);
//   * sigma(X_{t-1}) = (fidelity from K1) + sum_{j<l} w_jl ||X^(j) - X^(l)||^2 (Eq. stress,
//     Remark faststress), with X_{t-1} first centred per modality by its float-float
//     column means (Guttman outputs are centred in exact arithmetic; this removes
//     float32 drift);
//   * the column means of X_t (for the next centring) and, in the last CTA to finish,
//     the stress history entry and the stopping test of Algorithm 1 (read as "continue
//     while the decrease exceeds the tolerance").
#include "k_apply_common.cuh"

namespace fjofc {

constexpr int K2_THREADS = 256;

// One CTA per group of 32 consecutive objects (phase_b over its d units), then the last
// CTA to finish forms the totals.  Arithmetic is float32; cross-object sums are
// float-float (GB300's float64 rate is low).
__global__ void __launch_bounds__(K2_THREADS)
k_apply(const K2Params p) {
    extern __shared__ float s_dyn[];             // d * phase_b_floats_per_unit(m)
    __shared__ float s_mu[FJOFC_MAX_M * FJOFC_MAX_D];
    __shared__ bool s_last;

    if (ld_volatile(&p.st->done)) return;

    const int m = p.m, n = p.n, d = p.d;
    const int tid = threadIdx.x;
    const float* mu_prev = p.mu + ((p.t - 1) & 1) * (FJOFC_MAX_M * FJOFC_MAX_D);
    float* mu_next = p.mu + (p.t & 1) * (FJOFC_MAX_M * FJOFC_MAX_D);
    for (int e = tid; e < FJOFC_MAX_M * FJOFC_MAX_D; e += K2_THREADS) s_mu[e] = mu_prev[e];
    __syncthreads();

    PhaseBArgs a;
    a.tb = p.tb;
    a.Xprev = p.Xprev;
    a.Xnext = p.Xnext;
    a.bpart = p.bpart;
    a.mu_prev = s_mu;
    a.mu_stride = FJOFC_MAX_D;
    a.coef_g = p.coef_g;
    a.wcomm_g = p.wcomm_g;
    a.m = m; a.n = n; a.d = d; a.t = p.t; a.ngroups = p.nbx;
    a.centre = p.centre != 0;
    a.relax = p.relax;
    a.final_pass = p.final_pass != 0;
    phase_b(a, int(blockIdx.x) * d, int(blockIdx.x + 1) * d, d, s_dyn);

    const int npart = phase_b_parts(m, d);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(p.ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last CTA: totals in a fixed order (two quantities per warp; the persistent
    // kernel's phase C computes them the same way)
    __shared__ FF s_tot[FJOFC_MAX_M * FJOFC_MAX_D + FJOFC_MAX_D + 1];
    pass_totals(p.bpart, npart, int(gridDim.x), p.fid, p.G, s_tot);
    __syncthreads();
    for (int e = tid; e < m * d; e += K2_THREADS)
        mu_next[(e / d) * FJOFC_MAX_D + (e % d)] = (s_tot[e].hi + s_tot[e].lo) * p.inv_n;

    if (tid == 0) {
        const double sigma = stress_from_totals(s_tot, s_tot[npart], m, d);
        const int tp = p.t - 1;                 // index of the iterate whose stress this is
        p.hist[tp] = sigma;
        DevStatus* st = p.st;
        if (!isfinite(sigma)) {
            st->error = FJOFC_ERR_NONFINITE;    // final_iter keeps the last finite iterate
            st->done = 1;
        } else {
            st->final_iter = tp;
            st->stress = sigma;
            bool stop = p.final_pass != 0;
            if (!stop && tp >= 1 && p.tol >= 0.0) {
                const double prev = p.hist[tp - 1];
                const double dec = prev - sigma;
                const bool cont = (p.tol_mode == FJOFC_TOL_RELATIVE) ? (dec > p.tol * prev)
                                                                     : (dec > p.tol * p.npairs);
                stop = !cont;
            }
            if (stop) st->done = 1;
        }
        __threadfence();
        *p.ticket = 0u;                          // ready for the next launch
    }
}

int k2_blocks(int n) { return (n + kGroupObjects - 1) / kGroupObjects; }

cudaError_t launch_k2(const K2Params& p, cudaStream_t s) {
    const size_t smem = size_t(p.d) * phase_b_floats_per_unit(p.m) * sizeof(float);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    k_apply<<<p.nbx, K2_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

// Per-call initialisation (one CTA of kInitThreads): status block, ticket, mu_0 = 0, then
//   walk_off[P]  = sub-tiles before walk position P (prefix sums of the walk lengths),
//   cost_off[P]  = the modelled cost of those sub-tiles (kSplitCost*),
//   cta_start[b] = first sub-tile of CTA b: the ranges cut the modelled cost into G equal
//                  parts when every CTA gets at least 4 sub-tiles on average, else b*T/G,
//   tc           = the CTA with the least modelled cost (the first such),
//   cbase[I]     = first sub-tile (within a modality) of row block I's walk,
//   cont[l][I]   = the CTAs whose range starts strictly inside that walk.
// Each step reads only what earlier steps of this CTA wrote (global memory, ordered by
// __syncthreads).
constexpr int kInitThreads = 1024;

__device__ __forceinline__ int64_t walk_len(int P, const InitParams& p) {
    const int64_t cols = int64_t(p.n) - int64_t(walk_row(P, p.nRB)) * p.RB;
    return (cols + p.CW - 1) / p.CW;
}

// Modelled cost of walk position P's sub-tiles: each kSplitCostSub, the diagonal one and a
// ragged last one kSplitCostMask more, the walk's end kSplitCostWalkEnd.
__device__ __forceinline__ int64_t walk_cost(int P, const InitParams& p) {
    const int64_t cols = int64_t(p.n) - int64_t(walk_row(P, p.nRB)) * p.RB;
    const int64_t L = (cols + p.CW - 1) / p.CW;
    const int64_t masked = 1 + ((L >= 2 && cols % p.CW != 0) ? 1 : 0);
    return L * kSplitCostSub + masked * kSplitCostMask + kSplitCostWalkEnd;
}

// Modelled cost of sub-tiles [0, t) (walk_off and cost_off complete).
__device__ __forceinline__ int64_t cum_cost(int64_t t, const InitParams& p) {
    const int64_t Cm = p.cost_off[p.nRB];
    const int64_t l = t / p.Tm, r = t - l * p.Tm;
    if (r == 0) return l * Cm;
    int lo = 0, hi = p.nRB - 1;                        // last position with walk_off <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.walk_off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    const int64_t s = r - p.walk_off[lo];
    return l * Cm + p.cost_off[lo] + s * kSplitCostSub + (s >= 1 ? kSplitCostMask : 0);
}

__device__ __forceinline__ void init_problem(const InitParams& p) {
    __shared__ int64_t s_part[kInitThreads];
    __shared__ int64_t s_cost[kInitThreads];
    const int tid = threadIdx.x;
    for (int e = tid; e < p.m * p.m; e += kInitThreads) {
        p.coef_g[e] = p.coef[e];
        p.wcomm_g[e] = p.wcomm[e];
    }
    if (tid == 0) {
        p.st->done = 0;
        p.st->error = 0;
        p.st->final_iter = 0;
        p.st->timeout_site = 0;
        p.st->stress = 0.0;
        p.st->bad = kNoBadEntry;
        *p.ticket = 0u;
        if (p.bar) *p.bar = 0u;
        if (p.pub_seq) *p.pub_seq = 0u;
    }
    for (int e = tid; e < 2 * FJOFC_MAX_M * FJOFC_MAX_D; e += kInitThreads) p.mu[e] = 0.f;

    // walk_off: block scan over contiguous chunks of positions
    const int per = (p.nRB + kInitThreads - 1) / kInitThreads;
    const int P0 = tid * per, P1 = min(P0 + per, p.nRB);
    int64_t local = 0, lcost = 0;
    for (int P = P0; P < P1; ++P) {
        local += walk_len(P, p);
        lcost += walk_cost(P, p);
    }
    s_part[tid] = local;
    s_cost[tid] = lcost;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0, crun = 0;
        for (int e = 0; e < kInitThreads; ++e) {
            const int64_t v = s_part[e], c = s_cost[e];
            s_part[e] = run;
            s_cost[e] = crun;
            run += v;
            crun += c;
        }
    }
    __syncthreads();
    {
        int64_t run = s_part[tid], crun = s_cost[tid];
        for (int P = P0; P < P1; ++P) {
            p.walk_off[P] = run;
            p.cost_off[P] = crun;
            run += walk_len(P, p);
            crun += walk_cost(P, p);
        }
        if (P1 == p.nRB && P0 < P1) {
            p.walk_off[p.nRB] = run;
            p.cost_off[p.nRB] = crun;
        }
    }
    __syncthreads();

    // CTA ranges: equal parts of the modelled cost (a part holds more than the costliest
    // sub-tile when T >= 4 G, so no range is empty), else of the sub-tile count
    const bool weighted = p.T >= 4 * int64_t(p.G);
    const int64_t Ctot = int64_t(p.m) * p.cost_off[p.nRB];
    for (int b = tid; b <= p.G; b += kInitThreads) {
        int64_t start = int64_t(b) * p.T / p.G;
        if (weighted && b > 0 && b < p.G) {
            // the first t with cum_cost(t) >= target: the modality and the walk position
            // holding the target, then the sub-tile inside that walk in closed form
            const int64_t target = int64_t(b) * Ctot / p.G;
            const int64_t Cm = p.cost_off[p.nRB];
            const int64_t l = target / Cm, rem = target - l * Cm;
            int lo = 0, hi = p.nRB - 1;                // last position with cost_off <= rem
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.cost_off[mid] <= rem) lo = mid; else hi = mid - 1;
            }
            const int64_t need = rem - p.cost_off[lo];
            const int64_t L = p.walk_off[lo + 1] - p.walk_off[lo];
            int64_t sub = 0;
            if (need > 0) {
                sub = (need - kSplitCostMask + kSplitCostSub - 1) / kSplitCostSub;
                if (sub < 1) sub = 1;
                if (sub > L) sub = L;                  // the next walk's first sub-tile
            }
            start = l * p.Tm + p.walk_off[lo] + sub;
        }
        p.cta_start[b] = start;
    }
    __syncthreads();
    // the totals CTA: least modelled cost, then lowest index (key = cost * 2^20 + b)
    {
        int64_t key = INT64_MAX;
        for (int b = tid; b < p.G; b += kInitThreads) {
            const int64_t c = cum_cost(p.cta_start[b + 1], p) - cum_cost(p.cta_start[b], p);
            const int64_t k = (c << 20) + b;
            key = k < key ? k : key;
        }
        s_part[tid] = key;
        __syncthreads();
        for (int h = kInitThreads / 2; h > 0; h >>= 1) {
            if (tid < h && s_part[tid + h] < s_part[tid]) s_part[tid] = s_part[tid + h];
            __syncthreads();
        }
        if (tid == 0) *p.tc = int(s_part[0] & ((int64_t(1) << 20) - 1));
    }
    __syncthreads();

    // row-block tables
    for (int e = tid; e < p.m * p.nRB; e += kInitThreads) {
        const int l = e / p.nRB, I = e - l * p.nRB;
        const int64_t base = p.walk_off[walk_pos(I, p.nRB)];
        if (l == 0) p.cbase[I] = base;
        const int64_t ws = int64_t(l) * p.Tm + base;
        const int64_t we = ws + walk_len(walk_pos(I, p.nRB), p);
        // [lo, hi): CTAs b with ws < cta_start[b] < we
        int lo = 0, hi = p.G;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (p.cta_start[mid] > ws) hi = mid; else lo = mid + 1;
        }
        const int c_lo = lo;
        lo = c_lo; hi = p.G;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (p.cta_start[mid] >= we) hi = mid; else lo = mid + 1;
        }
        p.cont[e] = make_int2(c_lo, lo);
    }
}

__global__ void __launch_bounds__(kInitThreads) k_init(const __grid_constant__ InitParams p) { init_problem(p); }

// One CTA per problem of a batch.
__global__ void __launch_bounds__(kInitThreads) k_init_batched(const InitParams* __restrict__ ps) {
    init_problem(ps[blockIdx.x]);
}

cudaError_t launch_init(const InitParams& p, cudaStream_t s) {
    k_init<<<1, kInitThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_init_batched(const InitParams* ps, int count, cudaStream_t s) {
    if (count > 0) k_init_batched<<<count, kInitThreads, 0, s>>>(ps);
    return cudaGetLastError();
}

// Per-problem results of a batch: out[3 p] = error status, out[3 p + 1] = final
// iteration, out[3 p + 2] = where a bounded wait gave up (0 if none), stress[p] =
// sigma of the returned iterate.
__global__ void k_batch_results(const DevStatus* const* st, int count, int* out, double* stress) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const DevStatus* s = st[e];
    out[3 * e] = s->error;
    out[3 * e + 1] = s->final_iter;
    out[3 * e + 2] = s->timeout_site;
    stress[e] = s->stress;
}

cudaError_t launch_batch_results(const DevStatus* const* st, int count, int* out, double* stress, cudaStream_t s) {
    if (count > 0) k_batch_results<<<(count + 127) / 128, 128, 0, s>>>(st, count, out, stress);
    return cudaGetLastError();
}

// Copy the returned iterate to the caller's buffer when it lives in a workspace buffer
// (iterate t is stored in buffer t % 3; buffer 0 is the caller's X).
__global__ void k_finalize(float* Xout, const float* buf1, const float* buf2, int64_t count,
                           const DevStatus* st) {
    const int f = st->final_iter;
    const int slot = f % 3;
    if (slot == 0) return;
    const float* src = (slot == 1) ? buf1 : buf2;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x)
        Xout[e] = src[e];
}

// Input check (fjofc_opts.check_inputs): Delta_l must hold dissimilarities (Sec. 1.2):
// finite, non-negative and symmetric.  CTA (I, J, l) with I <= J compares the 32 x 32
// block (I, J) of Delta_l with block (J, I), both staged in shared memory by coalesced
// rows; every off-diagonal entry is read once.  A thread that finds an invalid entry
// lowers st->bad to that entry's key (atomicMin: the first entry in (l, row, column)
// order wins whatever the schedule) and marks the loop as stopped with FJOFC_ERR_ARG, so
// the kernels that follow on the stream return at once and leave X as given.
template <typename TD>
__device__ __forceinline__ float check_load(const void* base, int64_t ld, int64_t r, int64_t c) {
    return DeltaLoad<TD>::to_f32(static_cast<const TD*>(base)[r * ld + c]);
}

template <typename TD>
__global__ void __launch_bounds__(256) k_check_delta(const __grid_constant__ CheckParams p) {
    const int I = blockIdx.x, J = blockIdx.y, l = blockIdx.z;
    if (I > J) return;
    __shared__ float a[32][33], b[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n = p.n;
    const void* base = p.delta[l];
    for (int r = ty; r < 32; r += 8) {
        const int64_t ra = int64_t(I) * 32 + r, ca = int64_t(J) * 32 + tx;
        const int64_t rb = int64_t(J) * 32 + r, cb = int64_t(I) * 32 + tx;
        a[r][tx] = (ra < n && ca < n) ? check_load<TD>(base, p.ld, ra, ca) : 0.f;
        b[r][tx] = (rb < n && cb < n) ? check_load<TD>(base, p.ld, rb, cb) : 0.f;
    }
    __syncthreads();
    unsigned long long worst = kNoBadEntry;
    auto flag = [&](int64_t row, int64_t col, unsigned kind) {
        const unsigned long long key =
            ((unsigned long long)((int64_t(l) * n + row) * n + col) << 2) | (unsigned long long)kind;
        worst = key < worst ? key : worst;
    };
    for (int r = ty; r < 32; r += 8) {
        const int64_t row = int64_t(I) * 32 + r, col = int64_t(J) * 32 + tx;
        if (!(row < col && col < n)) continue;          // strict upper triangle of the block pair
        const float u = a[r][tx], v = b[tx][r];         // Delta[row][col], Delta[col][row]
        if (!isfinite(u)) flag(row, col, 2u);
        else if (u < 0.f) flag(row, col, 1u);
        if (!isfinite(v)) flag(col, row, 2u);
        else if (v < 0.f) flag(col, row, 1u);
        if (isfinite(u) && isfinite(v) && u != v) flag(row, col, 3u);
    }
    if (worst != kNoBadEntry) {
        atomicMin(&p.st->bad, worst);
        p.st->error = FJOFC_ERR_ARG;
        p.st->done = 1;
    }
}

cudaError_t launch_check_delta(const CheckParams& p, cudaStream_t s) {
    const int nt = int((p.n + 31) / 32);
    const dim3 grid(nt, nt, p.m);
    if (p.dtype == FJOFC_F32) k_check_delta<float><<<grid, 256, 0, s>>>(p);
    else if (p.dtype == FJOFC_F16) k_check_delta<__half><<<grid, 256, 0, s>>>(p);
    else k_check_delta<__nv_bfloat16><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Packed band layout of a symmetric Delta (pack_pos): CTA y writes packed row y; element x
// comes from band b = the pair's left band while x < its width, else the right band;
// padding and positions past n are zero.
template <typename TD>
__global__ void __launch_bounds__(256) k_pack_delta(const TD* __restrict__ D, int64_t n, int64_t ld, TD* __restrict__ P,
                                                    int64_t L) {
    const int64_t y = blockIdx.x;
    const int64_t nb = (n + kPackBand - 1) / kPackBand;
    const int64_t pair = y / kPackBand, ro = y - pair * kPackBand, other = nb - 1 - pair;
    const int es = int(sizeof(TD));
    const int64_t wl = pack_align(n - kPackBand * pair, es);
    const int64_t wr = other != pair ? pack_align(n - kPackBand * other, es) : 0;
    for (int64_t x = threadIdx.x; x < L; x += blockDim.x) {
        int64_t b = -1, rel = 0;
        if (x < wl) { b = pair; rel = x; }
        else if (x - wl < wr) { b = other; rel = x - wl; }
        TD v = TD(0.f);
        if (b >= 0) {
            const int64_t r = kPackBand * b + ro, c = kPackBand * b + rel;
            if (r < n && c < n) v = D[r * ld + c];
        }
        P[y * L + x] = v;
    }
}

cudaError_t launch_pack_delta(const void* D, int64_t n, int64_t ld, int dtype, void* P, cudaStream_t s) {
    const int es = dtype == FJOFC_F32 ? 4 : 2;
    const int64_t L = pack_width(n, es);
    const int64_t nb = (n + kPackBand - 1) / kPackBand;
    const int64_t rows = (nb + 1) / 2 * kPackBand;
    if (dtype == FJOFC_F32)
        k_pack_delta<float><<<unsigned(rows), 256, 0, s>>>(static_cast<const float*>(D), n, ld, static_cast<float*>(P), L);
    else if (dtype == FJOFC_F16)
        k_pack_delta<__half><<<unsigned(rows), 256, 0, s>>>(static_cast<const __half*>(D), n, ld, static_cast<__half*>(P), L);
    else
        k_pack_delta<__nv_bfloat16><<<unsigned(rows), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(D), n, ld,
                                                                   static_cast<__nv_bfloat16*>(P), L);
    return cudaGetLastError();
}

cudaError_t launch_finalize(float* Xout, const float* buf1, const float* buf2, int64_t count,
                            const DevStatus* st, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (count + threads - 1) / threads;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_finalize<<<int(blocks), threads, 0, s>>>(Xout, buf1, buf2, count, st);
    return cudaGetLastError();
}

}  // namespace fjofc

namespace fjofc {

// Out-of-sample set-up: X transposed to [m][d][nx] (row stride nx, a multiple of 4 so
// that vector loads stay aligned), the column sums of every X^(j) in float64 (fixed
// order per block), the group counter and the status block.
__global__ void k_oos_prep(const __grid_constant__ OOSPrepParams p) {
    const int j = blockIdx.x / p.d, kk = blockIdx.x - j * p.d;
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < p.m * p.m; e += blockDim.x) {
            p.winv_g[e] = p.winv[e];
            p.wcomm_g[e] = p.wcomm[e];
        }
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < p.nx; i += blockDim.x) {
        const float v = (i < p.n) ? p.X[(int64_t(j) * p.n + i) * p.d + kk] : 0.f;
        p.XT[(int64_t(j) * p.d + kk) * p.nx + i] = -v;       // K3 works with -x
        s += double(v);
    }
    s = warp_sum_f64(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
        p.SX[j * p.d + kk] = float(t);
        if (blockIdx.x == 0) {
            *p.next_block = 0ull;
            p.st->done = 0;
            p.st->error = 0;
            p.st->final_iter = 0;
            p.st->timeout_site = 0;
            p.st->stress = 0.0;
            p.st->bad = kNoBadEntry;
        }
    }
}

cudaError_t launch_oos_prep(const OOSPrepParams& p, cudaStream_t s) {
    k_oos_prep<<<p.m * p.d, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Fixed-order reduction of the per-object results: max iterations, total stress.
__global__ void k_oos_summary(const int32_t* iters, const double* stress, int64_t k, int32_t* it_out,
                              double* st_out) {
    __shared__ double sh[32];
    __shared__ int shi[32];
    double s = 0.0;
    int mx = 0;
    for (int64_t o = threadIdx.x; o < k; o += blockDim.x) {
        s += stress[o];
        mx = max(mx, iters[o]);
    }
    s = warp_sum_f64(s);
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = s; shi[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int m2 = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) { t += sh[w]; m2 = max(m2, shi[w]); }
        *st_out = t;
        *it_out = m2;
    }
}

cudaError_t launch_oos_summary(const int32_t* iters, const double* stress, int64_t k, int32_t* it_out,
                               double* st_out, cudaStream_t s) {
    k_oos_summary<<<1, 1024, 0, s>>>(iters, stress, k, it_out, st_out);
    return cudaGetLastError();
}

}  // namespace fjofc

namespace fjofc {

// Largest |Delta| of an n x n matrix (row stride ld) as float bits in *out (atomicMax on
// the bit patterns, which order like the values for non-negative floats; *out starts at 0).
__global__ void k_absmax(const float* __restrict__ D, int64_t n, int64_t ld, unsigned* out) {
    float mx = 0.f;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = e / n, c = e - r * n;
        mx = fmaxf(mx, fabsf(D[r * ld + c]));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// out (row stride ld16) = half(D * inv_scale).
__global__ void k_to_half(const float* __restrict__ D, int64_t n, int64_t ld, float inv_scale,
                          __half* __restrict__ out, int64_t ld16) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = e / n, c = e - r * n;
        out[r * ld16 + c] = __float2half_rn(D[r * ld + c] * inv_scale);
    }
}

cudaError_t launch_absmax(const float* D, int64_t n, int64_t ld, unsigned* out, cudaStream_t s) {
    k_absmax<<<256, 256, 0, s>>>(D, n, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_to_half(const float* D, int64_t n, int64_t ld, float inv_scale, void* out, int64_t ld16,
                           cudaStream_t s) {
    k_to_half<<<512, 256, 0, s>>>(D, n, ld, inv_scale, static_cast<__half*>(out), ld16);
    return cudaGetLastError();
}

}  // namespace fjofc

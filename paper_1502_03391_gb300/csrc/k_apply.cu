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
//     Remark faststress), with X_{t-1} first centred per modality in float64 (Guttman
//     outputs are centred in exact arithmetic; this removes float32 drift);
//   * the column means of X_t (for the next centring) and, in the last CTA to finish,
//     the stress history entry and the stopping test of Algorithm 1 (read as "continue
//     while the decrease exceeds the tolerance").
#include "fjofc_device.cuh"

namespace fjofc {

constexpr int K2_THREADS = 256;
constexpr int K2_OBJ = 32;                 // objects per CTA (one per lane)
constexpr int K2_TAB_SMEM_MAX = 4096;      // walk/CTA tables staged in shared memory up to this many

// Fixed-order float-float sum over the CTA; every thread receives the total.
__device__ __forceinline__ FF block_sum_ff(FF v, FF* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum_ff(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    FF t{0.f, 0.f};
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t = ff_add(t, sh[w]);
    return t;
}

// One CTA per 32 consecutive objects.  Phase 1: warp w sums the partials of (modality l,
// coordinate k) pairs w, w+8, ... for its 32 objects (lane = object), 16 independent loads
// in flight.  Phase 2: warp w handles coordinate k = w, w+8, ...: centre X_{t-1}, its
// commensurability, the Wmod^-1 mix into X_t and the per-block column sums.  Arithmetic
// is float32; cross-object sums are float-float (GB300's float64 rate is low).
__global__ void __launch_bounds__(K2_THREADS)
k_apply(const K2Params p) {
    extern __shared__ int64_t s_tab[];          // walk_off [nRB+1] then cta_start [G+1]
    __shared__ float s_bx[FJOFC_MAX_M * FJOFC_MAX_D][K2_OBJ];
    __shared__ FF s_ff[K2_THREADS / 32];
    __shared__ FF s_part[FJOFC_MAX_M * FJOFC_MAX_D];
    __shared__ bool s_last;

    if (ld_volatile(&p.st->done)) return;

    const int m = p.m, n = p.n, d = p.d;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i = blockIdx.x * K2_OBJ + lane;
    const bool tab_smem = (p.nRB + 1 + p.G + 1) <= K2_TAB_SMEM_MAX;
    const int64_t* woff = tab_smem ? s_tab : p.walk_off;
    const int64_t* cstart = tab_smem ? s_tab + (p.nRB + 1) : p.cta_start;
    if (tab_smem) {
        for (int e = tid; e <= p.nRB; e += K2_THREADS) s_tab[e] = p.walk_off[e];
        for (int e = tid; e <= p.G; e += K2_THREADS) s_tab[p.nRB + 1 + e] = p.cta_start[e];
    }
    __syncthreads();

    const float* mu_prev = p.mu + ((p.t - 1) & 1) * (FJOFC_MAX_M * FJOFC_MAX_D);
    float* mu_next = p.mu + (p.t & 1) * (FJOFC_MAX_M * FJOFC_MAX_D);

    if (!p.final_pass) {
        const int RB = p.RB, CW = p.CW, rbs = p.rb_shift, cws = p.cw_shift, nRB = p.nRB;
        for (int lk = warp; lk < m * d; lk += K2_THREADS / 32) {
            const int l = lk / d, k = lk - l * d;
            float acc = 0.f;
            if (i < n) {
                const int I = i >> rbs, ri = i & (RB - 1);
                acc = p.rowhead[((int64_t(l) * nRB + I) * d + k) * RB + ri];
                // continuation segments: CTAs whose range starts strictly inside this walk
                const int P = walk_pos(I, nRB);
                const int64_t ws = int64_t(l) * p.Tm + woff[P];
                const int64_t we = int64_t(l) * p.Tm + woff[P + 1];
                int lo = 0, hi = p.G;                 // first CTA b with cta_start[b] > ws
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cstart[mid] > ws) hi = mid; else lo = mid + 1;
                }
                for (int b = lo; b < p.G && cstart[b] < we; ++b)
                    acc += p.rowcont[(int64_t(b) * d + k) * RB + ri];
                // column partials of the walks of row blocks 0..I: 16 independent loads in
                // flight, summed in a fixed order
                const float* cp = p.colpart + int64_t(l) * p.Tm * d * CW;
                float csum = 0.f;
                for (int J0 = 0; J0 <= I; J0 += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int J = J0 + u;
                        v[u] = 0.f;
                        if (J <= I) {
                            const int rel = i - (J << rbs);
                            const int sidx = rel >> cws, c = rel & (CW - 1);
                            v[u] = cp[((woff[walk_pos(J, nRB)] + sidx) * d + k) * CW + c];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) csum += v[u];
                }
                acc += csum;
            }
            s_bx[lk][lane] = acc;
        }
    }
    __syncthreads();

    FF comm{0.f, 0.f};
    for (int k = warp; k < d; k += K2_THREADS / 32) {
        float xc[FJOFC_MAX_M];
        float cm = 0.f;
        if (i < n) {
            // centre X_{t-1} (in place) and its commensurability term
            for (int j = 0; j < m; ++j) {
                const int64_t off = (int64_t(j) * n + i) * d + k;
                xc[j] = p.Xprev[off] - mu_prev[j * FJOFC_MAX_D + k];
                if (p.t > 1) p.Xprev[off] = xc[j];   // X_0 (mu_0 = 0) is left untouched
            }
            for (int j = 0; j < m; ++j)
                for (int l = j + 1; l < m; ++l) {
                    const float df = xc[j] - xc[l];
                    cm = fmaf(p.wcomm[j][l] * df, df, cm);
                }
        }
        comm = ff_add(comm, cm);
        if (!p.final_pass) {
            for (int j = 0; j < m; ++j) {
                float v = 0.f;
                if (i < n) {
                    for (int l = 0; l < m; ++l) v = fmaf(p.coef[j][l], s_bx[l * d + k][lane], v);
                    p.Xnext[(int64_t(j) * n + i) * d + k] = v;
                }
                const FF cs = warp_sum_ff(FF{v, 0.f});
                if (lane == 0) s_part[j * d + k] = cs;
            }
        }
    }
    const FF ctot = block_sum_ff(comm, s_ff);
    const int npart = m * d + 1;
    if (tid == 0) {
        for (int e = 0; e < m * d; ++e)
            p.bpart[int64_t(blockIdx.x) * npart + e] = p.final_pass ? make_float2(0.f, 0.f)
                                                                     : make_float2(s_part[e].hi, s_part[e].lo);
        p.bpart[int64_t(blockIdx.x) * npart + m * d] = make_float2(ctot.hi, ctot.lo);
        __threadfence();
        const unsigned prev = atomicAdd(p.ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last CTA: totals in a fixed order (per-thread strided sums, then a tree)
    const int nblk = gridDim.x;
    for (int e = 0; e < m * d; ++e) {
        FF acc{0.f, 0.f};
        for (int b = tid; b < nblk; b += K2_THREADS) {
            const float2 v = __ldcg(p.bpart + int64_t(b) * npart + e);
            acc = ff_add(acc, FF{v.x, v.y});
        }
        const FF tot = block_sum_ff(acc, s_ff);
        if (tid == 0) mu_next[(e / d) * FJOFC_MAX_D + (e % d)] = (tot.hi + tot.lo) / float(n);
    }
    FF c{0.f, 0.f};
    for (int b = tid; b < nblk; b += K2_THREADS) {
        const float2 v = __ldcg(p.bpart + int64_t(b) * npart + m * d);
        c = ff_add(c, FF{v.x, v.y});
    }
    const FF comm_tot = block_sum_ff(c, s_ff);
    FF f{0.f, 0.f};
    for (int e = tid; e < p.G; e += K2_THREADS) {
        const float2 v = __ldcg(p.fid + e);
        f = ff_add(f, FF{v.x, v.y});
    }
    const FF fid_tot = block_sum_ff(f, s_ff);

    if (tid == 0) {
        const double sigma = (double(fid_tot.hi) + double(fid_tot.lo)) + (double(comm_tot.hi) + double(comm_tot.lo));
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
                                                                     : (dec / p.npairs > p.tol);
                stop = !cont;
            }
            if (stop) st->done = 1;
        }
        __threadfence();
        *p.ticket = 0u;                          // ready for the next launch
    }
}

int k2_blocks(int n) { return (n + K2_OBJ - 1) / K2_OBJ; }

cudaError_t launch_k2(const K2Params& p, cudaStream_t s) {
    const int tab = p.nRB + 1 + p.G + 1;
    const size_t smem = tab <= K2_TAB_SMEM_MAX ? size_t(tab) * sizeof(int64_t) : 0;
    k_apply<<<p.nbx, K2_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

// Per-call initialisation: status block, ticket, mu_0 = 0, walk offsets.
__global__ void k_init(const InitParams p) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        p.st->done = 0;
        p.st->error = 0;
        p.st->final_iter = 0;
        p.st->timeout_site = 0;
        p.st->stress = 0.0;
        *p.ticket = 0u;
        if (p.bar) *p.bar = 0u;
    }
    for (int e = tid; e < 2 * FJOFC_MAX_M * FJOFC_MAX_D; e += gridDim.x * blockDim.x) p.mu[e] = 0.f;
    for (int b = tid; b <= p.G; b += gridDim.x * blockDim.x) p.cta_start[b] = int64_t(b) * p.T / p.G;
    for (int P = tid; P <= p.nRB; P += gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int Q = 0; Q < P; ++Q) {
            const int64_t cols = int64_t(p.n) - int64_t(walk_row(Q, p.nRB)) * p.RB;
            s += (cols + p.CW - 1) / p.CW;
        }
        p.walk_off[P] = s;
    }
}

cudaError_t launch_init(const InitParams& p, cudaStream_t s) {
    const int threads = 256;
    const int mx = (p.nRB > p.G ? p.nRB : p.G) + 1;
    const int blocks = (mx + threads - 1) / threads;
    k_init<<<blocks, threads, 0, s>>>(p);
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
__global__ void k_oos_prep(const OOSPrepParams p) {
    const int j = blockIdx.x / p.d, kk = blockIdx.x - j * p.d;
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < p.nx; i += blockDim.x) {
        const float v = (i < p.n) ? p.X[(int64_t(j) * p.n + i) * p.d + kk] : 0.f;
        p.XT[(int64_t(j) * p.d + kk) * p.nx + i] = v;
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

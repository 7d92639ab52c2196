// K3r: the out-of-sample iterations of Sec. 3 (Eq. joosupdate) with one CTA per new
// object and the whole problem on chip, for in-sample sets small enough that -X^T
// (m d n floats) and one object's dissimilarities (m n floats) fit in shared memory.
//
// The streaming kernel (k_oos.cuh) gives every object one warp slot and reads its
// dissimilarities from memory again every iteration: right for many objects against a
// large in-sample set, but a few objects leave the GPU idle and every iteration waits
// on its own loads.  Here a CTA copies -X^T into shared memory once (it serves every
// object the CTA takes), copies an object's dissimilarities once, and runs that
// object's iterations out of shared memory: one pass of the CTA's threads over the m n
// (modality, point) pairs, a fixed-order reduction over the warps, the stopping test of
// the object's stress and the m x m mix.  Objects come from an atomic counter.  The
// arithmetic per pair, the stress and the stopping rule are the streaming kernel's:
//     d_jk = ||X^(j)_k - y_j||,  b_k = delta_j(k) / d_jk (0 when d_jk = 0, Eq. B),
//     xi_j = w_jj (sum_k X^(j)_k - s_j sum_k b_k X^(j)_k),  psi_j = w_jj s_j sum_k b_k,
//     y_t = Wmod^-1 (xi + psi o y_{t-1}),
//     sigma = sum_j w_jj sum_k (s_j delta_j(k) - d_jk)^2 + sum_{i<j} w_ij ||y_i - y_j||^2.
// No TMA, no mbarrier and no wait on another CTA: only CTA barriers.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"
#include "k3_decl.h"

namespace fjofc {

template <int D, typename TD>
__global__ void __launch_bounds__(kK3rThreads)
k_oos_resident(const K3Params p) {
    extern __shared__ float4 smem_f4[];
    float* xs = reinterpret_cast<float*>(smem_f4);        // [m][D][nx]  -x
    const int m = p.m, n = p.n, nx = p.nx;
    float* dl = xs + size_t(m) * D * nx;                  // [m][nx]     delta of the object
    float* s_y = dl + size_t(m) * nx;                     // [m][D]      y_{t-1}
    float* s_part = s_y + m * D;                          // [warps][m][D + 3]: -sum b x, sum b, fid (hi, lo)
    float* s_acc = s_part + kK3rWarps * m * (D + 3);      // [m][D + 1]
    double* s_fid = reinterpret_cast<double*>(s_y + k3r_state_floats(m, D));   // [m]
    double* s_comm = s_fid + m;                                                 // [m]
    __shared__ double s_sig;
    __shared__ long long s_obj;
    __shared__ int s_stop;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int passes = p.max_iter + 1;
    const TD* delta = static_cast<const TD*>(p.delta_new);

    // -X^T once per CTA ([m][D][nx], a multiple of 4 floats, 16-byte aligned)
    {
        const float4* src = reinterpret_cast<const float4*>(p.XT);
        float4* dst = reinterpret_cast<float4*>(xs);
        const int64_t nv = int64_t(m) * D * nx / 4;
        for (int64_t e = tid; e < nv; e += kK3rThreads) dst[e] = __ldg(src + e);
    }

    for (;;) {
        if (tid == 0) {
            const unsigned long long o = atomicAdd(p.next_block, 1ull);
            s_obj = (int64_t(o) < p.k && ld_volatile(&p.st->error) == 0) ? (long long)o : -1ll;
        }
        __syncthreads();                                   // also orders the -X^T copy
        const long long o = s_obj;
        if (o < 0) break;
        for (int64_t e = tid; e < int64_t(m) * n; e += kK3rThreads) {
            const int j = int(e / n), i = int(e - int64_t(j) * n);
            dl[int64_t(j) * nx + i] = DeltaLoad<TD>::to_f32(delta[(int64_t(o) * m + j) * p.ld + i]);
        }
        for (int e = tid; e < m * D; e += kK3rThreads) s_y[e] = p.Y[int64_t(o) * m * D + e];
        double sprev = 0.0;                                // read by thread 0 only
        __syncthreads();

        for (int pass = 1;; ++pass) {
            // sums over the in-sample points of every modality at y_{t-1}
            for (int j = 0; j < m; ++j) {
                float yj[D], bx[D];
#pragma unroll
                for (int kk = 0; kk < D; ++kk) { yj[kk] = s_y[j * D + kk]; bx[kk] = 0.f; }
                const float* xj = xs + size_t(j) * D * nx;
                const float* dj = dl + size_t(j) * nx;
                const float nsc = -p.dscale[j];
                float bs = 0.f, fs = 0.f;
                for (int i = tid; i < n; i += kK3rThreads) {
                    float xv[D];
                    float d2 = 0.f;
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        xv[kk] = xj[kk * nx + i];
                        const float df = yj[kk] + xv[kk];
                        d2 = fmaf(df, df, d2);
                    }
                    const float del = dj[i];
                    const float rinv = (d2 > 0.f) ? rsqrt_approx(d2) : 0.f;
                    const float bb = del * rinv;
                    const float e = fmaf(nsc, del, d2 * rinv);       // d - s delta
                    bs += bb;
                    fs = fmaf(e, e, fs);
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) bx[kk] = fmaf(bb, xv[kk], bx[kk]);   // -sum b x
                }
                const FF fr = warp_sum_ff(FF{fs, 0.f});
                bs = warp_sum_f32(bs);
#pragma unroll
                for (int kk = 0; kk < D; ++kk) bx[kk] = warp_sum_f32(bx[kk]);
                if (lane == 0) {
                    float* sp = s_part + (warp * m + j) * (D + 3);
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) sp[kk] = bx[kk];
                    sp[D] = bs;
                    sp[D + 1] = fr.hi;
                    sp[D + 2] = fr.lo;
                }
            }
            __syncthreads();
            // fixed-order totals over the warps: m (D + 1) float sums, then m float-float
            // fidelities, one per thread
            for (int e = tid; e < m * (D + 1) + m; e += kK3rThreads) {
                if (e < m * (D + 1)) {
                    const int j = e / (D + 1), c = e - j * (D + 1);
                    float v = 0.f;
                    for (int w = 0; w < kK3rWarps; ++w) v += s_part[(w * m + j) * (D + 3) + c];
                    s_acc[j * (D + 1) + c] = v;
                } else {
                    const int j = e - m * (D + 1);
                    FF f{0.f, 0.f};
                    for (int w = 0; w < kK3rWarps; ++w)
                        f = ff_add(f, FF{s_part[(w * m + j) * (D + 3) + D + 1], s_part[(w * m + j) * (D + 3) + D + 2]});
                    s_fid[j] = double(f.hi) + double(f.lo);
                }
            }
            // commensurability of y_{t-1}: thread a < m sums its pairs (a, b > a) in b order
            // (float64), thread 0 adds the m parts in a order after the fidelities
            if (tid < m) {
                const int a = tid;
                double ca = 0.0;
                for (int b2 = a + 1; b2 < m; ++b2) {
                    double s2 = 0.0;
                    for (int kk = 0; kk < D; ++kk) {
                        const double df = double(s_y[a * D + kk]) - double(s_y[b2 * D + kk]);
                        s2 += df * df;
                    }
                    ca += __ldg(p.wcomm + a * m + b2) * s2;
                }
                s_comm[a] = ca;
            }
            __syncthreads();
            // stress of y_{t-1} and the stopping test (the streaming kernel's rule)
            if (tid == 0) {
                double sig = 0.0;
                for (int j = 0; j < m; ++j) sig += double(p.wfid[j]) * s_fid[j];
                for (int a = 0; a < m; ++a) sig += s_comm[a];
                bool stop = (pass == passes) || !isfinite(sig);
                if (!stop && pass >= 2 && p.tol >= 0.0) {
                    const double dec = sprev - sig;
                    const bool cont = (p.tol_mode == FJOFC_TOL_RELATIVE) ? (dec > p.tol * sprev)
                                                                         : (dec / p.npairs > p.tol);
                    stop = !cont;
                }
                sprev = sig;
                s_sig = sig;
                s_stop = stop ? 1 : 0;
            }
            __syncthreads();
            if (s_stop) {
                for (int e = tid; e < m * D; e += kK3rThreads) p.Y[int64_t(o) * m * D + e] = s_y[e];
                if (tid == 0) {
                    if (p.iters_out) p.iters_out[o] = pass - 1;
                    p.stress_out[o] = s_sig;
                    if (!isfinite(s_sig)) atomicCAS(&p.st->error, 0, FJOFC_ERR_NONFINITE);
                }
                break;
            }
            // y_t = Wmod^-1 (xi + psi o y_{t-1}); m D <= FJOFC_MAX_M kK3rMaxD = kK3rThreads
            static_assert(FJOFC_MAX_M * kK3rMaxD <= kK3rThreads, "one thread per (j, k)");
            float v = 0.f;
            const bool mine = tid < m * D;
            if (mine) {
                const int j = tid / D, kk = tid - j * D;
                for (int i2 = 0; i2 < m; ++i2) {
                    const float wi = p.wfid[i2], si = p.dscale[i2];
                    const float xi = wi * fmaf(si, s_acc[i2 * (D + 1) + kk], p.SX[i2 * D + kk]);   // s_acc = -sum b x
                    const float psi = wi * si * s_acc[i2 * (D + 1) + D];
                    v = fmaf(__ldg(p.winv + j * m + i2), fmaf(psi, s_y[i2 * D + kk], xi), v);
                }
            }
            __syncthreads();
            if (mine) s_y[tid] = v;
            __syncthreads();
        }
        __syncthreads();                                   // the object's buffers are free again
    }
}

template <int D, typename TD>
cudaError_t k3r_launch_impl(int grid, const K3Params& p, cudaStream_t s) {
    const size_t smem = k3r_smem_bytes(p.m, p.nx, D);
    cudaError_t e = cudaFuncSetAttribute(k_oos_resident<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kK3rSmemBudget));
    if (e != cudaSuccess) return e;
    k_oos_resident<D, TD><<<grid, kK3rThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int D, typename TD>
int k3r_bps_impl(size_t smem) {
    cudaFuncSetAttribute(k_oos_resident<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kK3rSmemBudget));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_oos_resident<D, TD>, kK3rThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

#define FJOFC_INSTANTIATE_K3R(D)                                                          \
    template cudaError_t k3r_launch_impl<D, float>(int, const K3Params&, cudaStream_t);   \
    template cudaError_t k3r_launch_impl<D, __half>(int, const K3Params&, cudaStream_t);  \
    template cudaError_t k3r_launch_impl<D, __nv_bfloat16>(int, const K3Params&, cudaStream_t); \
    template int k3r_bps_impl<D, float>(size_t);                                          \
    template int k3r_bps_impl<D, __half>(size_t);                                         \
    template int k3r_bps_impl<D, __nv_bfloat16>(size_t);

}  // namespace fjofc

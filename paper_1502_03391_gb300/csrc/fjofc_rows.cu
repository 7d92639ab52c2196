// One Guttman transform restricted to a range of objects: the building block of
// row-block sharding across GPUs (fjofc_transform_rows).
//
// Eq. (update) mixes, per object i, the rows (B_l X^(l))_i of the m diagonal blocks of
// B(X) X: X_t^(j)_i = sum_l [Wmod^-1]_{jl} (B_l X^(l))_i.  A GPU that holds rows
// [r0, r1) of every Delta_l (all n columns) therefore computes the rows [r0, r1) of X_t
// from the whole X_{t-1}; the GPUs then exchange their rows (an all-gather of X) and add
// up the scalar parts below (an all-reduce) before the next transform.
//
// K6 (k_rows_pass<D, TD>): one CTA per group of 32 objects of the range, 8 warps of 4
// objects each.  For every modality l a warp walks the object's full Delta row: lane L
// takes columns L, L + 32, ..., forms d_ij = ||x_i - x_j|| (x centred by mu), b_ij =
// Delta_ij / d_ij (0 when d_ij = 0 or j = i, Eq. B) and accumulates b_ij (x_i - x_j) and
// (Delta_ij - d_ij)^2 (float32, folded into float-float every 8 columns); a butterfly
// gives the object's sums.  Then the CTA mixes the m rows of every object into X_t and
// forms its per-group parts in a fixed order: the fidelity share of the range (half of
// the full-row sum, every unordered pair being seen from both of its rows across the
// GPUs), the commensurability of the range's objects, and the column sums of the X_t
// rows.  The last CTA (ticket) adds the group parts in group order into float64 parts.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "fjofc_device.cuh"

namespace fjofc {
namespace {

constexpr int kRowsWarps = 8, kRowsPerWarp = 4, kRowsGroup = kRowsWarps * kRowsPerWarp;   // 32

struct RowsParams {
    const void* delta[FJOFC_MAX_M];   // rows r0..r1-1 of Delta_l, row stride ld
    int64_t ld;
    const float* X;                   // (m n) x d, X_{t-1}
    float* Xout;                      // m x (r1 - r0) x d
    float2* gpart;                    // [ngroups][2 + m d] float-float group parts
    double* parts;                    // [2 + m d] totals (device)
    unsigned* ticket;
    int m, n, d, r0, r1, ngroups;
    float mu[FJOFC_MAX_M * FJOFC_MAX_D];   // means of X_{t-1} per (modality, coordinate)
    float dscale[FJOFC_MAX_M];             // Delta scale s_l
    float coef[FJOFC_MAX_M * FJOFC_MAX_M]; // [Wmod^-1]_{jl} w_ll, m x m
    float wfid[FJOFC_MAX_M];               // w_ll
    float wcomm[FJOFC_MAX_M * FJOFC_MAX_M];// w_jl for j < l, else 0
};

template <int D, typename TD>
__global__ void __launch_bounds__(kRowsWarps * 32) k_rows_pass(const __grid_constant__ RowsParams p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, m = p.m, n = p.n;
    const int nr = p.r1 - p.r0;
    extern __shared__ float s_dyn[];
    float* s_bx = s_dyn;                                   // [32][m][D]  (B'_l X)_i
    __shared__ FF s_fid[kRowsGroup];
    for (int l = 0; l < m; ++l) {
        const float* Xl = p.X + int64_t(l) * n * D;
        const TD* Dl = static_cast<const TD*>(p.delta[l]);
        const float s = p.dscale[l];
        float xi[kRowsPerWarp][D], acc[kRowsPerWarp][D];
        FF fid[kRowsPerWarp];
        int gi[kRowsPerWarp];
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
            const int o = g * kRowsGroup + warp * kRowsPerWarp + r;        // object within the range
            gi[r] = (o < nr) ? p.r0 + o : -1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                xi[r][k] = gi[r] >= 0 ? __ldg(Xl + int64_t(gi[r]) * D + k) - p.mu[l * FJOFC_MAX_D + k] : 0.f;
                acc[r][k] = 0.f;
            }
            fid[r] = FF{0.f, 0.f};
        }
        float f32[kRowsPerWarp] = {};
        int cnt = 0;
        for (int j = lane; j < n; j += 32) {
            float xj[D];
#pragma unroll
            for (int k = 0; k < D; ++k) xj[k] = __ldg(Xl + int64_t(j) * D + k) - p.mu[l * FJOFC_MAX_D + k];
#pragma unroll
            for (int r = 0; r < kRowsPerWarp; ++r) {
                if (gi[r] < 0) continue;
                const float del = s * DeltaLoad<TD>::to_f32(Dl[int64_t(gi[r] - p.r0) * p.ld + j]);
                float diff[D], d2 = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    diff[k] = xi[r][k] - xj[k];
                    d2 = fmaf(diff[k], diff[k], d2);
                }
                if (j == gi[r]) continue;                    // the diagonal has weight 0 (Eq. W)
                const float dd = sqrtf(d2);
                const float b = dd > 0.f ? del / dd : 0.f;   // Eq. B: 0 when d_ij = 0
                const float e = del - dd;
                f32[r] = fmaf(e, e, f32[r]);
#pragma unroll
                for (int k = 0; k < D; ++k) acc[r][k] = fmaf(b, diff[k], acc[r][k]);
            }
            if (++cnt == 8) {
                cnt = 0;
#pragma unroll
                for (int r = 0; r < kRowsPerWarp; ++r) {
                    fid[r] = ff_add(fid[r], f32[r]);
                    f32[r] = 0.f;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
            fid[r] = warp_sum_ff(ff_add(fid[r], f32[r]));
#pragma unroll
            for (int k = 0; k < D; ++k) acc[r][k] = warp_sum_f32(acc[r][k]);
            const int row = warp * kRowsPerWarp + r;
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < D; ++k) s_bx[(row * m + l) * D + k] = acc[r][k];
                // fidelity of this row in modality l, weighted; accumulated over l in order
                const FF wf = ff_mul(fid[r], p.wfid[l]);
                s_fid[row] = (l == 0) ? wf : ff_add(s_fid[row], wf);
            }
        }
    }
    __syncthreads();
    // the mix, the commensurability and the column sums: thread e handles (row, k)
    float2* gp = p.gpart + int64_t(g) * (2 + m * D);
    for (int e = threadIdx.x; e < kRowsGroup * D; e += blockDim.x) {
        const int row = e / D, k = e - row * D;
        const int o = g * kRowsGroup + row;
        if (o >= nr) continue;
        for (int j = 0; j < m; ++j) {
            float v = 0.f;
            for (int l = 0; l < m; ++l) v = fmaf(p.coef[j * m + l], s_bx[(row * m + l) * D + k], v);
            p.Xout[(int64_t(j) * nr + o) * D + k] = v;
        }
    }
    __syncthreads();
    // group parts (one warp each, fixed order): fidelity (half of the full-row sums),
    // commensurability of the X_{t-1} rows, column sums of the X_t rows
    if (warp == 0) {
        const int o = g * kRowsGroup + lane;
        const bool in = o < nr;
        FF f = in ? s_fid[lane] : FF{0.f, 0.f};
        f = warp_sum_ff(f);
        float c = 0.f;
        if (in) {
            const int i = p.r0 + o;
            for (int j = 0; j < m; ++j)
                for (int l = j + 1; l < m; ++l)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float df = (__ldg(p.X + (int64_t(j) * n + i) * D + k) - p.mu[j * FJOFC_MAX_D + k]) -
                                         (__ldg(p.X + (int64_t(l) * n + i) * D + k) - p.mu[l * FJOFC_MAX_D + k]);
                        c = fmaf(p.wcomm[j * m + l] * df, df, c);
                    }
        }
        const FF cw = warp_sum_ff(FF{c, 0.f});
        if (lane == 0) {
            gp[0] = make_float2(0.5f * f.hi, 0.5f * f.lo);
            gp[1] = make_float2(cw.hi, cw.lo);
        }
        for (int e = 0; e < m * D; ++e) {
            const int j = e / D, k = e - j * D;
            const float v = in ? p.Xout[(int64_t(j) * nr + o) * D + k] : 0.f;
            const FF sv = warp_sum_ff(FF{v, 0.f});
            if (lane == 0) gp[2 + e] = make_float2(sv.hi, sv.lo);
        }
    }
    // the last CTA adds the group parts in group order
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(p.ticket, 1u) == unsigned(p.ngroups) - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int np = 2 + m * D;
    for (int e = warp; e < np; e += kRowsWarps) {
        const FF t = totals_ff(p.gpart + e, np, p.ngroups);
        if (lane == 0) p.parts[e] = double(t.hi) + double(t.lo);
    }
    if (threadIdx.x == 0) *p.ticket = 0u;
}

template <typename TD>
cudaError_t launch_rows_dt(int d, const RowsParams& p, cudaStream_t s) {
    const size_t smem = size_t(kRowsGroup) * p.m * d * sizeof(float);
    switch (d) {
#define C_(D)                                                                                                \
    case D: {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(k_rows_pass<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             int(smem));                                                     \
        if (e != cudaSuccess) return e;                                                                      \
        k_rows_pass<D, TD><<<p.ngroups, kRowsWarps * 32, smem, s>>>(p);                                      \
        return cudaGetLastError();                                                                           \
    }
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace fjofc

using namespace fjofc;

extern "C" int fjofc_transform_rows(int32_t m, int64_t n, int32_t d, int64_t r0, int64_t r1,
                                    const void* const* delta_rows, int64_t ld, int32_t delta_dtype,
                                    const float* delta_scale, const double* weights, const float* X, const double* mu,
                                    float* Xout, double* parts, void* cuda_stream) {
    char msg[256];
    auto fail = [&](int code, const char* text) {
        set_message(text);
        return code;
    };
    if (m < 1 || m > FJOFC_MAX_M) return fail(m < 1 ? FJOFC_ERR_ARG : FJOFC_ERR_UNSUPPORTED, "m outside 1..FJOFC_MAX_M");
    if (n < 2 || n > (int64_t(1) << 30)) return fail(FJOFC_ERR_ARG, "n must be in 2..2^30");
    if (d < 1 || d > FJOFC_MAX_D) return fail(d < 1 ? FJOFC_ERR_ARG : FJOFC_ERR_UNSUPPORTED, "d outside 1..FJOFC_MAX_D");
    if (r0 < 0 || r1 <= r0 || r1 > n) return fail(FJOFC_ERR_ARG, "object range must satisfy 0 <= r0 < r1 <= n");
    if (!delta_rows || !X || !Xout || !parts) return fail(FJOFC_ERR_ARG, "NULL pointer");
    if (ld < n) return fail(FJOFC_ERR_ARG, "ld must be >= n");
    if (delta_dtype != FJOFC_F32 && delta_dtype != FJOFC_F16 && delta_dtype != FJOFC_BF16)
        return fail(FJOFC_ERR_ARG, "unknown delta_dtype");
    for (int l = 0; l < m; ++l)
        if (!delta_rows[l]) return fail(FJOFC_ERR_ARG, "Delta pointer is NULL");
    if (delta_scale)
        for (int l = 0; l < m; ++l)
            if (!(delta_scale[l] > 0.f) || !std::isfinite(delta_scale[l]))
                return fail(FJOFC_ERR_ARG, "delta_scale must be finite and > 0");
    if (mu)
        for (int e = 0; e < m * d; ++e)
            if (!std::isfinite(mu[e])) return fail(FJOFC_ERR_ARG, "mu must be finite");
    double winv[FJOFC_MAX_M * FJOFC_MAX_M];
    int rc = modified_weights_inverse(m, n, weights, winv);
    if (rc) return rc;
    const size_t smem = size_t(kRowsGroup) * m * d * sizeof(float);
    if (smem > 200 * 1024) return fail(FJOFC_ERR_UNSUPPORTED, "m d too large for one group's staging");

    const cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    RowsParams p{};
    for (int l = 0; l < m; ++l) {
        p.delta[l] = delta_rows[l];
        p.dscale[l] = delta_scale ? delta_scale[l] : 1.f;
        p.wfid[l] = float(weights[l * m + l]);
        for (int k = 0; k < d; ++k) p.mu[l * FJOFC_MAX_D + k] = mu ? float(mu[l * d + k]) : 0.f;
    }
    for (int j = 0; j < m; ++j)
        for (int l = 0; l < m; ++l) {
            p.coef[j * m + l] = float(winv[j * m + l] * weights[l * m + l]);
            p.wcomm[j * m + l] = (j < l) ? float(weights[j * m + l]) : 0.f;
        }
    p.ld = ld;
    p.X = X;
    p.Xout = Xout;
    p.m = m; p.n = int(n); p.d = d; p.r0 = int(r0); p.r1 = int(r1);
    p.ngroups = int((r1 - r0 + kRowsGroup - 1) / kRowsGroup);
    const int np = 2 + m * d;
    // scratch: group parts, totals, ticket (stream-ordered)
    size_t bytes = size_t(p.ngroups) * np * sizeof(float2);
    const size_t o_parts = (bytes + 255) & ~size_t(255);
    bytes = o_parts + np * sizeof(double);
    const size_t o_ticket = (bytes + 255) & ~size_t(255);
    bytes = o_ticket + 256;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        snprintf(msg, sizeof(msg), "cudaMallocAsync(%zu bytes) failed", bytes);
        return fail(FJOFC_ERR_NOMEM, msg);
    }
    char* base = static_cast<char*>(mem);
    p.gpart = reinterpret_cast<float2*>(base);
    p.parts = reinterpret_cast<double*>(base + o_parts);
    p.ticket = reinterpret_cast<unsigned*>(base + o_ticket);
    cudaError_t e = cudaMemsetAsync(p.ticket, 0, sizeof(unsigned), stream);
    if (e == cudaSuccess)
        e = (delta_dtype == FJOFC_F32) ? launch_rows_dt<float>(d, p, stream)
          : (delta_dtype == FJOFC_F16) ? launch_rows_dt<__half>(d, p, stream)
                                       : launch_rows_dt<__nv_bfloat16>(d, p, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(parts, p.parts, np * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(mem, stream);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "%s (fjofc_transform_rows)", cudaGetErrorString(e));
        cudaGetLastError();
        return fail(FJOFC_ERR_CUDA, msg);
    }
    return FJOFC_OK;
}

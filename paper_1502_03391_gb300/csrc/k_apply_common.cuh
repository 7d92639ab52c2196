// Per-object work of a Guttman pass after the all-pairs tiles (Eq. update, Cor. 1,
// Remark faststress), shared by K2 (k_apply) and phase B of the persistent kernel so that
// both paths sum every partial in exactly the same order (bitwise equal results).
//
// Objects are handled in groups of 32 (lane = object).  For every group g the CTA
//   1. sums (B'_l X_l)_{i,k} for all (l, k) from the K1 partials and stages x_{t-1} of the
//      group in shared memory (one warp per (l, k) unit),
//   2. per coordinate k (one warp each): centres X_{t-1} with the previous pass's means,
//      forms its commensurability, mixes X_t^(j) = sum_l coef[j][l] (B'_l X_l) and writes
//      the float-float column sums of X_t -> bpart[g][j*d + k],
//   3. sums the commensurability over k in order -> bpart[g][m*d].
#pragma once

#include "fjofc_device.cuh"

namespace fjofc {

constexpr int kGroupObjects = 32;
constexpr int kBxBatch = 16;     // column partials in flight per lane

// (B'_l X_l)_{i,k}: the walk-head row partial of object i, the continuation row partials
// in CTA order, then the column partials of the walks of row blocks 0..I(i) in order.
// Data written earlier in the same launch is read through L2 (ld.global.cg); the tables
// are read-only for the whole launch (ld.global.nc).  This code runs once per pass after
// the long all-pairs loop, so it is kept small (rolled loops) to limit instruction-cache
// refills; kBxBatch loads are issued before their sum.
__device__ __forceinline__ float bx_sum(const BxTables& tb, int l, int k, int i) {
    const int d = tb.d, RB = tb.RB, CW = tb.CW, rbs = tb.rb_shift, cws = tb.cw_shift, nRB = tb.nRB;
    const int I = i >> rbs, ri = i & (RB - 1);
    const int2 cr = __ldg(tb.cont + int64_t(l) * nRB + I);
    const float* cp = tb.colpart + int64_t(l) * tb.Tm * d * CW;
    float acc = __ldcg(tb.rowhead + ((int64_t(l) * nRB + I) * d + k) * RB + ri);
#pragma unroll 1
    for (int b = cr.x; b < cr.y; ++b) acc += __ldcg(tb.rowcont + (int64_t(b) * d + k) * RB + ri);
    float csum = 0.f;
#pragma unroll 1
    for (int J0 = 0; J0 <= I; J0 += kBxBatch) {
        float v[kBxBatch];
#pragma unroll
        for (int u = 0; u < kBxBatch; ++u) {
            const int J = J0 + u, rel = i - (J << rbs);
            v[u] = (J <= I) ? __ldcg(cp + ((__ldg(tb.cbase + J) + (rel >> cws)) * d + k) * CW + (rel & (CW - 1)))
                            : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kBxBatch; ++u) csum += v[u];
    }
    return acc + csum;
}

// What phase B needs besides the partial tables.
struct PhaseBArgs {
    BxTables tb;
    float* Xprev;                               // X_{t-1}, centred in place (t > 1)
    float* Xnext;                               // X_t
    float2* bpart;                              // [ngroups][m*d + 1]
    const float* mu_prev;                       // [MAX_M][MAX_D] means of X_{t-1} (shared memory)
    const float (*coef)[FJOFC_MAX_M];           // Wmod^-1 w_ll s_l (shared memory)
    const float (*wcomm)[FJOFC_MAX_M];          // w_jl for j < l, else 0 (shared memory)
    int m, n, d, t;
    bool final_pass;                            // only centre and score X_{t-1}
};

// Shared-memory floats phase B needs per group (staged values, then d float-float sums).
__host__ __device__ constexpr int phase_b_floats_per_group(int m, int d) { return 2 * m * d * kGroupObjects + 2 * d; }

// Phase B for the groups g = g0, g0 + gstride, ... (< ngroups), processed in chunks of at
// most `cap` groups; s holds cap * phase_b_floats_per_group(m, d) floats (8-byte aligned).
// Every thread of the CTA must call it.
__device__ __forceinline__ void phase_b(const PhaseBArgs& a, int g0, int gstride, int ngroups, int cap, float* s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int m = a.m, n = a.n, d = a.d, md = m * d, npart = md + 1;
    const int mine = (g0 < ngroups) ? (ngroups - g0 + gstride - 1) / gstride : 0;
#pragma unroll 1
    for (int c0 = 0; c0 < mine; c0 += cap) {
        const int nc = min(cap, mine - c0);
        float* s_bx = s;                                   // [nc][m][d][32]
        float* s_xp = s + nc * md * kGroupObjects;         // [nc][m][d][32]
        FF* s_comm = reinterpret_cast<FF*>(s + 2 * nc * md * kGroupObjects);   // [nc][d]
        // 1. partial sums and staged x_{t-1}, one (group, l, k) unit per warp
#pragma unroll 1
        for (int u = warp; u < nc * md; u += nwarps) {
            const int gi = u / md, lk = u - gi * md, l = lk / d, k = lk - l * d;
            const int i = (g0 + (c0 + gi) * gstride) * kGroupObjects + lane;
            const bool in = i < n;
            s_xp[u * kGroupObjects + lane] = in ? __ldcg(a.Xprev + (int64_t(l) * n + i) * d + k) : 0.f;
            s_bx[u * kGroupObjects + lane] = (in && !a.final_pass) ? bx_sum(a.tb, l, k, i) : 0.f;
        }
        __syncthreads();
        // 2. per (group, coordinate): centre, commensurability, mix, column sums
#pragma unroll 1
        for (int w = warp; w < nc * d; w += nwarps) {
            const int gi = w / d, k = w - gi * d;
            const int g = g0 + (c0 + gi) * gstride;
            const int i = g * kGroupObjects + lane;
            const bool in = i < n;
            float xc[FJOFC_MAX_M];
            float c = 0.f;
            for (int j = 0; j < m; ++j) {
                xc[j] = in ? s_xp[((gi * m + j) * d + k) * kGroupObjects + lane] - a.mu_prev[j * FJOFC_MAX_D + k] : 0.f;
                if (in && a.t > 1) a.Xprev[(int64_t(j) * n + i) * d + k] = xc[j];
            }
            if (in)
                for (int j = 0; j < m; ++j)
                    for (int l = j + 1; l < m; ++l) {
                        const float df = xc[j] - xc[l];
                        c = fmaf(a.wcomm[j][l] * df, df, c);
                    }
            const FF cw = warp_sum_ff(FF{c, 0.f});
            if (lane == 0) s_comm[gi * d + k] = cw;
            for (int j = 0; j < m; ++j) {
                float v = 0.f;
                if (!a.final_pass && in) {
                    for (int l = 0; l < m; ++l) v = fmaf(a.coef[j][l], s_bx[((gi * m + l) * d + k) * kGroupObjects + lane], v);
                    a.Xnext[(int64_t(j) * n + i) * d + k] = v;
                }
                const FF cs = warp_sum_ff(FF{v, 0.f});
                if (lane == 0)
                    a.bpart[int64_t(g) * npart + j * d + k] = a.final_pass ? make_float2(0.f, 0.f) : make_float2(cs.hi, cs.lo);
            }
        }
        __syncthreads();
        // 3. commensurability of each group, summed over k in order
        for (int gi = threadIdx.x; gi < nc; gi += blockDim.x) {
            FF tot{0.f, 0.f};
            for (int k = 0; k < d; ++k) tot = ff_add(tot, s_comm[gi * d + k]);
            a.bpart[int64_t(g0 + (c0 + gi) * gstride) * npart + md] = make_float2(tot.hi, tot.lo);
        }
        __syncthreads();
    }
}

}  // namespace fjofc

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
constexpr int kBxBatch = 16;     // column partials in flight per lane (default)

// (B'_l X_l)_{i,k} for U units (l[u], k[u], object i[u]) at once: the walk-head row
// partial of the object, the continuation row partials in CTA order, then the column
// partials of the walks of row blocks 0..I(i) in order.  Every unit's loads of a round
// (BATCH column partials each) are issued before any sum, so U units cost the latency of
// one; each unit's sum is formed in the same order whatever U and BATCH are.  Data
// written earlier in the same launch is read through L2 (ld.global.cg); the tables are
// read-only for the whole launch (ld.global.nc).  This code runs once per pass after the
// long all-pairs loop, so its loops stay rolled to limit instruction-cache refills.
template <int BATCH, int U>
__device__ __forceinline__ void bx_sum(const BxTables& tb, const int (&l)[U], const int (&k)[U], const int (&i)[U],
                                       const bool (&on)[U], float (&out)[U]) {
    const int d = tb.d, RB = tb.RB, CW = tb.CW, rbs = tb.rb_shift, cws = tb.cw_shift, nRB = tb.nRB;
    int I[U];
    float acc[U], csum[U];
    int Imax = -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        I[u] = on[u] ? (i[u] >> rbs) : -1;
        Imax = max(Imax, I[u]);
        acc[u] = on[u] ? __ldcg(tb.rowhead + ((int64_t(l[u]) * nRB + I[u]) * d + k[u]) * RB + (i[u] & (RB - 1))) : 0.f;
        csum[u] = 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (!on[u]) continue;
        const int2 cr = __ldg(tb.cont + int64_t(l[u]) * nRB + I[u]);
#pragma unroll 1
        for (int b = cr.x; b < cr.y; ++b)
            acc[u] += __ldcg(tb.rowcont + (int64_t(b) * d + k[u]) * RB + (i[u] & (RB - 1)));
    }
#pragma unroll 1
    for (int J0 = 0; J0 <= Imax; J0 += BATCH) {
        float v[U][BATCH];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float* cp = tb.colpart + int64_t(l[u]) * tb.Tm * d * CW;
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int J = J0 + j, rel = i[u] - (J << rbs);
                v[u][j] = (J <= I[u]) ? __ldcg(cp + ((__ldg(tb.cbase + J) + (rel >> cws)) * d + k[u]) * CW +
                                               (rel & (CW - 1)))
                                      : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < BATCH; ++j) csum[u] += v[u][j];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) out[u] = acc[u] + csum[u];
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
template <int BATCH = kBxBatch>
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
        // 1. partial sums and staged x_{t-1}: (group, l, k) units, two per warp per round
#pragma unroll 1
        for (int u0 = warp; u0 < nc * md; u0 += 2 * nwarps) {
            int uu[2], ll[2], kk[2], ii[2];
            bool on[2], in[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uu[h] = u0 + h * nwarps;
                const bool unit = uu[h] < nc * md;
                const int gi = unit ? uu[h] / md : 0, lk = unit ? uu[h] - gi * md : 0;
                ll[h] = lk / d;
                kk[h] = lk - ll[h] * d;
                ii[h] = (g0 + (c0 + gi) * gstride) * kGroupObjects + lane;
                in[h] = unit && ii[h] < n;
                on[h] = in[h] && !a.final_pass;
            }
            float xp[2], bx[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) xp[h] = in[h] ? __ldcg(a.Xprev + (int64_t(ll[h]) * n + ii[h]) * d + kk[h]) : 0.f;
            bx_sum<BATCH, 2>(a.tb, ll, kk, ii, on, bx);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (uu[h] < nc * md) {
                    s_xp[uu[h] * kGroupObjects + lane] = xp[h];
                    s_bx[uu[h] * kGroupObjects + lane] = on[h] ? bx[h] : 0.f;
                }
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

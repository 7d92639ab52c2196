// Per-object work of a Guttman pass after the all-pairs tiles (Eq. update, Cor. 1,
// Remark faststress), shared by K2 (k_apply) and phase B of the persistent kernel so that
// both paths sum every partial in exactly the same order (bitwise equal results).
//
// Objects are handled in groups of 32 (lane = object) and per coordinate: a unit is one
// (group g, coordinate k).  For every unit the CTA
//   1. sums (B'_l X_l)_{i,k} for every modality l from the K1 partials and stages x_{t-1}
//      of the group in shared memory (one warp per (unit, l)),
//   2. (one warp per unit) centres X_{t-1} with the previous pass's means (plain
//      transform only), forms its commensurability in coordinate k, mixes
//      X_t^(j) = sum_l coef[j][l] (B'_l X_l) (relaxed: X_{t-1} + relax (that - X_{t-1})) and
//      writes the group's sums (part-major bpart): column sums of X_t (float32; they only
//      feed the next centring) -> part j*d + k, commensurability (float-float) -> part
//      m*d + k.
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

// Walks whose column partials one warp gathers in a round of bx_sum_wide: 8 lanes read
// one walk's 128-byte row (16 bytes each), so a load instruction covers 4 walks; 12
// loads per lane in flight.
constexpr int kWideUnroll = 12;
constexpr int kWideWalksPerRound = 4 * kWideUnroll;
// largest number of walks (row blocks) for which phase B gathers by rows (beyond it: lane
// = object, for any walk count the row gather measured faster)
#ifndef FJOFC_WIDE_MAX_WALKS
#define FJOFC_WIDE_MAX_WALKS (1 << 30)
#endif

// (B'_l X_l)_{i,k} for the 32 objects i = 32g + lane of one group (all in row block I):
// the walk-head row partial and the continuation row partials of each object (lane =
// object), plus the column partials of the walks of row blocks 0..I: lane (q, s) of the
// four 8-lane groups q reads objects 4s..4s+3 of walks q, q+4, q+8, ... (fully coalesced
// 128-byte rows), adds them in walk order, the four groups are combined by a fixed
// butterfly and a gather leaves object o's total in lane o.  The order of every sum is
// fixed.  Requires RB >= 32 (a group inside one row block).  Every lane of the warp must
// call it.
__device__ __forceinline__ float bx_sum_wide(const BxTables& tb, int l, int k, int g, bool on) {
    const int lane = threadIdx.x & 31, q = lane >> 3, sq = lane & 7;
    const int d = tb.d, RB = tb.RB, CW = tb.CW, rbs = tb.rb_shift, cws = tb.cw_shift, nRB = tb.nRB;
    const int i0 = g * kGroupObjects, i = i0 + lane;
    const int I = i0 >> rbs;
    const float* cp = tb.colpart + int64_t(l) * tb.Tm * d * CW;
    const int nJ = on ? I + 1 : 0;
    // every load of the first round goes out before any sum: the walk-head row partial, the
    // continuation row partials (up to kContBatch of them) and the column partials of up to
    // kWideWalksPerRound walks; the sums are then formed in the fixed order (head, the
    // continuations in CTA order, the walks in order)
    constexpr int kContBatch = 8;
    const int2 cr = on ? __ldg(tb.cont + int64_t(l) * nRB + I) : make_int2(0, 0);
    const float h0 = on ? __ldcg(tb.rowhead + ((int64_t(l) * nRB + I) * d + k) * RB + (i & (RB - 1))) : 0.f;
    auto col_round = [&](int J0, float4 (&v)[kWideUnroll]) {
#pragma unroll
        for (int u = 0; u < kWideUnroll; ++u) {
            const int J = J0 + 4 * u + q;
            if (J < nJ) {
                const int rel0 = i0 - (J << rbs);
                v[u] = __ldcg(reinterpret_cast<const float4*>(
                                  cp + ((__ldg(tb.cbase + J) + (rel0 >> cws)) * d + k) * CW + (rel0 & (CW - 1))) +
                              sq);
            } else {
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    float4 v[kWideUnroll];
    col_round(0, v);
    float cont[kContBatch];
#pragma unroll
    for (int u = 0; u < kContBatch; ++u)
        cont[u] = (cr.x + u < cr.y) ? __ldcg(tb.rowcont + (int64_t(cr.x + u) * d + k) * RB + (i & (RB - 1))) : 0.f;
    float head = h0;
#pragma unroll
    for (int u = 0; u < kContBatch; ++u)
        if (cr.x + u < cr.y) head += cont[u];
#pragma unroll 1
    for (int b = cr.x + kContBatch; b < cr.y; ++b) head += __ldcg(tb.rowcont + (int64_t(b) * d + k) * RB + (i & (RB - 1)));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int J0 = 0; J0 < nJ; J0 += kWideWalksPerRound) {
        if (J0 > 0) col_round(J0, v);
#pragma unroll
        for (int u = 0; u < kWideUnroll; ++u) {
            acc.x += v[u].x;
            acc.y += v[u].y;
            acc.z += v[u].z;
            acc.w += v[u].w;
        }
    }
    // combine the four walk groups (partners xor 8, then xor 16; every lane gets the sum)
#pragma unroll
    for (int o = 8; o <= 16; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    // object o = lane sits in component o & 3 of lane o >> 2
    const int src = lane >> 2, comp = lane & 3;
    const float cx = __shfl_sync(0xffffffffu, acc.x, src), cy = __shfl_sync(0xffffffffu, acc.y, src);
    const float cz = __shfl_sync(0xffffffffu, acc.z, src), cw = __shfl_sync(0xffffffffu, acc.w, src);
    const float col = comp == 0 ? cx : (comp == 1 ? cy : (comp == 2 ? cz : cw));
    return head + col;
}

// What phase B needs besides the partial tables.
struct PhaseBArgs {
    BxTables tb;
    float* Xprev;                               // X_{t-1}, centred in place (t > 1)
    float* Xnext;                               // X_t
    float2* bpart;                              // [npart][ngroups] (part-major), npart = m*d + d
    const float* mu_prev;                       // means of X_{t-1}: mean of (j, k) at j*mu_stride + k (shared memory)
    int mu_stride;
    const float* coef_g;                        // [Wmod^-1]_{jl} w_ll s_l, m x m row-major (global)
    const float* wcomm_g;                       // w_jl for j < l, else 0
    int m, n, d, t, ngroups;
    bool final_pass;                            // only centre and score X_{t-1}
    bool centre;                                // centre X_{t-1} in place (plain transform)
    float relax;                                // X_t = X_{t-1} + relax (G - X_{t-1})
#ifdef FJOFC_STAMPS
    long long* stamp = nullptr;                 // instrumented builds: clock after step 1
#endif
};

// Per-group float-float sums written by phase B: the column sums of X_t^(j) for every
// (j, k) at index j*d + k, then the commensurability of coordinate k at index m*d + k.
__host__ __device__ constexpr int phase_b_parts(int m, int d) { return m * d + d; }
// Shared-memory floats phase B needs per unit (staged partial sums and x_{t-1}).
__host__ __device__ constexpr int phase_b_floats_per_unit(int m) { return 2 * m * kGroupObjects; }

// Phase B for the units u in [u0, u1), unit u = (group g = u / d, coordinate k = u % d),
// processed in chunks of at most `cap` units; s holds cap * phase_b_floats_per_unit(m)
// floats.  Every thread of the CTA must call it.
//   1. one warp per (unit, modality l): (B'_l X_l)_{i,k} for the group's 32 objects (lane
//      = object) from the partials, and x_{t-1}; two such at once per warp;
//   2. one warp per unit: centre X_{t-1} with the previous pass's means (written back),
//      its commensurability in coordinate k, the mix X_t^(j) = sum_l coef[j][l] (B'_l X_l)
//      and the group's sums -> bpart.
template <int BATCH = kBxBatch>
__device__ __forceinline__ void phase_b(const PhaseBArgs& a, int u0, int u1, int cap, float* s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int m = a.m, n = a.n, d = a.d, md = m * d, npart = phase_b_parts(m, d);
#pragma unroll 1
    for (int c0 = u0; c0 < u1; c0 += cap) {
        const int nc = min(cap, u1 - c0);
        float* s_bx = s;                                   // [nc][m][32]
        float* s_xp = s + nc * m * kGroupObjects;          // [nc][m][32]
        // 1. (unit, l) pairs: one per warp per round, column partials gathered by walk
        //    rows (bx_sum_wide; RB >= 32), else two per warp per round with lane = object
        //    (bx_sum)
        if (a.tb.RB >= kGroupObjects && a.tb.nRB <= FJOFC_WIDE_MAX_WALKS) {
#pragma unroll 1
            for (int w = warp; w < nc * m; w += nwarps) {
                const int ui = w / m, l = w - ui * m;
                const int u = c0 + ui, g = u / d, k = u - g * d;
                const int i = g * kGroupObjects + lane;
                const bool in = i < n;
                const float xp = in ? __ldcg(a.Xprev + (int64_t(l) * n + i) * d + k) : 0.f;
                const float bx = bx_sum_wide(a.tb, l, k, g, !a.final_pass);
                s_xp[w * kGroupObjects + lane] = xp;
                s_bx[w * kGroupObjects + lane] = (in && !a.final_pass) ? bx : 0.f;
            }
        } else {
#pragma unroll 1
        for (int w0 = warp; w0 < nc * m; w0 += 2 * nwarps) {
            int ww[2], ll[2], kk[2], ii[2];
            bool on[2], in[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                ww[h] = w0 + h * nwarps;
                const bool unit = ww[h] < nc * m;
                const int ui = unit ? ww[h] / m : 0;
                ll[h] = unit ? ww[h] - ui * m : 0;
                const int u = c0 + ui, g = u / d;
                kk[h] = u - g * d;
                ii[h] = g * kGroupObjects + lane;
                in[h] = unit && ii[h] < n;
                on[h] = in[h] && !a.final_pass;
            }
            float xp[2], bx[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) xp[h] = in[h] ? __ldcg(a.Xprev + (int64_t(ll[h]) * n + ii[h]) * d + kk[h]) : 0.f;
            bx_sum<BATCH, 2>(a.tb, ll, kk, ii, on, bx);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (ww[h] < nc * m) {
                    s_xp[ww[h] * kGroupObjects + lane] = xp[h];
                    s_bx[ww[h] * kGroupObjects + lane] = on[h] ? bx[h] : 0.f;
                }
        }
        }
        __syncthreads();
#ifdef FJOFC_STAMPS
        if (a.stamp && threadIdx.x == 0 && c0 == u0) *a.stamp = clock64();
#endif
        // 2. per unit: centre, commensurability, mix, column sums.  The group's column
        //    sums of X_t (used only for the next centring) are float32 butterflies; the
        //    commensurability (part of sigma) is float-float; all m+1 in one butterfly.
        // rolled loops (this code runs once per pass: a compact body is fetched faster than
        // one unrolled for every m); the centred x_{t-1} stay in s_xp, the tables come from
        // global memory
#pragma unroll 1
        for (int ui = warp; ui < nc; ui += nwarps) {
            const int u = c0 + ui, g = u / d, k = u - g * d;
            const int i = g * kGroupObjects + lane;
            const bool in = i < n;
            float* xcs = s_xp + ui * m * kGroupObjects + lane;      // x of modality j at xcs[j * 32]
#pragma unroll 1
            for (int j = 0; j < m; ++j) {
                const float x = in ? xcs[j * kGroupObjects] - (a.centre ? a.mu_prev[j * a.mu_stride + k] : 0.f) : 0.f;
                xcs[j * kGroupObjects] = x;
                if (in && a.centre && a.t > 1) a.Xprev[(int64_t(j) * n + i) * d + k] = x;
            }
            float c = 0.f;
#pragma unroll 1
            for (int j = 0; j < m; ++j) {
                const float xj = xcs[j * kGroupObjects];
#pragma unroll 1
                for (int l = j + 1; l < m; ++l) {
                    const float df = xj - xcs[l * kGroupObjects];
                    c = fmaf(__ldg(a.wcomm_g + j * m + l) * df, df, c);
                }
            }
            FF cw{c, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const FF w{__shfl_xor_sync(0xffffffffu, cw.hi, o), __shfl_xor_sync(0xffffffffu, cw.lo, o)};
                cw = ((lane & o) == 0) ? ff_add(cw, w) : ff_add(w, cw);
            }
            if (lane == 0) a.bpart[int64_t(md + k) * a.ngroups + g] = make_float2(cw.hi, cw.lo);
#pragma unroll 1
            for (int j = 0; j < m; ++j) {
                float v = 0.f;
                if (!a.final_pass && in) {
                    const float* bxs = s_bx + ui * m * kGroupObjects + lane;
#pragma unroll 1
                    for (int l = 0; l < m; ++l) v = fmaf(__ldg(a.coef_g + j * m + l), bxs[l * kGroupObjects], v);
                    if (a.relax != 1.f) v = fmaf(1.f - a.relax, xcs[j * kGroupObjects], a.relax * v);
                    a.Xnext[(int64_t(j) * n + i) * d + k] = v;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) a.bpart[int64_t(j * d + k) * a.ngroups + g] = make_float2(a.final_pass ? 0.f : v, 0.f);
            }
        }
        __syncthreads();
    }
}

// Float-float totals of two strided float2 sequences (p0[g*s0], g < c0 and p1[g*s1],
// g < c1; c1 == 0: none) by one warp: lane l sums entries l, l+32, ... with 8 loads of
// each in flight, then a fixed-order butterfly.  Every CTA that calls it gets the same
// totals.
__device__ __forceinline__ void totals2_ff(const float2* p0, int s0, int c0, const float2* p1, int s1, int c1,
                                           FF& t0, FF& t1) {
    const int lane = threadIdx.x & 31;
    const int cmax = max(c0, c1);
    FF a0{0.f, 0.f}, a1{0.f, 0.f};
#pragma unroll 1
    for (int g0 = lane; g0 < cmax; g0 += 8 * 32) {
        float2 x0[8], x1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int g = g0 + 32 * j;
            x0[j] = g < c0 ? __ldcg(p0 + int64_t(g) * s0) : make_float2(0.f, 0.f);
            x1[j] = g < c1 ? __ldcg(p1 + int64_t(g) * s1) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            a0 = ff_add(a0, FF{x0[j].x, x0[j].y});
            a1 = ff_add(a1, FF{x1[j].x, x1[j].y});
        }
    }
    t0 = warp_sum_ff(a0);
    t1 = warp_sum_ff(a1);
}

// The per-pass totals in a fixed order, the same in every CTA that calls it (every thread
// must call it): out[e] for e < npart = the float-float sum over the ngroups groups of
// phase B's part e (bpart is part-major), out[npart] = the sum of the nfid fidelity
// partials.  Two totals per
// warp at once.
__device__ __forceinline__ void pass_totals(const float2* bpart, int npart, int ngroups, const float2* fid, int nfid,
                                            FF* out) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nt = npart + 1;
#pragma unroll 1
    for (int e = warp; e < nt; e += 2 * nwarps) {
        const int e1 = e + nwarps;
        const float2* p0 = e < npart ? bpart + int64_t(e) * ngroups : fid;
        const int c0 = e < npart ? ngroups : nfid;
        const float2* p1 = e1 < npart ? bpart + int64_t(e1) * ngroups : fid;
        const int c1 = e1 < npart ? ngroups : (e1 == npart ? nfid : 0);
        FF t0, t1;
        totals2_ff(p0, 1, c0, p1, 1, c1, t0, t1);
        if ((threadIdx.x & 31) == 0) {
            out[e] = t0;
            if (e1 < nt) out[e1] = t1;
        }
    }
}

// sigma from the pass totals (pass_totals' out) and the fidelity total of the same
// iterate: the fidelity plus the commensurability of every coordinate, summed over k in
// order.
__device__ __forceinline__ double stress_from_totals(const FF* tot, FF fid, int m, int d) {
    FF comm{0.f, 0.f};
    for (int k = 0; k < d; ++k) comm = ff_add(comm, tot[m * d + k]);
    return (double(fid.hi) + double(fid.lo)) + (double(comm.hi) + double(comm.lo));
}

}  // namespace fjofc

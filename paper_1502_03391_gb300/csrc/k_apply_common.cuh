// Per-object work of a Guttman pass after the all-pairs tiles (Eq. update, Cor. 1,
// Remark faststress), shared by K2 (k_apply) and phase B of the persistent kernel so that
// both paths sum every partial in exactly the same order (bitwise equal results).
#pragma once

#include "fjofc_device.cuh"

namespace fjofc {


// (B'_l X_l)_{i,k}: the walk-head row partial of object i, the continuation row partials
// in CTA order, then the column partials of the walks of row blocks 0..I(i) in order.
// Loads are issued 32 at a time; data written earlier in the same launch is read through
// L2 (ld.global.cg).
__device__ __forceinline__ float bx_partials(const BxTables& tb, int l, int k, int i) {
    const int d = tb.d, RB = tb.RB, CW = tb.CW, rbs = tb.rb_shift, cws = tb.cw_shift, nRB = tb.nRB;
    const int I = i >> rbs, ri = i & (RB - 1);
    float acc = __ldcg(tb.rowhead + ((int64_t(l) * nRB + I) * d + k) * RB + ri);
    const int2 cr = __ldg(tb.cont + int64_t(l) * nRB + I);
    for (int b = cr.x; b < cr.y; ++b) acc += __ldcg(tb.rowcont + (int64_t(b) * d + k) * RB + ri);
    const float* cp = tb.colpart + int64_t(l) * tb.Tm * d * CW;
    float csum = 0.f;
    for (int J0 = 0; J0 <= I; J0 += 32) {
        float v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int J = J0 + u;
            v[u] = 0.f;
            if (J <= I) {
                const int rel = i - (J << rbs);
                v[u] = __ldcg(cp + ((__ldg(tb.cbase + J) + (rel >> cws)) * d + k) * CW + (rel & (CW - 1)));
            }
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) csum += v[u];
    }
    return acc + csum;
}

// Coordinate k of object i: centre X_{t-1} in place (X_0 is left as given), add its
// commensurability term to *comm, and (unless final) write X_t^(j) = sum_l coef[j][l] bx[l]
// for every modality j.  xn[j] receives X_t^(j) (0 for i >= n) for the column sums.
__device__ __forceinline__ void mix_and_centre(float* Xprev, float* Xnext, int m, int n, int d, int i, int k,
                                               int t, bool final_pass, const float* mu_prev,
                                               const float (*coef)[FJOFC_MAX_M],
                                               const float (*wcomm)[FJOFC_MAX_M], const float* bx_col,
                                               int bx_stride, float* cm, float* xn) {
    float xc[FJOFC_MAX_M];
    float c = 0.f;
    if (i < n) {
        for (int j = 0; j < m; ++j) {
            const int64_t off = (int64_t(j) * n + i) * d + k;
            xc[j] = __ldcg(Xprev + off) - mu_prev[j * FJOFC_MAX_D + k];
            if (t > 1) Xprev[off] = xc[j];
        }
        for (int j = 0; j < m; ++j)
            for (int l = j + 1; l < m; ++l) {
                const float df = xc[j] - xc[l];
                c = fmaf(wcomm[j][l] * df, df, c);
            }
    }
    *cm = c;
    for (int j = 0; j < m; ++j) {
        float v = 0.f;
        if (!final_pass && i < n) {
            for (int l = 0; l < m; ++l) v = fmaf(coef[j][l], bx_col[l * bx_stride], v);
            Xnext[(int64_t(j) * n + i) * d + k] = v;
        }
        xn[j] = v;
    }
}

}  // namespace fjofc

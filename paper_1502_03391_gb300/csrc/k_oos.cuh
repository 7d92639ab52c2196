// K3: out-of-sample Guttman iterations (Sec. 3, Eq. joosupdate) for k independent
// new objects against a fixed in-sample configuration X.
//
// One pass over the in-sample points of modality j gives, for a new object with
// current position y_j,
//     d_jk = ||X^(j)_k - y_j||,   b_k = delta_j(k) / d_jk   (0 when d_jk = 0, Eq. B),
//     psi_j = w_jj s_j sum_k b_k,
//     xi_j  = w_jj ( sum_k X^(j)_k - s_j sum_k b_k X^(j)_k )   (= w_jj sum_k (1 - delta/d) X_k),
//     fid_j = sum_k (s_j delta_j(k) - d_jk)^2,
// after which y_t = Wmod^-1 (xi + psi o y_{t-1}) (for Eq. W, L22^-1 = I/(n+mw) + wJ/(n(n+mw)),
// Sec. 3; with general weights L22 is the modified weight matrix of Eq. modW) and the
// stress is sum_j w_jj fid_j + sum_{i<j} w_ij ||y_i - y_j||^2 (Eq. joos).
//
// GB300 layout: a persistent grid; every warp keeps R slots, each holding one new object
// at its own pass.  A round is one pass of every occupied slot over all (modality,
// sub-tile); a slot whose object stops is refilled from an atomic object counter at
// the end of the round, so a warp never idles on objects that converged early.  Each
// warp owns a private STAGES-deep ring; a stage holds one TMA box {CW points, 1
// modality, 1 object} per occupied slot, all completing on the stage's mbarrier, so
// warps never wait for one another (prefetch stays within a round).  Lanes own C
// consecutive points of each box; X is read transposed ([m][d][n]) so the C points of
// a lane are one vector load per coordinate, fetched one sub-tile ahead.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"

namespace fjofc {

template <int D> struct K3Cfg;
#define FJOFC_K3CFG(D_, R_) template <> struct K3Cfg<D_> { static constexpr int R = R_; };
FJOFC_K3CFG(1, 8) FJOFC_K3CFG(2, 8) FJOFC_K3CFG(3, 8) FJOFC_K3CFG(4, 8)
#ifndef FJOFC_K3_R_D5_8
#define FJOFC_K3_R_D5_8 8
#endif
FJOFC_K3CFG(5, FJOFC_K3_R_D5_8) FJOFC_K3CFG(6, FJOFC_K3_R_D5_8) FJOFC_K3CFG(7, FJOFC_K3_R_D5_8)
FJOFC_K3CFG(8, FJOFC_K3_R_D5_8)
FJOFC_K3CFG(9, 2) FJOFC_K3CFG(10, 2) FJOFC_K3CFG(11, 2) FJOFC_K3CFG(12, 2)
FJOFC_K3CFG(13, 2) FJOFC_K3CFG(14, 2) FJOFC_K3CFG(15, 2) FJOFC_K3CFG(16, 2)
#undef FJOFC_K3CFG

template <int D, typename TD>
struct K3Shape {
    // C points per lane (4 up to d = 8, 2 beyond: registers); stages keep about 16 KB of
    // boxes in flight per warp (at least 4)
    static constexpr int R = K3Cfg<D>::R, C = (D <= 8) ? 4 : 2, WARPS = 8;
    static constexpr int NT = WARPS * 32;
    static constexpr int CW = 32 * C;
    static constexpr int STAGE_ELEMS = R * CW;
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(TD);
    static constexpr int STAGES = (16384 / int(STAGE_BYTES)) < 4 ? 4 : ((16384 / int(STAGE_BYTES)) > 8 ? 8 : (16384 / int(STAGE_BYTES)));
    // per warp: ring, y state, reduced sums (sum b x: D, sum b: 1), fid (double); the
    // per-slot arrays hold m modalities, so a warp's share depends on m
    static constexpr size_t RING_BYTES = size_t(STAGES) * STAGE_BYTES;
    // y_j of the slots as (y, y) pairs: YB float4 per slot
    static constexpr int YB = (D + 1) / 2;
    static constexpr size_t YB_FLOATS = size_t(R) * YB * 4;
    static __host__ __device__ size_t warp_bytes(int m) {
        const size_t y = size_t(R) * m * D, acc = size_t(R) * m * (D + 1);
        return ((RING_BYTES + YB_FLOATS * 4 + (2 * y + acc) * 4 + size_t(R) * m * 8 + 2 * R * 8 + R * 8 +
                 STAGES * 8 + R * 8 + R * 4) + 127) & ~size_t(127);
    }
    // shared memory of a CTA (at most 227 KB, less its static variables)
    static constexpr size_t BUDGET = 232448 - 1024;
    // warps per CTA for m modalities: all WARPS when they fit, else as many as fit
    static __host__ int warps_for(int m) {
        const size_t wb = warp_bytes(m);
        const size_t fit = (BUDGET - 128) / wb;
        return int(fit < size_t(WARPS) ? fit : size_t(WARPS));
    }
};

template <int D, typename TD>
__global__ void __launch_bounds__(K3Shape<D, TD>::NT, 1)
k_oos_solve(const __grid_constant__ CUtensorMap tmap, const K3Params p) {
    using S = K3Shape<D, TD>;
    constexpr int R = S::R, C = S::C, STAGES = S::STAGES, CW = S::CW, YB = S::YB;
    static_assert(C % 2 == 0, "points are processed in pairs");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = p.m, n = p.n;
    unsigned char* wb = smem + size_t(warp) * p.warp_bytes;
    TD* ring = reinterpret_cast<TD*>(wb);
    float* yb = reinterpret_cast<float*>(wb + S::RING_BYTES);          // [R][YB] float4 (y, y) pairs
    float* ys = yb + S::YB_FLOATS;                                       // [R][m][D]  y_{t-1}
    float* yn = ys + size_t(R) * m * D;                                  // [R][m][D]  y_t
    float* acc = yn + size_t(R) * m * D;                                 // [R][m][D+1]
    double* fidj = reinterpret_cast<double*>(acc + size_t(R) * m * (D + 1));   // [R][m]
    double* sprev = fidj + R * m;                                        // [R]
    double* scur = sprev + R;                                            // [R]
    int* flags = reinterpret_cast<int*>(scur + R);                       // [R] state, [R] iters
    uint64_t* full = reinterpret_cast<uint64_t*>(flags + 2 * R);         // [STAGES]
    long long* slot_obj = reinterpret_cast<long long*>(full + STAGES);  // [R] object (-1: empty)
    int* slot_pass = reinterpret_cast<int*>(slot_obj + R);               // [R] pass of the slot's object

    const int nsub = (n + CW - 1) / CW;
    const int passes = p.max_iter + 1;
    const int64_t per_pass = int64_t(m) * nsub;

    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&full[s]), 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmap);
    }
    __syncwarp();

    uint32_t q_cons = 0;   // sub-tiles consumed by this warp, drives stage/parity
    uint32_t q_iss = 0;    // sub-tiles issued
    const uint32_t box_bytes = uint32_t(CW * sizeof(TD));

    // Slots: every slot holds one object (or none) and its own pass count; a slot whose
    // object stops is refilled from the global object counter at the end of the round.
    auto fetch = [&](int r) {              // one lane: next object into slot r
        const unsigned long long o = atomicAdd(p.next_block, 1ull);
        slot_obj[r] = (int64_t(o) < p.k) ? (long long)o : -1ll;
    };
    auto init_slot = [&](int r) {          // all lanes: state of slot r's new object
        const long long o = slot_obj[r];
        for (int e = lane; e < m * D; e += 32) {
            const int j = e / D, kk = e - j * D;
            ys[(r * m + j) * D + kk] = (o >= 0) ? p.Y[(int64_t(o) * m + j) * D + kk] : 0.f;
        }
        if (lane == 0) {
            flags[r] = (o >= 0) ? 0 : 1;   // 0 iterating, 1 empty
            flags[R + r] = 0;
            sprev[r] = 0.0;
            slot_pass[r] = 1;
        }
    };
    if (lane == 0)
        for (int r = 0; r < R; ++r) fetch(r);
    __syncwarp();
    for (int r = 0; r < R; ++r) init_slot(r);
    __syncwarp();

    bool failed = false;
    // sub-tile qq of a round: modality qq / nsub, points (qq % nsub) * CW; one box per
    // occupied slot, all completing on the stage's mbarrier.  Every lane of the warp calls
    // it: lane r issues slot r's box, lane 0 first announces the bytes of all of them.
    auto issue_sub = [&](int64_t qq) {
        const int j = int(qq / nsub), s = int(qq % nsub);
        const int stage = int(q_iss % STAGES);
        const uint32_t bar = smem_u32(&full[stage]);
        const bool act = lane < R && slot_obj[lane] >= 0;
        const unsigned occ = __ballot_sync(0xffffffffu, act);
        if (lane == 0) mbar_arrive_expect_tx(bar, uint32_t(__popc(occ)) * box_bytes);
        __syncwarp();
        if (act)
            tma_load_3d(smem_u32(ring + size_t(stage) * S::STAGE_ELEMS + size_t(lane) * CW), &tmap, s * CW, j,
                        int(slot_obj[lane]), bar);
    };

    for (;;) {
        // the round: one pass of every occupied slot over all (modality, sub-tile)
        int any = 0;
        if (lane < R) any = slot_obj[lane] >= 0;
        if (!__any_sync(0xffffffffu, any)) break;
        // an error raised elsewhere ends the loop after this round: the flag is read now and
        // tested at the round's end, so that its load latency overlaps the round
        const int err_seen = ld_volatile(&p.st->error);
        int64_t issued_in_round = 0;
        for (int e = 0; e < STAGES && issued_in_round < per_pass; ++e) {
            issue_sub(issued_in_round);
            ++issued_in_round;
            ++q_iss;
        }
        {
            for (int j = 0; j < m; ++j) {
                // the slots' y_j as (y, y) pairs (one packed operand for two points), read
                // by every lane from the same address
                for (int e = lane; e < R * D; e += 32) {
                    const int r = e / D, kk = e - r * D;
                    const float y = ys[(r * m + j) * D + kk];
                    *reinterpret_cast<float2*>(yb + (r * YB + kk / 2) * 4 + 2 * (kk & 1)) = make_float2(y, y);
                }
                __syncwarp();
                const float2 nsc = make_float2(-p.dscale[j], -p.dscale[j]);
                float2 bx[R][D], bs[R], f2[R];   // per point-parity halves; bx holds -sum b x
                FF fff[R];                        // float-float fidelity (GB300's float64 rate is low)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    bs[r] = make_float2(0.f, 0.f); f2[r] = make_float2(0.f, 0.f); fff[r] = FF{0.f, 0.f};
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) bx[r][kk] = make_float2(0.f, 0.f);
                }
                const float* XTj = p.XT + int64_t(j) * D * p.nx;
                // -x of the C points of this lane in sub-tile s as point pairs (X^T holds -x;
                // its rows are padded to a multiple of 4 points, so whole vectors stay inside
                // the row; points >= n are masked below)
                auto load_xp = [&](int s, float2 (&xv)[C / 2][D]) {
                    const int pt = s * CW + lane * C;
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        const float* src = XTj + int64_t(kk) * p.nx + pt;
                        if (pt + C <= p.nx) {
                            if constexpr (C == 4) {
                                const float4 v = __ldg(reinterpret_cast<const float4*>(src));
                                xv[0][kk] = make_float2(v.x, v.y);
                                xv[1][kk] = make_float2(v.z, v.w);
                            } else {
                                xv[0][kk] = __ldg(reinterpret_cast<const float2*>(src));
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < C / 2; ++c) xv[c][kk] = make_float2(0.f, 0.f);
                        }
                    }
                };
                float2 xpn[C / 2][D];
                load_xp(0, xpn);
                const uint32_t ybs = smem_u32(yb);
                for (int s = 0; s < nsub; ++s) {
                    const int pt0 = s * CW + lane * C;
                    float2 xp[C / 2][D];
#pragma unroll
                    for (int c = 0; c < C / 2; ++c)
#pragma unroll
                        for (int kk = 0; kk < D; ++kk) xp[c][kk] = xpn[c][kk];
                    if (s + 1 < nsub) load_xp(s + 1, xpn);
                    const int stage = int(q_cons % STAGES);
                    const uint32_t par = (q_cons / STAGES) & 1u;
                    failed |= !mbar_wait_bounded(smem_u32(&full[stage]), par);
                    const uint32_t tile = smem_u32(ring + size_t(stage) * S::STAGE_ELEMS);
                    const bool ragged = (s * CW + CW > n);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float2 y2[2 * YB];
#pragma unroll
                        for (int h = 0; h < YB; ++h) {
                            const float4 v = lds_f4(ybs + 16 * (r * YB + h));
                            y2[2 * h] = make_float2(v.x, v.y);
                            y2[2 * h + 1] = make_float2(v.z, v.w);
                        }
                        float dl[C];
                        lds_delta_row<TD, C>(tile + uint32_t((r * CW + lane * C) * sizeof(TD)), dl);
#pragma unroll
                        for (int cp = 0; cp < C / 2; ++cp) {
                            const float2 del = make_float2(dl[2 * cp], dl[2 * cp + 1]);
                            float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
                            for (int kk = 0; kk < D; ++kk) {
                                const float2 df = __fadd2_rn(y2[kk], xp[cp][kk]);
                                d2 = __ffma2_rn(df, df, d2);
                            }
                            const float2 rinv = make_float2((d2.x > 0.f) ? rsqrt_approx(d2.x) : 0.f,
                                                            (d2.y > 0.f) ? rsqrt_approx(d2.y) : 0.f);
                            float2 bb = __fmul2_rn(del, rinv);
                            float2 e = __ffma2_rn(nsc, del, __fmul2_rn(d2, rinv));    // d - s delta
                            if (ragged) {
                                if (pt0 + 2 * cp >= n) { bb.x = 0.f; e.x = 0.f; }
                                if (pt0 + 2 * cp + 1 >= n) { bb.y = 0.f; e.y = 0.f; }
                            }
                            bs[r] = __fadd2_rn(bs[r], bb);
                            f2[r] = __ffma2_rn(e, e, f2[r]);
#pragma unroll
                            for (int kk = 0; kk < D; ++kk) bx[r][kk] = __ffma2_rn(bb, xp[cp][kk], bx[r][kk]);
                        }
                    }
                    if ((s & 3) == 3) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            fff[r] = ff_add(fff[r], f2[r].x + f2[r].y);
                            f2[r] = make_float2(0.f, 0.f);
                        }
                    }
                    __syncwarp();
                    ++q_cons;
                    if (issued_in_round < per_pass) {
                        issue_sub(issued_in_round);
                        ++issued_in_round;
                        ++q_iss;
                    }
                }
                // reduce this modality's sums over the warp
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const FF fr = warp_sum_ff(ff_add(fff[r], f2[r].x + f2[r].y));
                    const float br = warp_sum_f32(bs[r].x + bs[r].y);
                    if (lane == 0) {
                        fidj[r * m + j] = double(fr.hi) + double(fr.lo);
                        acc[(r * m + j) * (D + 1) + D] = br;
                    }
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        const float v = warp_sum_f32(bx[r][kk].x + bx[r][kk].y);
                        if (lane == ((r * D + kk) & 31)) acc[(r * m + j) * (D + 1) + kk] = v;
                    }
                }
                __syncwarp();
            }
            failed = __any_sync(0xffffffffu, failed);
            if (failed) break;
            __syncwarp();

            // stress of every occupied slot's y_{t-1} and its stopping test, one lane per slot
            if (lane < R && flags[lane] == 0) {
                const int r = lane;
                const int pass = slot_pass[r];
                double sig = 0.0;
                for (int j = 0; j < m; ++j) sig += double(p.wfid[j]) * fidj[r * m + j];
                for (int a = 0; a < m; ++a)
                    for (int b2 = a + 1; b2 < m; ++b2) {
                        double s2 = 0.0;
                        for (int kk = 0; kk < D; ++kk) {
                            const double df = double(ys[(r * m + a) * D + kk]) -
                                              double(ys[(r * m + b2) * D + kk]);
                            s2 += df * df;
                        }
                        sig += __ldg(p.wcomm + a * m + b2) * s2;
                    }
                bool stop = (pass == passes) || !isfinite(sig);
                if (!stop && pass >= 2 && p.tol >= 0.0) {
                    const double dec = sprev[r] - sig;
                    const bool cont = (p.tol_mode == FJOFC_TOL_RELATIVE) ? (dec > p.tol * sprev[r])
                                                                         : (dec / p.npairs > p.tol);
                    stop = !cont;
                }
                scur[r] = sig;
                sprev[r] = sig;
                flags[R + r] = pass - 1;            // iterate index of the current y
                if (stop) flags[r] = 2;             // 2 = stopped at this pass
            }
            __syncwarp();
            // y_t = Wmod^-1 (xi + psi o y_{t-1}) for objects still iterating
            for (int e = lane; e < R * m * D; e += 32) {
                const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
                if (flags[r] != 0) continue;
                float v = 0.f;
                for (int i2 = 0; i2 < m; ++i2) {
                    const float* a = acc + (r * m + i2) * (D + 1);
                    const float wi = p.wfid[i2], si = p.dscale[i2];
                    const float xi = wi * fmaf(si, a[kk], p.SX[i2 * D + kk]);   // a[kk] = -sum_k b_k x_k
                    const float psi = wi * si * a[D];
                    v = fmaf(__ldg(p.winv + j * m + i2), fmaf(psi, ys[(r * m + i2) * D + kk], xi), v);
                }
                yn[(r * m + j) * D + kk] = v;
            }
            __syncwarp();
            for (int e = lane; e < R * m * D; e += 32) {
                const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
                if (flags[r] == 0) ys[(r * m + j) * D + kk] = yn[(r * m + j) * D + kk];
            }
            __syncwarp();
            // outputs of the objects that stopped at this pass
            for (int e = lane; e < R * m * D; e += 32) {
                const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
                if (flags[r] == 2) p.Y[(slot_obj[r] * m + j) * D + kk] = ys[(r * m + j) * D + kk];
            }
            __syncwarp();
            if (lane < R) {
                if (flags[lane] == 2) {
                    const int64_t o = slot_obj[lane];
                    if (p.iters_out) p.iters_out[o] = flags[R + lane];
                    p.stress_out[o] = scur[lane];
                    if (!isfinite(scur[lane])) atomicCAS(&p.st->error, 0, FJOFC_ERR_NONFINITE);
                } else if (flags[lane] == 0) {
                    slot_pass[lane] += 1;
                }
            }
            __syncwarp();
            // refill the slots whose object stopped: their claims on the object counter go
            // out together (lane r for slot r), then each new object's state
            if (lane < R && flags[lane] == 2) fetch(lane);
            __syncwarp();
            for (int r = 0; r < R; ++r) {
                if (flags[r] != 2) continue;       // uniform across the warp (shared memory)
                init_slot(r);
                __syncwarp();                      // (init_slot rewrites flags[r])
            }
        }
        if (__any_sync(0xffffffffu, err_seen != 0)) break;
    }

    // drain the sub-tiles issued but not consumed (only after a failure)
    while (q_cons < q_iss) {
        const int stage = int(q_cons % STAGES);
        failed |= !mbar_wait_bounded(smem_u32(&full[stage]), (q_cons / STAGES) & 1u);
        __syncwarp();
        ++q_cons;
    }
    if (__any_sync(0xffffffffu, failed) && lane == 0) raise_error(p.st, FJOFC_ERR_TIMEOUT, 3);
}

template <int D, typename TD>
cudaError_t k3_launch_impl(int grid, const CUtensorMap& tmap, const K3Params& p, cudaStream_t s) {
    using S = K3Shape<D, TD>;
    const int warps = S::warps_for(p.m);
    if (warps < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = size_t(warps) * p.warp_bytes + 128;
    cudaError_t e = cudaFuncSetAttribute(k_oos_solve<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_oos_solve<D, TD><<<grid, warps * 32, smem, s>>>(tmap, p);
    return cudaGetLastError();
}

// CTAs per SM for m modalities (0: not launchable)
template <int D, typename TD>
int k3_bps_impl(int m) {
    using S = K3Shape<D, TD>;
    const int warps = S::warps_for(m);
    if (warps < 1) return 0;
    const size_t smem = size_t(warps) * S::warp_bytes(m) + 128;
    cudaFuncSetAttribute(k_oos_solve<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_oos_solve<D, TD>, warps * 32, smem) != cudaSuccess) return 0;
    return nb;
}

// Geometry for m modalities: WARPS = warps per CTA, smem_bytes = one warp's share.
template <int D, typename TD>
K3Geom k3_geom_impl(int m) {
    using S = K3Shape<D, TD>;
    const int warps = S::warps_for(m);
    return K3Geom{S::R, S::C, warps, S::STAGES, S::R, S::CW, warps * 32, S::warp_bytes(m)};
}

#define FJOFC_INSTANTIATE_K3(D)                                                                        \
    template cudaError_t k3_launch_impl<D, float>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template cudaError_t k3_launch_impl<D, __half>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template cudaError_t k3_launch_impl<D, __nv_bfloat16>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template int k3_bps_impl<D, float>(int);                                                           \
    template int k3_bps_impl<D, __half>(int);                                                          \
    template int k3_bps_impl<D, __nv_bfloat16>(int);                                                   \
    template K3Geom k3_geom_impl<D, float>(int);                                                       \
    template K3Geom k3_geom_impl<D, __half>(int);                                                      \
    template K3Geom k3_geom_impl<D, __nv_bfloat16>(int);

}  // namespace fjofc

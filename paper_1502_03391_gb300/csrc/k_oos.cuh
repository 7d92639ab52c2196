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
// GB300 layout: a persistent grid; every warp takes groups of R new objects from an
// atomic counter and iterates them until all R have stopped.  Each warp owns a
// private STAGES-deep ring of TMA boxes {CW points, 1 modality, R objects} with its
// own mbarriers, so warps never wait for one another.  Lanes own C consecutive
// points of each box; X is read transposed ([m][d][n]) so the C points of a lane are
// one vector load per coordinate.
#pragma once

#include <float.h>

#include "fjofc_device.cuh"

namespace fjofc {

template <int D> struct K3Cfg;
#define FJOFC_K3CFG(D_, R_) template <> struct K3Cfg<D_> { static constexpr int R = R_; };
FJOFC_K3CFG(1, 8) FJOFC_K3CFG(2, 8) FJOFC_K3CFG(3, 8) FJOFC_K3CFG(4, 8)
FJOFC_K3CFG(5, 4) FJOFC_K3CFG(6, 4) FJOFC_K3CFG(7, 4) FJOFC_K3CFG(8, 4)
FJOFC_K3CFG(9, 2) FJOFC_K3CFG(10, 2) FJOFC_K3CFG(11, 2) FJOFC_K3CFG(12, 2)
FJOFC_K3CFG(13, 2) FJOFC_K3CFG(14, 2) FJOFC_K3CFG(15, 2) FJOFC_K3CFG(16, 2)
#undef FJOFC_K3CFG

template <int D, typename TD>
struct K3Shape {
    static constexpr int R = K3Cfg<D>::R, C = 2, WARPS = 8, STAGES = 4;
    static constexpr int NT = WARPS * 32;
    static constexpr int CW = 32 * C;
    static constexpr int STAGE_ELEMS = R * CW;
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(TD);
    // per warp: ring, y state, reduced sums (sum b x: D, sum b: 1), fid (double)
    static constexpr size_t RING_BYTES = size_t(STAGES) * STAGE_BYTES;
    static constexpr size_t Y_FLOATS = size_t(R) * FJOFC_MAX_M * D;
    static constexpr size_t ACC_FLOATS = size_t(R) * FJOFC_MAX_M * (D + 1);
    static constexpr size_t WARP_BYTES =
        ((RING_BYTES + (2 * Y_FLOATS + ACC_FLOATS) * 4 + size_t(R) * FJOFC_MAX_M * 8 + 2 * R * 8 + R * 8 +
          STAGES * 8) + 127) & ~size_t(127);
    static constexpr size_t SMEM = WARPS * WARP_BYTES + 128;
};

template <int D, typename TD>
__global__ void __launch_bounds__(K3Shape<D, TD>::NT, 1)
k_oos_solve(const __grid_constant__ CUtensorMap tmap, const K3Params p) {
    using S = K3Shape<D, TD>;
    constexpr int R = S::R, C = S::C, STAGES = S::STAGES, CW = S::CW;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wb = smem + size_t(warp) * S::WARP_BYTES;
    TD* ring = reinterpret_cast<TD*>(wb);
    float* ys = reinterpret_cast<float*>(wb + S::RING_BYTES);          // [R][MAXM][D]  y_{t-1}
    float* yn = ys + S::Y_FLOATS;                                        // [R][MAXM][D]  y_t
    float* acc = yn + S::Y_FLOATS;                                       // [R][MAXM][D+1]
    double* fidj = reinterpret_cast<double*>(acc + S::ACC_FLOATS);       // [R][MAXM]
    double* sprev = fidj + R * FJOFC_MAX_M;                              // [R]
    double* scur = sprev + R;                                            // [R]
    int* flags = reinterpret_cast<int*>(scur + R);                       // [R] done, [R] iters
    uint64_t* full = reinterpret_cast<uint64_t*>(flags + 2 * R);         // [STAGES]

    const int m = p.m, n = p.n;
    const int nsub = (n + CW - 1) / CW;
    const int passes = p.max_iter + 1;
    const int64_t per_pass = int64_t(m) * nsub;
    const int64_t ngroups = (p.k + R - 1) / R;

    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&full[s]), 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmap);
    }
    __syncwarp();

    uint32_t q_cons = 0;   // sub-tiles consumed by this warp (all groups), drives stage/parity
    uint32_t q_iss = 0;    // sub-tiles issued

    for (;;) {
        int64_t g = 0;
        if (lane == 0) g = static_cast<int64_t>(atomicAdd(p.next_block, 1ull));
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        if (ld_volatile(&p.st->error)) break;
        const int64_t o0 = g * R;

        // initial state of the R objects
        for (int e = lane; e < R * m * D; e += 32) {
            const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
            const int64_t o = o0 + r;
            ys[(r * FJOFC_MAX_M + j) * D + kk] = (o < p.k) ? p.Y[(o * m + j) * D + kk] : 0.f;
        }
        if (lane < R) {
            flags[lane] = (o0 + lane < p.k) ? 0 : 1;   // objects past k start "done"
            flags[R + lane] = 0;
            sprev[lane] = 0.0;
        }
        __syncwarp();

        // producer: sub-tile sequence (pass, j, s) of this group, in order
        int64_t issued_in_group = 0;
        const int64_t group_total = int64_t(passes) * per_pass;
        auto issue_next = [&]() {
            const int64_t qq = issued_in_group;
            const int j = int((qq % per_pass) / nsub);
            const int s = int(qq % nsub);
            const int stage = int(q_iss % STAGES);
            const uint32_t bar = smem_u32(&full[stage]);
            mbar_arrive_expect_tx(bar, S::STAGE_BYTES);
            tma_load_3d(smem_u32(ring + size_t(stage) * S::STAGE_ELEMS), &tmap, s * CW, j, int(o0), bar);
        };
        if (lane == 0) {
            for (int e = 0; e < STAGES && issued_in_group < group_total; ++e) {
                issue_next();
                ++issued_in_group;
                ++q_iss;
            }
        }
        issued_in_group = __shfl_sync(0xffffffffu, issued_in_group, 0);
        q_iss = __shfl_sync(0xffffffffu, q_iss, 0);

        bool failed = false;
        int pass = 1;
        for (; pass <= passes; ++pass) {
            for (int j = 0; j < m; ++j) {
                const float sc = p.dscale[j];
                float yr[R][D];
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) yr[r][kk] = ys[(r * FJOFC_MAX_M + j) * D + kk];
                float bx[R][D], bs[R], f32[R];
                FF fff[R];                  // float-float fidelity (GB300's float64 rate is low)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    bs[r] = 0.f; f32[r] = 0.f; fff[r] = FF{0.f, 0.f};
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) bx[r][kk] = 0.f;
                }
                const float* XTj = p.XT + int64_t(j) * D * p.nx;
                for (int s = 0; s < nsub; ++s) {
                    const int pt0 = s * CW + lane * C;
                    float xp[C][D];
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        if (pt0 + 1 < n) {
                            const float2 v = *reinterpret_cast<const float2*>(XTj + int64_t(kk) * p.nx + pt0);
                            xp[0][kk] = v.x; xp[1][kk] = v.y;
                        } else {
                            xp[0][kk] = (pt0 < n) ? XTj[int64_t(kk) * p.nx + pt0] : 0.f;
                            xp[1][kk] = 0.f;
                        }
                    }
                    const int stage = int(q_cons % STAGES);
                    const uint32_t par = (q_cons / STAGES) & 1u;
                    failed |= !mbar_wait_bounded(smem_u32(&full[stage]), par);
                    const TD* tile = ring + size_t(stage) * S::STAGE_ELEMS;
                    const bool ragged = (s * CW + CW > n);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float dl[C];
                        load_delta_row<TD, C>(tile + r * CW + lane * C, dl);
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            float d2 = 0.f;
#pragma unroll
                            for (int kk = 0; kk < D; ++kk) {
                                const float df = yr[r][kk] - xp[c][kk];
                                d2 = fmaf(df, df, d2);
                            }
                            const float rinv = (d2 > 0.f) ? rsqrt_approx(d2) : 0.f;
                            float bb = dl[c] * rinv;
                            float e = fmaf(sc, dl[c], -(d2 * rinv));
                            if (ragged && pt0 + c >= n) { bb = 0.f; e = 0.f; }
                            bs[r] += bb;
                            f32[r] = fmaf(e, e, f32[r]);
#pragma unroll
                            for (int kk = 0; kk < D; ++kk) bx[r][kk] = fmaf(bb, xp[c][kk], bx[r][kk]);
                        }
                    }
                    if ((s & 3) == 3) {
#pragma unroll
                        for (int r = 0; r < R; ++r) { fff[r] = ff_add(fff[r], f32[r]); f32[r] = 0.f; }
                    }
                    __syncwarp();
                    ++q_cons;
                    if (lane == 0 && issued_in_group < group_total) {
                        issue_next();
                        ++issued_in_group;
                        ++q_iss;
                    }
                    issued_in_group = __shfl_sync(0xffffffffu, issued_in_group, 0);
                    q_iss = __shfl_sync(0xffffffffu, q_iss, 0);
                }
                // reduce this modality's sums over the warp
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const FF fr = warp_sum_ff(ff_add(fff[r], f32[r]));
                    const float br = warp_sum_f32(bs[r]);
                    if (lane == 0) {
                        fidj[r * FJOFC_MAX_M + j] = double(fr.hi) + double(fr.lo);
                        acc[(r * FJOFC_MAX_M + j) * (D + 1) + D] = br;
                    }
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        const float v = warp_sum_f32(bx[r][kk]);
                        if (lane == ((r * D + kk) & 31)) acc[(r * FJOFC_MAX_M + j) * (D + 1) + kk] = v;
                    }
                }
            }
            failed = __any_sync(0xffffffffu, failed);
            if (failed) break;
            __syncwarp();

            // stress of y_{t-1} and the stopping test, one lane per object
            if (lane < R && !flags[lane]) {
                const int r = lane;
                double sig = 0.0;
                for (int j = 0; j < m; ++j) sig += double(p.wfid[j]) * fidj[r * FJOFC_MAX_M + j];
                for (int a = 0; a < m; ++a)
                    for (int b2 = a + 1; b2 < m; ++b2) {
                        double s2 = 0.0;
                        for (int kk = 0; kk < D; ++kk) {
                            const double df = double(ys[(r * FJOFC_MAX_M + a) * D + kk]) -
                                              double(ys[(r * FJOFC_MAX_M + b2) * D + kk]);
                            s2 += df * df;
                        }
                        sig += p.wcomm[a][b2] * s2;
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
                    const float* a = acc + (r * FJOFC_MAX_M + i2) * (D + 1);
                    const float wi = p.wfid[i2], si = p.dscale[i2];
                    const float xi = wi * (p.SX[i2 * D + kk] - si * a[kk]);
                    const float psi = wi * si * a[D];
                    v = fmaf(p.winv[j][i2], fmaf(psi, ys[(r * FJOFC_MAX_M + i2) * D + kk], xi), v);
                }
                yn[(r * FJOFC_MAX_M + j) * D + kk] = v;
            }
            __syncwarp();
            for (int e = lane; e < R * m * D; e += 32) {
                const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
                if (flags[r] == 0) ys[(r * FJOFC_MAX_M + j) * D + kk] = yn[(r * FJOFC_MAX_M + j) * D + kk];
            }
            __syncwarp();
            // outputs of the objects that stopped at this pass
            for (int e = lane; e < R * m * D; e += 32) {
                const int r = e / (m * D), rem = e - r * m * D, j = rem / D, kk = rem - j * D;
                if (flags[r] == 2) p.Y[((o0 + r) * m + j) * D + kk] = ys[(r * FJOFC_MAX_M + j) * D + kk];
            }
            __syncwarp();
            int alldone = 1;
            if (lane < R) {
                if (flags[lane] == 2) {
                    const int64_t o = o0 + lane;
                    if (p.iters_out) p.iters_out[o] = flags[R + lane];
                    p.stress_out[o] = scur[lane];
                    if (!isfinite(scur[lane])) atomicCAS(&p.st->error, 0, FJOFC_ERR_NONFINITE);
                    flags[lane] = 1;
                }
                alldone = flags[lane] != 0;
            }
            __syncwarp();
            if (__all_sync(0xffffffffu, alldone)) break;
        }

        // drain the sub-tiles issued ahead for passes that will not run
        while (__shfl_sync(0xffffffffu, q_cons, 0) < q_iss) {
            const int stage = int(q_cons % STAGES);
            failed |= !mbar_wait_bounded(smem_u32(&full[stage]), (q_cons / STAGES) & 1u);
            __syncwarp();
            ++q_cons;
        }
        if (__any_sync(0xffffffffu, failed)) {
            if (lane == 0) raise_error(p.st, FJOFC_ERR_TIMEOUT, 3);
            return;
        }
    }
}

template <int D, typename TD>
cudaError_t k3_launch_impl(int grid, const CUtensorMap& tmap, const K3Params& p, cudaStream_t s) {
    using S = K3Shape<D, TD>;
    cudaError_t e = cudaFuncSetAttribute(k_oos_solve<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
    if (e != cudaSuccess) return e;
    k_oos_solve<D, TD><<<grid, S::NT, S::SMEM, s>>>(tmap, p);
    return cudaGetLastError();
}

template <int D, typename TD>
int k3_bps_impl() {
    using S = K3Shape<D, TD>;
    cudaFuncSetAttribute(k_oos_solve<D, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_oos_solve<D, TD>, S::NT, S::SMEM) != cudaSuccess) return 0;
    return nb;
}

template <int D, typename TD>
K3Geom k3_geom_impl() {
    using S = K3Shape<D, TD>;
    return K3Geom{S::R, S::C, S::WARPS, S::STAGES, S::R, S::CW, S::NT, S::SMEM};
}

#define FJOFC_INSTANTIATE_K3(D)                                                                        \
    template cudaError_t k3_launch_impl<D, float>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template cudaError_t k3_launch_impl<D, __half>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template cudaError_t k3_launch_impl<D, __nv_bfloat16>(int, const CUtensorMap&, const K3Params&, cudaStream_t); \
    template int k3_bps_impl<D, float>();                                                              \
    template int k3_bps_impl<D, __half>();                                                             \
    template int k3_bps_impl<D, __nv_bfloat16>();                                                      \
    template K3Geom k3_geom_impl<D, float>();                                                          \
    template K3Geom k3_geom_impl<D, __half>();                                                         \
    template K3Geom k3_geom_impl<D, __nv_bfloat16>();

}  // namespace fjofc

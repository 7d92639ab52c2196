// Algorithm 2's initialisation: the initial configuration X_(0) of fJOFC.
//
//   xi_0 = cMDS of the average dissimilarity (sum_i Delta_i) / m, centred;
//   for every modality i: xi_i = cMDS of Delta_i, centred, and X^(i)_(0) its orthogonal
//   Procrustes fit onto xi_0 (the rotation R minimising ||xi_i R - xi_0||: with
//   xi_0' xi_i = U S V', R = V U'; the printed xi_i U V' is the inverse rotation).
//
// Classical MDS (Torgerson; the initialisation of Algorithm 1) takes the d leading
// eigenpairs of S = -1/2 J D2 J (D2 the elementwise squared dissimilarities, J = I - 11'/n) and
// returns v_k sqrt(max(lambda_k, 0)), each column's largest-magnitude entry made
// positive.  The eigenpairs come from subspace iteration with p = 2d + 4 vectors:
// Y = S V by one pass over Delta (the average and its square formed on the fly, no n x n
// intermediate), a Rayleigh-Ritz step on V'Y, V <- Y R^-1 with Y'Y = R'R (Cholesky), until
// the d leading Ritz values change by less than the tolerance.  The p x p and d x d
// algebra (Jacobi eigenvalues, Cholesky, the Procrustes SVD) runs on the host in float64;
// every n-length reduction runs on the device as per-block partials the host sums in a
// fixed order, so results are reproducible run to run.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fjofc_device.cuh"
#include "fjofc_internal.h"

namespace fjofc {
namespace {

constexpr int kSqWarps = 8;          // warps per CTA of the product kernel
constexpr int kSqRows = 4;           // rows per warp
constexpr int kSqChunk = 128;        // columns j staged per round (4 per lane)
constexpr int kRedRows = 128;        // rows per block of the small reductions
constexpr int kPMax = 32;            // widest subspace

struct SqParams {
    const void* delta[FJOFC_MAX_M];
    float w[FJOFC_MAX_M];            // scale_l / count: the average of the scaled Delta_l
    int count;                       // modalities averaged
    int64_t ld;
    int n;
    const float* V;                  // [n][P]
    float* A;                        // [n][P]  sum_j D2_ij V_jc
    float* S;                        // [n]     sum_j D2_ij
};

// Four consecutive elements j..j+3 of a Delta row as float (zero at and beyond n).
template <typename TD>
__device__ __forceinline__ void load4(const TD* row, int j, int n, float (&v)[4]) {
    if (j + 3 < n) {
        if constexpr (sizeof(TD) == 4) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(row + j));
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else {
            const uint2 x = __ldg(reinterpret_cast<const uint2*>(row + j));
            const TD* h = reinterpret_cast<const TD*>(&x);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = DeltaLoad<TD>::to_f32(h[q]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (j + q < n) ? DeltaLoad<TD>::to_f32(row[j + q]) : 0.f;
    }
}

// A = D2 V and S = D2 1 for D = sum_l w_l Delta_l: CTA = 8 warps x 4 rows; the columns in
// chunks of 128 (V chunk staged in shared memory, lane = 4 consecutive columns, 16-byte
// Delta loads); per-row sums over the lanes by a fixed butterfly.
template <int P, typename TD>
__global__ void __launch_bounds__(kSqWarps * 32) k_sq_product(const SqParams p) {
    __shared__ __align__(16) float sV[kSqChunk][P];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n;
    const int i0 = (blockIdx.x * kSqWarps + warp) * kSqRows;
    float a[kSqRows][P], s[kSqRows];
#pragma unroll
    for (int r = 0; r < kSqRows; ++r) {
        s[r] = 0.f;
#pragma unroll
        for (int c = 0; c < P; ++c) a[r][c] = 0.f;
    }
    for (int j0 = 0; j0 < n; j0 += kSqChunk) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSqChunk * P; e += kSqWarps * 32) {
            const int jj = e / P, c = e - jj * P;
            sV[jj][c] = (j0 + jj < n) ? __ldg(p.V + int64_t(j0 + jj) * P + c) : 0.f;
        }
        __syncthreads();
        const int j = j0 + lane * 4;
        float D2[kSqRows][4];
#pragma unroll
        for (int r = 0; r < kSqRows; ++r) {
            const int i = i0 + r;
            float D[4] = {0.f, 0.f, 0.f, 0.f};
            if (i < n && j < n) {
                for (int l = 0; l < p.count; ++l) {
                    float v[4];
                    load4<TD>(static_cast<const TD*>(p.delta[l]) + int64_t(i) * p.ld, j, n, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) D[q] = fmaf(p.w[l], v[q], D[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                D2[r][q] = D[q] * D[q];
                s[r] += D2[r][q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float vj[P];
#pragma unroll
            for (int c = 0; c < P; c += 4) {
                const float4 x = *reinterpret_cast<const float4*>(&sV[lane * 4 + q][c]);
                vj[c] = x.x; vj[c + 1] = x.y; vj[c + 2] = x.z; vj[c + 3] = x.w;
            }
#pragma unroll
            for (int r = 0; r < kSqRows; ++r)
#pragma unroll
                for (int c = 0; c < P; ++c) a[r][c] = fmaf(D2[r][q], vj[c], a[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < kSqRows; ++r) {
        const int i = i0 + r;
        const float sr = warp_sum_f32(s[r]);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float v = warp_sum_f32(a[r][c]);
            if (lane == 0 && i < n) p.A[int64_t(i) * P + c] = v;
        }
        if (lane == 0 && i < n) p.S[i] = sr;
    }
}

// Column sums of X (n x P) by one CTA of 1024 threads in a fixed order (float64):
// thread t sums column t % P over rows t / P, t / P + 1024 / P, ...; then per column over
// the threads in index order.
template <int P>
__device__ __forceinline__ void colsums_f64(const float* X, int n, double* s_part, double* out) {
    const int t = threadIdx.x, c = t % P, r0 = t / P, step = blockDim.x / P;
    double acc = 0.0;
    for (int i = r0; i < n; i += step) acc += double(X[int64_t(i) * P + c]);
    s_part[t] = acc;
    __syncthreads();
    if (t < P) {
        double tot = 0.0;
        for (int k = 0; k < step; ++k) tot += s_part[k * P + t];
        out[t] = tot;
    }
    __syncthreads();
}

// Y = -1/2 J (A - S vbar'), vbar = column means of V: -1/2 J D2 J V for the A and S of
// k_sq_product.  One CTA (the column means are two fixed-order reductions).
template <int P>
__global__ void __launch_bounds__(1024) k_sq_finish(const float* V, const float* A, const float* S, float* Y, int n) {
    __shared__ double s_part[1024];
    __shared__ double s_vbar[P], s_zbar[P];
    colsums_f64<P>(V, n, s_part, s_vbar);
    if (threadIdx.x < P) s_vbar[threadIdx.x] /= double(n);
    __syncthreads();
    for (int e = threadIdx.x; e < n * P; e += blockDim.x) {
        const int i = e / P, c = e - i * P;
        Y[e] = A[e] - S[i] * float(s_vbar[c]);
    }
    __syncthreads();
    colsums_f64<P>(Y, n, s_part, s_zbar);
    if (threadIdx.x < P) s_zbar[threadIdx.x] /= double(n);
    __syncthreads();
    for (int e = threadIdx.x; e < n * P; e += blockDim.x) {
        const int c = e % P;
        Y[e] = -0.5f * (Y[e] - float(s_zbar[c]));
    }
}

// Per-block partial products out[b][c1 * P2 + c2] = sum over the block's rows of
// X1[i][c1] X2[i][c2] (X1 with row stride P1, X2 with row stride P2).
__global__ void __launch_bounds__(256) k_cross_partials(const float* X1, int P1, const float* X2, int P2, int n,
                                                        float* out) {
    __shared__ float s1[kRedRows][kPMax], s2[kRedRows][kPMax];
    const int i0 = blockIdx.x * kRedRows;
    for (int e = threadIdx.x; e < kRedRows * kPMax; e += blockDim.x) {
        const int r = e / kPMax, c = e - r * kPMax, i = i0 + r;
        s1[r][c] = (i < n && c < P1) ? X1[int64_t(i) * P1 + c] : 0.f;
        s2[r][c] = (i < n && c < P2) ? X2[int64_t(i) * P2 + c] : 0.f;
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < P1 * P2; pr += blockDim.x) {
        const int c1 = pr / P2, c2 = pr - c1 * P2;
        float acc = 0.f;
        for (int r = 0; r < kRedRows; ++r) acc = fmaf(s1[r][c1], s2[r][c2], acc);
        out[int64_t(blockIdx.x) * P1 * P2 + pr] = acc;
    }
}

struct RotParams {
    float M[kPMax * kPMax];          // P1 x P2, row-major
};

// out[i][c] = sum_k X[i][k] M[k][c] (X with row stride P1, out with row stride P2).
__global__ void __launch_bounds__(256) k_rotate(const float* X, int P1, const __grid_constant__ RotParams R, int P2,
                                                int n, float* out, int out_stride, int out_col0) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * P2) return;
    const int i = int(e / P2), c = int(e - int64_t(i) * P2);
    float acc = 0.f;
    for (int k = 0; k < P1; ++k) acc = fmaf(X[int64_t(i) * P1 + k], R.M[k * P2 + c], acc);
    out[int64_t(i) * out_stride + out_col0 + c] = acc;
}

// Per block and column: the entry of largest magnitude (lowest row on ties), as
// out[b][c] = (value, row).
__global__ void __launch_bounds__(256) k_absmax_partials(const float* X, int P, int n, float2* out) {
    __shared__ float s_v[256];
    __shared__ int s_i[256];
    const int c = blockIdx.y;
    const int i0 = blockIdx.x * 256 * 8;
    float best = 0.f;
    int bi = 0x7fffffff;
    for (int k = 0; k < 8; ++k) {
        const int i = i0 + k * 256 + threadIdx.x;
        if (i < n) {
            const float v = X[int64_t(i) * P + c];
            if (fabsf(v) > fabsf(best) || (fabsf(v) == fabsf(best) && i < bi)) { best = v; bi = i; }
        }
    }
    s_v[threadIdx.x] = best;
    s_i[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bv = 0.f;
        int b = 0x7fffffff;
        for (int t = 0; t < 256; ++t)
            if (s_i[t] != 0x7fffffff && (fabsf(s_v[t]) > fabsf(bv) || (fabsf(s_v[t]) == fabsf(bv) && s_i[t] < b))) {
                bv = s_v[t];
                b = s_i[t];
            }
        out[int64_t(blockIdx.x) * gridDim.y + c] = make_float2(bv, __int_as_float(b));
    }
}

// V0: a fixed pseudo-random start (SplitMix64 of the element index), entries in [-1, 1).
__global__ void k_random_start(float* V, int P, int p, int n) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * P) return;
    const int c = int(e % P);
    uint64_t z = uint64_t(e) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    V[e] = (c < p) ? float(double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0) : 0.f;
}

// ------------------------------------------------------------------ host algebra (float64)

// Eigen-decomposition of a symmetric k x k matrix by cyclic Jacobi rotations: on return
// lam[0..k) are the eigenvalues in decreasing order and Q (k x k, row-major) holds the
// matching eigenvectors as columns.
void jacobi_eigen(int k, std::vector<double> A, std::vector<double>& lam, std::vector<double>& Q) {
    Q.assign(size_t(k) * k, 0.0);
    for (int i = 0; i < k; ++i) Q[size_t(i) * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                tot += A[size_t(i) * k + j] * A[size_t(i) * k + j];
                if (i != j) off += A[size_t(i) * k + j] * A[size_t(i) * k + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[size_t(p) * k + q];
                if (apq == 0.0) continue;
                const double app = A[size_t(p) * k + p], aqq = A[size_t(q) * k + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {
                    const double arp = A[size_t(r) * k + p], arq = A[size_t(r) * k + q];
                    A[size_t(r) * k + p] = c * arp - s * arq;
                    A[size_t(r) * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {
                    const double apr = A[size_t(p) * k + r], aqr = A[size_t(q) * k + r];
                    A[size_t(p) * k + r] = c * apr - s * aqr;
                    A[size_t(q) * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    const double qrp = Q[size_t(r) * k + p], qrq = Q[size_t(r) * k + q];
                    Q[size_t(r) * k + p] = c * qrp - s * qrq;
                    Q[size_t(r) * k + q] = s * qrp + c * qrq;
                }
            }
    }
    std::vector<int> idx(k);
    for (int i = 0; i < k; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[size_t(a) * k + a] > A[size_t(b) * k + b]; });
    lam.resize(k);
    std::vector<double> Qs(size_t(k) * k);
    for (int j = 0; j < k; ++j) {
        lam[j] = A[size_t(idx[j]) * k + idx[j]];
        for (int r = 0; r < k; ++r) Qs[size_t(r) * k + j] = Q[size_t(r) * k + idx[j]];
    }
    Q.swap(Qs);
}

// R^-1 for G = R'R (upper-triangular R, G symmetric positive definite, k x k); a column
// whose pivot is not positive (rank deficiency) is dropped (its row of R^-1 left zero).
void cholesky_inverse_upper(int k, const std::vector<double>& G, std::vector<double>& Rinv) {
    std::vector<double> R(size_t(k) * k, 0.0);
    std::vector<char> ok(k, 1);
    for (int j = 0; j < k; ++j) {
        double dsum = G[size_t(j) * k + j];
        for (int i = 0; i < j; ++i) dsum -= R[size_t(i) * k + j] * R[size_t(i) * k + j];
        const double scale = std::fabs(G[size_t(j) * k + j]);
        if (!(dsum > 1e-12 * scale) || !(scale > 0.0)) { ok[j] = 0; continue; }
        const double rjj = std::sqrt(dsum);
        R[size_t(j) * k + j] = rjj;
        for (int c = j + 1; c < k; ++c) {
            double v = G[size_t(j) * k + c];
            for (int i = 0; i < j; ++i) v -= R[size_t(i) * k + j] * R[size_t(i) * k + c];
            R[size_t(j) * k + c] = v / rjj;
        }
    }
    Rinv.assign(size_t(k) * k, 0.0);
    for (int c = k - 1; c >= 0; --c) {          // solve R X = I column by column (upper-triangular)
        for (int r = c; r >= 0; --r) {
            if (!ok[r]) continue;
            double v = (r == c) ? 1.0 : 0.0;
            for (int t = r + 1; t <= c; ++t)
                if (ok[t]) v -= R[size_t(r) * k + t] * Rinv[size_t(t) * k + c];
            Rinv[size_t(r) * k + c] = v / R[size_t(r) * k + r];
        }
    }
}

struct InitBuffers {
    float *V, *Y, *A, *S, *part, *xi0, *xi;
    float2* amax;
};

#define FJ_TRY(call)                                                                                   \
    do {                                                                                               \
        const cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                       \
            char b_[256];                                                                              \
            snprintf(b_, sizeof(b_), "%s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__);        \
            set_message(b_);                                                                           \
            return FJOFC_ERR_CUDA;                                                                     \
        }                                                                                              \
    } while (0)

// sum over the blocks of X1' X2 (P1 x P2) in float64, blocks in index order
int cross(const float* X1, int P1, const float* X2, int P2, int n, const InitBuffers& B, cudaStream_t st,
          std::vector<double>& out) {
    const int nb = (n + kRedRows - 1) / kRedRows;
    k_cross_partials<<<nb, 256, 0, st>>>(X1, P1, X2, P2, n, B.part);
    FJ_TRY(cudaGetLastError());
    std::vector<float> h(size_t(nb) * P1 * P2);
    FJ_TRY(cudaMemcpyAsync(h.data(), B.part, h.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    FJ_TRY(cudaStreamSynchronize(st));
    out.assign(size_t(P1) * P2, 0.0);
    for (int b = 0; b < nb; ++b)
        for (int e = 0; e < P1 * P2; ++e) out[e] += double(h[size_t(b) * P1 * P2 + e]);
    return FJOFC_OK;
}

int rotate(const float* X, int P1, const std::vector<double>& M, int P2, int n, float* out, int out_stride,
           int out_col0, cudaStream_t st) {
    RotParams R{};
    for (int e = 0; e < P1 * P2; ++e) R.M[e] = float(M[e]);
    const int64_t total = int64_t(n) * P2;
    k_rotate<<<unsigned((total + 255) / 256), 256, 0, st>>>(X, P1, R, P2, n, out, out_stride, out_col0);
    FJ_TRY(cudaGetLastError());
    return FJOFC_OK;
}

template <int P>
int sq_apply(SqParams sp, int dtype, const float* V, const InitBuffers& B, float* Y, cudaStream_t st) {
    sp.V = V;
    sp.A = B.A;
    sp.S = B.S;
    const int rows_per_cta = kSqWarps * kSqRows;
    const unsigned grid = unsigned((sp.n + rows_per_cta - 1) / rows_per_cta);
    if (dtype == FJOFC_F32) k_sq_product<P, float><<<grid, kSqWarps * 32, 0, st>>>(sp);
    else if (dtype == FJOFC_F16) k_sq_product<P, __half><<<grid, kSqWarps * 32, 0, st>>>(sp);
    else k_sq_product<P, __nv_bfloat16><<<grid, kSqWarps * 32, 0, st>>>(sp);
    FJ_TRY(cudaGetLastError());
    k_sq_finish<P><<<1, 1024, 0, st>>>(V, B.A, B.S, Y, sp.n);
    FJ_TRY(cudaGetLastError());
    return FJOFC_OK;
}

// cMDS of the dissimilarity described by sp into xi (n x d, device, row stride d),
// centred and with the sign convention.  Returns the number of subspace iterations in
// *iters.
__global__ void k_fill(float* X, int count, float v) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) X[e] = v;
}

// out[i][k] = s_k (X[i][k] - mu_k) in place (X with row stride P).
struct AffParams {
    float s[kPMax], mu[kPMax];
};
__global__ void __launch_bounds__(256) k_affine_cols(float* X, int P, int n, const __grid_constant__ AffParams a) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * P) return;
    const int k = int(e % P);
    X[e] = a.s[k] * (X[e] - a.mu[k]);
}

// Centre the columns of xi (n x d) and make each column's entry of largest magnitude
// (lowest row on ties) positive; sums and the search on the device, the d results on the
// host.
int centre_and_sign(float* xi, int d, int n, const InitBuffers& B, cudaStream_t st) {
    int rc;
    // column sums as xi' 1 through the partial-product kernel, with a column of ones
    k_fill<<<unsigned((n + 255) / 256), 256, 0, st>>>(B.S, n, 1.f);
    FJ_TRY(cudaGetLastError());
    std::vector<double> cs;
    if ((rc = cross(xi, d, B.S, 1, n, B, st, cs))) return rc;
    AffParams a{};
    for (int k = 0; k < d; ++k) {
        a.s[k] = 1.f;
        a.mu[k] = float(cs[k] / double(n));
    }
    const int64_t total = int64_t(n) * d;
    k_affine_cols<<<unsigned((total + 255) / 256), 256, 0, st>>>(xi, d, n, a);
    FJ_TRY(cudaGetLastError());
    const int nbm = (n + 256 * 8 - 1) / (256 * 8);
    k_absmax_partials<<<dim3(nbm, d), 256, 0, st>>>(xi, d, n, B.amax);
    FJ_TRY(cudaGetLastError());
    std::vector<float2> h(size_t(nbm) * d);
    FJ_TRY(cudaMemcpyAsync(h.data(), B.amax, h.size() * sizeof(float2), cudaMemcpyDeviceToHost, st));
    FJ_TRY(cudaStreamSynchronize(st));
    AffParams sg{};
    for (int k = 0; k < d; ++k) {
        float bv = 0.f;
        int bi = 0x7fffffff;
        for (int b = 0; b < nbm; ++b) {
            const float v = h[size_t(b) * d + k].x;
            int i;
            std::memcpy(&i, &h[size_t(b) * d + k].y, sizeof(int));
            if (i == 0x7fffffff) continue;
            if (std::fabs(v) > std::fabs(bv) || (std::fabs(v) == std::fabs(bv) && i < bi)) { bv = v; bi = i; }
        }
        sg.s[k] = (bv < 0.f) ? -1.f : 1.f;
        sg.mu[k] = 0.f;
    }
    k_affine_cols<<<unsigned((total + 255) / 256), 256, 0, st>>>(xi, d, n, sg);
    FJ_TRY(cudaGetLastError());
    return FJOFC_OK;
}

template <int P>
int cmds_device(const SqParams& sp, int dtype, int n, int d, int p, int max_iter, double tol, const InitBuffers& B,
                float* xi, cudaStream_t st, int* iters) {
    int rc;
    {
        const int64_t total = int64_t(n) * P;
        k_random_start<<<unsigned((total + 255) / 256), 256, 0, st>>>(B.V, P, p, n);
        FJ_TRY(cudaGetLastError());
    }
    std::vector<double> G, H, Rinv, lam, Q, prev(d, 0.0);
    // orthonormal start
    if ((rc = cross(B.V, P, B.V, P, n, B, st, G))) return rc;
    cholesky_inverse_upper(P, G, Rinv);
    if ((rc = rotate(B.V, P, Rinv, P, n, B.Y, P, 0, st))) return rc;
    FJ_TRY(cudaMemcpyAsync(B.V, B.Y, size_t(n) * P * sizeof(float), cudaMemcpyDeviceToDevice, st));
    int it = 0;
    for (;;) {
        if ((rc = sq_apply<P>(sp, dtype, B.V, B, B.Y, st))) return rc;          // Y = S V
        if ((rc = cross(B.V, P, B.Y, P, n, B, st, H))) return rc;              // Rayleigh quotient V'SV
        for (int i = 0; i < P; ++i)
            for (int j = i + 1; j < P; ++j) H[size_t(i) * P + j] = H[size_t(j) * P + i] = 0.5 * (H[size_t(i) * P + j] + H[size_t(j) * P + i]);
        jacobi_eigen(P, H, lam, Q);
        ++it;
        double change = 0.0;
        for (int k = 0; k < d; ++k)
            change = std::max(change, std::fabs(lam[k] - prev[k]) / std::max(std::fabs(lam[k]), 1e-300));
        for (int k = 0; k < d; ++k) prev[k] = lam[k];
        if ((it > 1 && change <= tol) || it >= max_iter) break;
        if ((rc = cross(B.Y, P, B.Y, P, n, B, st, G))) return rc;              // V <- Y R^-1
        cholesky_inverse_upper(P, G, Rinv);
        if ((rc = rotate(B.Y, P, Rinv, P, n, B.V, P, 0, st))) return rc;
    }
    *iters = it;
    // xi = V Q_d diag(sqrt(max(lambda, 0)))
    std::vector<double> M(size_t(P) * d, 0.0);
    for (int r = 0; r < P; ++r)
        for (int k = 0; k < d; ++k) M[size_t(r) * d + k] = Q[size_t(r) * P + k] * std::sqrt(std::max(lam[k], 0.0));
    if ((rc = rotate(B.V, P, M, d, n, xi, d, 0, st))) return rc;
    // centring (column means, float64 sums of device partials) and the sign convention
    if ((rc = centre_and_sign(xi, d, n, B, st))) return rc;
    return FJOFC_OK;
}

// Procrustes rotation R (d x d) of xi onto xi0: with T = xi0' xi = U S V', R = V U'.  The
// SVD from the Jacobi eigenvectors of T'T (V, S^2); U = T V S^-1, columns of a vanishing
// singular value completed by Gram-Schmidt.
void procrustes_rotation(int d, const std::vector<double>& T, std::vector<double>& R) {
    std::vector<double> TtT(size_t(d) * d, 0.0), lam, V;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = 0.0;
            for (int r = 0; r < d; ++r) v += T[size_t(r) * d + i] * T[size_t(r) * d + j];
            TtT[size_t(i) * d + j] = v;
        }
    jacobi_eigen(d, TtT, lam, V);
    const double smax = std::sqrt(std::max(lam[0], 0.0));
    std::vector<double> U(size_t(d) * d, 0.0);
    std::vector<char> have(d, 0);
    for (int k = 0; k < d; ++k) {
        const double sk = std::sqrt(std::max(lam[k], 0.0));
        if (!(sk > 1e-12 * smax) || !(smax > 0.0)) continue;
        for (int r = 0; r < d; ++r) {
            double v = 0.0;
            for (int c = 0; c < d; ++c) v += T[size_t(r) * d + c] * V[size_t(c) * d + k];
            U[size_t(r) * d + k] = v / sk;
        }
        have[k] = 1;
    }
    for (int k = 0; k < d; ++k) {             // complete an orthonormal U
        if (have[k]) continue;
        for (int e = 0; e < d && !have[k]; ++e) {
            std::vector<double> u(d, 0.0);
            u[e] = 1.0;
            for (int j = 0; j < d; ++j) {
                if (!have[j]) continue;
                double dot = 0.0;
                for (int r = 0; r < d; ++r) dot += U[size_t(r) * d + j] * u[r];
                for (int r = 0; r < d; ++r) u[r] -= dot * U[size_t(r) * d + j];
            }
            double nn = 0.0;
            for (int r = 0; r < d; ++r) nn += u[r] * u[r];
            if (nn > 1e-6) {
                for (int r = 0; r < d; ++r) U[size_t(r) * d + k] = u[r] / std::sqrt(nn);
                have[k] = 1;
            }
        }
    }
    R.assign(size_t(d) * d, 0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = 0.0;
            for (int k = 0; k < d; ++k) v += V[size_t(i) * d + k] * U[size_t(j) * d + k];
            R[size_t(i) * d + j] = v;
        }
}

template <int P>
int init_with_width(int m, int n, int d, int p, const void* const* delta, int64_t ld, int dtype,
                    const float* delta_scale, float* X, int max_iter, double tol, const InitBuffers& B,
                    cudaStream_t st, int32_t* iters_out) {
    int rc, it = 0;
    SqParams sp{};
    sp.ld = ld;
    sp.n = n;
    sp.count = m;
    for (int l = 0; l < m; ++l) {
        sp.delta[l] = delta[l];
        sp.w[l] = (delta_scale ? delta_scale[l] : 1.f) / float(m);
    }
    if ((rc = cmds_device<P>(sp, dtype, n, d, p, max_iter, tol, B, B.xi0, st, &it))) return rc;
    if (iters_out) iters_out[0] = it;
    for (int i = 0; i < m; ++i) {
        SqParams si{};
        si.ld = ld;
        si.n = n;
        si.count = 1;
        si.delta[0] = delta[i];
        si.w[0] = delta_scale ? delta_scale[i] : 1.f;
        if ((rc = cmds_device<P>(si, dtype, n, d, p, max_iter, tol, B, B.xi, st, &it))) return rc;
        if (iters_out) iters_out[i + 1] = it;
        std::vector<double> T, R;
        if ((rc = cross(B.xi0, d, B.xi, d, n, B, st, T))) return rc;          // xi0' xi
        procrustes_rotation(d, T, R);
        if ((rc = rotate(B.xi, d, R, d, n, X + int64_t(i) * n * d, d, 0, st))) return rc;
    }
    FJ_TRY(cudaStreamSynchronize(st));
    return FJOFC_OK;
}

}  // namespace
}  // namespace fjofc

extern "C" int fjofc_init_cmds(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld,
                               int32_t delta_dtype, const float* delta_scale, float* X, const fjofc_init_opts* opts,
                               int32_t* iters_out, void* cuda_stream) {
    using namespace fjofc;
    int rc = validate_problem(m, n, d, delta, ld, delta_dtype, delta_scale, X);
    if (rc) return rc;
    int max_iter = 200;
    double tol = 1e-6;
    if (opts) {
        if (opts->max_iter < 0) { set_message("max_iter must be >= 0"); return FJOFC_ERR_ARG; }
        if (!(opts->tol >= 0.0)) { set_message("tol must be >= 0"); return FJOFC_ERR_ARG; }
        for (int r = 0; r < 4; ++r)
            if (opts->reserved[r] != 0) { set_message("opts.reserved must be zero"); return FJOFC_ERR_ARG; }
        if (opts->max_iter > 0) max_iter = opts->max_iter;
        if (opts->tol > 0.0) tol = opts->tol;
    }
    if (n > (int64_t(1) << 24)) { set_message("n too large for the initialisation"); return FJOFC_ERR_UNSUPPORTED; }
    const int nn = int(n);
    const int p = int(std::min<int64_t>(2 * int64_t(d) + 4, n));
    const int pw = std::max(p, int(d));                 // the width holds d columns even when n < d
    const int P = pw <= 8 ? 8 : (pw <= 16 ? 16 : 32);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nb = (nn + kRedRows - 1) / kRedRows;
    const size_t nP = size_t(nn) * P, nd = size_t(nn) * d;
    const size_t bytes = (3 * nP + nn + size_t(nb) * kPMax * kPMax + 2 * nd + 64) * sizeof(float) +
                         size_t(nb + 1) * kPMax * sizeof(float2) + 8 * 256;
    void* base = nullptr;
    if (cudaMallocAsync(&base, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_message("cudaMallocAsync failed for the initialisation scratch");
        return FJOFC_ERR_NOMEM;
    }
    char* c = static_cast<char*>(base);
    auto take = [&](size_t nbytes) {
        char* r = c;
        c += (nbytes + 255) & ~size_t(255);
        return r;
    };
    InitBuffers B{};
    B.V = reinterpret_cast<float*>(take(nP * 4));
    B.Y = reinterpret_cast<float*>(take(nP * 4));
    B.A = reinterpret_cast<float*>(take(nP * 4));
    B.S = reinterpret_cast<float*>(take(size_t(nn) * 4 + 64));
    B.part = reinterpret_cast<float*>(take(size_t(nb) * kPMax * kPMax * 4));
    B.xi0 = reinterpret_cast<float*>(take(nd * 4));
    B.xi = reinterpret_cast<float*>(take(nd * 4));
    B.amax = reinterpret_cast<float2*>(take(size_t(nb + 1) * kPMax * sizeof(float2)));
    if (P == 8) rc = init_with_width<8>(m, nn, d, p, delta, ld, delta_dtype, delta_scale, X, max_iter, tol, B, st, iters_out);
    else if (P == 16) rc = init_with_width<16>(m, nn, d, p, delta, ld, delta_dtype, delta_scale, X, max_iter, tol, B, st, iters_out);
    else rc = init_with_width<32>(m, nn, d, p, delta, ld, delta_dtype, delta_scale, X, max_iter, tol, B, st, iters_out);
    cudaFreeAsync(base, st);
    if (rc == FJOFC_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_message("CUDA error after the initialisation");
        return FJOFC_ERR_CUDA;
    }
    return rc;
}

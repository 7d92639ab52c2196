// Learned warm start for the out-of-sample update (no counterpart in the paper): a
// 2-hidden-layer GELU network that maps a new object's dissimilarities to fixed in-sample
// landmarks to a starting position y_j(0) for the Guttman iterations of Sec. 3.
//
// Everything runs in the kernels of this file: landmark gather (float16 features),
// forward, backward, loss, Adam, parameter initialisation, batch gather.  The matrix
// products are small (at most 512 x 512 x batch) and are computed by one SIMT float32
// kernel, k_gemm, over strided operand views:
//   C[i][j] = sum_k A(i, k) B(k, j),  A(i,k) = a[i*sar + k*sac],  B(k,j) = b[k*sbr + j*sbc],
// 64 x 64 output tiles, 16-deep k slices staged in shared memory in the order of each
// view's unit stride (coalesced), the next slice prefetched into registers, 4 x 4 outputs
// per thread accumulated in a fixed k order; products with few tiles split k into up to 4
// ranges whose partial sums are added in range order (deterministic results).  Epilogues:
// + bias (per column), GELU (storing the pre-activation too), or x GELU'(z) (backward).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fjofc.h"
#include "fjofc_internal.h"

namespace fjofc {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, GEMM_THREADS = 256;

enum class Epi { Plain, BiasGelu, Bias, GeluGrad };

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

template <typename TA>
__device__ __forceinline__ float ld_as_float(const TA* p) { return float(*p); }
template <>
__device__ __forceinline__ float ld_as_float<__half>(const __half* p) { return __half2float(*p); }

// Epilogue of one output element (the pre-activation z goes to zout for BiasGelu).
template <Epi E>
__device__ __forceinline__ float epilogue(float v, int64_t o, int j, const float* __restrict__ bias,
                                          float* __restrict__ zout, const float* __restrict__ zin) {
    if constexpr (E == Epi::BiasGelu) {
        v += bias[j];
        zout[o] = v;
        v = gelu_f(v);
    } else if constexpr (E == Epi::Bias) {
        v += bias[j];
    } else if constexpr (E == Epi::GeluGrad) {
        v *= gelu_grad_f(zin[o]);
    }
    return v;
}

// C (M x N, row stride ldc) = A B with the epilogue E, over the k range [kb, ke) of
// split blockIdx.z (ke - kb a multiple of TK except at K).  With splits > 1 the kernel
// writes raw partial products to part[z][M][N] and k_gemm_reduce applies the epilogue.
//   BiasGelu: Z = AB + bias[j] -> zout, C = gelu(Z)
//   Bias:     C = AB + bias[j]
//   GeluGrad: C = AB * gelu'(zin[i*ldc + j])
// Operand slabs are staged in shared memory in the order of their unit stride (k or i for
// A, j or k for B) so that a warp's loads are coalesced for every view, and the next slab
// is loaded into registers while the current one is used (two shared buffers).
template <typename TA, typename TB, Epi E>
__global__ void __launch_bounds__(GEMM_THREADS)
k_gemm(int M, int N, int K, int kspan, const TA* __restrict__ a, int64_t sar, int64_t sac, const TB* __restrict__ b,
       int64_t sbr, int64_t sbc, float* __restrict__ c, int64_t ldc, const float* __restrict__ bias,
       float* __restrict__ zout, const float* __restrict__ zin, float* __restrict__ part) {
    __shared__ float As[2][TK][TM + 4];
    __shared__ float Bs[2][TK][TN + 4];
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;          // 16 x 16 threads, 4 x 4 outputs each
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    const int kb = blockIdx.z * kspan, ke = min(K, kb + kspan);
    const bool a_kfast = (sac == 1), b_jfast = (sbc == 1);
    constexpr int PER = TM * TK / GEMM_THREADS;      // 4 elements of each operand per thread
    float ra[PER], rb[PER];
    auto load = [&](int k0) {
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = t * GEMM_THREADS + tid;
            const int ii = a_kfast ? e / TK : e % TM, kk = a_kfast ? e % TK : e / TM;
            const int i = i0 + ii, k = k0 + kk;
            ra[t] = (i < M && k < ke) ? ld_as_float(a + int64_t(i) * sar + int64_t(k) * sac) : 0.f;
            const int jj = b_jfast ? e % TN : e / TK, kb2 = b_jfast ? e / TN : e % TK;
            const int j = j0 + jj, k2 = k0 + kb2;
            rb[t] = (k2 < ke && j < N) ? ld_as_float(b + int64_t(k2) * sbr + int64_t(j) * sbc) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = t * GEMM_THREADS + tid;
            const int ii = a_kfast ? e / TK : e % TM, kk = a_kfast ? e % TK : e / TM;
            As[buf][kk][ii] = ra[t];
            const int jj = b_jfast ? e % TN : e / TK, kb2 = b_jfast ? e / TN : e % TK;
            Bs[buf][kb2][jj] = rb[t];
        }
    };
    float acc[4][4] = {};
    int buf = 0;
    load(kb);
    store(0);
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += TK) {
        const bool more = k0 + TK < ke;
        if (more) load(k0 + TK);
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a4[r], b4[q], acc[r][q]);
        }
        if (more) {
            store(buf ^ 1);
            buf ^= 1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
        if (i >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (j >= N) continue;
            if (part) {
                part[(int64_t(blockIdx.z) * M + i) * N + j] = acc[r][q];
            } else {
                const int64_t o = int64_t(i) * ldc + j;
                c[o] = epilogue<E>(acc[r][q], o, j, bias, zout, zin);
            }
        }
    }
}

// Sum of the split partial products in split order, then the epilogue.
template <Epi E>
__global__ void __launch_bounds__(256) k_gemm_reduce(int M, int N, int splits, const float* __restrict__ part,
                                                     float* __restrict__ c, int64_t ldc, const float* __restrict__ bias,
                                                     float* __restrict__ zout, const float* __restrict__ zin) {
    const int64_t total = int64_t(M) * N;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < splits; ++z) v += part[int64_t(z) * total + e];
        const int i = int(e / N), j = int(e - int64_t(i) * N);
        const int64_t o = int64_t(i) * ldc + j;
        c[o] = epilogue<E>(v, o, j, bias, zout, zin);
    }
}

// Split-K workspace (floats) a training step uses: at most 4 splits of a 256 x 512 or 2
// of a 512 x 512 product, reused call after call (stream order).
constexpr int64_t kSplitFloats = int64_t(4) * 256 * 512;

// Splits of the k range so that the tiles and splits fill about 128 CTAs, each split at
// least 4 slabs long; 1 when no workspace is available.
int choose_splits(int M, int N, int K, const float* ws, int64_t ws_floats) {
    const int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    int s = 1;
    while (s < 4 && tiles * s * 2 <= 160 && K / (2 * s) >= 4 * TK && int64_t(2 * s) * M * N <= ws_floats) s *= 2;
    return ws ? s : 1;
}

template <typename TA, typename TB, Epi E>
cudaError_t gemm(int M, int N, int K, const TA* a, int64_t sar, int64_t sac, const TB* b, int64_t sbr, int64_t sbc,
                 float* c, int64_t ldc, const float* bias, float* zout, const float* zin, cudaStream_t s,
                 float* ws = nullptr, int64_t ws_floats = 0) {
    const int splits = choose_splits(M, N, K, ws, ws_floats);
    const int kspan = splits == 1 ? K : ((K + splits - 1) / splits + TK - 1) / TK * TK;
    const dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, splits);
    k_gemm<TA, TB, E><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, kspan, a, sar, sac, b, sbr, sbc, c, ldc, bias, zout, zin,
                                                    splits > 1 ? ws : nullptr);
    if (splits > 1) {
        const int64_t total = int64_t(M) * N;
        const int blocks = int((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
        k_gemm_reduce<E><<<blocks, 256, 0, s>>>(M, N, splits, ws, c, ldc, bias, zout, zin);
    }
    return cudaGetLastError();
}

// out[j] = sum_i x[i*ld + j] for i < rows (bias gradients).  CTA c takes columns
// 32c .. 32c+31 (lane = column); warp w sums rows w, w + 8, ... in row order, then lane j
// adds the eight warp sums in warp order (a fixed order: deterministic).
constexpr int kColsumWarps = 8;
__global__ void __launch_bounds__(kColsumWarps * 32) k_colsum(int rows, int cols, const float* __restrict__ x,
                                                              int64_t ld, float* __restrict__ out) {
    __shared__ float part[kColsumWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (j < cols)
        for (int i = warp; i < rows; i += kColsumWarps) s += x[int64_t(i) * ld + j];
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && j < cols) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kColsumWarps; ++w) t += part[w][lane];
        out[j] = t;
    }
}
void colsum(int rows, int cols, const float* x, int64_t ld, float* out, cudaStream_t s) {
    k_colsum<<<(cols + 31) / 32, kColsumWarps * 32, 0, s>>>(rows, cols, x, ld, out);
}

// dY = (yhat - y) / B and the batch loss sum ||yhat - y||^2 / (2B) (one CTA, fixed order).
// With idx (training graphs) the loss goes to loss_out[*idx].
__global__ void k_mse(int B, int O, const float* __restrict__ yhat, const float* __restrict__ y,
                      float* __restrict__ dy, float* __restrict__ loss_out, const long long* __restrict__ idx = nullptr) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int e = threadIdx.x; e < B * O; e += blockDim.x) {
        const float r = yhat[e] - y[e];
        dy[e] = r / float(B);
        acc = fmaf(r, r, acc);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) loss_out[idx ? *idx : 0] = s[0] / (2.f * float(B));
}

// Adam with bias correction; c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t) from the host (with
// idx: from the host-made tables c1t[*idx], c2t[*idx], step t = *idx + 1).
__global__ void k_adam(int64_t P, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float beta1, float beta2, float eps, float c1, float c2,
                       const float* __restrict__ c1t = nullptr, const float* __restrict__ c2t = nullptr,
                       const long long* __restrict__ idx = nullptr) {
    if (idx) {
        c1 = c1t[*idx];
        c2 = c2t[*idx];
    }
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < P; e += int64_t(gridDim.x) * blockDim.x) {
        const float ge = g[e];
        const float me = beta1 * m[e] + (1.f - beta1) * ge;
        const float ve = beta2 * v[e] + (1.f - beta2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        theta[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014): a counter-based 64-bit generator; element e of a
// stream draws splitmix64(seed + (e + 1) * golden gamma).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// theta[off + e] ~ U(-r, r) for e < count (weights and biases of one layer: r = 1/sqrt(fan_in)).
__global__ void k_init_uniform(float* __restrict__ theta, int64_t off, int64_t count, float r, uint64_t seed) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t h = splitmix64(seed + uint64_t(off + e) * 0x9E3779B97F4A7C15ull);
        const float u = float(h >> 40) * (1.0f / 16777216.0f);      // [0, 1) from 24 bits
        theta[off + e] = (2.f * u - 1.f) * r;
    }
}

// The batch of training step *step (steps counted over all epochs, nb batches per epoch):
// epoch ep = step / nb uses the order i -> (pa[ep] i + pc[ep]) mod N; the same rows as
// rows (pa[ep] i + pc[ep]) mod N for i in [(step % nb) B, (step % nb + 1) B).
__global__ void k_gather_step(int B, int ni, int no, int64_t N, int64_t nb, const long long* __restrict__ step,
                              const uint64_t* __restrict__ pa, const uint64_t* __restrict__ pc,
                              const __half* __restrict__ x, const float* __restrict__ y, __half* __restrict__ xb,
                              float* __restrict__ yb) {
    const int row = blockIdx.x;
    if (row >= B) return;
    const long long st = *step;
    const long long ep = st / nb, bi = st - ep * nb;
    const int64_t src = int64_t((pa[ep] * uint64_t(bi * B + row) + pc[ep]) % uint64_t(N));
    for (int e = threadIdx.x; e < ni; e += blockDim.x) xb[int64_t(row) * ni + e] = x[src * ni + e];
    for (int e = threadIdx.x; e < no; e += blockDim.x) yb[int64_t(row) * no + e] = y[src * no + e];
}

__global__ void k_step_advance(long long* step) { *step += 1; }

// Features of new objects: out[o][j*L + t] = half(delta_new[o][j][landmark[t]] * inv_mean[j]).
struct FeatParams {
    const float* delta;
    int64_t ld;
    const int32_t* landmarks;
    float inv_mean[FJOFC_MAX_M];
    __half* out;
    int64_t k;
    int m, L;
};
__global__ void k_features(const FeatParams p) {
    const int64_t total = p.k * p.m * p.L;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = e / (int64_t(p.m) * p.L);
        const int r = int(e - o * p.m * p.L), j = r / p.L, t = r - j * p.L;
        const float v = p.delta[(o * p.m + j) * p.ld + p.landmarks[t]] * p.inv_mean[j];
        p.out[e] = __float2half_rn(v);
    }
}

// Y[o][j][:] = yhat[o][:] for every modality j.
__global__ void k_broadcast(int64_t k, int m, int d, const float* __restrict__ yhat, float* __restrict__ Y) {
    const int64_t total = k * m * d;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = e / (int64_t(m) * d);
        const int kk = int(e % d);
        Y[e] = yhat[o * d + kk];
    }
}

// Per object, the start with the lower stress: the warm start when s_warm <= s_std.
__global__ void k_select(int64_t k, int m, int d, const float* __restrict__ Yw, const double* __restrict__ sw,
                         const double* __restrict__ ss, float* __restrict__ Y, int32_t* __restrict__ used) {
    const int64_t total = k * m * d;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = e / (int64_t(m) * d);
        const bool warm = sw[o] <= ss[o];
        if (warm) Y[e] = Yw[e];
        if (used && e % (int64_t(m) * d) == 0) used[o] = warm ? 1 : 0;
    }
}

// ------------------------------------------------------------------ network passes

struct Net {
    int ni, nh, no;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, P;
    Net(const float* th, int ni_, int nh_, int no_) : ni(ni_), nh(nh_), no(no_) {
        oW1 = 0; ob1 = oW1 + int64_t(nh) * ni; oW2 = ob1 + nh; ob2 = oW2 + int64_t(nh) * nh; oW3 = ob2 + nh;
        ob3 = oW3 + int64_t(no) * nh; P = ob3 + no;
        W1 = th + oW1; b1 = th + ob1; W2 = th + oW2; b2 = th + ob2; W3 = th + oW3; b3 = th + ob3;
    }
};

// Activations of a batch of B rows: z1, h1, z2, h2 (B x nh each), yhat (B x no), then the
// backward buffers dz2, dz1 (B x nh), dy (B x no).
struct Acts {
    float *z1, *h1, *z2, *h2, *y, *dz2, *dz1, *dy;
    static int64_t floats(int B, int nh, int no) { return int64_t(B) * (6 * int64_t(nh) + 2 * no); }
    Acts(float* w, int B, int nh, int no) {
        const int64_t H = int64_t(B) * nh, O = int64_t(B) * no;
        z1 = w; h1 = z1 + H; z2 = h1 + H; h2 = z2 + H; y = h2 + H; dz2 = y + O; dz1 = dz2 + H; dy = dz1 + H;
    }
};

cudaError_t forward(const Net& n, const __half* x, int B, Acts& a, cudaStream_t s, float* ws = nullptr,
                    int64_t wsf = 0) {
    cudaError_t e;
    // z1 = x W1^T + b1: A = x (B x ni), B(k, j) = W1[j][k]
    if ((e = gemm<__half, float, Epi::BiasGelu>(B, n.nh, n.ni, x, n.ni, 1, n.W1, 1, n.ni, a.h1, n.nh, n.b1, a.z1,
                                                nullptr, s, ws, wsf)))
        return e;
    if ((e = gemm<float, float, Epi::BiasGelu>(B, n.nh, n.nh, a.h1, n.nh, 1, n.W2, 1, n.nh, a.h2, n.nh, n.b2, a.z2,
                                               nullptr, s, ws, wsf)))
        return e;
    return gemm<float, float, Epi::Bias>(B, n.no, n.nh, a.h2, n.nh, 1, n.W3, 1, n.nh, a.y, n.no, n.b3, nullptr,
                                         nullptr, s, ws, wsf);
}

// Gradient of the batch loss into g (P floats), given dL/dyhat in a.dy.
// A second stream for the bias-gradient sums, which depend only on the layer's output
// gradient: forked from the main stream after that gradient and joined before the
// caller's next kernel, so they run beside the following products (used while a training
// step is captured into a graph, where the fork becomes parallel branches).
struct SideSums {
    cudaStream_t side = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

cudaError_t backward(const Net& n, const __half* x, int B, Acts& a, float* g, cudaStream_t s, float* ws = nullptr,
                     int64_t wsf = 0, const SideSums* ss = nullptr) {
    cudaError_t e;
    int fork = 0;
    auto bias_sum = [&](int rows, int cols, const float* v, int64_t ld, float* out) -> cudaError_t {
        if (!ss) {
            colsum(rows, cols, v, ld, out, s);
            return cudaSuccess;
        }
        cudaError_t r = cudaEventRecord(ss->ev[fork], s);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(ss->side, ss->ev[fork], 0);
        ++fork;
        if (r == cudaSuccess) colsum(rows, cols, v, ld, out, ss->side);
        return r;
    };
    // gW3 = dy^T h2 (no x nh): A(i, k=b) = dy[b][i], B(b, j) = h2[b][j]
    if ((e = gemm<float, float, Epi::Plain>(n.no, n.nh, B, a.dy, 1, n.no, a.h2, n.nh, 1, g + n.oW3, n.nh, nullptr,
                                            nullptr, nullptr, s, ws, wsf)))
        return e;
    if ((e = bias_sum(B, n.no, a.dy, n.no, g + n.ob3))) return e;
    // dz2 = (dy W3) * gelu'(z2): A = dy (B x no), B = W3 (no x nh)
    if ((e = gemm<float, float, Epi::GeluGrad>(B, n.nh, n.no, a.dy, n.no, 1, n.W3, n.nh, 1, a.dz2, n.nh, nullptr,
                                               nullptr, a.z2, s, ws, wsf)))
        return e;
    if ((e = gemm<float, float, Epi::Plain>(n.nh, n.nh, B, a.dz2, 1, n.nh, a.h1, n.nh, 1, g + n.oW2, n.nh, nullptr,
                                            nullptr, nullptr, s, ws, wsf)))
        return e;
    if ((e = bias_sum(B, n.nh, a.dz2, n.nh, g + n.ob2))) return e;
    // dz1 = (dz2 W2) * gelu'(z1)
    if ((e = gemm<float, float, Epi::GeluGrad>(B, n.nh, n.nh, a.dz2, n.nh, 1, n.W2, n.nh, 1, a.dz1, n.nh, nullptr,
                                               nullptr, a.z1, s, ws, wsf)))
        return e;
    // gW1 = dz1^T x (nh x ni): A(i, k=b) = dz1[b][i], B(b, j) = x[b][j] (float16)
    if ((e = gemm<float, __half, Epi::Plain>(n.nh, n.ni, B, a.dz1, 1, n.nh, x, n.ni, 1, g + n.oW1, n.ni, nullptr,
                                             nullptr, nullptr, s, ws, wsf)))
        return e;
    if ((e = bias_sum(B, n.nh, a.dz1, n.nh, g + n.ob1))) return e;
    if (ss) {                                      // join the side stream
        if ((e = cudaEventRecord(ss->ev[3], ss->side)) || (e = cudaStreamWaitEvent(s, ss->ev[3], 0))) return e;
    }
    return cudaGetLastError();
}

constexpr int kChunk = 8192;     // rows per forward chunk (activation scratch ~100 MB at 512 wide)

int dims_ok(int ni, int nh, int no) {
    if (ni < 1 || nh < 1 || no < 1 || ni > 65536 || nh > 65536 || no > 65536) {
        set_message("network sizes must be in [1, 65536]");
        return FJOFC_ERR_ARG;
    }
    return FJOFC_OK;
}

// Scratch of the given float count from the stream-ordered allocator.
struct Scratch {
    float* p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t s_) : s(s_) {}
    cudaError_t alloc(int64_t floats) { return cudaMallocAsync(reinterpret_cast<void**>(&p), size_t(floats) * 4, s); }
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

int cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FJOFC_OK;
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    set_message(msg);
    return e == cudaErrorMemoryAllocation ? FJOFC_ERR_NOMEM : FJOFC_ERR_CUDA;
}

}  // namespace
}  // namespace fjofc

using namespace fjofc;

extern "C" int64_t fjofc_mlp_param_count(int32_t n_in, int32_t hidden, int32_t n_out) {
    if (dims_ok(n_in, hidden, n_out) != FJOFC_OK) return -1;
    return int64_t(hidden) * n_in + hidden + int64_t(hidden) * hidden + hidden + int64_t(n_out) * hidden + n_out;
}

extern "C" int fjofc_mlp_init(float* params, int32_t n_in, int32_t hidden, int32_t n_out, uint64_t seed,
                              void* cuda_stream) {
    int rc = dims_ok(n_in, hidden, n_out);
    if (rc) return rc;
    if (!params) {
        set_message("params is NULL");
        return FJOFC_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Net n(params, n_in, hidden, n_out);
    // every layer's weights and bias ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in))
    const int64_t off[6] = {n.oW1, n.ob1, n.oW2, n.ob2, n.oW3, n.ob3};
    const int64_t cnt[6] = {n.ob1 - n.oW1, n.oW2 - n.ob1, n.ob2 - n.oW2, n.oW3 - n.ob2, n.ob3 - n.oW3, n.P - n.ob3};
    const int fan[6] = {n_in, n_in, hidden, hidden, hidden, hidden};
    for (int l = 0; l < 6; ++l)
        k_init_uniform<<<256, 256, 0, s>>>(params, off[l], cnt[l], 1.0f / std::sqrt(float(fan[l])), seed);
    return cuda_status(cudaGetLastError(), "fjofc_mlp_init");
}

extern "C" int fjofc_mlp_features(int32_t m, int64_t n, int64_t k, const float* delta_new, int64_t ld,
                                  const int32_t* landmarks, int32_t n_land, const float* inv_mean, uint16_t* features,
                                  void* cuda_stream) {
    if (m < 1 || m > FJOFC_MAX_M || n < 1 || k < 0 || n_land < 1 || ld < n || !delta_new || !landmarks || !inv_mean ||
        !features) {
        set_message("fjofc_mlp_features: invalid argument");
        return FJOFC_ERR_ARG;
    }
    if (k == 0) return FJOFC_OK;
    FeatParams p{};
    p.delta = delta_new;
    p.ld = ld;
    p.landmarks = landmarks;
    for (int j = 0; j < FJOFC_MAX_M; ++j) p.inv_mean[j] = j < m ? inv_mean[j] : 0.f;
    p.out = reinterpret_cast<__half*>(features);
    p.k = k;
    p.m = m;
    p.L = n_land;
    k_features<<<1024, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(p);
    return cuda_status(cudaGetLastError(), "fjofc_mlp_features");
}

extern "C" int fjofc_mlp_forward(const float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x,
                                 int64_t count, float* y, void* cuda_stream) {
    int rc = dims_ok(n_in, hidden, n_out);
    if (rc) return rc;
    if (!params || !x || !y || count < 0) {
        set_message("fjofc_mlp_forward: invalid argument");
        return FJOFC_ERR_ARG;
    }
    if (count == 0) return FJOFC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Net n(params, n_in, hidden, n_out);
    const int B = int(count < kChunk ? count : kChunk);
    Scratch w(s);
    if ((rc = cuda_status(w.alloc(Acts::floats(B, hidden, n_out)), "scratch"))) return rc;
    Acts a(w.p, B, hidden, n_out);
    const __half* xh = reinterpret_cast<const __half*>(x);
    for (int64_t r0 = 0; r0 < count; r0 += B) {
        const int rows = int(count - r0 < B ? count - r0 : B);
        if ((rc = cuda_status(forward(n, xh + r0 * n_in, rows, a, s), "forward"))) return rc;
        if ((rc = cuda_status(cudaMemcpyAsync(y + r0 * n_out, a.y, size_t(rows) * n_out * 4, cudaMemcpyDeviceToDevice, s),
                              "copy")))
            return rc;
    }
    return FJOFC_OK;
}

extern "C" int fjofc_mlp_gradient(const float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x,
                                  const float* y, int64_t count, float* grad, double* loss, void* cuda_stream) {
    int rc = dims_ok(n_in, hidden, n_out);
    if (rc) return rc;
    if (!params || !x || !y || !grad || count < 1 || count > kChunk) {
        set_message("fjofc_mlp_gradient: invalid argument (1 <= count <= 8192)");
        return FJOFC_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Net n(params, n_in, hidden, n_out);
    const int B = int(count);
    Scratch w(s);
    const int64_t act = Acts::floats(B, hidden, n_out);
    if ((rc = cuda_status(w.alloc(act + 4 + kSplitFloats), "scratch"))) return rc;
    Acts a(w.p, B, hidden, n_out);
    float* dloss = a.dy + int64_t(B) * n_out;
    float* ws = w.p + act + 4;
    const __half* xh = reinterpret_cast<const __half*>(x);
    if ((rc = cuda_status(forward(n, xh, B, a, s, ws, kSplitFloats), "forward"))) return rc;
    k_mse<<<1, 256, 0, s>>>(B, n_out, a.y, y, a.dy, dloss);
    if ((rc = cuda_status(backward(n, xh, B, a, grad, s, ws, kSplitFloats), "backward"))) return rc;
    float hl = 0.f;
    if ((rc = cuda_status(cudaMemcpyAsync(&hl, dloss, 4, cudaMemcpyDeviceToHost, s), "copy"))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(s), "sync"))) return rc;
    if (loss) *loss = hl;
    return FJOFC_OK;
}

extern "C" int fjofc_mlp_train(float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x,
                               const float* y, int64_t count, const fjofc_mlp_train_opts* opts, float* loss_history,
                               void* cuda_stream) {
    int rc = dims_ok(n_in, hidden, n_out);
    if (rc) return rc;
    if (!params || !x || !y || !opts || opts->epochs < 0 || opts->batch < 1 || opts->batch > kChunk ||
        count < opts->batch || !(opts->lr > 0.f)) {
        set_message("fjofc_mlp_train: invalid argument (1 <= batch <= min(count, 8192), lr > 0)");
        return FJOFC_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Net n(params, n_in, hidden, n_out);
    const int B = opts->batch;
    const int64_t nb = count / B;                 // full batches per epoch
    const int64_t P = n.P;
    const int64_t act = Acts::floats(B, hidden, n_out);
    const int64_t xb_floats = (int64_t(B) * n_in + 1) / 2;    // float16 batch rows
    const int64_t steps = nb * opts->epochs;
    // scratch: activations, gradient, Adam moments, batch, losses, split-K workspace, and the
    // step tables of the training graph (counter, epoch orders, bias corrections)
    const int64_t tab_floats = 2 + 4 * int64_t(opts->epochs) + 2 * steps;
    const int64_t total = act + 3 * P + xb_floats + int64_t(B) * n_out + steps + 4 + kSplitFloats + tab_floats + 4;
    Scratch w(s);
    if ((rc = cuda_status(w.alloc(total), "scratch"))) return rc;
    Acts a(w.p, B, hidden, n_out);
    float* g = w.p + act;
    float* mom = g + P;
    float* vel = mom + P;
    __half* xb = reinterpret_cast<__half*>(vel + P);
    float* yb = vel + P + xb_floats;
    float* losses = yb + int64_t(B) * n_out;
    float* ws = losses + steps + 4;
    float* tabs = ws + kSplitFloats;
    // 8-byte aligned tables
    tabs = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tabs) + 7) & ~uintptr_t(7));
    long long* ctl = reinterpret_cast<long long*>(tabs);
    uint64_t* tpa = reinterpret_cast<uint64_t*>(ctl + 1);
    uint64_t* tpc = tpa + opts->epochs;
    float* tc1 = reinterpret_cast<float*>(tpc + opts->epochs);
    float* tc2 = tc1 + steps;
    if ((rc = cuda_status(cudaMemsetAsync(mom, 0, size_t(2 * P) * 4, s), "memset"))) return rc;
    const __half* xh = reinterpret_cast<const __half*>(x);
    const float beta1 = opts->beta1 > 0.f ? opts->beta1 : 0.9f, beta2 = opts->beta2 > 0.f ? opts->beta2 : 0.999f;
    const float eps = opts->eps > 0.f ? opts->eps : 1e-8f;
    if (steps == 0) return FJOFC_OK;
    // the epoch orders (i -> (a i + c) mod count, gcd(a, count) = 1) and the bias
    // corrections of every step, made on the host
    std::vector<uint64_t> hpa(size_t(opts->epochs)), hpc(size_t(opts->epochs));
    std::vector<float> hc1(static_cast<size_t>(steps)), hc2(static_cast<size_t>(steps));
    uint64_t rng = opts->seed;
    for (int ep = 0; ep < opts->epochs; ++ep) {
        uint64_t pa = 1;
        for (;;) {
            rng = splitmix64(rng);
            pa = (rng % uint64_t(count)) | 1u;
            uint64_t x0 = pa, y0 = uint64_t(count);
            while (y0) { const uint64_t t = x0 % y0; x0 = y0; y0 = t; }
            if (x0 == 1) break;
        }
        rng = splitmix64(rng);
        hpa[size_t(ep)] = pa;
        hpc[size_t(ep)] = rng % uint64_t(count);
    }
    for (int64_t st = 0; st < steps; ++st) {
        hc1[size_t(st)] = float(1.0 / (1.0 - std::pow(double(beta1), double(st + 1))));
        hc2[size_t(st)] = float(1.0 / (1.0 - std::pow(double(beta2), double(st + 1))));
    }
    if ((rc = cuda_status(cudaMemsetAsync(ctl, 0, sizeof(long long), s), "memset"))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(tpa, hpa.data(), hpa.size() * 8, cudaMemcpyHostToDevice, s), "copy")) ||
        (rc = cuda_status(cudaMemcpyAsync(tpc, hpc.data(), hpc.size() * 8, cudaMemcpyHostToDevice, s), "copy")) ||
        (rc = cuda_status(cudaMemcpyAsync(tc1, hc1.data(), hc1.size() * 4, cudaMemcpyHostToDevice, s), "copy")) ||
        (rc = cuda_status(cudaMemcpyAsync(tc2, hc2.data(), hc2.size() * 4, cudaMemcpyHostToDevice, s), "copy")))
        return rc;
    // one training step, captured once into a CUDA graph on a private stream: every kernel
    // takes its step from the device counter, which the last node advances; the graph is
    // then launched once per step on the caller's stream
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SideSums ss;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (ss.side) cudaStreamDestroy(ss.side);
        for (cudaEvent_t ev : ss.ev)
            if (ev) cudaEventDestroy(ev);
    };
    if ((rc = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream"))) return rc;
    {
        cudaError_t se = cudaStreamCreateWithFlags(&ss.side, cudaStreamNonBlocking);
        for (int i = 0; i < 4 && se == cudaSuccess; ++i) se = cudaEventCreateWithFlags(&ss.ev[i], cudaEventDisableTiming);
        if ((rc = cuda_status(se, "side stream"))) {
            cleanup();
            return rc;
        }
    }
    if ((rc = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "capture"))) {
        cleanup();
        return rc;
    }
    k_gather_step<<<B, 128, 0, cs>>>(B, n_in, n_out, count, nb, ctl, tpa, tpc, xh, y, xb, yb);
    cudaError_t ce = forward(n, xb, B, a, cs, ws, kSplitFloats);
    k_mse<<<1, 256, 0, cs>>>(B, n_out, a.y, yb, a.dy, losses, ctl);
    if (ce == cudaSuccess) ce = backward(n, xb, B, a, g, cs, ws, kSplitFloats, &ss);
    k_adam<<<512, 256, 0, cs>>>(P, params, g, mom, vel, opts->lr, beta1, beta2, eps, 1.f, 1.f, tc1, tc2, ctl);
    k_step_advance<<<1, 1, 0, cs>>>(ctl);
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    for (int64_t st = 0; ce == cudaSuccess && st < steps; ++st) ce = cudaGraphLaunch(exec, s);
    cleanup();
    if ((rc = cuda_status(ce, "training graph"))) return rc;
    if ((rc = cuda_status(cudaGetLastError(), "train launches"))) return rc;
    if (loss_history && opts->epochs > 0) {
        std::vector<float> hl(size_t(nb) * opts->epochs);
        if ((rc = cuda_status(cudaMemcpyAsync(hl.data(), losses, hl.size() * 4, cudaMemcpyDeviceToHost, s), "copy")))
            return rc;
        if ((rc = cuda_status(cudaStreamSynchronize(s), "sync"))) return rc;
        for (int ep = 0; ep < opts->epochs; ++ep) {
            double acc = 0.0;
            for (int64_t bi = 0; bi < nb; ++bi) acc += hl[size_t(ep * nb + bi)];
            loss_history[ep] = float(acc / double(nb));
        }
    }
    return FJOFC_OK;
}

extern "C" int fjofc_mlp_broadcast(int64_t k, int32_t m, int32_t d, const float* yhat, float* Y, void* cuda_stream) {
    if (k < 0 || m < 1 || d < 1 || (k > 0 && (!yhat || !Y))) {
        set_message("fjofc_mlp_broadcast: invalid argument");
        return FJOFC_ERR_ARG;
    }
    if (k == 0) return FJOFC_OK;
    k_broadcast<<<1024, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(k, m, d, yhat, Y);
    return cuda_status(cudaGetLastError(), "fjofc_mlp_broadcast");
}

extern "C" int fjofc_mlp_select(int64_t k, int32_t m, int32_t d, const float* Y_warm, const double* s_warm,
                                const double* s_std, float* Y, int32_t* used, void* cuda_stream) {
    if (k < 0 || m < 1 || d < 1 || (k > 0 && (!Y_warm || !s_warm || !s_std || !Y))) {
        set_message("fjofc_mlp_select: invalid argument");
        return FJOFC_ERR_ARG;
    }
    if (k == 0) return FJOFC_OK;
    k_select<<<1024, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(k, m, d, Y_warm, s_warm, s_std, Y, used);
    return cuda_status(cudaGetLastError(), "fjofc_mlp_select");
}

// Host side of the fJOFC C ABI: argument validation, the m x m weight algebra of
// Sec. 2.1 in float64, TMA descriptors, workspace layout and the launch sequence of
// the in-sample loop and of the out-of-sample solver.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "fjofc_device.cuh"
#include "k1_decl.h"
#include "k3_decl.h"

using namespace fjofc;

namespace {

// ------------------------------------------------------------------ errors
#define FJ_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            set_last_error(cudaGetErrorString(e_), #call);    \
            return FJOFC_ERR_CUDA;                            \
        }                                                     \
    } while (0)

thread_local char g_last_msg[512] = "";

void set_last_error(const char* what, const char* where) {
    snprintf(g_last_msg, sizeof(g_last_msg), "%s (%s)", what, where);
}

int arg_error(const char* msg) {
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg);
    return FJOFC_ERR_ARG;
}

// ------------------------------------------------------------------ weights (Sec. 2.1)
// Validates the m x m weights of Eq. (W2) and returns Wmod^-1 (Eq. modW inverted by
// Gauss-Jordan elimination with partial pivoting, float64).  Wmod is strictly
// diagonally dominant when every w_ii > 0 (proof of Thm 1), hence invertible.
int weights_inverse(int m, int64_t n, const double* w, double* winv) {
    if (!w) return arg_error("weights is NULL");
    if (m < 1 || m > FJOFC_MAX_M) return arg_error("m outside 1..FJOFC_MAX_M");
    for (int i = 0; i < m; ++i) {
        if (!(w[i * m + i] > 0.0) || !std::isfinite(w[i * m + i]))
            return arg_error("fidelity weights w_ii must be finite and > 0");
        for (int j = 0; j < m; ++j) {
            if (i == j) continue;
            const double a = w[i * m + j], b = w[j * m + i];
            if (!(a >= 0.0) || !std::isfinite(a)) return arg_error("commensurability weights must be finite and >= 0");
            if (a != b) return arg_error("weights must be symmetric (w_ij == w_ji)");
        }
    }
    // [m][2m] augmented matrix on the stack: no heap allocation (fjofc_embed_noalloc
    // relies on this)
    double A[FJOFC_MAX_M * 2 * FJOFC_MAX_M];
    for (int e = 0; e < 2 * m * m; ++e) A[e] = 0.0;
    for (int i = 0; i < m; ++i) {
        double diag = double(n) * w[i * m + i];
        for (int j = 0; j < m; ++j)
            if (j != i) {
                diag += w[i * m + j];
                A[size_t(i) * 2 * m + j] = -w[i * m + j];
            }
        A[size_t(i) * 2 * m + i] = diag;
        A[size_t(i) * 2 * m + m + i] = 1.0;
    }
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(A[size_t(r) * 2 * m + c]) > std::fabs(A[size_t(piv) * 2 * m + c])) piv = r;
        if (A[size_t(piv) * 2 * m + c] == 0.0) return arg_error("modified weight matrix is singular");
        if (piv != c)
            for (int j = 0; j < 2 * m; ++j) std::swap(A[size_t(c) * 2 * m + j], A[size_t(piv) * 2 * m + j]);
        const double inv = 1.0 / A[size_t(c) * 2 * m + c];
        for (int j = 0; j < 2 * m; ++j) A[size_t(c) * 2 * m + j] *= inv;
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = A[size_t(r) * 2 * m + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * m; ++j) A[size_t(r) * 2 * m + j] -= f * A[size_t(c) * 2 * m + j];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) winv[i * m + j] = A[size_t(i) * 2 * m + m + j];
    return FJOFC_OK;
}

size_t dtype_size(int dt) { return dt == FJOFC_F32 ? 4 : 2; }

int check_delta_layout(const void* const* ptrs, int count, int64_t n, int64_t ld, int dtype) {
    if (dtype != FJOFC_F32 && dtype != FJOFC_F16 && dtype != FJOFC_BF16) return arg_error("unknown delta_dtype");
    if (ld < n) return arg_error("ld must be >= n");
    if ((ld * int64_t(dtype_size(dtype))) % 16 != 0)
        return arg_error("Delta row stride must be a multiple of 16 bytes (ld*elem_size % 16 == 0)");
    for (int i = 0; i < count; ++i) {
        if (!ptrs[i]) return arg_error("Delta pointer is NULL");
        if (reinterpret_cast<uintptr_t>(ptrs[i]) % 16 != 0) return arg_error("Delta base pointer must be 16-byte aligned");
    }
    return FJOFC_OK;
}

// ------------------------------------------------------------------ TMA descriptors
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        set_last_error("cuTensorMapEncodeTiled unavailable", "cudaGetDriverEntryPointByVersion");
        return FJOFC_ERR_CUDA;
    }
    return FJOFC_OK;
}

CUtensorMapDataType tma_dtype(int dt) {
    return dt == FJOFC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
         : dt == FJOFC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

// rank-r tiled map; dims/strides innermost first, strides in bytes (rank-1 entries)
int encode_map(CUtensorMap* map, int dtype, int rank, const void* base, const cuuint64_t* dims,
               const cuuint64_t* strides, const cuuint32_t* box, bool swizzle128 = false) {
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode(map, tma_dtype(dtype), cuuint32_t(rank), const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_msg, sizeof(g_last_msg), "cuTensorMapEncodeTiled failed (CUresult %d)", int(r));
        return FJOFC_ERR_CUDA;
    }
    return FJOFC_OK;
}

// ------------------------------------------------------------------ K1 dispatch
template <typename TD>
cudaError_t k1_launch_dt(int d, int grid, const TMaps& tm, const K1Params& p, cudaStream_t s) {
    switch (d) {
#define C_(D) case D: return k1_launch_impl<D, TD>(grid, tm, p, s);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return cudaErrorInvalidValue;
}
template <typename TD>
int k1_bps_dt(int d) {
    switch (d) {
#define C_(D) case D: return k1_bps_impl<D, TD>();
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return 0;
}
template <typename TD>
K1Geom k1_geom_dt(int d) {
    switch (d) {
#define C_(D) case D: return k1_geom_impl<D, TD>();
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return K1Geom{};
}

template <typename TD>
cudaError_t persist_launch_dt(int d, int grid, const TMaps& tm, const PersistParams& P, cudaStream_t s) {
    switch (d) {
#define C_(D) case D: return persist_launch_impl<D, TD>(grid, tm, P, s);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return cudaErrorInvalidValue;
}
template <typename TD>
int persist_bps_dt(int d) {
    switch (d) {
#define C_(D) case D: return persist_bps_impl<D, TD>();
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return 0;
}

// ------------------------------------------------------------------ K3 dispatch
template <typename TD>
cudaError_t k3_launch_dt(int d, int grid, const CUtensorMap& tm, const K3Params& p, cudaStream_t s) {
    switch (d) {
#define C_(D) case D: return k3_launch_impl<D, TD>(grid, tm, p, s);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return cudaErrorInvalidValue;
}
template <typename TD>
int k3_bps_dt(int d, int m) {
    switch (d) {
#define C_(D) case D: return k3_bps_impl<D, TD>(m);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return 0;
}
template <typename TD>
K3Geom k3_geom_dt(int d, int m) {
    switch (d) {
#define C_(D) case D: return k3_geom_impl<D, TD>(m);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13) C_(14) C_(15) C_(16)
#undef C_
    }
    return K3Geom{};
}

template <typename TD>
cudaError_t k3r_launch_dt(int d, int grid, const K3Params& p, cudaStream_t s) {
    switch (d) {
#define C_(D) case D: return k3r_launch_impl<D, TD>(grid, p, s);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8)
#undef C_
    }
    return cudaErrorInvalidValue;
}
template <typename TD>
int k3r_bps_dt(int d, size_t smem) {
    switch (d) {
#define C_(D) case D: return k3r_bps_impl<D, TD>(smem);
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8)
#undef C_
    }
    return 0;
}

// ------------------------------------------------------------------ device scratch
// One stream-ordered allocation per call, carved into 256-byte aligned pieces.
struct Carver {
    size_t off = 0;
    template <typename T> size_t take(size_t count) {
        const size_t o = (off + 255) & ~size_t(255);
        off = o + count * sizeof(T);
        return o;
    }
};

struct ScopedDeviceMem {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~ScopedDeviceMem() { if (p) cudaFreeAsync(p, s); }
};

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

bool cooperative_ok() {
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return false;
    return coop != 0;
}

int persist_blocks_per_sm(int d, int dtype) {
    return dtype == FJOFC_F32 ? persist_bps_dt<float>(d) : dtype == FJOFC_F16 ? persist_bps_dt<__half>(d)
                                                                               : persist_bps_dt<__nv_bfloat16>(d);
}

EmbedPlan make_plan(int m, int64_t n, int d, int dtype, bool persistent, int G_override = 0) {
    EmbedPlan P;
    P.g = fjofc::k1_geometry(d, dtype);
    P.nRB = int((n + P.g.RB - 1) / P.g.RB);
    int64_t Tm = 0;
    for (int I = 0; I < P.nRB; ++I) Tm += (n - int64_t(I) * P.g.RB + P.g.CW - 1) / P.g.CW;
    P.Tm = Tm;
    P.T = Tm * m;
    const int bps = std::max(1, persistent ? persist_blocks_per_sm(d, dtype) : fjofc::k1_blocks_per_sm(d, dtype));
    int64_t G = G_override > 0 ? int64_t(G_override) : int64_t(bps) * sm_count();
    if (G > P.T) G = P.T;
    P.G = int(G);
    P.nbx = fjofc::k2_blocks(int(n));
    return P;
}

// The option fields every entry point that takes fjofc_opts validates the same way.
int check_common_opts(const fjofc_opts& o) {
    if (o.check_inputs != 0 && o.check_inputs != 1) return arg_error("check_inputs must be 0 or 1");
    if (o.deterministic != 0 && o.deterministic != 1) return arg_error("deterministic must be 0 or 1");
    if (o.wait_limit_us < 0) return arg_error("wait_limit_us must be >= 0");
    if (o.delta_layout != FJOFC_LAYOUT_FULL && o.delta_layout != FJOFC_LAYOUT_PACKED)
        return arg_error("unknown delta_layout");
    for (int r = 0; r < 2; ++r)
        if (o.reserved[r] != 0) return arg_error("opts.reserved must be zero");
    return FJOFC_OK;
}

// Bound of the grid-wide waits in nanoseconds (0 = the default).
uint64_t wait_limit_ns(const fjofc_opts& o) {
    return o.wait_limit_us > 0 ? uint64_t(o.wait_limit_us) * 1000ull : kWaitLimitNs;
}

// Extra arrivals added to the first grid-wide wait of the next in-sample loop (test
// support, fjofc_test_barrier_skew).
std::atomic<int> g_barrier_skew{0};

// Message for an error the in-sample kernels raised (status block copied to the host).
void device_status_message(const DevStatus& h, int64_t n) {
    if (h.error == FJOFC_ERR_TIMEOUT)
        snprintf(g_last_msg, sizeof(g_last_msg), "device wait timed out (site %d)", h.timeout_site);
    if (h.error == FJOFC_ERR_NONFINITE) snprintf(g_last_msg, sizeof(g_last_msg), "stress became non-finite");
    if (h.error == FJOFC_ERR_ARG && h.bad != kNoBadEntry) {
        const unsigned long long pos = h.bad >> 2;
        const int kind = int(h.bad & 3ull);
        const long long col = (long long)(pos % (unsigned long long)n);
        const long long row = (long long)((pos / (unsigned long long)n) % (unsigned long long)n);
        const int l = int(pos / ((unsigned long long)n * (unsigned long long)n));
        snprintf(g_last_msg, sizeof(g_last_msg), "check_inputs: Delta_%d[%lld][%lld] %s", l + 1, row, col,
                 kind == 1 ? "is negative" : kind == 2 ? "is not finite" : "differs from its transposed entry");
    }
}

// Common validation of the in-sample arguments.
int validate_insample(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                      const float* delta_scale, const void* X) {
    if (m < 1) return arg_error("m must be >= 1");
    if (m > FJOFC_MAX_M) { snprintf(g_last_msg, sizeof(g_last_msg), "m > %d is not built", FJOFC_MAX_M); return FJOFC_ERR_UNSUPPORTED; }
    if (n < 2) return arg_error("n must be >= 2");
    if (n > (int64_t(1) << 30)) return arg_error("n too large");
    if (d < 1) return arg_error("d must be >= 1");
    if (d > FJOFC_MAX_D) { snprintf(g_last_msg, sizeof(g_last_msg), "d > %d is not built", FJOFC_MAX_D); return FJOFC_ERR_UNSUPPORTED; }
    if (!delta) return arg_error("delta is NULL");
    if (!X) return arg_error("X is NULL");
    if (reinterpret_cast<uintptr_t>(X) & 15u) return arg_error("X must be 16-byte aligned");
    if (delta_scale)
        for (int i = 0; i < m; ++i)
            if (!(delta_scale[i] > 0.f) || !std::isfinite(delta_scale[i])) return arg_error("delta_scale must be finite and > 0");
    return check_delta_layout(delta, m, n, ld, dtype);
}

}  // namespace

namespace fjofc {

int modified_weights_inverse(int m, int64_t n, const double* w, double* winv) { return weights_inverse(m, n, w, winv); }
int validate_problem(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                     const float* delta_scale, const void* X) {
    return validate_insample(m, n, d, delta, ld, dtype, delta_scale, X);
}
int tensor_map_encoder() { return get_encoder(); }

int InsampleSetup::plan(int m_, int64_t n_, int d_, int dtype_, const fjofc_opts& opts, bool persistent,
                        int G_override) {
    m = m_; n = n_; d = d_; dtype = dtype_; o = opts;
    P = make_plan(m, n, d, dtype, persistent, G_override);
    if (P.g.RB == 0) {
        snprintf(g_last_msg, sizeof(g_last_msg), "no kernel for d=%d", d);
        return FJOFC_ERR_UNSUPPORTED;
    }
    const int RB = P.g.RB, CW = P.g.CW;
    const int64_t mnd = int64_t(m) * n * d;
    Carver cv;
    o_buf1 = cv.take<float>(mnd);
    o_buf2 = cv.take<float>(mnd);
    o_col = cv.take<float>(size_t(P.T) * d * CW);
    o_head = cv.take<float>(size_t(m) * P.nRB * d * RB);
    o_cont = cv.take<float>(size_t(P.G) * d * RB);
    o_fid = cv.take<float2>(P.G);
    o_woff = cv.take<int64_t>(P.nRB + 1);
    o_cta = cv.take<int64_t>(size_t(P.G) + 1);
    o_mu = cv.take<float>(2 * FJOFC_MAX_M * FJOFC_MAX_D);
    o_bpart = cv.take<float2>(2 * size_t(P.nbx) * (size_t(m) * d + d));   // two pass parities
    o_ticket = cv.take<unsigned>(1);
    o_st = cv.take<DevStatus>(1);
    o_hist = cv.take<double>(size_t(o.max_iter) + 2);
    o_fid2 = cv.take<float2>(2 * size_t(P.G));
    o_cbase = cv.take<int64_t>(size_t(P.nRB));
    o_contr = cv.take<int2>(size_t(m) * P.nRB);
    o_bar = cv.take<unsigned>(1);
    o_tab = cv.take<float>(2 * size_t(m) * m);
    o_pub = cv.take<float2>(size_t(m) * d + d + 1);
    o_coff = cv.take<int64_t>(size_t(P.nRB) + 1);
    o_tcs = cv.take<int>(1);
    o_pseq = cv.take<unsigned>(1);
    bytes = (cv.off + 255) & ~size_t(255);
    return FJOFC_OK;
}

int InsampleSetup::bind(char* base, const void* const* delta, int64_t ld, const float* delta_scale,
                        const double* weights, const double* winv, float* X) {
    int rc;
    const int RB = P.g.RB, CW = P.g.CW;
    // TMA descriptors: Delta_l as a 2-D tensor {n cols, n rows} (packed layout: {L cols,
    // packed rows}), box {CW, RB} (row-band layout) or {128 bytes, RB} with the 128-byte
    // swizzle (column-strip layout)
    std::memset(&tm, 0, sizeof(tm));
    const bool packed = o.delta_layout == FJOFC_LAYOUT_PACKED;
    if (packed && ld != pack_width(n, int(dtype_size(dtype)))) {
        snprintf(g_last_msg, sizeof(g_last_msg), "packed Delta needs ld = %lld (fjofc_packed_size)",
                 (long long)pack_width(n, int(dtype_size(dtype))));
        return FJOFC_ERR_ARG;
    }
    const int64_t nbands = (n + kPackBand - 1) / kPackBand;
    for (int l = 0; l < m; ++l) {
        const cuuint64_t dims[2] = {cuuint64_t(packed ? ld : n),
                                    cuuint64_t(packed ? (nbands + 1) / 2 * kPackBand : n)};
        const cuuint64_t strides[1] = {cuuint64_t(ld) * dtype_size(dtype)};
        const bool strip = P.g.box_elems > 0;
        const cuuint32_t box[2] = {cuuint32_t(strip ? P.g.box_elems : CW), cuuint32_t(RB)};
        if ((rc = encode_map(&tm.map[l], dtype, 2, delta[l], dims, strides, box, strip))) return rc;
    }
    DevStatus* st = reinterpret_cast<DevStatus*>(base + o_st);
    double* hist = reinterpret_cast<double*>(base + o_hist);
    k1 = K1Params{};
    k1.colpart = reinterpret_cast<float*>(base + o_col);
    k1.rowhead = reinterpret_cast<float*>(base + o_head);
    k1.rowcont = reinterpret_cast<float*>(base + o_cont);
    k1.fid = reinterpret_cast<float2*>(base + o_fid);
    k1.walk_off = reinterpret_cast<int64_t*>(base + o_woff);
    k1.cta_start = reinterpret_cast<int64_t*>(base + o_cta);
    k1.st = st;
    k1.m = m; k1.n = int(n); k1.d = d; k1.nRB = P.nRB; k1.G = P.G;
    k1.Tm = P.Tm; k1.T = P.T;
    k1.packed = packed ? 1 : 0;
    // the all-pairs pass works in Delta's stored units (x / s_l), so its fidelity sum
    // carries s_l^2
    double dsc[FJOFC_MAX_M];
    for (int l = 0; l < FJOFC_MAX_M; ++l) {
        dsc[l] = (l < m && delta_scale) ? double(delta_scale[l]) : 1.0;
        k1.wfid[l] = l < m ? float(weights[l * m + l] * dsc[l] * dsc[l]) : 0.f;
        k1.xscale[l] = float(1.0 / dsc[l]);
    }

    k2 = K2Params{};
    k2.colpart = k1.colpart; k2.rowhead = k1.rowhead; k2.rowcont = k1.rowcont; k2.fid = k1.fid;
    k2.walk_off = k1.walk_off;
    k2.cta_start = k1.cta_start;
    k2.mu = reinterpret_cast<float*>(base + o_mu);
    k2.bpart = reinterpret_cast<float2*>(base + o_bpart);
    k2.ticket = reinterpret_cast<unsigned*>(base + o_ticket);
    k2.st = st;
    k2.hist = hist;
    k2.m = m; k2.n = int(n); k2.d = d; k2.RB = RB; k2.CW = CW; k2.nRB = P.nRB; k2.G = P.G; k2.nbx = P.nbx;
    k2.rb_shift = 0;
    while ((1 << k2.rb_shift) < RB) ++k2.rb_shift;
    k2.cw_shift = 0;
    while ((1 << k2.cw_shift) < CW) ++k2.cw_shift;
    if ((1 << k2.rb_shift) != RB || (1 << k2.cw_shift) != CW) {
        snprintf(g_last_msg, sizeof(g_last_msg), "internal: tile sizes must be powers of two");
        return FJOFC_ERR_UNSUPPORTED;
    }
    k2.Tm = P.Tm; k2.T = P.T;
    k2.tol_mode = o.tol_mode; k2.tol = o.tol;
    // relaxed updates: 0 and 1 are the plain transform, whose iterates are centred
    k2.relax = (o.relax == 0.f) ? 1.f : o.relax;
    k2.centre = (k2.relax == 1.f) ? 1 : 0;
    k2.npairs = double(m * n) * double(m * n - 1) / 2.0;
    k2.inv_n = float(1.0 / double(n));
    float* coef_g = reinterpret_cast<float*>(base + o_tab);
    float* wcomm_g = coef_g + size_t(m) * m;
    k2.coef_g = coef_g;
    k2.wcomm_g = wcomm_g;
    unsigned* bar = reinterpret_cast<unsigned*>(base + o_bar);
    k2.tb.colpart = k1.colpart;
    k2.tb.rowhead = k1.rowhead;
    k2.tb.rowcont = k1.rowcont;
    k2.tb.cbase = reinterpret_cast<int64_t*>(base + o_cbase);
    k2.tb.cont = reinterpret_cast<int2*>(base + o_contr);
    k2.tb.Tm = P.Tm;
    k2.tb.d = d; k2.tb.RB = RB; k2.tb.CW = CW; k2.tb.rb_shift = k2.rb_shift; k2.tb.cw_shift = k2.cw_shift;
    k2.tb.nRB = P.nRB;
    ip = InitParams{coef_g, wcomm_g, {}, {}, st, k2.ticket, k2.mu, const_cast<int64_t*>(k1.walk_off), const_cast<int64_t*>(k2.cta_start),
                    bar, const_cast<int64_t*>(k2.tb.cbase), const_cast<int2*>(k2.tb.cont), m, int(n), RB, CW,
                    P.nRB, P.G, P.T, P.Tm, reinterpret_cast<int64_t*>(base + o_coff),
                    reinterpret_cast<int*>(base + o_tcs), reinterpret_cast<unsigned*>(base + o_pseq)};
    // the per-object mix: [Wmod^-1]_{jl} w_ll s_l and the commensurability weights, in
    // the set-up kernel's parameters (it writes them to global memory for the kernels)
    for (int j = 0; j < m; ++j)
        for (int l = 0; l < m; ++l) {
            ip.coef[j * m + l] = float(winv[j * m + l] * weights[l * m + l] * dsc[l]);
            ip.wcomm[j * m + l] = (j < l) ? float(weights[j * m + l]) : 0.f;
        }

    pp = PersistParams{};
    pp.k1 = k1;
    pp.buf[0] = X;
    pp.buf[1] = reinterpret_cast<float*>(base + o_buf1);
    pp.buf[2] = reinterpret_cast<float*>(base + o_buf2);
    pp.cta_start = k2.cta_start;
    pp.fid2 = reinterpret_cast<float2*>(base + o_fid2);
    pp.bpart = k2.bpart;
    pp.bar = bar;
    pp.hist = hist;
    pp.ngroups = P.nbx;
    pp.rb_shift = k2.rb_shift; pp.cw_shift = k2.cw_shift;
    pp.max_iter = o.max_iter; pp.tol_mode = o.tol_mode; pp.tol = o.tol; pp.npairs = k2.npairs; pp.inv_n = k2.inv_n;
    pp.relax = k2.relax; pp.centre = k2.centre;
    pp.bar_skew = 0;
    pp.wait_ns = wait_limit_ns(o);
    pp.pub = reinterpret_cast<float2*>(base + o_pub);
    pp.pub_seq = ip.pub_seq;
    pp.tc = ip.tc;   // written by the set-up kernel with the CTA ranges
    pp.coef_g = k2.coef_g;
    pp.wcomm_g = k2.wcomm_g;
    pp.tb = k2.tb;
    return FJOFC_OK;
}

}  // namespace fjofc

namespace {
// The in-sample loop.  stress_only: sigma(X) of X only.  ext: run in a caller-supplied
// scratch region with no allocation of any kind (no events, no host buffers).
int run_insample_impl(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                      const float* delta_scale, const double* weights, float* X, const fjofc_opts* opts,
                      fjofc_result* res, cudaStream_t stream, bool stress_only, double* stress_out,
                      const fjofc::ExtScratch* ext) {
    int rc = validate_insample(m, n, d, delta, ld, dtype, delta_scale, X);
    if (rc) return rc;
    fjofc_opts o{};
    if (!stress_only) {
        if (!opts) return arg_error("opts is NULL");
        o = *opts;
        if (o.max_iter < 0) return arg_error("max_iter must be >= 0");
        if (o.tol_mode != FJOFC_TOL_ABS_NORMALIZED && o.tol_mode != FJOFC_TOL_RELATIVE) return arg_error("unknown tol_mode");
        if (std::isnan(o.tol)) return arg_error("tol is NaN");
        if (o.profile < 0 || o.profile > 2) return arg_error("profile must be 0, 1 or 2");
        if (!(o.relax >= 0.f && o.relax <= 2.f)) return arg_error("relax must be in [0, 2]");
        if ((rc = check_common_opts(o))) return rc;
    } else {
        o.max_iter = 0;
        o.tol = -1.0;
        o.tol_mode = FJOFC_TOL_RELATIVE;
    }
    if (ext && o.profile) return arg_error("profile timing is not available without allocation");
    if (o.delta_layout == FJOFC_LAYOUT_PACKED && o.check_inputs) {
        snprintf(g_last_msg, sizeof(g_last_msg), "check_inputs is not available with the packed Delta layout");
        return FJOFC_ERR_UNSUPPORTED;
    }
    if (o.delta_layout == FJOFC_LAYOUT_PACKED && ld != pack_width(n, int(dtype_size(dtype)))) {
        snprintf(g_last_msg, sizeof(g_last_msg), "packed Delta needs ld = %lld (fjofc_packed_size)",
                 (long long)pack_width(n, int(dtype_size(dtype))));
        return FJOFC_ERR_ARG;
    }
    double winv[FJOFC_MAX_M * FJOFC_MAX_M];
    rc = weights_inverse(m, n, weights, winv);
    if (rc) return rc;
    if ((rc = get_encoder())) return rc;

    // One persistent cooperative launch runs the whole loop; profile == 1 (per-kernel
    // timing) uses one launch per all-pairs pass and per W^-1 pass instead.
    const bool persist = (o.profile != 1) && cooperative_ok() && persist_blocks_per_sm(d, dtype) >= 1;
    fjofc::InsampleSetup S;
    if ((rc = S.plan(m, n, d, dtype, o, persist, 0))) return rc;
    const int64_t mnd = int64_t(m) * n * d;
    const size_t total = S.bytes;

    ScopedDeviceMem mem;
    mem.s = stream;
    char* base = nullptr;
    if (ext) {
        if (total > ext->capacity) {
            snprintf(g_last_msg, sizeof(g_last_msg),
                     "problem needs %zu bytes of scratch; the fixed scratch array holds %zu bytes", total,
                     ext->capacity);
            return FJOFC_ERR_UNSUPPORTED;
        }
        base = static_cast<char*>(ext->base);
    } else {
        if (cudaMallocAsync(&mem.p, total, stream) != cudaSuccess) {
            cudaGetLastError();
            snprintf(g_last_msg, sizeof(g_last_msg), "cudaMallocAsync(%zu bytes) failed", total);
            return FJOFC_ERR_NOMEM;
        }
        base = static_cast<char*>(mem.p);
    }
    if ((rc = S.bind(base, delta, ld, delta_scale, weights, winv, X))) return rc;
    const EmbedPlan& P = S.P;
    const TMaps& tm = S.tm;
    K1Params& k1 = S.k1;
    K2Params& k2 = S.k2;
    float* buf1 = S.pp.buf[1];
    float* buf2 = S.pp.buf[2];
    DevStatus* st = k1.st;
    double* hist = k2.hist;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (!ext) {
        FJ_CUDA(cudaEventCreate(&ev0));
        FJ_CUDA(cudaEventCreate(&ev1));
        FJ_CUDA(cudaEventRecord(ev0, stream));
    }

    int launches = 2;   // init + finalize (or init + the persistent kernel)
    FJ_CUDA(launch_init(S.ip, stream));
    if (o.check_inputs) {
        CheckParams cp{};
        for (int l = 0; l < m; ++l) cp.delta[l] = delta[l];
        cp.n = n; cp.ld = ld; cp.m = m; cp.dtype = dtype; cp.st = st;
        if ((n + 31) / 32 > 65535) return arg_error("check_inputs supports n <= 2097120");
        FJ_CUDA(launch_check_delta(cp, stream));
        ++launches;
    }

    float* bufs[3] = {X, buf1, buf2};
    const bool prof = o.profile == 1;
    std::vector<cudaEvent_t> pev;
    if (prof) {
        pev.resize(size_t(3) * (o.max_iter + 1));
        for (auto& e : pev) FJ_CUDA(cudaEventCreate(&e));
    }
    cudaEvent_t pe0 = nullptr, pe1 = nullptr;
    if (persist) {
        S.pp.bar_skew = unsigned(g_barrier_skew.exchange(0));
        const PersistParams& pp = S.pp;
        if (o.profile == 2) {
            FJ_CUDA(cudaEventCreate(&pe0));
            FJ_CUDA(cudaEventCreate(&pe1));
            FJ_CUDA(cudaEventRecord(pe0, stream));
        }
        const cudaError_t e = (dtype == FJOFC_F32) ? persist_launch_dt<float>(d, P.G, tm, pp, stream)
                            : (dtype == FJOFC_F16) ? persist_launch_dt<__half>(d, P.G, tm, pp, stream)
                                                   : persist_launch_dt<__nv_bfloat16>(d, P.G, tm, pp, stream);
        FJ_CUDA(e);
        if (o.profile == 2) FJ_CUDA(cudaEventRecord(pe1, stream));
    }
    auto k1_launch = [&](cudaError_t& e) {
        e = (dtype == FJOFC_F32) ? k1_launch_dt<float>(d, P.G, tm, k1, stream)
          : (dtype == FJOFC_F16) ? k1_launch_dt<__half>(d, P.G, tm, k1, stream)
                                 : k1_launch_dt<__nv_bfloat16>(d, P.G, tm, k1, stream);
    };
    for (int t = 1; !persist && t <= o.max_iter + 1; ++t) {
        const bool final_pass = (t == o.max_iter + 1);
        k1.X = bufs[(t - 1) % 3];
        cudaError_t e;
        if (prof) FJ_CUDA(cudaEventRecord(pev[3 * (t - 1)], stream));
        k1_launch(e);
        FJ_CUDA(e);
        if (prof) FJ_CUDA(cudaEventRecord(pev[3 * (t - 1) + 1], stream));
        k2.Xprev = bufs[(t - 1) % 3];
        k2.Xnext = bufs[t % 3];
        k2.t = t;
        k2.final_pass = final_pass ? 1 : 0;
        FJ_CUDA(launch_k2(k2, stream));
        if (prof) FJ_CUDA(cudaEventRecord(pev[3 * (t - 1) + 2], stream));
        launches += 2;
    }
    if (!persist) FJ_CUDA(launch_finalize(X, buf1, buf2, mnd, st, stream));
    if (!ext) FJ_CUDA(cudaEventRecord(ev1, stream));

    DevStatus hst;
    if (ext) {
        // no host buffers: the history goes straight into the caller's array
        FJ_CUDA(cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, stream));
        if (res && res->stress_history)
            FJ_CUDA(cudaMemcpyAsync(res->stress_history, hist, (size_t(o.max_iter) + 1) * sizeof(double),
                                    cudaMemcpyDeviceToHost, stream));
        FJ_CUDA(cudaStreamSynchronize(stream));
        rc = hst.error;
        device_status_message(hst, n);
        if (res) {
            res->status = rc;
            res->iters = hst.final_iter;
            res->stress = hst.stress;
            res->stress_normalized = hst.stress / k2.npairs;
            res->ms_total = 0.f;
            res->passes = 0;
            res->ms_pass = 0.f;
            res->ms_apply = 0.f;
            res->launches = launches;
            if (res->stress_history) {
                const int upto = (hst.error == FJOFC_ERR_NONFINITE) ? hst.final_iter + 1 : hst.final_iter;
                for (int t = upto + 1; t <= o.max_iter; ++t) res->stress_history[t] = 0.0;
            }
        }
        return rc;
    }
    std::vector<double> hh(size_t(o.max_iter) + 1);
    FJ_CUDA(cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, stream));
    FJ_CUDA(cudaMemcpyAsync(hh.data(), hist, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
    FJ_CUDA(cudaStreamSynchronize(stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    // passes that did work: the one that computed sigma(X_final) and all before it
    const int worked = std::min(o.max_iter + 1, hst.final_iter + 1 + (hst.error == FJOFC_ERR_NONFINITE ? 1 : 0));
    float ms_pass = 0.f, ms_apply = 0.f;
    if (pe0) {
        cudaEventElapsedTime(&ms_pass, pe0, pe1);
        cudaEventDestroy(pe0);
        cudaEventDestroy(pe1);
    }
    if (prof) {
        for (int t = 0; t < worked; ++t) {
            float a = 0.f, b2 = 0.f;
            cudaEventElapsedTime(&a, pev[3 * t], pev[3 * t + 1]);
            cudaEventElapsedTime(&b2, pev[3 * t + 1], pev[3 * t + 2]);
            ms_pass += a;
            ms_apply += b2;
        }
        for (auto& e : pev) cudaEventDestroy(e);
    }

    rc = hst.error;
    device_status_message(hst, n);
    if (stress_out) *stress_out = (hst.error == FJOFC_ERR_NONFINITE) ? hh[0] : hst.stress;
    if (res) {
        res->status = rc;
        res->iters = hst.final_iter;
        res->stress = hst.stress;
        res->stress_normalized = hst.stress / k2.npairs;
        res->ms_total = ms;
        res->passes = (prof || o.profile == 2) ? worked : 0;
        res->ms_pass = ms_pass;
        res->ms_apply = ms_apply;
        res->launches = launches;
        if (res->stress_history) {
            const int upto = (hst.error == FJOFC_ERR_NONFINITE) ? hst.final_iter + 1 : hst.final_iter;
            for (int t = 0; t <= upto && t <= o.max_iter; ++t) res->stress_history[t] = hh[t];
        }
    }
    return rc;
}

// Out-of-sample solve (Sec. 3): k independent objects, each iterated to its own stop.
int run_oos(int32_t m, int64_t n, int32_t d, int64_t k, const float* X, const void* delta_new, int64_t ld,
            int32_t dtype, const float* delta_scale, const double* weights, float* Y, int32_t* iters_out,
            double* stress_out, const fjofc_opts* opts, fjofc_result* res, cudaStream_t stream) {
    if (m < 1) return arg_error("m must be >= 1");
    if (m > FJOFC_MAX_M) { snprintf(g_last_msg, sizeof(g_last_msg), "m > %d is not built", FJOFC_MAX_M); return FJOFC_ERR_UNSUPPORTED; }
    if (n < 1) return arg_error("n must be >= 1");
    if (n > (int64_t(1) << 30)) return arg_error("n too large");
    if (d < 1) return arg_error("d must be >= 1");
    if (d > FJOFC_MAX_D) { snprintf(g_last_msg, sizeof(g_last_msg), "d > %d is not built", FJOFC_MAX_D); return FJOFC_ERR_UNSUPPORTED; }
    if (k < 0) return arg_error("k must be >= 0");
    if (k > (int64_t(1) << 31)) return arg_error("k too large");
    if (!X || !Y) return arg_error("X or Y is NULL");
    if (!opts) return arg_error("opts is NULL");
    const fjofc_opts o = *opts;
    if (o.max_iter < 0) return arg_error("max_iter must be >= 0");
    if (o.tol_mode != FJOFC_TOL_ABS_NORMALIZED && o.tol_mode != FJOFC_TOL_RELATIVE) return arg_error("unknown tol_mode");
    if (std::isnan(o.tol)) return arg_error("tol is NaN");
    if (delta_scale)
        for (int i = 0; i < m; ++i)
            if (!(delta_scale[i] > 0.f) || !std::isfinite(delta_scale[i])) return arg_error("delta_scale must be finite and > 0");
    if (o.oos_form != FJOFC_OOS_AUTO && o.oos_form != FJOFC_OOS_STREAMING && o.oos_form != FJOFC_OOS_RESIDENT)
        return arg_error("unknown oos_form");
    {
        const int orc = check_common_opts(o);
        if (orc) return orc;
    }
    const int nx = int((n + 3) / 4 * 4);
    const bool resident_fits = k3r_fits(m, nx, d);
    if (o.oos_form == FJOFC_OOS_RESIDENT && !resident_fits) {
        snprintf(g_last_msg, sizeof(g_last_msg),
                 "the resident out-of-sample form needs d <= %d and %zu bytes of shared memory (at most %zu)", kK3rMaxD,
                 k3r_smem_bytes(m, nx, d), kK3rSmemBudget);
        return FJOFC_ERR_UNSUPPORTED;
    }
    int rc;
    if (k > 0) {
        const void* ptrs[1] = {delta_new};
        if ((rc = check_delta_layout(ptrs, 1, n, ld, dtype))) return rc;
    }
    double winv[FJOFC_MAX_M * FJOFC_MAX_M];
    if ((rc = weights_inverse(m, n, weights, winv))) return rc;
    if (k == 0) {
        if (res) { res->status = 0; res->iters = 0; res->stress = 0.0; res->stress_normalized = 0.0; res->ms_total = 0.f; }
        return FJOFC_OK;
    }
    // the form: resident when asked, or (auto) when it fits and every object gets its own
    // CTA in one wave; otherwise streaming
    const size_t r_smem = k3r_smem_bytes(m, nx, d);
    int r_bps = 0;
    if (resident_fits && o.oos_form != FJOFC_OOS_STREAMING)
        r_bps = (dtype == FJOFC_F32) ? k3r_bps_dt<float>(d, r_smem) : (dtype == FJOFC_F16) ? k3r_bps_dt<__half>(d, r_smem)
                                                                                         : k3r_bps_dt<__nv_bfloat16>(d, r_smem);
    const bool resident = (o.oos_form == FJOFC_OOS_RESIDENT) ||
                          (o.oos_form == FJOFC_OOS_AUTO && resident_fits && r_bps > 0 && k <= int64_t(r_bps) * sm_count());
    if (o.oos_form == FJOFC_OOS_RESIDENT && r_bps < 1) {
        snprintf(g_last_msg, sizeof(g_last_msg), "the resident out-of-sample form cannot be launched (%zu bytes of shared memory)", r_smem);
        return FJOFC_ERR_UNSUPPORTED;
    }
    if ((rc = get_encoder())) return rc;
    const K3Geom g = (dtype == FJOFC_F32) ? k3_geom_dt<float>(d, m) : (dtype == FJOFC_F16) ? k3_geom_dt<__half>(d, m)
                                                                                         : k3_geom_dt<__nv_bfloat16>(d, m);
    if (!resident && g.WARPS < 1) {
        snprintf(g_last_msg, sizeof(g_last_msg), "the streaming out-of-sample form does not fit m=%d at d=%d", m, d);
        return FJOFC_ERR_UNSUPPORTED;
    }

    Carver cv;
    const size_t o_xt = cv.take<float>(size_t(m) * d * nx);
    const size_t o_sx = cv.take<float>(size_t(m) * d);
    const size_t o_ctr = cv.take<unsigned long long>(1);
    const size_t o_st = cv.take<DevStatus>(1);
    const size_t o_it = cv.take<int32_t>(size_t(k));
    const size_t o_sig = cv.take<double>(size_t(k));
    const size_t o_sum = cv.take<double>(2);
    const size_t o_winv = cv.take<float>(size_t(m) * m);
    const size_t o_wcomm = cv.take<double>(size_t(m) * m);
    const size_t total = cv.off;
    ScopedDeviceMem mem;
    mem.s = stream;
    if (cudaMallocAsync(&mem.p, total, stream) != cudaSuccess) {
        cudaGetLastError();
        snprintf(g_last_msg, sizeof(g_last_msg), "cudaMallocAsync(%zu bytes) failed", total);
        return FJOFC_ERR_NOMEM;
    }
    char* base = static_cast<char*>(mem.p);
    DevStatus* st = reinterpret_cast<DevStatus*>(base + o_st);

    // delta_new as a 3-D tensor {n points, m modalities, k objects}, box {CW, 1, 1}
    // (the streaming form's TMA source)
    CUtensorMap tmap;
    if (!resident) {
        const cuuint64_t dims[3] = {cuuint64_t(n), cuuint64_t(m), cuuint64_t(k)};
        const cuuint64_t strides[2] = {cuuint64_t(ld) * dtype_size(dtype), cuuint64_t(ld) * m * dtype_size(dtype)};
        const cuuint32_t box[3] = {cuuint32_t(g.CW), 1u, 1u};
        if ((rc = encode_map(&tmap, dtype, 3, delta_new, dims, strides, box))) return rc;
    }

    K3Params p{};
    p.X = X;
    p.XT = reinterpret_cast<float*>(base + o_xt);
    p.SX = reinterpret_cast<float*>(base + o_sx);
    p.Y = Y;
    p.delta_new = delta_new;
    p.ld = ld;
    p.iters_out = iters_out ? iters_out : reinterpret_cast<int32_t*>(base + o_it);
    p.stress_out = stress_out ? stress_out : reinterpret_cast<double*>(base + o_sig);
    p.next_block = reinterpret_cast<unsigned long long*>(base + o_ctr);
    p.st = st;
    p.m = m; p.n = int(n); p.nx = nx; p.d = d; p.max_iter = o.max_iter; p.tol_mode = o.tol_mode; p.k = k;
    p.tol = o.tol;
    p.npairs = double(m) * double(n) + double(m) * (m - 1) / 2.0;
    for (int j = 0; j < FJOFC_MAX_M; ++j) {
        p.wfid[j] = j < m ? float(weights[j * m + j]) : 0.f;
        p.dscale[j] = (j < m && delta_scale) ? delta_scale[j] : 1.f;
    }
    p.winv = reinterpret_cast<const float*>(base + o_winv);
    p.wcomm = reinterpret_cast<const double*>(base + o_wcomm);
    p.warp_bytes = g.smem_bytes;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    FJ_CUDA(cudaEventCreate(&ev0));
    FJ_CUDA(cudaEventCreate(&ev1));
    FJ_CUDA(cudaEventRecord(ev0, stream));
    OOSPrepParams pp{};
    pp.X = X;
    pp.XT = const_cast<float*>(p.XT);
    pp.SX = const_cast<float*>(p.SX);
    pp.winv_g = reinterpret_cast<float*>(base + o_winv);
    pp.wcomm_g = reinterpret_cast<double*>(base + o_wcomm);
    for (int j = 0; j < m; ++j)
        for (int l = 0; l < m; ++l) {
            pp.winv[j * m + l] = float(winv[j * m + l]);
            pp.wcomm[j * m + l] = (j != l) ? weights[j * m + l] : 0.0;
        }
    pp.m = m; pp.n = int(n); pp.nx = nx; pp.d = d;
    pp.next_block = p.next_block;
    pp.st = st;
    FJ_CUDA(launch_oos_prep(pp, stream));
    cudaError_t e;
    if (resident) {
        // one CTA per object, at most one wave; CTAs take further objects from the counter
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(k, int64_t(r_bps) * sm_count()));
        e = (dtype == FJOFC_F32) ? k3r_launch_dt<float>(d, int(grid), p, stream)
          : (dtype == FJOFC_F16) ? k3r_launch_dt<__half>(d, int(grid), p, stream)
                                 : k3r_launch_dt<__nv_bfloat16>(d, int(grid), p, stream);
    } else {
        const int bps = std::max(1, (dtype == FJOFC_F32) ? k3_bps_dt<float>(d, m)
                                    : (dtype == FJOFC_F16) ? k3_bps_dt<__half>(d, m) : k3_bps_dt<__nv_bfloat16>(d, m));
        const int64_t groups = (k + g.R - 1) / g.R;
        int64_t grid = int64_t(bps) * sm_count();
        const int64_t need = (groups + g.WARPS - 1) / g.WARPS;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        e = (dtype == FJOFC_F32) ? k3_launch_dt<float>(d, int(grid), tmap, p, stream)
          : (dtype == FJOFC_F16) ? k3_launch_dt<__half>(d, int(grid), tmap, p, stream)
                                 : k3_launch_dt<__nv_bfloat16>(d, int(grid), tmap, p, stream);
    }
    FJ_CUDA(e);
    double* sums = reinterpret_cast<double*>(base + o_sum);
    FJ_CUDA(launch_oos_summary(p.iters_out, p.stress_out, k, reinterpret_cast<int32_t*>(sums + 1), sums, stream));
    FJ_CUDA(cudaEventRecord(ev1, stream));
    DevStatus hst;
    double hsum[2];
    FJ_CUDA(cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, stream));
    FJ_CUDA(cudaMemcpyAsync(hsum, sums, sizeof(hsum), cudaMemcpyDeviceToHost, stream));
    FJ_CUDA(cudaStreamSynchronize(stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    rc = hst.error;
    if (rc == FJOFC_ERR_TIMEOUT) snprintf(g_last_msg, sizeof(g_last_msg), "device wait timed out (site %d)", hst.timeout_site);
    if (res) {
        res->status = rc;
        int32_t it;
        std::memcpy(&it, &hsum[1], sizeof(it));
        res->iters = it;
        res->stress = hsum[0];
        res->stress_normalized = hsum[0] / p.npairs;
        res->ms_total = ms;
        res->passes = 0;
        res->ms_pass = 0.f;
        res->ms_apply = 0.f;
        res->launches = 3;
    }
    return rc;
}

}  // namespace

namespace fjofc {
int run_insample(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                 const float* delta_scale, const double* weights, float* X, const fjofc_opts* opts,
                 fjofc_result* res, cudaStream_t stream, bool stress_only, double* stress_out,
                 const ExtScratch* ext) {
    return run_insample_impl(m, n, d, delta, ld, dtype, delta_scale, weights, X, opts, res, stream, stress_only,
                             stress_out, ext);
}
const char* set_message(const char* msg) {
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg);
    return g_last_msg;
}
K1Geom k1_geometry(int d, int dtype) {
    if (d < 1 || d > FJOFC_MAX_D) return K1Geom{};
    return dtype == FJOFC_F32 ? k1_geom_dt<float>(d) : dtype == FJOFC_F16 ? k1_geom_dt<__half>(d) : k1_geom_dt<__nv_bfloat16>(d);
}
int k1_blocks_per_sm(int d, int dtype) {
    return dtype == FJOFC_F32 ? k1_bps_dt<float>(d) : dtype == FJOFC_F16 ? k1_bps_dt<__half>(d) : k1_bps_dt<__nv_bfloat16>(d);
}
}  // namespace fjofc

// ====================================================================== C ABI
extern "C" {

int fjofc_embed(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t delta_dtype,
                const float* delta_scale, const double* weights, float* X, const fjofc_opts* opts,
                fjofc_result* res, void* cuda_stream) {
    const int rc = run_insample_impl(m, n, d, delta, ld, delta_dtype, delta_scale, weights, X, opts, res,
                                     static_cast<cudaStream_t>(cuda_stream), false, nullptr, nullptr);
    if (res) res->status = rc;
    return rc;
}

int fjofc_stress(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t delta_dtype,
                 const float* delta_scale, const double* weights, const float* X, double* stress_out,
                 void* cuda_stream) {
    if (!stress_out) return arg_error("stress_out is NULL");
    // max_iter = 0: one pass over X; the kernels centre X in place only when a Guttman
    // output is returned, and X_0 is returned as given (mu_0 = 0), so X is not modified.
    return run_insample_impl(m, n, d, delta, ld, delta_dtype, delta_scale, weights, const_cast<float*>(X), nullptr,
                             nullptr, static_cast<cudaStream_t>(cuda_stream), true, stress_out, nullptr);
}

int fjofc_oos(int32_t m, int64_t n, int32_t d, int64_t k, const float* X, const void* delta_new, int64_t ld,
              int32_t delta_dtype, const float* delta_scale, const double* weights, float* Y, int32_t* iters_out,
              double* stress_out, const fjofc_opts* opts, fjofc_result* res, void* cuda_stream) {
    const int rc = run_oos(m, n, d, k, X, delta_new, ld, delta_dtype, delta_scale, weights, Y, iters_out, stress_out,
                           opts, res, static_cast<cudaStream_t>(cuda_stream));
    if (res) res->status = rc;
    return rc;
}

const char* fjofc_strerror(int status) {
    switch (status) {
        case FJOFC_OK: return "ok";
        case FJOFC_ERR_ARG: return g_last_msg[0] ? g_last_msg : "invalid argument";
        case FJOFC_ERR_CUDA: return g_last_msg[0] ? g_last_msg : "CUDA error";
        case FJOFC_ERR_NONFINITE: return g_last_msg[0] ? g_last_msg : "stress became non-finite (NaN/Inf)";
        case FJOFC_ERR_TIMEOUT: return g_last_msg[0] ? g_last_msg : "a bounded device-side wait timed out";
        case FJOFC_ERR_NOMEM: return g_last_msg[0] ? g_last_msg : "out of device memory";
        case FJOFC_ERR_UNSUPPORTED: return g_last_msg[0] ? g_last_msg : "unsupported configuration";
    }
    return "unknown status";
}

int64_t fjofc_packed_size(int64_t n, int32_t delta_dtype, int64_t* ld_out) {
    if (n < 1 || n > (int64_t(1) << 30) ||
        (delta_dtype != FJOFC_F32 && delta_dtype != FJOFC_F16 && delta_dtype != FJOFC_BF16))
        return -1;
    const int es = int(dtype_size(delta_dtype));
    const int64_t L = pack_width(n, es);
    const int64_t nb = (n + kPackBand - 1) / kPackBand;
    if (ld_out) *ld_out = L;
    return (nb + 1) / 2 * kPackBand * L;
}

int fjofc_pack_delta(int64_t n, const void* delta, int64_t ld, int32_t delta_dtype, void* packed, void* cuda_stream) {
    if (fjofc_packed_size(n, delta_dtype, nullptr) < 0) return arg_error("invalid n or delta_dtype");
    if (!delta || !packed) return arg_error("NULL pointer");
    if (ld < n) return arg_error("ld must be >= n");
    if (reinterpret_cast<uintptr_t>(packed) % 16 != 0) return arg_error("packed must be 16-byte aligned");
    FJ_CUDA(launch_pack_delta(delta, n, ld, delta_dtype, packed, static_cast<cudaStream_t>(cuda_stream)));
    return FJOFC_OK;
}

void fjofc_test_barrier_skew(int32_t extra) { g_barrier_skew.store(extra > 0 ? extra : 0); }

const char* fjofc_version(void) { return "fjofc-gb300 0.2 (sm_103a; d=1..16; m<=32; f32/f16/bf16 Delta)"; }

}  // extern "C"

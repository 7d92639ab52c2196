// Internal declarations of the fJOFC library: kernel parameter blocks, tile
// configurations and the host-side launch entry points of each translation unit.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fjofc.h"

namespace fjofc {

struct DevStatus;


// Tensor maps of the m dissimilarity matrices (one 2-D map per modality), passed to
// the kernels as a __grid_constant__ parameter.
struct TMaps {
    CUtensorMap map[FJOFC_MAX_M];
};

// ---------------------------------------------------------------------------
// Tile geometry of the all-pairs pass (K1)
//
// The upper triangle of each Delta_l is covered by "walks": row block I (RB rows
// starting at I*RB) visits the column sub-tiles [I*RB + s*CW, I*RB + (s+1)*CW) for
// s = 0 .. L(I)-1, L(I) = ceil((n - I*RB)/CW).  Sub-tiles are numbered linearly
// t = l*Tm + walk_off[I] + s; CTA b processes t in [b*T/G, (b+1)*T/G).
// ---------------------------------------------------------------------------
struct K1Geom {
    int R, C, WARPS, STAGES;    // rows per thread, columns per lane, warps, pipeline depth
    int RB, CW;                 // row-block height (WARPS*R), sub-tile width (32*C)
    int threads;
    size_t smem_bytes;
    int box_elems;              // > 0: Delta is staged as boxes of box_elems x RB with the 128-byte
                                // swizzle (column-strip layout); 0: one CW x RB box, no swizzle
};

// Geometry of the K1 instantiation used for embedding dimension d.
K1Geom k1_geometry(int d, int dtype);

// Packed storage of a symmetric Delta (fjofc_opts.delta_layout = FJOFC_LAYOUT_PACKED): the
// rows are cut into bands of kPackBand rows; band b keeps only its columns from the
// diagonal on, [kPackBand b, n), row stride aligned to 16 bytes (width W_b = align(n -
// kPackBand b)), and bands b and nB - 1 - b share packed rows side by side (b first), so
// the packed matrix is ceil(nB / 2) kPackBand rows of width L = max over pairs of the two
// widths: about half of n^2.  kPackBand is a multiple of every all-pairs row block.
constexpr int kPackBand = 128;
__host__ __device__ inline int64_t pack_align(int64_t w, int esize) {
    const int64_t a = 16 / esize;
    return (w + a - 1) / a * a;
}
// Width of the packed rows (elements).
__host__ __device__ inline int64_t pack_width(int64_t n, int esize) {
    const int64_t nb = (n + kPackBand - 1) / kPackBand;
    int64_t L = 0;
    for (int64_t b = 0; b <= (nb - 1) / 2; ++b) {
        const int64_t c = nb - 1 - b;
        const int64_t w = pack_align(n - kPackBand * b, esize) + (c != b ? pack_align(n - kPackBand * c, esize) : 0);
        L = w > L ? w : L;
    }
    return L;
}
// Packed position (x = column, y = row) of Delta[row r][column c >= the band's start].
__host__ __device__ inline void pack_pos(int64_t n, int esize, int64_t r, int64_t c, int64_t& x, int64_t& y) {
    const int64_t nb = (n + kPackBand - 1) / kPackBand;
    const int64_t b = r / kPackBand, pb = nb - 1 - b;
    const bool right = b > pb;                       // the second band of its pair
    const int64_t pair = right ? pb : b;
    x = (right ? pack_align(n - kPackBand * pb, esize) : 0) + (c - kPackBand * b);
    y = kPackBand * pair + (r - kPackBand * b);
}

struct K1Params {
    const float* X;            // X_{t-1}: (m*n) x d row-major
    float* colpart;            // [T][d][CW]   column partials of B'X per sub-tile
    float* rowhead;            // [m][nRB][d][RB] row partials of the segment that starts a walk
    float* rowcont;            // [G][d][RB]   row partial of a CTA whose range starts mid-walk
    float2* fid;               // [G]          weighted fidelity partial per CTA (float-float)
    const int64_t* walk_off;   // [nRB+1]      prefix sums of the walk lengths, by walk position
    const int64_t* cta_start;  // [G+1]        first sub-tile of every CTA's range
    DevStatus* st;
    int m, n, d, nRB, G;
    int64_t Tm, T;             // sub-tiles per modality, total
    float wfid[FJOFC_MAX_M];   // w_ll s_l^2: weight of the fidelity sum in scaled units
    float xscale[FJOFC_MAX_M]; // 1 / s_l: coordinates of modality l in Delta's stored units
    int packed;                // 1: Delta in the packed band layout (pack_pos)
};

// CTAs of the K1 instantiation that fit on one SM.
int k1_blocks_per_sm(int d, int dtype);

// Tables written once per call by the initialisation kernel.
struct BxTables {
    const float* colpart;      // [T][d][CW]
    const float* rowhead;      // [m][nRB][d][RB]
    const float* rowcont;      // [G][d][RB]
    const int64_t* cbase;      // [nRB]       first sub-tile (within a modality) of row block I's walk
    const int2* cont;          // [m][nRB]    CTAs [x, y) whose range starts strictly inside that walk
    int64_t Tm;
    int d, RB, CW, rb_shift, cw_shift, nRB;
};

// ---------------------------------------------------------------------------
// K2: apply Wmod^-1, centre, commensurability, stress, stopping test
// ---------------------------------------------------------------------------
struct K2Params {
    float* Xprev;              // X_{t-1}; its modality blocks are centred in place
    float* Xnext;              // X_t (written unless final_pass)
    const float* colpart;
    const float* rowhead;
    const float* rowcont;
    const float2* fid;         // float-float fidelity partials of the K1 CTAs
    const int64_t* walk_off;
    const int64_t* cta_start;  // [G+1] first sub-tile of every K1 CTA (b*T/G)
    float* mu;                 // [2][FJOFC_MAX_M][FJOFC_MAX_D] modality column means, by t parity
    float2* bpart;             // [m*d+d][nbx] per-group float-float sums (column sums, commensurability)
    unsigned* ticket;
    DevStatus* st;
    double* hist;              // sigma(X_0..X_max_iter)
    int m, n, d, RB, CW, rb_shift, cw_shift, nRB, G, nbx;   // nbx = number of K2 CTAs (k2_blocks(n))
    int64_t Tm, T;
    int t;                     // pass index: reads X_{t-1}, writes X_t
    int final_pass;            // 1: only sigma(X_{t-1}) and the centring
    int tol_mode;
    double tol, npairs;        // tolerance, C(mn,2)
    float inv_n;               // 1 / n (column means)
    float relax;               // relaxed update factor (1: the plain Guttman transform)
    int centre;                // 1: centre X_{t-1} in place with its column means (relax == 1)
    const float* coef_g;             // [Wmod^-1]_{jl} * w_ll * s_l, m x m row-major (global)
    const float* wcomm_g;            // w_jl for j < l, else 0
    BxTables tb;
};

cudaError_t launch_k2(const K2Params& p, cudaStream_t s);
int k2_blocks(int n);

// Parameters of the persistent in-sample loop kernel (k_embed_persistent.cuh).
struct PersistParams {
    K1Params k1;                // geometry, partial buffers, weights (k1.X unused)
    float* buf[3];              // iterate t lives in buf[t % 3]; buf[0] is the caller's X
    const int64_t* cta_start;   // [G+1]
    float2* fid2;               // [2][G] fidelity partials by pass parity
    float2* bpart;              // [2][m*d+d][ngroups] by pass parity
    unsigned* bar;              // grid barrier counter (zeroed before launch)
    double* hist;               // sigma(X_0..X_max_iter)
    int ngroups;                // ceil(n / 32)
    int rb_shift, cw_shift;
    int max_iter, tol_mode;
    double tol, npairs;
    float inv_n;
    float relax;                // relaxed update factor (1: the plain Guttman transform)
    int centre;                 // 1: centre X_{t-1} in place with its column means
    float2* pub;                // [m*d + d + 1] the pass totals published by the totals CTA
    unsigned* pub_seq;          // the pass whose totals pub holds (written after them, release)
    const int* tc;              // the totals CTA (chosen by the set-up kernel: the least work)
    unsigned bar_skew;          // extra arrivals the first grid-wide wait expects (0; test support)
    unsigned long long wait_ns; // bound of every grid-wide wait
    const float* coef_g;        // m x m tables in global memory (see K2Params)
    const float* wcomm_g;
    BxTables tb;
};

// One cooperative launch of many problems of the same embedding dimension and Delta type.
struct BatchLaunch {
    const TMaps* maps;            // [problems] tensor maps (global memory, 64-byte aligned)
    const PersistParams* probs;   // [problems]
    const int* cta_off;           // [grid + 1] offsets of every CTA's assignment list
    const int2* assign;           // (problem, rank in the problem's CTA group)
};

struct InitParams {
    float* coef_g;             // destinations of the m x m tables below (global memory)
    float* wcomm_g;
    float coef[FJOFC_MAX_M * FJOFC_MAX_M];    // [Wmod^-1]_{jl} w_ll s_l, row-major m x m
    float wcomm[FJOFC_MAX_M * FJOFC_MAX_M];   // w_jl for j < l, else 0
    DevStatus* st;
    unsigned* ticket;
    float* mu;
    int64_t* walk_off;
    int64_t* cta_start;
    unsigned* bar;             // grid barrier counter of the persistent kernel (may be NULL)
    int64_t* cbase;            // [nRB]
    int2* cont;                // [m][nRB]
    int m, n, RB, CW, nRB, G;
    int64_t T, Tm;
    int64_t* cost_off;         // [nRB+1] modelled cost before walk position P (split_cost units)
    int* tc;                   // out: the totals CTA
    unsigned* pub_seq;         // cleared: the pass whose totals were last published
};

// Modelled cost of the all-pairs sub-tiles, used to split them over the CTAs (units of
// 1/100 of an unmasked sub-tile; fitted to per-CTA clock stamps of the column-strip pass
// at m = 2, n = 5000, d = 3): a masked sub-tile (a diagonal or ragged one) costs 0.15
// more, a walk that ends inside a CTA's range 0.76 more (its row sums and the hand-over
// of the next walk's rows).  Ranges stay contiguous; only their lengths change.
constexpr int64_t kSplitCostSub = 100, kSplitCostMask = 15, kSplitCostWalkEnd = 76;
// Dissimilarity check of fjofc_opts.check_inputs (one pass over every Delta_l).
struct CheckParams {
    const void* delta[FJOFC_MAX_M];
    int64_t n, ld;
    int m, dtype;
    DevStatus* st;
};
cudaError_t launch_check_delta(const CheckParams& p, cudaStream_t s);
cudaError_t launch_pack_delta(const void* D, int64_t n, int64_t ld, int dtype, void* P, cudaStream_t s);
cudaError_t launch_init(const InitParams& p, cudaStream_t s);
cudaError_t launch_init_batched(const InitParams* ps, int count, cudaStream_t s);
// float32 Delta -> float16 storage for the batched tuner: largest |Delta| (float bits,
// *out zeroed by the caller) and the scaled conversion.
cudaError_t launch_absmax(const float* D, int64_t n, int64_t ld, unsigned* out, cudaStream_t s);
cudaError_t launch_to_half(const float* D, int64_t n, int64_t ld, float inv_scale, void* out, int64_t ld16,
                           cudaStream_t s);
cudaError_t launch_batch_results(const DevStatus* const* st, int count, int* out, double* stress, cudaStream_t s);
cudaError_t launch_finalize(float* Xout, const float* buf1, const float* buf2, int64_t count,
                            const DevStatus* st, cudaStream_t s);

// ---------------------------------------------------------------------------
// K3: out-of-sample Guttman iterations (one CTA per block of new objects)
// ---------------------------------------------------------------------------
struct K3Geom {
    int R, C, WARPS, STAGES, OB, CW, threads;
    size_t smem_bytes;
};

struct K3Params {
    const float* X;            // in-sample (m*n) x d
    const float* XT;           // in-sample transposed and negated, -X^T: [m][d][nx] (nx = n rounded up to 4)
    const float* SX;           // [m][d] column sums of each X^(j)
    float* Y;                  // k x m x d
    const void* delta_new;     // k x m x n, row stride ld elements (the resident form reads it directly)
    int64_t ld;
    int32_t* iters_out;        // may be NULL
    double* stress_out;        // never NULL (internal buffer when the caller passes NULL)
    unsigned long long* next_block;   // work counter (next new object)
    DevStatus* st;
    int m, n, nx, d, max_iter, tol_mode;
    int64_t k;
    double tol, npairs;
    float wfid[FJOFC_MAX_M];
    float dscale[FJOFC_MAX_M];
    const float* winv;         // Wmod^-1, m x m row-major (global memory, written by the set-up kernel)
    const double* wcomm;       // w_jl, j != l, m x m (per-object stress, once per pass)
    size_t warp_bytes;         // streaming form: shared memory of one warp (depends on m)
};

// ---------------------------------------------------------------------------
// In-sample driver (fjofc_api.cu).  ext != NULL runs it in a caller-supplied scratch
// region without any allocation, event or host buffer (fjofc_embed_noalloc).
// ---------------------------------------------------------------------------
struct ExtScratch {
    void* base;
    size_t capacity;
};
int run_insample(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                 const float* delta_scale, const double* weights, float* X, const fjofc_opts* opts,
                 fjofc_result* res, cudaStream_t stream, bool stress_only, double* stress_out,
                 const ExtScratch* ext);
// Stores msg as the text fjofc_strerror returns for the next error; returns it.
const char* set_message(const char* msg);

// Geometry of one in-sample problem's all-pairs pass on G CTAs.
struct EmbedPlan {
    K1Geom g;
    int nRB = 0, G = 0, nbx = 0;
    int64_t Tm = 0, T = 0;
};

// Scratch layout and kernel parameters of one in-sample problem (shared by fjofc_embed
// and the batched plans).  plan() sizes the scratch for G CTAs (G_override > 0: at most
// that many, else one per SM times the resident CTAs per SM); bind() places it at base,
// encodes the Delta tensor maps and fills the parameter blocks.
struct InsampleSetup {
    EmbedPlan P;
    int m = 0, d = 0, dtype = 0;
    int64_t n = 0;
    fjofc_opts o{};
    size_t o_buf1 = 0, o_buf2 = 0, o_col = 0, o_head = 0, o_cont = 0, o_fid = 0, o_woff = 0, o_cta = 0, o_mu = 0,
           o_bpart = 0, o_ticket = 0, o_st = 0, o_hist = 0, o_fid2 = 0, o_cbase = 0, o_contr = 0, o_bar = 0,
           o_coff = 0, o_tcs = 0, o_pseq = 0,
           o_tab = 0, o_pub = 0;
    size_t bytes = 0;
    TMaps tm;
    K1Params k1;
    K2Params k2;
    PersistParams pp;
    InitParams ip;
    int plan(int m, int64_t n, int d, int dtype, const fjofc_opts& opts, bool persistent, int G_override);
    int bind(char* base, const void* const* delta, int64_t ld, const float* delta_scale, const double* weights,
             const double* winv, float* X);
};
// Gauss-Jordan inverse of Wmod (Eq. modW) for the m x m weights; FJOFC_ERR_ARG if singular.
int modified_weights_inverse(int m, int64_t n, const double* w, double* winv);
// The argument checks of fjofc_embed for one problem.
int validate_problem(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t dtype,
                     const float* delta_scale, const void* X);
// cuTensorMapEncodeTiled from the driver (once per process).
int tensor_map_encoder();

struct OOSPrepParams {
    const float* X;
    float* XT;
    float* SX;
    float* winv_g;             // destinations of the m x m tables below
    double* wcomm_g;
    float winv[FJOFC_MAX_M * FJOFC_MAX_M];
    double wcomm[FJOFC_MAX_M * FJOFC_MAX_M];
    int m, n, nx, d;
    unsigned long long* next_block;
    DevStatus* st;
};
cudaError_t launch_oos_prep(const OOSPrepParams& p, cudaStream_t s);
cudaError_t launch_oos_summary(const int32_t* iters, const double* stress, int64_t k, int32_t* it_out,
                               double* st_out, cudaStream_t s);

}  // namespace fjofc

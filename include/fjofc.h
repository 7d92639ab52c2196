/*
 * fjofc.h -- C ABI of the GB300 (sm_103a) fJOFC library.
 *
 * fJOFC (Lyzinski, Park, Priebe, Trosset: "Fast Embedding for JOFC Using the Raw
 * Stress Criterion") embeds m matched dissimilarity matrices Delta_1..Delta_m on the
 * same n objects into R^d by minimising the JOFC raw stress (Eq. stress) with
 * successive Guttman transforms X_t = L^+ B(X_{t-1}) X_{t-1} (Algorithm 1), where the
 * pseudoinverse is applied in the closed form of Sec. 2.1 / Cor. 1 so that each
 * iteration is X_t^(j) = sum_l [Wmod^-1]_{jl} B_l X_{t-1}^(l) (Eq. update), with B_l the
 * l-th diagonal block of B(X) (Eq. B).  New objects are embedded by the
 * out-of-sample Guttman transform of Sec. 3 (Eq. joosupdate).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them and never keeps them after the call returns.
 *  - Pointers named "host" are ordinary host memory read (or written) during the call.
 *  - Calls are ordered on the CUDA stream passed as `cuda_stream` (a cudaStream_t;
 *    NULL = legacy default stream).  A call enqueues its kernels and then waits for
 *    that stream once, to copy the small result block back; it allocates temporary
 *    device memory with the stream-ordered allocator and releases it on the stream.
 *  - Return value: FJOFC_OK (0) or a negative FJOFC_ERR_* status; fjofc_strerror()
 *    gives a message.  Argument errors are detected before anything is enqueued.
 *  - Floating point: Delta is read as float32 (or float16/bfloat16 scaled by a
 *    per-modality factor), all distance/B(X) arithmetic is float32, stress sums and
 *    the m x m weight algebra are float64.
 *  - At most FJOFC_MAX_M modalities and 1 <= d <= FJOFC_MAX_D.
 *  - Delta row strides (`ld`, in elements) must make each row start on a 16-byte
 *    boundary (ld * element size % 16 == 0) and each Delta base pointer must be
 *    16-byte aligned: the kernels stage Delta tiles with the Tensor Memory
 *    Accelerator, which requires it.
 */
#ifndef FJOFC_H
#define FJOFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FJOFC_MAX_M 32
#define FJOFC_MAX_D 16

/* status codes */
#define FJOFC_OK             0
#define FJOFC_ERR_ARG       -1   /* invalid argument (sizes, weights, pointers, alignment) */
#define FJOFC_ERR_CUDA      -2   /* a CUDA runtime call failed */
#define FJOFC_ERR_NONFINITE -3   /* the stress became NaN/Inf; the last finite iterate is returned */
#define FJOFC_ERR_TIMEOUT   -4   /* a bounded device-side wait gave up (no GPU hang) */
#define FJOFC_ERR_NOMEM     -5   /* temporary device memory could not be allocated */
#define FJOFC_ERR_UNSUPPORTED -6 /* valid but not supported here (e.g. d or m beyond the built range) */

/* element type of Delta */
#define FJOFC_F32  0
#define FJOFC_F16  1
#define FJOFC_BF16 2

/* stopping rule (Algorithm 1, Remark eps).  Iteration continues while the stress
 * DECREASE sigma(X_{t-1}) - sigma(X_t) exceeds the tolerance (the paper prints the
 * difference with the opposite sign, which a descent method never satisfies):
 *   FJOFC_TOL_ABS_NORMALIZED: decrease / C(mn, 2) > tol   (the paper's setting, Remark eps)
 *   FJOFC_TOL_RELATIVE:       decrease / sigma(X_{t-1}) > tol
 * A negative tol disables the test: exactly max_iter transforms are applied. */
#define FJOFC_TOL_ABS_NORMALIZED 0
#define FJOFC_TOL_RELATIVE       1

/* Out-of-sample kernel forms (fjofc_opts.oos_form).  STREAMING: every object is one warp
 * slot of a persistent kernel that streams its dissimilarities from memory every
 * iteration (any m, n, d; built for many objects).  RESIDENT: one CTA per object with
 * -X^T and the object's dissimilarities held in shared memory for all its iterations
 * (d <= 8 and 4 m ceil4(n) (d + 1) <= 200 KB; built for few objects against a small
 * in-sample set); FJOFC_ERR_UNSUPPORTED when it does not fit. */
#define FJOFC_OOS_AUTO 0
#define FJOFC_OOS_STREAMING 1
#define FJOFC_OOS_RESIDENT 2

typedef struct fjofc_opts {
    int32_t max_iter;     /* maximum number of Guttman transforms (>= 0) */
    double  tol;          /* tolerance of the stopping rule; < 0 = run max_iter transforms */
    int32_t tol_mode;     /* FJOFC_TOL_* */
    int32_t profile;      /* 0: no timing.  The loop runs as one persistent cooperative kernel.
                             1: one launch per all-pairs pass (K1) and per W^-1 pass (K2),
                                each timed with CUDA events on cuda_stream (ms_pass, ms_apply).
                             2: the persistent kernel, its launch timed (ms_pass). */
    float   relax;        /* relaxed updates (the Conclusion's suggested acceleration of the
                             majorization): X_t = X_{t-1} + relax (L^+ B(X_{t-1}) X_{t-1} -
                             X_{t-1}).  0 or 1: the plain Guttman transform.  Otherwise in
                             (0, 2]: the stress still does not increase (the relaxed point
                             stays inside the majorizer's level set).  With relax != 1 the
                             iterates are not centred (the oracle's definition: a relaxed
                             iterate keeps (1 - relax) times the previous one's column
                             means).  FJOFC_ERR_ARG outside [0, 2]. */
    int32_t oos_form;     /* fjofc_oos only (other entry points ignore it): FJOFC_OOS_*.
                             FJOFC_OOS_AUTO picks the resident form when it fits and every
                             object gets its own CTA in one wave, else the streaming form. */
    int32_t check_inputs; /* in-sample entry points: 1 = one extra pass over every Delta_i
                             before the loop checks that it is a dissimilarity (Sec. 1.2):
                             every entry finite and >= 0 and Delta[a][b] == Delta[b][a]
                             exactly (the diagonal is not read).  A violation returns
                             FJOFC_ERR_ARG naming the modality and the entry; X is left
                             as given.  0 = no check (the kernels then read only the strict
                             upper triangle, so an asymmetric input is used through it). */
    int32_t deterministic;/* 0 or 1.  Every reduction of every entry point runs in a fixed
                             order (no floating-point atomics), so results are bitwise
                             reproducible run to run on the same GPU model whatever this
                             is set to; the field records the caller's requirement and is
                             checked for a valid value only. */
    int32_t wait_limit_us;/* bound of the in-sample loop's grid-wide waits, microseconds
                             (0 = 2 000 000, i.e. 2 s).  A wait that does not complete in
                             time ends the kernel with FJOFC_ERR_TIMEOUT instead of
                             spinning; X then holds X_0 or an earlier iterate of the call
                             (the loop keeps every third iterate in the caller's buffer),
                             X_0 as given when the first pass timed out. */
    int32_t delta_layout; /* in-sample entry points: FJOFC_LAYOUT_FULL (each Delta_i a whole n x n
                             matrix, row stride ld) or FJOFC_LAYOUT_PACKED (each Delta_i in
                             the packed band layout of fjofc_pack_delta, ld = the packed row
                             stride fjofc_packed_size returns): about half the memory, the same
                             results bit for bit.  check_inputs is not available with it. */
    int32_t reserved[2];  /* must be zero */
} fjofc_opts;

/* Delta storage layouts (fjofc_opts.delta_layout) */
#define FJOFC_LAYOUT_FULL   0
#define FJOFC_LAYOUT_PACKED 1

typedef struct fjofc_result {
    int32_t status;             /* copy of the return value */
    int32_t iters;              /* number of transforms T applied to produce the returned X */
    double  stress;             /* raw stress sigma(X_T) (Eq. stress), float64 */
    double  stress_normalized;  /* sigma(X_T) / C(mn, 2) (Remark eps) */
    double* stress_history;     /* host, caller-owned, length >= max_iter + 1, or NULL:
                                   receives sigma(X_0) .. sigma(X_T) */
    float   ms_total;           /* device time of the call, milliseconds (CUDA events) */
    /* filled when opts->profile != 0 (else 0): */
    int32_t passes;             /* all-pairs passes that did work (= iters + 1) */
    float   ms_pass;            /* profile 1: summed device time of those all-pairs passes (K1);
                                   profile 2: device time of the persistent loop kernel */
    float   ms_apply;           /* profile 1: summed device time of the matching W^-1 passes */
    int32_t launches;           /* kernels this call launched */
} fjofc_result;

/*
 * fjofc_embed -- in-sample fJOFC (Algorithm 2's loop from a given X_0).
 *
 *  m, n, d      : modalities (1..FJOFC_MAX_M), objects (>= 2), embedding dimension
 *                 (1..FJOFC_MAX_D).
 *  delta        : host array of m DEVICE pointers; delta[i] is Delta_{i+1}, an n x n
 *                 row-major matrix with row stride `ld` elements (ld >= n) of element
 *                 type `delta_dtype`.  Delta must be symmetric with finite non-negative
 *                 entries (the dissimilarities of Sec. 1.2); the kernels read only the
 *                 strictly upper triangle (the diagonal is ignored, Eq. W has w=0 there).
 *  delta_scale  : host array of m float scales, or NULL (= all 1).  The dissimilarity
 *                 used is delta_scale[i] * Delta_i[a][b]; meant for float16/bfloat16
 *                 storage of data whose range needs rescaling.
 *  weights      : host m x m row-major float64 matrix of Eq. (W2): w_ii > 0 is the
 *                 fidelity weight of modality i, w_ij = w_ji >= 0 (i != j) the
 *                 commensurability weight of matched pairs across modalities i and j.
 *                 Eq. (W) is w_ii = 1, w_ij = w.
 *  X            : DEVICE float32 (m*n) x d row-major, rows modality-major (the n rows of
 *                 X^(1), then X^(2), ...), 16-byte aligned.  In: X_0.  Out: the final
 *                 iterate X_T, with each modality block's column means removed (Guttman
 *                 outputs are centred in exact arithmetic, Sec. 1.2.2; not with
 *                 relaxed updates, see opts.relax).  X_0 itself is used as given (its
 *                 stress is that of the uncentred input).
 *  opts, res    : host; see above.  res may be NULL.
 *  cuda_stream  : cudaStream_t.
 *
 * Errors: FJOFC_ERR_ARG (sizes, NULL pointers, w_ii <= 0, w_ij < 0, asymmetric
 * weights, misaligned Delta), FJOFC_ERR_UNSUPPORTED (d or m beyond the built range),
 * FJOFC_ERR_NONFINITE (X holds the last iterate whose stress was finite),
 * FJOFC_ERR_TIMEOUT, FJOFC_ERR_NOMEM, FJOFC_ERR_CUDA.  Reaching max_iter is not an
 * error.
 */
int fjofc_embed(int32_t m, int64_t n, int32_t d,
                const void* const* delta, int64_t ld, int32_t delta_dtype,
                const float* delta_scale, const double* weights,
                float* X, const fjofc_opts* opts, fjofc_result* res, void* cuda_stream);

/*
 * fjofc_init_cmds -- Algorithm 2's initial configuration X_(0): xi_0 = classical
 * MDS of the average dissimilarity (sum_i Delta_i)/m, centred; for every modality i,
 * xi_i = classical MDS of Delta_i, centred, and X^(i)_(0) = its orthogonal Procrustes fit
 * onto xi_0 (the rotation R minimising ||xi_i R - xi_0||_F; with xi_0' xi_i = U S V',
 * R = V U' -- the printed xi_i U V' is the inverse rotation).  Classical MDS (Torgerson, the
 * initialisation of Algorithm 1): the d leading eigenpairs of -1/2 J D2 J (D2 the elementwise squared
 * dissimilarities), coordinates v_k sqrt(max(lambda_k, 0)), each column's entry of largest
 * magnitude made positive.  Eigenpairs by subspace iteration on the device (one pass over
 * Delta per iteration, p = min(2d + 4, n) vectors) until the d leading Ritz values change
 * by less than opts->tol (relative).
 *
 *  m, n, d, delta, ld, delta_dtype, delta_scale : as in fjofc_embed.
 *  X          : DEVICE float32 (m*n) x d, 16-byte aligned; out: X_(0), rows modality-major.
 *  opts       : host, may be NULL (max_iter 200, tol 1e-6); max_iter <= 0 and tol <= 0
 *               select those defaults; reserved must be zero.
 *  iters_out  : host array of m + 1 ints or NULL: subspace iterations of the average's and
 *               of every modality's eigenproblem.
 *  cuda_stream: cudaStream_t.  Synchronises the stream (the small eigenproblems are solved
 *               on the host between device passes); allocates its scratch with the
 *               stream-ordered allocator.
 * Errors as fjofc_embed (FJOFC_ERR_ARG for invalid arguments).
 */
typedef struct fjofc_init_opts {
    int32_t max_iter;     /* subspace iterations per eigenproblem (<= 0: 200) */
    double  tol;          /* relative change of the d leading Ritz values to stop (<= 0: 1e-6) */
    int32_t reserved[4];  /* must be zero */
} fjofc_init_opts;

int fjofc_init_cmds(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld, int32_t delta_dtype,
                    const float* delta_scale, float* X, const fjofc_init_opts* opts, int32_t* iters_out,
                    void* cuda_stream);

/*
 * fjofc_stress -- the raw stress sigma(X) of Eq. (stress) for a configuration X, by the
 * same all-pairs pass (fidelity over the upper triangle of each Delta_i, Remark
 * faststress) plus the commensurability term.  Arguments as in fjofc_embed; X is
 * read only.  *stress_out (host) receives sigma(X).
 */
int fjofc_stress(int32_t m, int64_t n, int32_t d,
                 const void* const* delta, int64_t ld, int32_t delta_dtype,
                 const float* delta_scale, const double* weights,
                 const float* X, double* stress_out, void* cuda_stream);

/*
 * fjofc_oos -- out-of-sample embedding of k new objects (Sec. 3, Eq. joosupdate),
 * each an independent problem against the fixed in-sample configuration X.
 *
 *  X          : DEVICE float32 (m*n) x d in-sample configuration (read only).
 *  delta_new  : DEVICE k x m x n dissimilarities, element type `delta_dtype`, row
 *               stride `ld` elements (ld >= n, 16-byte aligned rows): delta_new[o][j][:]
 *               holds delta_j of new object o to the n in-sample objects of modality j.
 *  weights    : host m x m float64 as in fjofc_embed (fidelity w_jj towards the
 *               in-sample points of modality j, commensurability w_ij between the new
 *               object's m points).
 *  Y          : DEVICE float32 k x m x d.  In: y_0 per object.  Out: final y per object.
 *  iters_out  : DEVICE int32[k] or NULL: transforms applied per object.
 *  stress_out : DEVICE float64[k] or NULL: final out-of-sample stress (Eq. joos).
 *  opts       : max_iter and the stopping rule, applied per object; the normalised
 *               mode divides by the number of weighted terms m*n + C(m,2).  oos_form
 *               picks the kernel form (FJOFC_OOS_*); both give the same results up to
 *               float32 summation order.
 *  res        : res->iters receives the largest per-object count, res->stress the sum
 *               of the final stresses.  May be NULL.
 */
int fjofc_oos(int32_t m, int64_t n, int32_t d, int64_t k,
              const float* X, const void* delta_new, int64_t ld, int32_t delta_dtype,
              const float* delta_scale, const double* weights,
              float* Y, int32_t* iters_out, double* stress_out,
              const fjofc_opts* opts, fjofc_result* res, void* cuda_stream);

/*
 * fjofc_embed_noalloc -- fjofc_embed without any allocation at call time.
 *
 * Some callers cannot allocate device memory while they run: real-time or embedded
 * loops that must not enter an allocator (CUDA's or a framework's caching allocator)
 * once start-up is over, processes whose device memory was carved up once at launch by
 * another component, and code that must not fail part-way for lack of memory.  This
 * entry point takes exactly the arguments of fjofc_embed and works in the caller's
 * buffers plus one fixed device array of FJOFC_NOALLOC_SCRATCH_BYTES inside the library
 * (the paper has no counterpart: this is a deployment variant of the same
 * computation).  It calls no cudaMalloc, cudaFree, stream-ordered allocator, event
 * creation or host heap allocation.  Like fjofc_embed it launches kernels and then
 * synchronises cuda_stream, so it is called from ordinary host code (not from a host
 * callback such as cudaLaunchHostFunc, where CUDA calls are not allowed).
 *
 *  - The array is part of the library's device code: every GPU on which that code is
 *    loaded holds it until the process exits.
 *  - The first call on a device looks up the array's device address on that device
 *    (cudaGetSymbolAddress) and caches it; with CUDA's lazy module loading (the default
 *    since CUDA 12.2) that first call, and the first launch of each kernel it uses, also
 *    load the library's device code, which does allocate.  So make one call per device
 *    at start-up, before the period in which nothing may allocate, and before any
 *    stream capture on the device (or set CUDA_MODULE_LOADING=EAGER so that the device
 *    code is loaded when the context is created).
 *  - Calls share the array: two calls that overlap on the GPU (different streams, or
 *    different host threads on the same device) race and corrupt each other's results.
 *    Serialise them.  Each call clears what must start at zero.
 *  - A problem whose scratch does not fit is rejected with FJOFC_ERR_UNSUPPORTED and a
 *    message naming the bytes it would need.  The scratch is, per call: the column
 *    partials, 4 d CW bytes per all-pairs sub-tile, about 2 m d n^2 / RB bytes (RB = CW =
 *    128 for d <= 4, 64 x 128 for d = 5-6, smaller beyond); two iterate buffers of 4 m n d
 *    bytes each; 8 (max_iter + 2) bytes of stress history; and tables of about
 *    4 m n d + (m + 1) d n / 2 bytes.  At m = 2, d = 3, float32 Delta that allows n up to
 *    12800 with max_iter = 200 (12416 with max_iter = 100000).
 *  - opts->profile must be 0; res->ms_total and the profiling fields are returned as 0;
 *    res->stress_history, when given, receives max_iter + 1 entries (those past iters
 *    are 0).
 * Otherwise the results are those of fjofc_embed on the same inputs.
 */
#define FJOFC_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int fjofc_embed_noalloc(int32_t m, int64_t n, int32_t d,
                        const void* const* delta, int64_t ld, int32_t delta_dtype,
                        const float* delta_scale, const double* weights,
                        float* X, const fjofc_opts* opts, fjofc_result* res, void* cuda_stream);

/*
 * fjofc_transform_rows -- one Guttman transform (Eq. update) for the objects [r0, r1) of
 * every modality: the building block of row-block sharding across GPUs.  The mix
 * X_t^(j)_i = sum_l [Wmod^-1]_{jl} (B_l X^(l))_i of Eq. (update) / Cor. 1 is per object,
 * and (B_l X^(l))_i needs only row i of Delta_l (Eq. B) and the whole X_{t-1}; so a GPU
 * holding rows [r0, r1) of every Delta_l computes those rows of X_t, and the GPUs then
 * all-gather X_t and add up the parts below before the next transform.
 *
 *  m, n, d      : as fjofc_embed; 0 <= r0 < r1 <= n.
 *  delta_rows   : host array of m DEVICE pointers; delta_rows[l] holds rows r0..r1-1 of
 *                 Delta_{l+1} (all n columns), row stride ld >= n, element type delta_dtype,
 *                 used as delta_scale[l] * value (delta_scale may be NULL).  Delta must be
 *                 symmetric: a row is used whole (both triangles), once from each side.
 *  weights      : host m x m float64, as fjofc_embed.
 *  X            : DEVICE float32 (m n) x d: the whole X_{t-1} (read only).
 *  mu           : host m x d float64 or NULL: column means subtracted from X_{t-1}^(j) before
 *                 use (the centring of the previous transform's output; NULL = 0).
 *  Xout         : DEVICE float32 m x (r1 - r0) x d: rows [r0, r1) of X_t, modality-major.
 *  parts        : host float64[2 + m d] out: [0] the range's share of the fidelity term of
 *                 sigma(X_{t-1}) (sum over its objects i of w_ll sum_{j != i}
 *                 (Delta_l,ij - d_ij)^2 / 2), [1] the commensurability of its objects
 *                 (sum_{j<l} w_jl ||x_i^(j) - x_i^(l)||^2), [2 + j d + k] the column sums of its
 *                 X_t^(j) rows.  Summed over ranges that cover [0, n): sigma(X_{t-1}) =
 *                 parts[0] + parts[1], and n times the means of X_t.
 * Float32 distances and sums, float-float group sums, float64 parts.  Allocates its small
 * scratch with the stream-ordered allocator; synchronises the stream.  Errors as
 * fjofc_embed.
 */
int fjofc_transform_rows(int32_t m, int64_t n, int32_t d, int64_t r0, int64_t r1, const void* const* delta_rows,
                         int64_t ld, int32_t delta_dtype, const float* delta_scale, const double* weights,
                         const float* X, const double* mu, float* Xout, double* parts, void* cuda_stream);

/* ------------------------------------------------------------------------------------
 * Batched in-sample embedding (the paper has no counterpart: a deployment form that
 * runs many independent fJOFC problems, Algorithm 1 with Eq. update each, of uneven
 * size together).  A plan fixes the problems' pointers, sizes, weights and the loop
 * options (the same fjofc_opts for every problem; profile must be 0) and captures the
 * whole computation into one CUDA graph: a per-problem set-up kernel, one cooperative
 * launch per (d, delta_dtype) class in which every SM runs its list of problems (large
 * problems on groups of SMs of their own), and a result gather.  fjofc_plan_run
 * re-runs it from the current contents of every X (in X_0, out the returned X_T, as
 * fjofc_embed).  Results are per problem, with the same status codes as fjofc_embed.
 * The plan owns one device allocation (cudaMalloc) until fjofc_plan_destroy; Delta and
 * X stay owned by the caller and must outlive the plan.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int32_t m;                  /* modalities, 1..FJOFC_MAX_M */
    int64_t n;                  /* objects, >= 2 */
    int32_t d;                  /* embedding dimension, 1..FJOFC_MAX_D */
    const void* const* delta;   /* m device pointers to n x n Delta (as fjofc_embed); the
                                   host array is read by fjofc_plan_create only */
    int64_t ld;                 /* row stride of Delta in elements */
    int32_t delta_dtype;        /* FJOFC_F32 / FJOFC_F16 / FJOFC_BF16 */
    const float* delta_scale;   /* m host scales or NULL (read at create) */
    const double* weights;      /* m x m host weights (read at create) */
    float* X;                   /* device (m n) x d, in X_0, out X_T */
} fjofc_problem;

typedef struct fjofc_plan fjofc_plan;

/* Validates every problem (FJOFC_ERR_ARG / _UNSUPPORTED as fjofc_embed), schedules and
 * captures the plan; *plan receives it (NULL on error). */
int fjofc_plan_create(const fjofc_problem* problems, int32_t count, const fjofc_opts* opts, fjofc_plan** plan);

/* Enqueues the captured plan on the stream (no synchronisation). */
int fjofc_plan_run(fjofc_plan* plan, void* cuda_stream);

/* Per-problem results of the last run (host arrays of count entries, each may be NULL):
 * status, iters (T of the returned X_T), stress sigma(X_T).  Synchronises the stream;
 * returns the first non-zero status, else FJOFC_OK. */
int fjofc_plan_results(const fjofc_plan* plan, int32_t* status, int32_t* iters, double* stress, void* cuda_stream);

/* Schedule facts: groups[count] = SMs given to each problem (may be NULL), *graphed = 1
 * when the plan runs as one CUDA graph, *launches = kernels per run. */
int fjofc_plan_info(const fjofc_plan* plan, int32_t* groups, int32_t* graphed, int32_t* launches);

void fjofc_plan_destroy(fjofc_plan* plan);

typedef struct {
    int32_t probe_iters;   /* transforms per timed probe run (<= 0: 8) */
    int32_t allow_f16;     /* 1: float32 Delta may be stored as float16 (scaled by max/2^10) */
    int32_t reserved[6];
} fjofc_tune_opts;

typedef struct {
    float pass_cost;       /* chosen schedule constants (sub-tile units) */
    float barrier_cost;
    int32_t delta_dtype;   /* FJOFC_F16 when the float16 copies won, else -1 (as given) */
    float probe_ms;        /* the winner's probe run */
    int32_t candidates;    /* candidates timed */
    int32_t reserved[3];
} fjofc_tune_result;

/* Autotuned plan: times a probe run (probe_iters transforms) of each candidate -- the
 * schedule's cost constants, which fix how problems are cut into per-SM (problem,
 * sub-tile range) work, and, when allowed, float16 storage of float32 Delta in
 * plan-owned buffers -- and creates the plan of the fastest with opts.  Every problem's
 * X is restored after each probe (X holds X_0 again on return).  result may be NULL. */
int fjofc_plan_autotune(const fjofc_problem* problems, int32_t count, const fjofc_opts* opts,
                        const fjofc_tune_opts* tune, fjofc_plan** plan, fjofc_tune_result* result,
                        void* cuda_stream);

/* ------------------------------------------------------------------------------------
 * Learned warm start for fjofc_oos.  The paper has no counterpart: this is the learned
 * form added beside the method.  A network with two hidden GELU layers
 *     h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), yhat = W3 h2 + b3,
 * gelu(z) = z Phi(z), maps a new object's dissimilarities to in-sample landmarks to a
 * start for the out-of-sample Guttman iterations of Sec. 3, which refine it: either
 * every modality's position (n_out = m d, rows of the k x m x d layout of fjofc_oos) or
 * one shared position yhat in R^d used as y_j(0) = yhat for every j (n_out = d).  Parameters are one flat float32 device vector:
 * W1 (hidden x n_in), b1, W2 (hidden x hidden), b2, W3 (n_out x hidden), b3, matrices
 * row-major.  Inputs x are IEEE binary16 (uint16_t bit patterns), count x n_in
 * row-major; targets and outputs are float32 count x n_out.  All pointers except
 * loss_history/loss/inv_mean are device pointers owned by the caller.  Scratch comes
 * from the stream-ordered allocator.  Errors: FJOFC_ERR_ARG (sizes outside [1, 65536],
 * NULL pointers, bad counts), FJOFC_ERR_NOMEM, FJOFC_ERR_CUDA.
 * ------------------------------------------------------------------------------------ */

/* Number of parameters (floats), or -1 for invalid sizes. */
int64_t fjofc_mlp_param_count(int32_t n_in, int32_t hidden, int32_t n_out);

/* Every weight and bias of a layer ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a
 * counter-based SplitMix64 stream keyed by seed (deterministic). */
int fjofc_mlp_init(float* params, int32_t n_in, int32_t hidden, int32_t n_out, uint64_t seed, void* cuda_stream);

/* Network inputs of k new objects: features[o][j*n_land + t] =
 * binary16(delta_new[o][j][landmarks[t]] * inv_mean[j]); delta_new is the float32
 * (k, m, ld) layout of fjofc_oos; landmarks: n_land device int32 in-sample indices;
 * inv_mean: m host floats (1 / mean of Delta_j). */
int fjofc_mlp_features(int32_t m, int64_t n, int64_t k, const float* delta_new, int64_t ld, const int32_t* landmarks,
                       int32_t n_land, const float* inv_mean, uint16_t* features, void* cuda_stream);

/* y = network(x) for count rows. */
int fjofc_mlp_forward(const float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x,
                      int64_t count, float* y, void* cuda_stream);

/* Gradient (P floats, device) and value (*loss, host, may be NULL) of
 * L = 1/(2 count) sum_o ||network(x_o) - y_o||^2 over 1 <= count <= 8192 rows.
 * Synchronises the stream. */
int fjofc_mlp_gradient(const float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x,
                       const float* y, int64_t count, float* grad, double* loss, void* cuda_stream);

/* The warm start y_j(0) = yhat for every modality: Y[o][j][:] = yhat[o][:] (Y is the
 * k x m x d layout of fjofc_oos). */
int fjofc_mlp_broadcast(int64_t k, int32_t m, int32_t d, const float* yhat, float* Y, void* cuda_stream);

/* Fallback to the standard start: per object o, if s_warm[o] <= s_std[o] (stresses of the
 * two starts, e.g. from fjofc_oos with max_iter = 0) Y[o] = Y_warm[o], else Y[o] keeps
 * the standard start it holds on entry; used[o] (may be NULL) = 1 when the warm start
 * was kept. */
int fjofc_mlp_select(int64_t k, int32_t m, int32_t d, const float* Y_warm, const double* s_warm, const double* s_std,
                     float* Y, int32_t* used, void* cuda_stream);

typedef struct {
    int32_t epochs;      /* passes over the training rows */
    int32_t batch;       /* rows per Adam step (1..8192, <= count); the remainder is dropped */
    float lr;            /* Adam step size (> 0) */
    float beta1, beta2;  /* Adam moment decays; <= 0 selects 0.9 / 0.999 */
    float eps;           /* Adam epsilon; <= 0 selects 1e-8 */
    uint64_t seed;       /* epoch orders: row i -> (a i + c) mod count with gcd(a, count) = 1 */
    int32_t reserved[4];
} fjofc_mlp_train_opts;

/* Adam on L over minibatches, in place on params (Adam moments start at zero).
 * loss_history (host, may be NULL) receives each epoch's mean batch loss; when it is
 * non-NULL the call synchronises the stream. */
int fjofc_mlp_train(float* params, int32_t n_in, int32_t hidden, int32_t n_out, const uint16_t* x, const float* y,
                    int64_t count, const fjofc_mlp_train_opts* opts, float* loss_history, void* cuda_stream);

/*
 * Packed storage of a symmetric Delta (the paper's Delta_i are symmetric, Sec. 1.2, and the
 * all-pairs pass reads each unordered pair once, Remark faststress).  The rows are cut
 * into bands of 128 rows; band b keeps its columns from the diagonal on, [128 b, n), and
 * bands b and nB - 1 - b (nB = ceil(n / 128)) share packed rows side by side, so the
 * packed matrix has ceil(nB / 2) * 128 rows of *ld_out elements (about n (n + 128) / 2
 * elements in all; each band's width rounded up to 16 bytes).
 *
 * fjofc_packed_size: elements of one packed matrix for n objects and element type
 * delta_dtype; *ld_out (may be NULL) receives its row stride.  -1 for invalid arguments.
 * fjofc_pack_delta: writes the packed form of the DEVICE n x n matrix delta (row stride
 * ld, element type delta_dtype) into the DEVICE buffer packed (fjofc_packed_size elements,
 * 16-byte aligned); stream-ordered, no synchronisation.  Padding elements are zero.
 */
int64_t fjofc_packed_size(int64_t n, int32_t delta_dtype, int64_t* ld_out);
int fjofc_pack_delta(int64_t n, const void* delta, int64_t ld, int32_t delta_dtype, void* packed, void* cuda_stream);

/* Test support for the bounded-wait error path (the paper has no counterpart).  The
 * next in-sample loop started by fjofc_embed or fjofc_embed_noalloc in this process
 * expects `extra` more arrivals at the first grid-wide wait of its first pass than its
 * CTAs make, so that wait cannot complete: every CTA gives up after
 * opts->wait_limit_us, waits for its own copies in flight and returns, and the call
 * returns FJOFC_ERR_TIMEOUT with X as given.  The setting is consumed by that one call
 * (later calls run normally); extra <= 0 clears it.  Loops with a single CTA have no
 * grid-wide wait and ignore it. */
void fjofc_test_barrier_skew(int32_t extra);

/* Message for a status code (static string). */
const char* fjofc_strerror(int status);

/* Library version string and the list of compiled embedding dimensions. */
const char* fjofc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FJOFC_H */

/*
 * dm.h -- C ABI of the GB300 (sm_103a) library for implicit distance-matrix
 * products, after Indyk & Silwal, "Faster Linear Algebra for Distance
 * Matrices" (arXiv 2210.15114).
 *
 * Given n points x_1..x_n in R^d (the rows of X) and a block Z of k query
 * columns, the library returns
 *
 *     out = A Z,    A_ij = f(x_i, x_j),
 *
 * for f = ||x - y||_1 (Section 2, Algorithms 1 and 2, Theorem "p=1") or
 * f = ||x - y||_2^2 (Appendix A, Theorem "l2_squared_upper_bound" with the
 * Gram decomposition of Section 1.2).  A is never formed.  A block Z is k
 * independent queries sharing one preprocessing (Lemma "matrixmult").
 *
 * Conventions shared by every call:
 *  - All array arguments are DEVICE pointers (caller-owned, any CUDA
 *    allocation reachable from the context's device) unless the name ends in
 *    _host.  Matrices are row-major with a leading dimension in elements:
 *    X is n x d (ldx >= d), Z is n x k (ldz >= k), out is n x k (ldo >= k).
 *  - Element types: DM_F32 points take F32 queries and give F32 results;
 *    DM_F64 -> F64; DM_I32 points take I32 queries and give INT64 results
 *    (exact: two's-complement arithmetic is exact whenever the true result
 *    fits in int64).
 *  - Every call is asynchronous on the context's stream.  Argument errors are
 *    returned at once.  Errors found on the device (non-finite coordinates,
 *    a bounded wait that ran out, an index check) are latched in the
 *    context's error word and returned by the next dm_sync (dm_prepare and
 *    dm_matmat_host synchronize and return them too).
 *  - n >= 1, d >= 1, k >= 1, n < 2^30 (positions and tile counts are 32-bit).
 *  - A call never reads outside the rows and columns described by its sizes
 *    and leading dimensions.
 */
#ifndef DM_H
#define DM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DM_OK = 0,
    DM_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad leading dimension */
    DM_ERR_UNSUPPORTED = 2,   /* valid call that this build does not handle    */
    DM_ERR_NONFINITE = 3,     /* NaN or Inf among the point coordinates        */
    DM_ERR_OOM = 4,           /* device allocation failed                      */
    DM_ERR_CUDA = 5,          /* CUDA runtime error (launch, copy, device)     */
    DM_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out            */
    DM_ERR_INTERNAL = 7       /* a device-side consistency check failed (an
                                 index out of range was skipped)              */
} dm_status;

typedef enum { DM_F32 = 0, DM_F64 = 1, DM_I32 = 2 } dm_dtype;
/* DM_L1: ||x - y||_1 (Section 2).  DM_L2SQ: ||x - y||_2^2 (Appendix A).
 * DM_TV: total variation of distributions, ||x - y||_1 / 2 (Appendix A,
 * Theorem "tv"; FP32/FP64 only).  DM_LPP: ||x - y||_p^p, 2 <= p <= 16
 * (Appendix A, "General p"; plans from dm_prepare_lpp).  DM_L2_EMBED: the
 * approximate ||x - y||_2 of Appendix A (plans from dm_prepare_l2_embed). */
typedef enum { DM_L1 = 0, DM_L2SQ = 1, DM_TV = 2, DM_LPP = 3, DM_L2_EMBED = 4 } dm_metric;

typedef struct dm_ctx dm_ctx;     /* opaque: device, stream, scratch, error word */
typedef struct dm_plan dm_plan;   /* opaque: one preprocessed point set          */

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is borrowed:
 * the caller keeps it alive for the context's lifetime.  The context owns a
 * scratch arena (grown on demand, reused across calls) and a device error
 * word. */
dm_status dm_create(dm_ctx** ctx, int device, void* cuda_stream);

/* Synchronize the stream and free the context.  Plans and batches made from
 * it may be destroyed before or after it, in any order: while any of them is
 * alive the context's memory is kept, every other call on the context or on
 * its plans and batches returns DM_ERR_INVALID_ARG, and the memory is
 * released with the last of them (the stream is not used again, so it may be
 * gone by then).  Calling dm_destroy twice on one context is an error unless
 * children kept it alive in between. */
void dm_destroy(dm_ctx* ctx);

/* Switch the stream later calls are issued on (borrowed, as in dm_create). */
dm_status dm_set_stream(dm_ctx* ctx, void* cuda_stream);

/* Accumulation order of the l1 query's d per-coordinate contributions
 * (Algorithm 2 sums them over the coordinates).  on = 0 (the default): each
 * contribution is added with a reduction in L2 as soon as it is ready; the
 * order of the d additions of one output element varies from run to run, so
 * results can differ in the last bits between runs.  on = 1: the
 * contributions of coordinate c are added only after all of coordinate c-1,
 * in a fixed order, so repeated runs give identical bits (slower: each
 * coordinate waits for the previous one).  The squared-l2 path and integer
 * data are deterministic in both settings (integer sums are exact). */
dm_status dm_set_deterministic(dm_ctx* ctx, int on);

/* Units that run the two contractions of the squared-l2 product (Appendix
 * A): the reduce [X - mu, 1, s]^T Z (also of squared-l2 gradients and of
 * even-p DM_LPP products) and the apply -2 (X - mu) W of
 * out = s u^T + 1 v^T - 2 (X - mu) W.  Both tensor-core kernels use tcgen05
 * with TF32 operands split as hi + lo and FP32 accumulation (the reduce forms
 * all four partial products in one MMA per K step, its accumulator drained
 * every 32 points into FP32 runs and FP64 sums; the apply three products).
 *   DM_ENGINE_TENSOR_CORES: the reduce for FP32 data with d and k multiples
 *     of 4, d <= 60, k <= 32 and contiguous, 16-byte aligned rows of X and Z;
 *     the apply for FP32 data with d a multiple of 4 up to 32, k <= 32 and
 *     contiguous rows of X; other shapes and types keep the CUDA-core
 *     kernels.
 *   DM_ENGINE_CUDA_CORES: always the CUDA-core kernels.
 *   DM_ENGINE_AUTO (the default): the tensor cores where they measured at
 *     least as fast: the apply when k >= 16 and d k >= 512; the reduce when
 *     k <= 16 or d >= 48.
 * Results agree with the FP64 oracle within the FP32 tolerance either way;
 * the bits differ between engines. */
typedef enum { DM_ENGINE_AUTO = 0, DM_ENGINE_CUDA_CORES = 1, DM_ENGINE_TENSOR_CORES = 2 } dm_engine;
dm_status dm_set_engine(dm_ctx* ctx, dm_engine engine);

/* Preprocess a point set (Algorithm 1, Section 2, for DM_L1; Appendix A for
 * DM_L2SQ).
 *   DM_L1:   every coordinate column of X is sorted ascending with a stable
 *            LSD radix sort; the plan owns the sorted values (d x n) and the
 *            sorting permutation (d x n, int32).  X may be freed afterwards.
 *   DM_L2SQ: the plan records the pointer X (the caller keeps X alive and
 *            unchanged for the plan's lifetime) and the column means mu (a
 *            shift: the product is translation invariant).
 * DM_L1 synchronizes the context's stream once (it reads the digit
 * histograms back to skip radix passes whose digit is constant) and returns
 * DM_ERR_NONFINITE if X holds NaN or Inf; DM_L2SQ is asynchronous and reports
 * non-finite coordinates through dm_sync. */
dm_status dm_prepare(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* X,
                     int64_t n, int64_t d, int64_t ldx, dm_plan** plan);
/* (dm_prepare takes DM_L1, DM_L2SQ and DM_TV; DM_TV plans are l1 plans whose
 * products and gradients are halved.) */

/* ||x - y||_p^p plan, 2 <= p <= 16 (Appendix A, "General p").
 *
 * Even p (the printed query read with the binomial coefficients C(p, t) and
 * the weights y_j, t = 0..p): the plan records X (kept alive by the caller,
 * as for DM_L2SQ) and its column means; dm_matmat forms the moments
 * sum_j y_j (x_j(c) - mu_c)^s, s = 0..p, and evaluates
 * (Ay)_k = sum_c sum_t C(p,t) (-1)^(p-t) (x_k(c) - mu_c)^t M_{c,p-t}.
 * DM_ERR_UNSUPPORTED when d * p exceeds what one reduce launch holds.
 *
 * Odd p, 3 <= p <= 15 (Theorem "odd_p"): the plan is an l1 plan (sorted
 * coordinates, Algorithm 1; X is not kept).  With x~ = x - m_c, m_c the
 * coordinate's median, and for the point at sorted position r inside the tie
 * group a..b, dm_matmat evaluates
 *     sum_j y_j |x~ - x~_j|^p = sum_s C(p, s) x~^(p-s) (L_s - R_s),
 * L_s / R_s the sums of y_j (-x~_j)^s over the strictly smaller / larger
 * values (prefix sums in sorted order, p + 1 per query column).  The result
 * block is written with atomic adds (summation order not fixed).
 *
 * Exact for DM_I32 when the result fits in int64 (wrap-around arithmetic).
 * Both expansions cancel more as p grows; on centred Gaussian data FP32
 * results stayed near 1e-7 relative up to p = 8 (even). */
dm_status dm_prepare_lpp(dm_ctx* ctx, dm_dtype dtype, const void* X, int64_t n, int64_t d,
                         int64_t ldx, int p, dm_plan** plan);

/* Approximate ||x - y||_2 plan (Appendix A, "Approximate Matrix-Vector
 * Query for l2"): the points are mapped by T(x) = G x / (beta m) with
 * beta = sqrt(2/pi) (Theorem "l2embed") and the plan is the l1 plan of the
 * mapped points, so A Z is approximated by B Z with B_ij = ||T x_i - T x_j||_1.
 * G: m x d row-major device matrix (caller-drawn N(0, 1) entries, element
 * type of the plan; only read during this call).  FP32/FP64 only;
 * DM_ERR_UNSUPPORTED when G does not fit in shared memory (m * (d + 1)
 * elements beyond about 200 KB). */
dm_status dm_prepare_l2_embed(dm_ctx* ctx, dm_dtype dtype, const void* X, int64_t n, int64_t d,
                              int64_t ldx, const void* G, int64_t m, dm_plan** plan);

/* Release a plan.  Its device buffers go back to the context, which reuses
 * them for later plans in stream order (no wait; buffers beyond 8 GiB per
 * context are freed).  Work already queued that uses the plan still runs. */
void dm_plan_destroy(dm_plan* plan);

/* out = A z for one query column z (n elements, contiguous) on an l1 plan
 * (Algorithm 2: prefix sums of z and x.z in sorted order, evaluated per
 * point and summed over coordinates).  out has n elements. */
dm_status dm_matvec_l1(dm_plan* plan, const void* z, void* out);

/* out = A z for one query column on a squared-l2 plan (Appendix A:
 * (Az)_i = ||x_i||^2 (1^T z) + (||x||^2)^T z - 2 <x_i, X^T z>, in the mu-shifted
 * frame). */
dm_status dm_matvec_l2sq(dm_plan* plan, const void* z, void* out);

/* out = A Z for a block of k query columns on a plan of either metric
 * (Lemma "matrixmult": k independent queries sharing one preprocessing). */
dm_status dm_matmat(dm_plan* plan, const void* Z, int64_t k, int64_t ldz,
                    void* out, int64_t ldo);

/* Gradient of L = sum_q w_q^T A(X) z_q with respect to the points X, for a
 * plan of either metric (the paper states no gradient; this is the chain rule
 * applied to the definition of A):
 *     G[i, c] = sum_q sum_j (W[i,q] Z[j,q] + Z[i,q] W[j,q]) phi'(x_i(c) - x_j(c)),
 * phi'(t) = sgn(t) for DM_L1, with sgn(0) = 0 (tied coordinates contribute
 * nothing: the symmetric subgradient), phi'(t) = sgn(t) / 2 for DM_TV and
 * phi'(t) = 2t for DM_L2SQ (DM_LPP and DM_L2_EMBED: DM_ERR_UNSUPPORTED).
 *   W, Z: n x k (leading dimensions ldw, ldz >= k), 1 <= k <= 64, element type
 *         of the plan (int32 for DM_I32 plans);
 *   G:    n x d result (ldg >= d), element type of the plan's results (FP32,
 *         FP64, or exact int64 for DM_I32).
 * The l1 gradient runs through the plan's sorted coordinates (Algorithm 1)
 * with prefix sums of w and z in sorted order (as in Algorithm 2), so its X
 * need not be alive; the squared-l2 plan reads its recorded X.  DM_L2SQ
 * returns DM_ERR_UNSUPPORTED where its reduce does not fit (large d * k).
 * Asynchronous on the context's stream; scratch comes from the context. */
dm_status dm_grad(dm_plan* plan, const void* W, int64_t ldw, const void* Z, int64_t ldz,
                  int64_t k, void* G, int64_t ldg);

/* ------------------------------------------------------------- batches
 * Many independent point sets, each with its own block of query vectors,
 * processed as one unit: every run preprocesses every set (Algorithm 1 for
 * DM_L1, the column means for DM_L2SQ) and computes out_s = A_s Z_s for each
 * (Lemma "matrixmult" per set), all replayed from one CUDA graph.
 *
 * dm_batch_create takes host arrays of length nsets: sizes n[s], d[s], k[s],
 * leading dimensions, and DEVICE pointers X[s] (n x d), Z[s] (n x k) and
 * out[s] (n x k; element types as for dm_matmat).  The pointers are baked
 * into the graph: later runs read whatever X[s] and Z[s] hold then, and the
 * buffers must stay alive until dm_batch_destroy.  Creation allocates every
 * plan and scratch buffer, spreads the sets over `lanes` concurrent streams
 * (largest sets first, each to the least loaded lane) and captures the graph.
 * lanes = 0 asks for the autotuner: it captures the batch with 1, 2, 4, 8
 * and 16 lanes, times four replays of each, keeps the fastest (so creation
 * runs the whole batch about 20 times) and remembers the choice for batches
 * of the same shape in this process.  Inside the graph nothing synchronizes:
 * all radix passes run (no histogram read-back) and non-finite coordinates
 * are reported by dm_sync, not by the run.
 *
 * dm_batch_run launches the graph, ordered after earlier work on the
 * context's stream and before later work there (asynchronous).  Runs of one
 * batch must not overlap each other (they share the plans and scratch). */
typedef struct dm_batch dm_batch;

dm_status dm_batch_create(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, int64_t nsets,
                          const int64_t* n, const int64_t* d, const void* const* X,
                          const int64_t* ldx, const int64_t* k, const void* const* Z,
                          const int64_t* ldz, void* const* out, const int64_t* ldo, int lanes,
                          dm_batch** batch);
dm_status dm_batch_run(dm_batch* batch);
/* Number of concurrent lanes the batch runs on (the autotuner's choice when
 * it was created with lanes = 0). */
int dm_batch_lanes(const dm_batch* batch);
/* Synchronize, then free the batch's graph, streams, plans and scratch. */
void dm_batch_destroy(dm_batch* batch);

/* Wait for the context's stream and return (then clear) the first device-side
 * error latched since the last dm_sync. */
dm_status dm_sync(dm_ctx* ctx);

/* ------------------------------------------------- dense tall-skinny products
 * The dense steps of the block Krylov iteration that the paper draws from
 * fast products (Appendix C, Theorems "musco" and "singular_values_system"):
 * projections of a block against the earlier ones, Gram matrices of Cholesky
 * QR, the Rayleigh-Ritz matrix and the Ritz vectors.  FP32 device matrices,
 * row-major with a leading dimension (rows contiguous), n rows in the
 * millions, the other dimensions small; FP32 arithmetic.  Asynchronous on the
 * context's stream.
 *
 * dm_dense_tn: C (m x k, ldc) = alpha A^T B with A n x m (lda), B n x k (ldb).
 *   The rows are split into chunks whose FP32 partial products are added in
 *   FP64 in a fixed order (reproducible); the partials live in the context's
 *   scratch arena.  C must not overlap A or B. */
dm_status dm_dense_tn(dm_ctx* ctx, const float* A, int64_t n, int64_t m, int64_t lda, const float* B,
                      int64_t k, int64_t ldb, float* C, int64_t ldc, float alpha);

/* dm_dense_nn: C (n x k, ldc) = beta C + alpha A T with A n x m (lda) and T
 * m x k (ldt), 1 <= k <= 64 (DM_ERR_UNSUPPORTED beyond); beta = 0 does not
 * read C.  C may be the same block as the one read through beta but must not
 * overlap A or T. */
dm_status dm_dense_nn(dm_ctx* ctx, const float* A, int64_t n, int64_t m, int64_t lda, const float* T,
                      int64_t k, int64_t ldt, float* C, int64_t ldc, float alpha, float beta);

/* Rounds a device-side wait of this context's kernels may spin before it
 * gives up (the radix passes' decoupled look-back over earlier tiles of a
 * column, Algorithm 1's sort; the ordered mode of the l1 query waiting for
 * the previous coordinate).  A wait that runs out latches DM_ERR_TIMEOUT for
 * dm_sync and lets its kernel finish (its results are then wrong); the
 * context stays usable.  rounds = 0 restores the default (2^20 rounds of a
 * short sleep, about a second). */
dm_status dm_set_wait_limit(dm_ctx* ctx, uint32_t rounds);

/* Test hook for the bounded wait (no counterpart in the paper): launches one
 * CTA of a radix pass over a two-tile FP32 column, started as the second
 * tile, so the predecessor it looks back to never publishes its counts.  The
 * CTA gives up after the context's wait limit, latches DM_ERR_TIMEOUT (read
 * it with dm_sync) and returns; it touches only the context's scratch arena.
 * Use a small limit (dm_set_wait_limit) to keep the call short. */
dm_status dm_test_unpublished_wait(dm_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* dm_status_string(dm_status status);

/* Copy a sorted plan's coordinates (d x n, element type of the plan) and
 * sorting permutation (d x n int32; row c lists the point indices in
 * ascending order of coordinate c, ties in index order) into caller device
 * buffers.  Sorted plans: DM_L1, DM_TV, DM_L2_EMBED (the mapped points) and
 * DM_LPP with odd p.  DM_ERR_INVALID_ARG for the others. */
dm_status dm_plan_export(dm_plan* plan, void* sorted_values, int32_t* perm);

/* The plain method: out = A Z with every entry f(x_i, x_j) computed on the
 * fly, O(n^2 (d + k)) work (the paper's naive baseline of Section 4, without
 * materializing A).  Needs d <= 64. */
dm_status dm_bruteforce(dm_ctx* ctx, dm_metric metric, dm_dtype dtype,
                        const void* X, int64_t n, int64_t d, int64_t ldx,
                        const void* Z, int64_t k, int64_t ldz,
                        void* out, int64_t ldo);

/* End to end with HOST buffers: copies X and Z to the device, preprocesses,
 * computes out = A Z, copies out back and synchronizes.  Host buffers may be
 * pageable or pinned (pinned is faster).  Device buffers are taken from the
 * context's device buffers for host calls, grown on demand.
 *
 * Host-to-device copies of calls on one device (any contexts, any threads)
 * cross the host link in the order the calls issue them: a call's copies of
 * X and Z start when the previous call's copies have finished, so that every
 * call's preprocessing starts as soon as its own inputs are in. */
dm_status dm_matmat_host(dm_ctx* ctx, dm_metric metric, dm_dtype dtype,
                         const void* X_host, int64_t n, int64_t d, int64_t ldx,
                         const void* Z_host, int64_t k, int64_t ldz,
                         void* out_host, int64_t ldo);

/* dm_matmat_host without the final wait: the copies, preprocessing, product
 * and copy back are issued on the context's streams and the call returns
 * (for l1 plans after the key histograms have been read back, which waits
 * for the copy of X and the key pass).  out_host holds the result, and
 * device-side errors are reported, after the next dm_sync(ctx).  X_host,
 * Z_host and out_host must stay allocated, and X_host and Z_host unchanged,
 * until then; with pageable buffers the copies are synchronous, so pinned
 * buffers are the useful case.  Issuing the calls of several contexts one
 * after the other from one thread and then calling dm_sync on each runs
 * them concurrently, their copies in issue order.  A later host call on the
 * same context waits for this call's copy of Z. */
dm_status dm_matmat_host_async(dm_ctx* ctx, dm_metric metric, dm_dtype dtype,
                               const void* X_host, int64_t n, int64_t d, int64_t ldx,
                               const void* Z_host, int64_t k, int64_t ldz,
                               void* out_host, int64_t ldo);

/* Several products of the same points and queries end to end with HOST
 * buffers: out_host[i] = A_i Z for the distance matrix A_i of metrics[i]
 * (DM_L1 or DM_L2SQ; 1 <= count <= 8), each out_host[i] an n x k buffer with
 * leading dimension ldo.  X and Z cross the host link once (in the device's
 * link order, as for dm_matmat_host); each product is preprocessed and
 * computed on a context of its own (this one for the first, internal peer
 * contexts with their own streams and scratch for the others, created on
 * first use and released with this context), so the products run side by
 * side, and each result is copied back as soon as it is done.  Returns when
 * every result is in place; the first error of any product is returned.
 * The context's settings (dm_set_deterministic, dm_set_wait_limit,
 * dm_set_engine) apply to every product. */
dm_status dm_matmat_host_multi(dm_ctx* ctx, int count, const dm_metric* metrics, dm_dtype dtype,
                               const void* X_host, int64_t n, int64_t d, int64_t ldx,
                               const void* Z_host, int64_t k, int64_t ldz,
                               void* const* out_host, int64_t ldo);

/* Number of kernels this context has launched so far (all calls). */
int64_t dm_launch_count(const dm_ctx* ctx);

/* Kernel timing.  While enabled, every group of launches a call makes
 * ("sort_keygen_hist", "sort_onesweep", "l1_rowsum", "l1_prologue",
 * "l1_aggregate", "l1_query", "l1_finalize", "l2_prepare", "l2_reduce",
 * "l2_apply", "bruteforce", "grad_pack", "grad_l1_tiles", "grad_l1_scan",
 * "grad_l1_eval", "grad_l1_transpose", "grad_l2_reduce", "grad_l2_apply",
 * "tv_scale", "lpp_features", "lpp_reduce", "lpp_apply", "lpp_odd_tiles",
 * "lpp_odd_scan", "lpp_odd_eval", "l2_embed_project") is
 * bracketed by two CUDA events
 * recorded on the context's stream.  Enabling (or disabling) clears what was
 * collected.  Off by default; costs two event records per group. */
dm_status dm_profile_enable(dm_ctx* ctx, int enable);

/* Resolve the recorded events (synchronizes the stream) and report, for up to
 * `max` groups, the name (NUL-terminated, 32 bytes per slot of `names`), the
 * number of kernel launches and their total device time in milliseconds.
 * *count receives the number of groups filled in. */
dm_status dm_profile_read(dm_ctx* ctx, int max, int* count, char* names,
                          int64_t* launches, double* total_ms);

/* out = A Z for the squared-l2 metric (the same product as dm_prepare with
 * DM_L2SQ followed by dm_matmat) for callers that cannot allocate device
 * memory when they call in -- code running inside a memory pool or arena it
 * does not own, or on a path where an allocation (which can synchronize the
 * device) is not allowed.  The paper has no counterpart: this is an
 * interface variant only.
 *   - Needs no context and allocates nothing (no cudaMalloc / cudaFree, no
 *     allocating library call).  Its scratch is one file-scope device array
 *     of a little under 3 MiB that every GPU loading this library holds
 *     until the process exits.
 *   - Limits: 1 <= d <= 32 and 1 <= k <= 32 (larger sizes return
 *     DM_ERR_UNSUPPORTED before any work), n < 2^30; X, Z, out are device
 *     pointers as in the other calls; the work is issued on cuda_stream on
 *     the current device.
 *   - The first call on a device looks up the scratch's device address once
 *     (with that device current); make that first call before any stream
 *     capture.
 *   - Every call shares the one scratch array and it keeps the last call's
 *     contents (nothing in it needs to start at zero).  Calls that overlap on
 *     the GPU -- on different streams, or from different host threads --
 *     race on it and give wrong results: order them.
 *   - Non-finite coordinates are not reported (there is no error word); the
 *     result is then non-finite.  Launch failures return DM_ERR_CUDA. */
dm_status dm_l2sq_matmat_noalloc(dm_dtype dtype, const void* X, int64_t n, int64_t d,
                                 int64_t ldx, const void* Z, int64_t k, int64_t ldz,
                                 void* out, int64_t ldo, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DM_H */

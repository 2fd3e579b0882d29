/*
 * pod.h -- C ABI of the GB300 iterative sampling-and-merging POD library.
 *
 * The library computes the dominant left singular vectors (POD modes) and
 * singular values of a tall m x n snapshot matrix A (column j = snapshot j,
 * rows mean-centred by the caller) with the iterative sampling-and-merging
 * algorithm ISMA of Charumathi, Ramakrishna and Vasudevan, arXiv 1905.05107:
 * Algorithm 1 (sampling loop, GET UPDATE, SAMPLE AND SCALE UNIQUE ROWS),
 * Algorithm 2 (BLOCK MERGE, Eqs. 8-9) and the closing refinement
 * QR(A^T U), SVD(R) of Algorithm 1.
 *
 * Conventions shared by every entry point:
 *  - Matrices are column-major.  A is m x n with leading dimension lda >= m;
 *    U-type outputs are m x k with leading dimension m.
 *  - Pointers named *_dev are device pointers on the current CUDA device;
 *    pointers named *_host are host pointers.  The library never frees or
 *    keeps caller pointers beyond what each entry point documents.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is ordered on that stream; only calls documented as
 *    synchronising wait for the device.
 *  - Every entry point returns a pod_status and never aborts the process.
 *    After POD_ECUDA, POD_ETIMEOUT, POD_ENAN or POD_ERANK from a context
 *    call the context is poisoned: pod_destroy and the host-only queries
 *    (pod_counters, pod_row_draws) stay valid, every other call returns
 *    POD_ESTATE.
 */
#ifndef POD_GB300_H
#define POD_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define POD_API __attribute__((visibility("default")))
#else
#define POD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pod_status {
    POD_OK = 0,
    POD_EINVAL = 1,       /* an argument is out of range or inconsistent    */
    POD_ENOMEM = 2,       /* device or host allocation failed               */
    POD_ECUDA = 3,        /* a CUDA runtime call failed                     */
    POD_ERANK = 4,        /* Cholesky breakdown that shifting did not cure  */
    POD_ETIMEOUT = 5,     /* a bounded device wait gave up                  */
    POD_ENAN = 6,         /* a non-finite value reached the core            */
    POD_ESTATE = 7,       /* call not valid in the context's current state  */
    POD_EUNSUPPORTED = 8  /* size or option combination not built           */
} pod_status;

/* storage type of A and of the modes */
enum { POD_F32 = 0, POD_F64 = 1 };
/* column strategy after round 0 (Sec. 3.1; round 0 is always L2N, Eq. 2) */
enum { POD_L2N = 0, POD_UNF = 1, POD_ORT = 2 };
/* row strategy for ICRS (Sec. 3.1): L2 norms of D's rows, or leverage scores */
enum { POD_ROW_L2N = 0, POD_ROW_LS = 1 };
/* convergence criterion (Algorithm 1): principal angles, or mode cosines */
enum { POD_SUBSPACE = 0, POD_MODES = 1 };
/* arithmetic of the core SVD of E (Algorithm 2):
 * POD_CORE_AUTO = FP64 for POD_F64 data, FP32 for POD_F32 data */
enum { POD_CORE_AUTO = 0, POD_CORE_F32 = 1, POD_CORE_F64 = 2 };
/* arithmetic of the dense contractions U^T C (BLOCK MERGE's projection of
 * the sampled columns, Algorithm 2) and A^T U (refinement, ORT weights):
 * POD_PREC_F32    FP32 SIMT products, FP64 sums of FP32 partials
 * POD_PREC_TF32X3 tcgen05 tensor cores, split-TF32 products (x = hi + lo
 *                 exactly, three TF32 products hi hi + hi lo + lo hi):
 *                 FP32-level products
 * POD_PREC_BF16X3 tcgen05 tensor cores, split-BF16 products (x ~ b0 + b1,
 *                 b0 = bf16(x), b1 = bf16(x - b0); b0 b0 + b0 b1 + b1 b0):
 *                 about 2^-16 relative per product
 * POD_PREC_BF16   tcgen05 tensor cores, one BF16 product: about 2^-8
 * The tensor-core forms accumulate in FP32 over 64-row groups and in
 * double-float / FP64 across groups; they need FP32 data, m and lda
 * multiples of 4, 16-byte aligned A, r <= 64 (else POD_EUNSUPPORTED).  The
 * residual's second projection (CGS2), the CholeskyQR Grams, the core SVD
 * and the convergence test keep FP32 products with FP64-level sums, so the
 * low-precision U^T C is corrected by the second projection. */
enum { POD_PREC_F32 = 0, POD_PREC_BF16 = 1, POD_PREC_BF16X3 = 2, POD_PREC_TF32X3 = 3 };

/*
 * Parameters of one POD problem; mirrors ISMA's inputs (A, p, k, c, w, r,
 * tau, rows) in Algorithm 1.
 */
typedef struct pod_params {
    int64_t m, n, lda;     /* A is m x n, column-major, lda >= m             */
    int32_t k;             /* modes wanted, 1 <= k <= min(m, n)              */
    int32_t c;             /* column draws per iteration (with replacement)  */
    int32_t w;             /* row draws per iteration when rows = 1; 0 ->
                              Eq. 5 with epsilon = delta = 0.6, at most m    */
    int32_t r;             /* carried rank after each merge; 0 -> k; r >= k  */
    int32_t rows;          /* 0 = columns only (ICS), 1 = columns+rows (ICRS):
                              the new block is C = D V_r, V_r the top r right
                              singular vectors of the scaled row sample W of
                              D (GET UPDATE with rows, SAMPLE AND SCALE
                              UNIQUE ROWS)                                  */
    int32_t col_strategy;  /* POD_L2N | POD_UNF | POD_ORT                    */
    int32_t row_strategy;  /* POD_ROW_L2N | POD_ROW_LS                       */
    int32_t criterion;     /* POD_SUBSPACE | POD_MODES                       */
    double  tol;           /* subspace: stop when max sin(theta) <= tol;
                              modes: stop when min |cos| >= tol              */
    int32_t max_iter;      /* merges after round 0 (<= 0: until S is empty)  */
    int32_t refine;        /* 1: pod_modes runs QR(A^T U), SVD(R) first      */
    int32_t dtype;         /* POD_F32 | POD_F64                              */
    int32_t core;          /* POD_CORE_AUTO | POD_CORE_F32 | POD_CORE_F64    */
    uint64_t seed;         /* Philox4x32-10 key                              */
    int32_t block_trunc;   /* 1: GET UPDATE truncates the new block to rank r
                              through SVD(D^T D) before the merge (the paper's
                              literal Algorithm 1); 0: D merges directly     */
    int32_t precision;     /* POD_PREC_* (see above); a tensor-core form with
                              FP64 data or an unsupported shape is
                              POD_EUNSUPPORTED                               */
    int32_t keep_tape;     /* 1: record, per round, the basis U_t entering
                              the merge and the merge core (E, its singular
                              values and left vectors, Ptot, R^{-1}) so that
                              pod_backward can run; O(T m r) device memory,
                              grown between batches of rounds; ICS only     */
    int32_t reserved;      /* must be 0                                      */
} pod_params;

typedef struct pod_ctx pod_ctx;

/*
 * pod_init -- create a context for one POD problem (Algorithm 1, "S <- all
 * columns", first GET UPDATE not yet run).
 *   ctx_out : receives the new context (NULL on failure).
 *   p       : parameters, copied.
 *   A_dev   : device pointer to A (dtype p->dtype).  Borrowed: it is read,
 *             never written or freed, and must stay valid and unchanged
 *             until pod_destroy.
 *   stream  : cudaStream_t all work of this context is ordered on.
 * Allocates every device workspace the context needs (O(m r + m c + n c)),
 * computes the column norms of A (Eq. 2 numerators) on `stream`.
 * Errors: POD_EINVAL for inconsistent parameters, POD_ENOMEM, POD_ECUDA.
 */
POD_API pod_status pod_init(pod_ctx **ctx_out, const pod_params *p, const void *A_dev,
                    void *stream);

/*
 * pod_iterate -- run up to max_steps ISMA iterations (round 0 counts as one):
 * probabilities, draws, GET UPDATE, BLOCK MERGE, convergence test
 * (Algorithm 1 while-loop).  Synchronises `stream` at least once.
 *   max_steps : > 0.
 *   done      : (host, may be NULL) 1 once converged, S is empty or
 *               max_iter merges have run.
 *   sin_max   : (host, may be NULL) last max sin(theta) (subspace) or
 *               1 - min |cos| (modes); 1.0 before a comparison exists.
 *   steps_run : (host, may be NULL) iterations actually executed.
 * Errors: POD_ERANK, POD_ENAN, POD_ECUDA, POD_ESTATE (poisoned context).
 */
POD_API pod_status pod_iterate(pod_ctx *ctx, int32_t max_steps, int32_t *done,
                       double *sin_max, int32_t *steps_run);

/*
 * pod_modes -- the k dominant POD modes (Algorithm 1 return values).  When
 * p->refine is 1 the refinement QR(A^T U) = Q R, SVD(R) = U_R S_R V_R^T,
 * U <- U V_R, sigma <- S_R, V <- Q U_R runs first (once; later calls reuse
 * it).  Signs are fixed so that u_i^T z > 0 for the reference vector
 * z_i = int32(Philox(i, 0, 3, 0).x0) / 2^31.
 *   U_dev     : device, m x k, leading dimension m, dtype p->dtype.
 *   sigma_dev : device, k doubles.
 *   V_dev     : device, n x k, leading dimension n, dtype p->dtype, or NULL;
 *               requires refine = 1.
 * Synchronises once (to read the number of modes carried), then enqueues the
 * rest on the stream.  Fewer than k modes exist only if A has numerical rank
 * < k; the missing columns are written as zeros.
 */
POD_API pod_status pod_modes(pod_ctx *ctx, void *U_dev, double *sigma_dev, void *V_dev);

/*
 * pod_get_trace -- the draw set of iteration t (sorted distinct column
 * indices I_c of Algorithm 1, GET UPDATE) and that iteration's convergence
 * measure.  Synchronises `stream`.
 *   idx_host : capacity >= p->c int32, may be NULL; g_host : count written.
 *   measure_host : max sin(theta) (subspace) / 1 - min|cos| (modes), may be NULL.
 * Errors: POD_EINVAL if t has not run yet.
 */
POD_API pod_status pod_get_trace(pod_ctx *ctx, int32_t t, int32_t *idx_host,
                         int32_t *g_host, double *measure_host);

/*
 * pod_wedin -- the quality measure of the converged solution (Sec. 3.3,
 * Eq. 7): with the refined top-k triplets (U~_k, sigma~_k, V~_k),
 * R = A V~_k - U~_k Sigma~_k and S = A^T U~_k - V~_k Sigma~_k, and
 * omega = min(|sigma~_k - sigma~_{k+1}|, sigma~_k) estimated from the carried
 * singular values, out4 (host, 4 doubles) receives
 *   { sqrt(|R|_F^2 + |S|_F^2) / omega, |R|_F, |S|_F, omega }.
 * One extra pass over A (R); S comes from the refinement's A^T U.
 * Needs pod_modes to have run with refine = 1 (else POD_ESTATE) and r >= k + 1
 * carried modes (else POD_EUNSUPPORTED: sigma~_{k+1} does not exist).
 * Allocates its O(n k) workspace for the call; synchronises the stream.
 * Errors: POD_EINVAL, POD_ESTATE, POD_EUNSUPPORTED, POD_ENOMEM, POD_ECUDA.
 */
POD_API pod_status pod_wedin(pod_ctx *ctx, double *out4);

/*
 * pod_robust_rounds -- how many rounds so far needed the guarded rerun of the
 * first CholeskyQR pass with a compensated Gram (their residual block was too
 * ill-conditioned for an FP32 Gram: the second pass's Gram was not within 0.1
 * of I).  Synchronises.
 */
POD_API pod_status pod_robust_rounds(pod_ctx *ctx, int32_t *robust_rounds);

/*
 * pod_last_rows -- the row sample of the most recent ICRS iteration (SAMPLE
 * AND SCALE UNIQUE ROWS of Algorithm 1): the h distinct rows I_r in
 * ascending order and their draw counts t_hat (sum = w).  Synchronises.
 *   rows_host, counts_host : host arrays of cap entries (each may be NULL).
 *   h                      : (host) receives h; 0 before the first round.
 * Errors: POD_ESTATE when rows = 0, POD_EINVAL when h > cap (h is still
 * written), POD_ECUDA.
 */
POD_API pod_status pod_last_rows(pod_ctx *ctx, int32_t *rows_host, int32_t *counts_host,
                                 int32_t cap, int32_t *h);

/*
 * pod_row_draws -- the number w of row draws per iteration this context
 * uses (p->w, or the Eq. 5 default); 0 when rows = 0.  No GPU work.
 */
POD_API pod_status pod_row_draws(pod_ctx *ctx, int32_t *w);

/*
 * pod_replay_indices -- freeze the draws: iteration t merges exactly the
 * columns idx_host[offsets[t] .. offsets[t+1]) instead of drawing (used to
 * compare runs on identical index sets).  Copies the lists; T iterations
 * are available, after which the run stops as if S were empty.
 * Must be called before the first pod_iterate.
 */
POD_API pod_status pod_replay_indices(pod_ctx *ctx, const int32_t *idx_host,
                              const int32_t *offsets_host, int32_t T);

/*
 * pod_backward -- adjoint of the truncated POD of a finished run, with the
 * run's draws held fixed (the draws are discrete; the derivative is that of
 * the map A -> (U, sigma) for those index sets).  Given dL/dU and dL/dsigma
 * of the k returned modes (pod_modes' outputs, signs included), computes
 * dL/dA: reverse-mode through the closing refinement (the SVD of U^T A) and
 * every merge of Algorithm 2 (the SVD of [U Sigma, D], Eqs. 8-9) using the
 * SVD adjoint with the 1 / (sigma_j^2 - sigma_i^2) coupling (broadened:
 * d / (d^2 + (1e-12 sigma_1^2)^2)), the sampled blocks D re-gathered from A by
 * the recorded indices.
 *   dU_dev     : device, m x k, ld m, dtype.
 *   dsigma_dev : device, k doubles, or NULL (zero).
 *   dA_dev     : device, m x n, ld lda, dtype; overwritten (accumulate = 0)
 *                or added to (accumulate = 1).
 * Needs keep_tape = 1 (else POD_ESTATE) and pod_modes to have run.
 * Allocates O(m r) workspace for the call; synchronises the stream.
 * Errors: POD_EINVAL, POD_ESTATE, POD_EUNSUPPORTED (tape overflow), POD_ENOMEM,
 * POD_ECUDA.
 */
POD_API pod_status pod_backward(pod_ctx *ctx, const void *dU_dev, const double *dsigma_dev,
                        void *dA_dev, int32_t accumulate);

/*
 * pod_reset -- start a new problem of the same shape on an existing context:
 * S <- all columns, U <- empty, column norms of A recomputed (Algorithm 1,
 * first lines).  Keeps every workspace and, when A_dev is NULL or equal to
 * the current matrix, the captured per-round CUDA graph.  A_dev (device,
 * same m, n, lda, dtype; borrowed as in pod_init) replaces the matrix when
 * not NULL.  Frozen draw lists set by pod_replay_indices stay in force.
 * Stream-ordered, does not synchronise.
 */
POD_API pod_status pod_reset(pod_ctx *ctx, const void *A_dev);

/*
 * pod_round_timings -- run the next ISMA round (as pod_iterate with
 * max_steps = 1 would) launch by launch, with a CUDA event recorded on the
 * context's stream after every kernel, and return each kernel's duration in
 * milliseconds in launch order (with ORT: A^T U, ORT values; then
 * probabilities and draws, U^T C, C - U P with U^T Z and Z^T Z, first
 * Cholesky, second CholeskyQR Gram, core SVD, update, end of round).
 * Synchronises.
 *   ms_host : capacity cap floats;  count : entries written.
 */
POD_API pod_status pod_round_timings(pod_ctx *ctx, float *ms_host, int32_t cap, int32_t *count);

/*
 * pod_refine_timings -- run the closing refinement of Algorithm 1 (the step
 * pod_modes runs first when p->refine is 1: Y = A^T U, CholeskyQR2 of Y,
 * SVD(R), U <- U V_R) launch by launch with a CUDA event recorded after
 * every kernel, and return each kernel's duration in milliseconds in launch
 * order: state, A^T U, state, Gram of Y, first Cholesky, state, second
 * CholeskyQR pass, SVD of R, state, U V_R.  A later pod_modes reuses the
 * refinement.  Synchronises.
 *   ms_host : capacity cap floats;  count : entries written.
 * Errors: POD_EINVAL, POD_ESTATE (refine = 0, refinement already run, or a
 * poisoned context), POD_ECUDA, POD_ETIMEOUT.
 */
POD_API pod_status pod_refine_timings(pod_ctx *ctx, float *ms_host, int32_t cap, int32_t *count);

/*
 * pod_counters -- number of kernels this context has launched (graph
 * replays count every kernel node) and ISMA rounds completed as of the last
 * synchronisation.  Host-only, never synchronises.
 */
POD_API pod_status pod_counters(pod_ctx *ctx, int64_t *kernel_launches, int32_t *rounds);

/*
 * pod_core_stats -- diagnostics of the last core SVD of E (Algorithm 2):
 * Jacobi sweeps run, and SM clock cycles spent in its phases
 * (cycles[0] second CholeskyQR factor and E, [1] Jacobi sweeps, [2] top-r
 * vectors and singular values, [3] convergence measure, [4] update
 * coefficients, [5] whole kernel).  Synchronises.  Either pointer may be
 * NULL.
 */
POD_API pod_status pod_core_stats(pod_ctx *ctx, int32_t *sweeps, int64_t *cycles);

/*
 * pod_set_wait_limit -- bound, in polls, of each pipeline wait (on an
 * mbarrier) in this context's tensor-core kernels before the kernel gives up
 * with POD_ETIMEOUT; 0 restores the default of 2^24 polls, far above any
 * wait that can complete.  A small bound makes the waits run out on purpose,
 * so that a caller can check that a kernel gives up cleanly: it records
 * POD_ETIMEOUT, stops issuing work, lets its own copies and tensor-core
 * operations in flight complete (those waits keep the default bound), frees
 * its tensor memory and returns; the call that ran it returns POD_ETIMEOUT
 * and poisons the context.  Applies to launches enqueued after the call
 * (the round graph is captured at the first pod_iterate and keeps the bound
 * it was captured with).  Host only, no GPU work.  The paper has no
 * counterpart: it is a testing aid for the bounded-wait design.
 * Errors: POD_EINVAL (NULL ctx), POD_ESTATE (poisoned context).
 */
POD_API pod_status pod_set_wait_limit(pod_ctx *ctx, uint32_t polls);

/* pod_destroy -- free every workspace of ctx (NULL is a no-op). Synchronises. */
POD_API void pod_destroy(pod_ctx *ctx);

/* pod_strerror -- static description of a status code. */
POD_API const char *pod_strerror(pod_status s);

/* ------------------------------------------------------------------------
 * Step-level entry points (one step of the hot path each; stream-ordered,
 * no synchronisation, scratch allocated and freed inside unless noted).
 * ------------------------------------------------------------------------ */

/*
 * pod_colnorms -- s_j = sum_i a_ij^2 for every column (numerators of the
 * column-norm probabilities, Eq. 2), accumulated with FP64-level accuracy.
 *   A_dev : device, m x n, ld lda, dtype;  s_dev : device, n doubles.
 */
POD_API pod_status pod_colnorms(const void *A_dev, int32_t dtype, int64_t m, int64_t n,
                        int64_t lda, double *s_dev, void *stream);

/*
 * pod_atu -- Y = A^T U, the dense contraction of the closing refinement
 * (Algorithm 1, QR(A^T U)) and of the ORT weights (Eq. 6), as a step.
 *   A_dev : device, m x n column-major (lda), dtype.
 *   U_dev : device, m x r column-major (ld m), dtype.
 *   Y_dev : device, n x r FP64 column-major (ld n), overwritten.
 *   precision : POD_PREC_F32 (FP32 SIMT / FP64 SIMT for FP64 data) or a
 *               tensor-core form POD_PREC_TF32X3 / BF16X3 / BF16 (FP32
 *               data, m and lda multiples of 4, 16-byte aligned A and U,
 *               r <= 64; else POD_EUNSUPPORTED).
 * Allocates its workspace for the call; synchronises the stream.
 * Errors: POD_EINVAL, POD_EUNSUPPORTED, POD_ENOMEM, POD_ECUDA, POD_ETIMEOUT.
 */
POD_API pod_status pod_atu(const void *A_dev, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                           const void *U_dev, int32_t r, double *Y_dev, int32_t precision, void *stream);

/*
 * pod_sample -- draw c column indices with replacement with probability
 * w_j / sum(w) restricted to mask_j != 0 (uniform over the mask if every
 * such weight is 0), keep the sorted distinct draws and clear them from
 * the mask (Algorithm 1, GET UPDATE: I_s, I_c, S <- S \ I_c).  Draw j of
 * iteration t uses Philox4x32-10(counter = (j, t, stream_id, 0),
 * key = seed); v = floor(u * W / 2^64) with u = (x0 << 32) | x1 selects the
 * smallest i whose inclusive prefix sum of weights exceeds v.
 *   w_dev    : device, n uint64 weights with sum < 2^62.
 *   mask_dev : device, n bytes, updated in place.
 *   idx_dev  : device, >= c int32;  g_dev : device int32, distinct count.
 */
POD_API pod_status pod_sample(const uint64_t *w_dev, uint8_t *mask_dev, int64_t n, int32_t c,
                      uint64_t seed, int32_t t, int32_t stream_id, int32_t *idx_dev,
                      int32_t *g_dev, void *stream);

/*
 * pod_incremental -- Algorithm 3 (incremental POD for matrices that do not
 * fit in device memory): A is split into `blocks` column ranges
 * [b n / t, (b + 1) n / t); each range is copied to the device on a side
 * stream while the previous one is processed (two device buffers), ISMA
 * (Algorithm 1 with p's parameters, r modes kept, no refinement) runs on it,
 * and BLOCK MERGE (Algorithm 2) folds its r scaled modes into the running
 * U, Sigma.  One pass over A.
 *   p       : parameters (p->n, p->lda describe the whole host matrix;
 *             keep_tape must be 0).
 *   A_host  : host m x n column-major (lda), dtype; pinned memory lets the
 *             copies overlap the computation.  Borrowed, read only.
 *   U_dev   : device m x k (ld m), the first k modes with the sign
 *             convention of pod_modes; sigma_dev : device k doubles.
 * Allocates two m x ceil(n / t) device buffers and the per-block contexts
 * for the call; synchronises the stream.
 * Errors: as pod_init and pod_iterate; POD_EINVAL for blocks < 1 or > n.
 */
POD_API pod_status pod_incremental(const pod_params *p, const void *A_host, int32_t blocks, void *U_dev,
                                   double *sigma_dev, void *stream);

/*
 * pod_block_merge -- Algorithm 2 (BLOCK MERGE) with the new block given as
 * its scaled left factor C = U_2 Sigma_2 (m x g):
 * U_t = C - U_1 (U_1^T C) (computed twice), U_t = U_o R (CholeskyQR2),
 * E = [[diag(s_1), U_1^T C], [0, R]], E = U_E Sigma_E V_E^T,
 * U = [U_1 U_o] U_E truncated to r and to the non-zero singular values.
 *   U1_dev : device m x r1 (ld m) or NULL when r1 = 0; s1_dev device r1 doubles.
 *   C_dev  : device m x g (ld ldc).
 *   U_out_dev : device m x r (ld m); s_out_dev : device r doubles;
 *   r_out_host : number of modes kept.  dtype applies to U1, C and U_out.
 *   core : POD_CORE_* arithmetic of the core SVD.
 * Synchronises `stream` (to return r_out).
 */
POD_API pod_status pod_block_merge(int32_t dtype, int64_t m, const void *U1_dev,
                           const double *s1_dev, int32_t r1, const void *C_dev,
                           int64_t ldc, int32_t g, int32_t r, int32_t core,
                           void *U_out_dev, double *s_out_dev, int32_t *r_out_host,
                           void *stream);

/*
 * pod_sample_noalloc -- the same draw step as pod_sample (same inputs, same
 * outputs, bit-identical results), for callers that cannot allocate device
 * memory when they draw: processes whose device memory pool is capped or
 * fully reserved by another framework, and latency-critical loops that must
 * not touch the allocator.  It allocates nothing: its scratch lives in fixed
 * arrays compiled into the library, which every GPU that loads the library
 * holds (about 1.1 MB) until the process exits.  It does make CUDA API calls
 * (an address lookup, two copies, a launch), so it must not be called from
 * a host callback (cudaLaunchHostFunc, cudaStreamAddCallback), where CUDA
 * forbids them.  The paper has no counterpart to this entry point.
 *   Limits: n <= 65536 columns and c <= 4096 draws; larger sizes return
 *   POD_EUNSUPPORTED without doing anything.
 *   The first call on each device looks up the arrays' device addresses
 *   (cudaGetSymbolAddress) with that device current; under CUDA's lazy
 *   module loading that lookup is also when the arrays are placed in device
 *   memory, so it can fail with POD_ECUDA where nothing may be allocated.
 *   Make one call per device at set-up, outside any stream capture and
 *   while allocation is still possible.
 *   All calls share the arrays: calls that overlap on the GPU (different
 *   streams or host threads on one device) race and must be serialised by
 *   the caller.  Each call re-initialises the parts it needs.
 * Arguments, layout and errors as pod_sample.  Stream-ordered, does not
 * synchronise.
 */
POD_API pod_status pod_sample_noalloc(const uint64_t *w_dev, uint8_t *mask_dev, int64_t n, int32_t c,
                                      uint64_t seed, int32_t t, int32_t stream_id, int32_t *idx_dev,
                                      int32_t *g_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* POD_GB300_H */

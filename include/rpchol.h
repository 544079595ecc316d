/*
 * rpchol.h -- C ABI of the GB300 (sm_103a) implementation of accelerated
 * randomly pivoted Cholesky (Epperly, Tropp, Webber, arXiv 2410.03969).
 *
 * The library turns a kernel matrix A = K(X, X) that is never formed into a
 * rank-k factor F with A ~= F F^*, by the block rounds of Algorithm 2
 * ("Accelerated RPCholesky: standard implementation", Sec. 2.3):
 *   (a) propose T pivots iid from the residual diagonal d (Algorithm 2,
 *       step 1; Eq. 1.3),
 *   (b) form H = A(S',S') - F(S',:) F(S',:)^* and thin the proposals with
 *       RejectionSampleSubmatrix (Algorithm 1, Sec. 2.2),
 *   (c) G = (A(:,S) - F F(S,:)^*) L^{-*}, F <- [F G] (Algorithm 2, step 3),
 *   (d) d <- max(d - rowsumsq(G), 0) (Algorithm 2, last two lines).
 * Simple RPCholesky (Algorithm 6, appendix) is provided as the GPU baseline.
 * Every step runs in the library's own CUDA kernels; there is no CPU path.
 *
 * Conventions shared by every entry point:
 *   - Status codes only; nothing throws or aborts across this boundary.
 *     rpchol_last_error() returns a thread-local description of the last
 *     failure on the calling thread.
 *   - Device memory is owned by the library (allocated at create, released
 *     at destroy) through the allocator given in rpchol_opts, or
 *     cudaMallocAsync/cudaFreeAsync on the context's stream when none is
 *     given.
 *   - Every call that launches work is asynchronous on the context's
 *     stream, unless stated otherwise.  A context must not be used from two
 *     threads at once.
 *   - Points X are row-major N x d (the paper's d x N column matrix
 *     X = [x_1 ... x_N] of App. A.1, stored point by point).
 *   - The factor F is row-major N x ldF (ldF >= k_max, a multiple of 32);
 *     column j holds the j-th accepted pivot's column; columns >= rank are
 *     unspecified.  Pivots are 0-based row indices (int64).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed low 32 bits, seed high 32 bits); round r, proposal slot j of
 *     instance m uses counter (j, r, 0, m); words (w0,w1) give the proposal
 *     uniform, (w2,w3) the acceptance uniform, each as
 *     ((w_a >> 5) 2^26 + (w_b >> 6)) 2^-53.  Simple RPCholesky step i uses
 *     counter (0, i, 0, m), words (w0,w1).
 */
#ifndef RPCHOL_H
#define RPCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RPCHOL_OK = 0,
    RPCHOL_EINVAL = 1,     /* invalid argument; nothing was launched */
    RPCHOL_ENOMEM = 2,     /* device or host allocation failed */
    RPCHOL_ECUDA = 3,      /* a CUDA runtime call failed; see rpchol_last_error */
    RPCHOL_ETIMEOUT = 4,   /* round limit reached or a bounded device wait expired */
    RPCHOL_EBUSY = 5,      /* resource in use (server slots, budget) */
    RPCHOL_ECANCELLED = 6, /* job cancelled before it ran */
    RPCHOL_ENUMERIC = 7    /* non-finite value or non-positive pivot met on the device */
} rpchol_status;

/* kappa(x, y) = phi(r), r = ||x - y||_2 (r1 = ||x - y||_1 for LAPLACE_L1),
 * phi(0) = 1 so diag A = 1.
 *   GAUSSIAN    exp(-r^2 / (2 sigma^2))                     (Sec. 1.2)
 *   LAPLACE_L2  exp(-r / sigma)
 *   MATERN52    (1 + sqrt5 r/sigma + 5 r^2/(3 sigma^2)) exp(-sqrt5 r/sigma)
 *                                                           (Sec. 3.2)
 *   MATERN32    (1 + sqrt3 r/sigma) exp(-sqrt3 r/sigma)     (named in Sec. 4's
 *                                         testbed; the formula is the textbook one)
 *   LAPLACE_L1  exp(-r1 / sigma)                            (Sec. 1.2)
 * LAPLACE_L1 has no inner-product form: its column step runs on CUDA cores
 * (in mixed mode too), the others use the tensor-core step in mixed mode.  */
typedef enum {
    RPCHOL_GAUSSIAN = 0,
    RPCHOL_LAPLACE_L2 = 1,
    RPCHOL_MATERN52 = 2,
    RPCHOL_MATERN32 = 3,
    RPCHOL_LAPLACE_L1 = 4
} rpchol_kernel_kind;

/* FP64: every step in IEEE double (parity mode).
 * MIXED: F stored in FP32; the kernel-column and Schur contractions run in
 * single-precision arithmetic with FP32 accumulation (compensated split
 * products on the tensor-core path); H is stored in FP64, its F(S',:) F(S',:)^*
 * part summed as float pairs (about 48 significant bits); the T x T
 * rejection-sampling Cholesky, L^{-1} and the residual-diagonal
 * accumulation stay in FP64.                                               */
typedef enum { RPCHOL_FP64 = 0, RPCHOL_MIXED = 1 } rpchol_precision;

typedef enum { RPCHOL_DT_F32 = 0, RPCHOL_DT_F64 = 1 } rpchol_dtype;

typedef void* (*rpchol_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*rpchol_free_fn)(void* ptr, void* stream, void* user);

typedef struct {
    int32_t precision;       /* rpchol_precision */
    int32_t use_graph;       /* 1: round loop as a CUDA graph with a device-side
                                while-condition (default); 0: host loop */
    uint32_t instance;       /* Philox counter word 3 (independent streams) */
    int32_t profile;         /* 1: host-driven loop with CUDA events around every
                                kernel phase on the context's stream; the per-phase
                                times appear in rpchol_run_stats (slower: one
                                launch per kernel instead of one graph) */
    void* stream;            /* cudaStream_t; NULL = legacy default stream */
    rpchol_alloc_fn dev_alloc; /* optional device allocator (e.g. torch's) */
    rpchol_free_fn dev_free;
    void* alloc_user;
} rpchol_opts;

typedef struct {
    int64_t rank;            /* columns of F produced by the last run */
    int64_t rounds;          /* rounds (accelerated) or steps (simple) */
    int64_t proposals;       /* pivots proposed in total */
    int64_t accepted;        /* pivots accepted (== rank) */
    int32_t status;          /* rpchol_status of the last run's device work */
    int32_t plain;           /* algorithm of the last run: 0 accelerated, 1 simple
                                RPCholesky, 2 block RPCholesky */
    double residual_trace;   /* sum of the clamped residual diagonal d */
    double trace_error;      /* tr(A - F F^*) / tr(A) from F itself, FP64
                                accumulation (filled by rpchol_stats) */
    double col_bytes;        /* algorithmic bytes of the column-step kernel(s) of
                                the run: per round N (rank b_F + s b_F + 4 d + 16),
                                b_F the bytes of one F element; for simple
                                RPCholesky the GEMV's N (i b_F + b_F + 4 d + 16) */
    double col_flops;        /* algorithmic flops of the same kernel(s): per round
                                2 N rank s + N s^2 + 3 N d s */
    double phase_ms[8];      /* profile mode: summed CUDA-event time per phase:
                                0 propose, 1 H, 2 Algorithm 1, 3 operand prep,
                                4 column step, 5 round control, 6 simple-RPC GEMV,
                                7 simple-RPC finish (scaling, d, tile sums, step
                                end) */
    int64_t phase_launches[8];
    int64_t kernel_launches; /* kernels the last run launched on the device (the
                                reset kernel plus every kernel of every loop body) */
    double mma_flops_tf32;   /* tensor-core flops the column steps executed with
                                tcgen05.mma kind::tf32 (split terms and padding
                                included), 0 on the CUDA-core paths */
    double mma_flops_f16;    /* the same for kind::f16 */
} rpchol_run_stats;

typedef struct rpchol_ctx rpchol_ctx;

/* Library version string. */
const char* rpchol_version(void);

/* Thread-local description of the last error on this thread ("" if none). */
const char* rpchol_last_error(void);

/* Create a factorisation context for the points X (N x d, row-major).
 *   kind, sigma  kernel (sigma > 0)
 *   X            x_dtype RPCHOL_DT_F32 or RPCHOL_DT_F64; FP64 points are
 *                rounded once to FP32, the precision every mode factorises
 *   x_on_device  1 if X is a device pointer, 0 if host memory
 *   k_max        largest rank any run on this context will ask for (<= N)
 *   T_max        largest block size (1 <= T_max <= 256)
 *   opts         may be NULL (defaults: FP64, graph on, instance 0)
 * X is copied; the caller may free it when this returns (the copy is
 * synchronous with respect to the host).  Errors: EINVAL for N < 1, d < 1,
 * d > 4096, sigma <= 0, k_max < 1 or > N, T_max outside [1, 256]; ENOMEM;
 * ECUDA.                                                                  */
rpchol_status rpchol_create(int32_t kind, double sigma, const void* X, int64_t N, int32_t d,
                            int32_t x_dtype, int32_t x_on_device, int64_t k_max, int32_t T_max,
                            const rpchol_opts* opts, rpchol_ctx** out);

/* Accelerated RPCholesky (Algorithm 2 with Algorithm 1), to rank exactly k
 * (the round that would pass k stops Algorithm 1 once k pivots are
 * accepted).  Stops earlier if the residual diagonal sums to zero
 * (status OK, rank < k).  1 <= k <= k_max, 1 <= T <= T_max.  Asynchronous;
 * the device-side status is read by rpchol_stats / rpchol_sync.          */
rpchol_status rpchol_run(rpchol_ctx* ctx, int64_t k, int32_t T, uint64_t seed);

/* Simple RPCholesky (Algorithm 6) to rank k on the same context: the GPU
 * baseline.  Asynchronous.                                                */
rpchol_status rpchol_run_plain(rpchol_ctx* ctx, int64_t k, uint64_t seed);

/* Block RPCholesky (Algorithm 7, appendix): each round draws b pivots iid
 * from the residual diagonal (the same draws as rpchol_run with T = b),
 * keeps the first draw of each index (Unique), and accepts every kept draw
 * whose Schur residual in the FP64 Cholesky of A(S',S') - F(S',:)F(S',:)*
 * is positive, in draw order (a non-positive residual is a zero column,
 * which the algorithm's last line removes); the round that would pass k
 * stops at k.  Same kernels as rpchol_run with the acceptance test of
 * Algorithm 1 replaced; same stopping rules, status and outputs.
 * 1 <= k <= k_max, 1 <= b <= T_max.  Asynchronous.                       */
rpchol_status rpchol_run_block(rpchol_ctx* ctx, int64_t k, int32_t b, uint64_t seed);

/* Wait for the context's stream; returns the device-side status of the
 * last run (OK, ETIMEOUT when the round limit was reached, ENUMERIC).    */
rpchol_status rpchol_sync(rpchol_ctx* ctx);

/* Borrowed device view of the result of the last run: F (N x ldF, dtype
 * F32 in MIXED, F64 in FP64), rank, pivots (int64, device).  Valid until
 * the next run or destroy.  Synchronises the stream.                      */
rpchol_status rpchol_factor(rpchol_ctx* ctx, const void** F_dev, int64_t* ldF, int32_t* F_dtype,
                            int64_t* rank, const int64_t** pivots_dev);

/* Copy the result to caller memory (host or device, any pointer the CUDA
 * runtime can address): F as FP64, N x ld_out (ld_out >= rank), the
 * pivots (rank entries) and the residual diagonal d (N entries).  Any of
 * the three pointers may be NULL.  Synchronous.                           */
rpchol_status rpchol_copy_factor(rpchol_ctx* ctx, double* F_out, int64_t ld_out,
                                 int64_t* pivots_out, double* d_out);

/* Copy the result to caller memory in the dtype F is stored in (FP32 in
 * MIXED, FP64 in FP64 mode): F as N x ld_out (ld_out >= rank) and the
 * pivots.  Either pointer may be NULL.  Synchronous.                      */
rpchol_status rpchol_copy_factor_raw(rpchol_ctx* ctx, void* F_out, int64_t ld_out,
                                     int64_t* pivots_out);

/* Accelerated RPCholesky (as rpchol_run) with the factor streamed to
 * caller memory while the rounds run.  Columns of F never change once
 * their round has ended (later rounds only append columns), so after each
 * round the columns it added are copied, by the copy engine on a stream of
 * the context's own, to F_out while the next rounds compute (whenever the
 * copy stream is idle, else once the pending columns make rows of 3200
 * bytes, so that each copy moves wide rows at the link's rate).  The rounds
 * are launched from the host, a few ahead of the one whose end the host
 * waits for (no CUDA graph).  On return F_out holds F as N x ld_out in the
 * dtype F is stored in (FP32 in MIXED, FP64 in FP64 mode) and pivots_out
 * the rank pivots; entries of F_out beyond the final rank are not written.
 * Results are bit-identical to rpchol_run followed by
 * rpchol_copy_factor_raw.  F_out and pivots_out: any memory the CUDA
 * runtime can address (pinned host memory gives the copy engine's full
 * rate); pivots_out may be NULL.  1 <= k <= k_max, 1 <= T <= T_max,
 * ld_out >= k.  Synchronous; returns the run status as rpchol_sync does.  */
rpchol_status rpchol_run_to_host(rpchol_ctx* ctx, int64_t k, int32_t T, uint64_t seed,
                                 void* F_out, int64_t ld_out, int64_t* pivots_out);

/* Statistics of the last run; computes the relative trace error
 * tr(A - F F^*)/tr(A) from F with FP64 accumulation.  Synchronous.        */
rpchol_status rpchol_stats(rpchol_ctx* ctx, rpchol_run_stats* out);

/* Relative trace error tr(A - F F^*) / tr(A) of a caller-provided factor,
 * without allocating any device memory.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory at all, such as code
 * inside a host runtime that reserves all device memory up front in its own
 * pool and forbids cudaMalloc outside it, or a latency-critical loop where
 * an allocation could block or fail.  It computes what rpchol_stats reports
 * as trace_error, for any factor.
 *   F_dev    device pointer, row-major N x ldF, dtype RPCHOL_DT_F32 or
 *            RPCHOL_DT_F64; only columns 0..rank-1 are read (diag A = 1)
 *   out_dev  device (or device-accessible) pointer to one double
 *   stream   cudaStream_t (NULL = legacy default stream); asynchronous
 * Scratch: per-tile partial sums in a static device array of 65,536 doubles
 * (512 KiB) that every GPU loading the library keeps until the process
 * exits; N > 8,388,608 is rejected with RPCHOL_EINVAL.  Every call looks
 * up the array's address on the current device (nothing is cached, so a
 * device reset between calls is harmless); the first call on a device loads
 * the module there, so make it before any stream capture on that device.
 * All calls share the array: calls whose
 * kernels overlap on the GPU race, so serialise them.  Each call overwrites
 * every partial it uses, so no state carries over between calls.
 * Errors: EINVAL (null pointer, N < 1, rank < 0, ldF < rank, bad dtype,
 * N too large), ECUDA.  Calls no allocator of any kind.                    */
rpchol_status rpchol_trace_error_noalloc(const void* F_dev, int32_t F_dtype, int64_t N,
                                         int64_t ldF, int64_t rank, double* out_dev,
                                         void* stream);

/* Checkpoints (no counterpart in the paper; the state saved is that of
 * Algorithm 2's loop between rounds).  rpchol_save writes the state of the
 * last run (run state,
 * residual diagonal, tile sums, pivots and the rank columns of F in the
 * stored dtype) to host_buf; with host_buf NULL it only sets *bytes to the
 * size needed.  Synchronous.  rpchol_restore loads such a buffer into a
 * context created with the same X, kernel, sigma, N, d and precision and
 * k_max >= the saved rank (T_max >= the saved T); afterwards
 * rpchol_factor / rpchol_copy_factor / rpchol_stats describe the saved run.
 * X itself is not saved.  Errors: EINVAL (no run yet, buffer too small
 * (*bytes then holds the size needed), foreign or mismatched checkpoint),
 * ECUDA.                                                                  */
rpchol_status rpchol_save(rpchol_ctx* ctx, void* host_buf, size_t* bytes);
rpchol_status rpchol_restore(rpchol_ctx* ctx, const void* host_buf, size_t bytes);

/* Continue the last run (or the restored one) from its current rank to rank
 * k > rank with the same algorithm, block size and random stream: the next
 * round is the saved round counter, so a resumed run draws what the
 * original context would have drawn had it been resumed itself.  The run's
 * status must be OK.  Asynchronous like rpchol_run.  Errors: EINVAL.       */
rpchol_status rpchol_resume(rpchol_ctx* ctx, int64_t k);

/* Failure-detection self-test (no counterpart in the paper): two
 * one-thread kernels each wait on an
 * mbarrier that nothing completes, one with the CTA-scope bounded wait of
 * the tensor-core column step, one with the cluster-scope bounded wait of
 * Algorithm 1.  Each wait must give up after limit_ms (1..2000) and report
 * it; the kernels then return and the CUDA context stays usable.  Returns
 * RPCHOL_ETIMEOUT when both waits expired as designed (the expected
 * outcome; waited_ms[0..1], if not NULL, receives the two waiting times),
 * ECUDA if one did not report its expiry or a CUDA call failed, EINVAL for
 * limit_ms out of range.  Synchronous, on the legacy default stream.       */
rpchol_status rpchol_selftest_wait(uint32_t limit_ms, double* waited_ms);

/* Release everything the context owns.  NULL is accepted.  A batch that
 * holds the context must be destroyed first.                              */
void rpchol_destroy(rpchol_ctx* ctx);

/* ---------------------------------------------------------- low memory
 * Algorithm 3 (arXiv 2410.03969, Sec. 2.4): accelerated RPCholesky that
 * keeps no N x k factor.  The context holds X, the residual diagonal, the
 * pivots S and the Cholesky factor L of A(S,S) (k_max x k_max, FP64, twice:
 * row- and column-major), and regenerates kernel entries A(R,S) as the
 * rounds need them: O(N d + k_max^2) device memory, O(N k^2 / T) kernel
 * evaluations.  It draws the same pivots as rpchol_run in FP64 mode (same
 * random stream); the implicit approximation is
 * A(:,S) L^{-*} L^{-1} A(S,:).  FP64 throughout, CUDA cores.
 * Limits: 1 <= k_max <= min(N, 16384), 1 <= T_max <= 256, d <= 4096.     */
typedef struct rpchol_lowmem rpchol_lowmem;

/* X: N x d row-major host or device memory (F32 or F64 by x_dtype; copied
 * to the device, F64 rounded once to F32 as in rpchol_create).  stream:
 * cudaStream_t (NULL = legacy default) used for every call.
 * Errors: EINVAL, ENOMEM, ECUDA.                                          */
rpchol_status rpchol_lowmem_create(int32_t kind, double sigma, const void* X, int64_t N,
                                   int32_t d, int32_t x_dtype, int64_t k_max, int32_t T_max,
                                   void* stream, rpchol_lowmem** out);

/* Algorithm 3 to rank k with T proposals per round.  Synchronous (the host
 * reads the done flag every 8 rounds).  Errors: EINVAL (k, T out of
 * range), ENUMERIC, ETIMEOUT (round limit 4k + 64), ECUDA.                 */
rpchol_status rpchol_lowmem_run(rpchol_lowmem* ctx, int64_t k, int32_t T, uint64_t seed);

/* Copy out the last run: L_out (rank x rank, row-major, leading dimension
 * ld_out >= rank, lower triangular with zeros above the diagonal),
 * pivots_out (rank), d_out (N: the residual diagonal diag(A - Ahat),
 * clamped at 0), rank and rounds.  Any pointer may be NULL.  Host or
 * device destinations.  Errors: EINVAL (ld_out < rank), ECUDA, and the
 * run's own status.                                                       */
rpchol_status rpchol_lowmem_copy(rpchol_lowmem* ctx, double* L_out, int64_t ld_out,
                                 int64_t* pivots_out, double* d_out, int64_t* rank,
                                 int64_t* rounds);

/* Release the context (NULL accepted).                                    */
rpchol_status rpchol_lowmem_destroy(rpchol_lowmem* ctx);

/* --------------------------------------------------- randomly pivoted QR
 * Algorithm 5 (arXiv 2410.03969, appendix): accelerated randomly pivoted
 * QR of a dense M x N matrix B, FP64 on CUDA cores.  Each round draws T
 * columns from the residual squared column norms u, accepts a subset by
 * Algorithm 1 on C^* C with C = B(:,S') - Q F(S',:)^*, orthonormalises the
 * accepted residual columns (a second Gram-Schmidt pass against Q, then the
 * thin-QR factor with positive diagonal by Cholesky QR twice) and appends
 * them to Q, appends G = B^* Q_perp to F, and subtracts the squared row
 * norms of G from u.  B ~ Q F^*.  Same random stream as rpchol_run, so that
 * it draws the pivots rpchol_run draws on A = B^* B.                      */
typedef struct rpchol_rpqr rpchol_rpqr;

/* B: column-major M x N, leading dimension ldb >= M, host or device; copied.
 * Device memory: N M + (k_max + 256) M + N k_max doubles, a split-K
 * workspace of max(4 k_max, 16384) x 256 doubles and O(N) vectors.
 * 1 <= k_max <= min(M, N), 1 <= T_max <= 256.  stream as in
 * rpchol_lowmem_create.  Errors: EINVAL, ENOMEM, ECUDA.                   */
rpchol_status rpchol_rpqr_create(const double* B, int64_t M, int64_t N, int64_t ldb,
                                 int64_t k_max, int32_t T_max, void* stream, rpchol_rpqr** out);

/* Algorithm 5 to rank k (the round that would pass k stops at k), T
 * proposals per round.  Synchronous (the host reads the accepted count
 * each round).  Errors: EINVAL, ENUMERIC, ETIMEOUT (round limit), ECUDA.   */
rpchol_status rpchol_rpqr_run(rpchol_rpqr* ctx, int64_t k, int32_t T, uint64_t seed);

/* Copy out the last run: Q_out (M x rank column-major, ldq >= M, orthonormal
 * columns), F_out (N x rank row-major, ldf >= rank, F = B^* Q), pivots_out
 * (rank), u_out (N residual squared column norms), rank, rounds.  Any
 * pointer may be NULL; host or device destinations.  Errors: EINVAL
 * (leading dimension too small), ECUDA, and the run's own status.         */
rpchol_status rpchol_rpqr_copy(rpchol_rpqr* ctx, double* Q_out, int64_t ldq, double* F_out,
                               int64_t ldf, int64_t* pivots_out, double* u_out, int64_t* rank,
                               int64_t* rounds);

/* Release the context (NULL accepted).                                    */
rpchol_status rpchol_rpqr_destroy(rpchol_rpqr* ctx);

/* ---------------------------------------------------------------- batches
 * Many independent factorisations (Algorithm 2 each, arXiv 2410.03969 §3)
 * in one launch.  Two executors:
 *
 *   RPCHOL_BATCH_ENGINE: one persistent kernel launch.  Its grid is made of
 *     clusters of 8 CTAs (one CTA per SM, as many clusters as can be
 *     resident).  Instances are admitted from a device queue in the order
 *     of their expected work N k^2, largest first.  Each round of an
 *     instance is one control job (sampler, H, Algorithm 1, operand prep)
 *     that a whole cluster runs, then a column step split into tile parts
 *     that any CTA of any cluster takes; the CTA finishing the last part
 *     closes the round and frees the next control job.  Needs every context
 *     in mixed precision with the tensor-core column step (N >= 128, not
 *     the l1-Laplace kernel) and T_max <= 256.
 *   RPCHOL_BATCH_GRAPH: one CUDA graph in which every context has its own
 *     branch, a reset kernel followed by a conditional while-loop over that
 *     context's rounds (the loop body is the kernel sequence rpchol_run
 *     launches).  Any precision.
 *
 * Both run each phase with the block decomposition rpchol_run uses, so an
 * instance's pivots and factor are bit-identical to rpchol_run's.  The
 * graph executor is the default (the faster of the two on the measured
 * batches: the engine's control phases hold whole SMs while they wait on
 * latency).  Each
 * context keeps its own buffers and results; after a batch run,
 * rpchol_stats / rpchol_factor / rpchol_copy_factor* on a context see that
 * context's run (its stream waits for the batch).
 * The paper runs one factorisation at a time; it has no batched form.     */
typedef struct rpchol_batch rpchol_batch;

#define RPCHOL_BATCH_GRAPH 0
#define RPCHOL_BATCH_ENGINE 1

/* Set up a batch of n >= 1 contexts (all on the current device) with block
 * sizes T[i] (1 <= T[i] <= that context's T_max), recording the graph
 * executor (the default mode).  The batch borrows the contexts:
 * destroy it before any of them.  Errors: EINVAL (n < 1, NULL context, T
 * out of range, a context twice), ENOMEM, ECUDA.                          */
rpchol_status rpchol_batch_create(rpchol_ctx* const* ctxs, int32_t n, const int32_t* T,
                                  rpchol_batch** out);

/* Switch the executor for later runs (RPCHOL_BATCH_ENGINE sets up the
 * engine's records on first use).  Errors: EINVAL (unknown mode, or the
 * engine when a member does not support it), ENOMEM, ECUDA.                */
rpchol_status rpchol_batch_set_mode(rpchol_batch* batch, int32_t mode);

/* The executor in use; -1 for NULL.                                        */
int32_t rpchol_batch_mode(const rpchol_batch* batch);

/* Run every instance once: instance i to rank k[i] (1 <= k[i] <= its
 * k_max) with Philox seed seeds[i] (the same stream contract as
 * rpchol_run, so instance i draws exactly what rpchol_run(ctx_i, k[i],
 * T[i], seeds[i]) draws).  Asynchronous on `stream` (cudaStream_t, NULL =
 * legacy default stream), which first waits for every context's stream.
 * Errors: EINVAL, ECUDA.                                                   */
rpchol_status rpchol_batch_run(rpchol_batch* batch, const int64_t* k, const uint64_t* seeds,
                               void* stream);

/* Release the batch (not the contexts).  NULL is accepted. */
void rpchol_batch_destroy(rpchol_batch* batch);

/* Device memory (bytes) a context of these sizes allocates: F, the points
 * and their TF32 planes (mixed mode), d, and the round work arrays.       */
int64_t rpchol_context_bytes(int64_t N, int32_t d, int64_t k_max, int32_t T_max,
                             int32_t precision);

/* ---------------------------------------------------------------- serving
 * A continuous-batching server for factorisation jobs (Algorithm 2 each)
 * of different N, d, kernel and k.  Jobs queue in arrival order; a worker
 * thread admits the oldest waiting job as soon as the device memory it
 * needs (rpchol_context_bytes) fits in the budget next to the jobs that hold
 * memory and a slot is free, gives it its own context and stream, and
 * launches its run, so that jobs admitted while others run overlap on the
 * GPU.  A finished job keeps its factor on the device (and its memory in
 * the budget) until it is released.  Results do not depend on what else
 * runs: each job is computed exactly as rpchol_run computes it alone.
 * The paper has no serving layer.                                          */
typedef struct rpchol_server rpchol_server;

typedef struct {
    int32_t kind;        /* rpchol_kernel_kind */
    double sigma;        /* bandwidth, > 0 */
    const void* X;       /* host points, N x d row-major; copied by submit */
    int64_t N;
    int32_t d;
    int32_t x_dtype;     /* RPCHOL_DT_F32 or RPCHOL_DT_F64 */
    int64_t k;           /* target rank, 1 <= k <= N */
    int32_t T;           /* block size, 0 = 120 (or N if smaller) */
    int32_t precision;   /* RPCHOL_FP64 or RPCHOL_MIXED */
    uint64_t seed;       /* Philox seed (same contract as rpchol_run) */
} rpchol_job;

typedef struct {
    int32_t state;       /* 0 waiting, 1 running, 2 finished, 3 failed */
    int32_t status;      /* rpchol_status of the job once finished or failed */
    int64_t rank;
    int64_t rounds;
    double trace_error;  /* tr(A - F F^*) / tr(A) */
    double queue_ms;     /* submit -> admitted */
    double run_ms;       /* admitted -> device work observed finished */
    double latency_ms;   /* submit -> finished */
    int64_t device_bytes;
} rpchol_job_result;

/* Start a server on the current device with a device-memory budget (bytes,
 * > 0) and at most max_slots jobs holding memory at once (>= 1).  Errors:
 * EINVAL, ECUDA.                                                           */
rpchol_status rpchol_server_create(int64_t mem_budget_bytes, int32_t max_slots,
                                   rpchol_server** out);

/* Queue a job; returns its ticket.  X is copied before this returns.
 * Errors: EINVAL (bad job, or a job that can never fit the budget),
 * ENOMEM (host copy).                                                      */
rpchol_status rpchol_server_submit(rpchol_server* srv, const rpchol_job* job, uint64_t* ticket);

/* State and timings of a job; waits up to wait_ms milliseconds (0: no
 * wait, < 0: until finished) for it to finish.  EINVAL for an unknown or
 * released ticket.                                                         */
rpchol_status rpchol_server_poll(rpchol_server* srv, uint64_t ticket, int32_t wait_ms,
                                 rpchol_job_result* out);

/* Copy a finished job's factor (stored dtype: FP32 in MIXED, FP64 in
 * FP64 mode; N x ld_out, ld_out >= rank) and pivots to caller memory
 * (either pointer may be NULL).  EBUSY if the job has not finished.        */
rpchol_status rpchol_server_copy_factor(rpchol_server* srv, uint64_t ticket, void* F_out,
                                        int64_t ld_out, int64_t* pivots_out);

/* Free a finished job's device memory (its result is gone afterwards).
 * EBUSY if the job has not finished.                                       */
rpchol_status rpchol_server_release(rpchol_server* srv, uint64_t ticket);

/* Stop the worker, wait for running jobs, free everything. */
void rpchol_server_destroy(rpchol_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* RPCHOL_H */

/*
 * pcdm.h -- C ABI of libpcdm, a GB300 (sm_103a) implementation of the parallel
 * coordinate descent method PCDM1 with tau-nice sampling (Richtarik & Takac,
 * "Parallel Coordinate Descent Methods for Big Data Optimization",
 * arXiv:1212.0873, Algorithm 1) specialised to LASSO:
 *
 *     minimise F(x) = 1/2 ||A x - b||^2 + lambda ||x||_1,   A sparse, stored by columns
 *
 * (eq. (P) with f = 1/2||Ax-b||^2 and Omega = lambda||.||_1; the LASSO instance of Sec. 8.1).
 *
 * One iteration k draws a tau-nice set S_k (Sec. 4.1, item 3), computes for every
 * i in S_k the partial derivative grad_i = a_i^T g against the maintained residual
 * g = A x - b, takes the step of eq. (h(x)) with w = L, L_i = ||a_i||^2 and
 * beta = 1 + (omega-1)(tau-1)/max(1,n-1) (Theorem ESO-nice, Table ESO), and then
 * moves x_i and g for all tau coordinates at once (Jacobi: every step reads x_k).
 *
 * Conventions for every entry point:
 *  - Sizes are int64_t; row and column indices are int32_t (m, n < 2^31).
 *  - "Device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary (pageable or pinned) host memory.
 *  - All work is enqueued on the stream given at pcdm_create.  Calls that return
 *    host values (gap, solve, get_* to host, stats) synchronise that stream.
 *  - Functions return a pcdm_status and never abort the process.  On failure
 *    pcdm_last_error(handle) describes the cause.  After PCDM_ECUDA or
 *    PCDM_ETIMEOUT the handle refuses further work (PCDM_ESTATE) until
 *    pcdm_reset is called.
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef PCDM_H
#define PCDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcdm_ctx *pcdm_handle;

typedef enum {
    PCDM_OK = 0,
    PCDM_EINVAL = 1,    /* an argument or the matrix is invalid; nothing was changed */
    PCDM_ENOMEM = 2,    /* device memory allocation failed */
    PCDM_ECUDA = 3,     /* a CUDA call failed */
    PCDM_ETIMEOUT = 4,  /* a bounded device-side wait (grid barrier) ran out */
    PCDM_ENOTCONV = 5,  /* pcdm_solve hit max_iters before the tolerance */
    PCDM_ESTATE = 6     /* the handle is in a failed state, or a call came out of order */
} pcdm_status;

typedef enum { PCDM_F64 = 0, PCDM_F32 = 1, PCDM_BF16 = 2 } pcdm_dtype;

/*
 * A in compressed sparse column form (the paper stores A = [a_1 .. a_n] by
 * columns, Sec. 8.1).  col_ptr has n+1 entries with col_ptr[0] = 0,
 * col_ptr[n] = nnz and col_ptr non-decreasing; the rows of column i are
 * row_idx[col_ptr[i] .. col_ptr[i+1]-1], strictly increasing, each in [0, m);
 * val holds the matching values in val_dtype, all finite.  Empty columns are
 * allowed.  The library copies everything it needs: the caller keeps ownership.
 */
typedef struct {
    int64_t m, n, nnz;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const void *val;
    int32_t val_dtype;    /* pcdm_dtype */
    int32_t on_device;    /* 1: the three arrays are device pointers, 0: host pointers */
} pcdm_csc;

/*
 * Options.  Fill with pcdm_default_opts and change what you need.
 * Precision pairs (val_dtype, xg_dtype): (F64, F64), (F32, F32), (BF16, F32).
 * The FP32 forms keep g in FP32 and accumulate gradients in FP32; x and the
 * proximal step are FP64 in every pair (an FP32 x alone bounds the reachable
 * relative duality gap near 1e-6); the residual refresh and the duality gap are
 * always computed in FP64.
 */
typedef struct {
    int32_t xg_dtype;            /* dtype of g and the gradient accumulator: PCDM_F64 or PCDM_F32 */
    int32_t fused;               /* 1: one persistent cooperative kernel per run of iterations,
                                    0: two kernels per iteration (gather/prox, scatter)          */
    int64_t refresh_every;       /* after iteration k with (k+1) % refresh_every == 0, recompute
                                    g = A x - b in FP64 (0: only when pcdm_gap runs)            */
    int64_t check_every;         /* pcdm_solve: iterations between duality-gap checks
                                    (0: adaptive, see pcdm_next_check_interval)                 */
    int64_t lanes_per_col;       /* threads that share one column: 0 (auto), 4, 8, 16 or 32     */
    uint64_t barrier_timeout_ns; /* bound on every grid-barrier wait of the fused kernel          */
    int32_t profile;             /* 1: time every iteration-kernel launch with CUDA events        */
    int32_t sampling;            /* PCDM_SAMPLING_NICE (default), _INDEPENDENT or _BINOMIAL       */
    double p_b;                  /* binomial sampling: probability that a position is kept, (0, 1] */
    int32_t l2_persist;          /* 1: raise the CUDA context's L2 persisting-lines limit
                                    (cudaLimitPersistingL2CacheSize) to the device maximum while
                                    the handle lives.  The handles of a device share the limit:
                                    the first l2_persist handle raises it, and destroying the last
                                    one restores the value from before the first and resets the
                                    persisting lines, whatever the order of create and destroy.
                                    The kernels mark the residual evict-last; the set-aside keeps
                                    more of it in L2.  The limit is context-wide: it holds for every
                                    kernel of the process while the handle lives.  Changing the
                                    limit costs milliseconds at create and destroy, so it pays off
                                    for handles that run many iterations.  0: leave it.
                                    Single-problem handles only (the batch and multi APIs ignore it). */
    int32_t deterministic_scatter;  /* 1: bitwise reproducible iterations (Algorithm 1, step 4, in a
                                    fixed order of operations).  Each gradient sums its column in
                                    storage order from 0, every product and addition rounded on its
                                    own (no FMA); beta L_i is one product, and u = x_i - grad/(beta L_i),
                                    t = lambda/(beta L_i) use correctly rounded divisions; x_i becomes
                                    soft(u, t).  Each g_r then receives the iteration's nonzero steps
                                    in increasing sampled position, g_r = g_r + a_ri h_j, with no
                                    atomics, and the residual refresh sums each row from -b_r in
                                    increasing column index.  In the FP64 form these are exactly the
                                    operations of a plain sequential FP64 run of Algorithm 1 that
                                    visits S_k[0], S_k[1], ... in turn.  Runs the two-kernel form
                                    (fused, lanes_per_col and the tuning calls are ignored), LASSO
                                    with the tau-nice sampling only (else EINVAL at create), and
                                    keeps a row-major copy of A (8(m+1) + nnz(4 + value bytes)) and
                                    8 n bytes of stamps.  0: atomics in arrival order.          */
} pcdm_opts;

/*
 * Samplings (Sec. 4.1).  All three are doubly uniform; beta follows Theorem
 * ESO-DU, 1 + (omega-1)(E|S|^2/E|S| - 1)/max(1, n-1), which for the tau-nice
 * sampling is the beta of Theorem ESO-nice.
 *  NICE         tau distinct blocks, uniform over tau-subsets (see pcdm_step).
 *  INDEPENDENT  tau picks, each uniform over [0, n) and independent: pick j is
 *               floor(W_j n / 2^64), W_j the low 64 bits (words 0, 1) of the
 *               Philox4x32-10 block with counter (j, 1, lo32 k, hi32 k) and key
 *               (lo32 seed, hi32 seed); a block picked more than once is updated
 *               once, by its first pick (the others are idle).
 *               E|S| = n(1 - a), E|S|^2 = E|S| + n(n-1)(1 - 2a + (1-2/n)^tau),
 *               a = (1-1/n)^tau.
 *  BINOMIAL     the tau-nice positions, each kept independently with
 *               probability p_b (the paper's unreliable-processor model, case 2):
 *               position j is kept iff word 0 of the Philox block with counter
 *               (j, 2, lo32 k, hi32 k) is below min(2^32, floor(p_b 2^32)).
 *               E|S| = tau p_b, E|S|^2 = tau p_b (1 + tau p_b - p_b).
 * INDEPENDENT and BINOMIAL run the two-kernel form (opts.fused is ignored).
 */
enum { PCDM_SAMPLING_NICE = 0, PCDM_SAMPLING_INDEPENDENT = 1, PCDM_SAMPLING_BINOMIAL = 2 };

/* Counters since pcdm_create or pcdm_reset_stats. */
typedef struct {
    int64_t iterations;        /* PCDM1 iterations run */
    int64_t updates;           /* coordinate updates (tau per iteration) */
    int64_t gathered_nnz;      /* nonzeros read by the gradient gathers */
    int64_t scattered_nnz;     /* nonzeros scattered into g (columns with h_i != 0) */
    int64_t nonzero_updates;   /* updates with h_i != 0 */
    int64_t iter_launches;     /* launches of the iteration kernel(s) */
    double iter_kernel_ms;     /* summed CUDA-event time of those launches (profile = 1), else 0 */
    int64_t refreshes;         /* FP64 residual refreshes */
    int64_t gaps;              /* duality-gap evaluations */
    int64_t val_bytes;         /* bytes of one stored value */
    int64_t xg_bytes;          /* bytes of one g entry (x entries are 8-byte doubles) */
    int64_t kernel_launches;   /* every kernel this handle launched (all phases) */
} pcdm_stats;

/* Default options: xg_dtype F64, fused 1, refresh_every 0, check_every 0,
 * lanes_per_col 0, barrier_timeout_ns 2e9, profile 0, sampling NICE, p_b 1,
 * l2_persist 0. */
void pcdm_default_opts(pcdm_opts *opts);

/*
 * Create a solver for one LASSO instance (eq. (P), Sec. 8.1) and run the set-up:
 * validation of A, L_i = ||a_i||^2 in FP64, omega = max_r #nonzeros of row r
 * (Sec. 1, examples of partially separable functions), x = 0 and g = -b.
 *   A          matrix (see pcdm_csc); copied
 *   b          right-hand side, m entries of b_dtype (PCDM_F64 or PCDM_F32), host or
 *              device as A->on_device says; copied and kept in FP64
 *   lambda     regularisation weight, finite and >= 0
 *   opts       NULL for defaults
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream)
 *   out        receives the handle
 * Errors: EINVAL for a NULL pointer, sizes out of range, a bad dtype pair,
 * lambda < 0 or not finite, col_ptr not monotone or not ending at nnz, a row
 * index out of range or not strictly increasing in its column, a non-finite
 * value in A or b.  ENOMEM, ECUDA.
 */
pcdm_status pcdm_create(const pcdm_csc *A, const void *b, int32_t b_dtype, double lambda,
                        const pcdm_opts *opts, void *cuda_stream, pcdm_handle *out);

/*
 * The two other objectives the paper runs PCDM1 on, with blocks of size 1:
 *
 *  PCDM_PROBLEM_SVM_DUAL (Sec. 8.3): A is d x n, column i the example A_i, y in
 *    {-1,+1}^n one label per column, lambda > 0.  Minimise the negated dual of
 *    the L2-regularised hinge-loss SVM over the box [0,1]^n:
 *      F(x) = 1/(2 lambda n^2) ||sum_i y_i x_i A_i||^2 - (1/n) sum_i x_i
 *    (the paper's f with Z_ij = y_i y_j <A_i, A_j>, Psi the box indicator).
 *    L_i = ||A_i||^2/(lambda n^2); omega = the largest number of examples sharing
 *    a feature (row counts).  The step clips x_i - grad_i/(beta L_i) to [0, 1];
 *    an all-zero example goes to 1.  The maintained vector is g = sum_i y_i x_i A_i
 *    (m = d entries); the primal point is w = g/(lambda n).
 *    pcdm_gap: primal = (1/n) sum_i max(0, 1 - y_i <w, A_i>) + lambda/2 ||w||^2,
 *    dual = -F(x), gap = primal - dual.
 *
 *  PCDM_PROBLEM_LOGISTIC (Sec. 8.4): A is m x n, row j the example A_j, y in
 *    {-1,+1}^m one label per row, lambda > 0.  Minimise
 *      F(x) = sum_j log(1 + exp(-y_j A_j^T x)) + lambda ||x||^2.
 *    L_i = ||a_i||^2/4 (the logistic loss has curvature at most 1/4); omega = the
 *    largest number of features of an example.  The step is
 *    x_i - (grad_i + 2 lambda x_i)/(beta L_i + 2 lambda).  The maintained vector
 *    is the margins g_j = y_j A_j^T x (m entries).
 *    pcdm_gap: primal = F(x), dual = the Fenchel dual at alpha_j = 1/(1 + exp(g_j)),
 *    gap = primal - dual = ||grad F(x)||^2/(4 lambda).
 *
 * pcdm_solve stops at gap/primal <= rel_gap_tol as for LASSO.  Layout,
 * ownership, dtypes and options are those of pcdm_create; y is n (SVM dual) or
 * m (logistic) doubles on the host or the device as A->on_device says, copied.
 * The labels are folded into the stored values (a sign flip, exact in every
 * dtype), so pcdm_get_residual returns the g above; pcdm_get_L returns ||A_i||^2
 * for the SVM dual (the paper's L_i times lambda n^2) and ||a_i||^2/4 for
 * logistic regression.  These handles run the tau-nice sampling in the pipelined
 * kernel, the fused kernel with lanes per column or the two-kernel form (not in
 * the rounds kernel); pcdm_polish, pcdm_backward, pcdm_set_b and the
 * asynchronous mode return EINVAL, and pcdm_set_tuning rejects kernel 3.
 * Errors: those of pcdm_create, plus EINVAL for an unknown problem, a NULL y,
 * lambda <= 0 or not finite, a sampling other than PCDM_SAMPLING_NICE, and a
 * label other than -1 or +1.
 */
enum { PCDM_PROBLEM_LASSO = 0, PCDM_PROBLEM_SVM_DUAL = 1, PCDM_PROBLEM_LOGISTIC = 2 };

pcdm_status pcdm_create_problem(const pcdm_csc *A, int32_t problem, const double *y, double lambda,
                                const pcdm_opts *opts, void *cuda_stream, pcdm_handle *out);

/*
 * Device memory of the single-problem handles (pcdm_create,
 * pcdm_create_problem) comes from a per-device stream-ordered pool owned by
 * the library: a handle's buffers are allocated and freed in order on its
 * stream, and freed memory stays in the pool for the next handle, so that
 * creating and destroying handles costs microseconds of allocation instead of
 * milliseconds of cudaMalloc and cudaFree.
 *   pcdm_set_memory_cache       the most memory the pool of the current device
 *                               keeps after it is freed (bytes; default 16 GiB);
 *                               the rest goes back to the device at the next
 *                               synchronisation
 *   pcdm_release_cached_memory  return the cached memory of the current
 *                               device's pool now (memory whose stream-ordered
 *                               free has not yet executed stays)
 * ECUDA on a CUDA error.
 */
pcdm_status pcdm_set_memory_cache(uint64_t bytes);
pcdm_status pcdm_release_cached_memory(void);

/* The PCDM_PROBLEM_* of a handle. */
pcdm_status pcdm_problem_kind(pcdm_handle h, int32_t *problem);

/*
 * Run `iters` iterations of Algorithm 1 (PCDM1) with the tau-nice sampling,
 * continuing the handle's iteration counter k.  S_k depends only on
 * (seed, k, n, tau), so step(a) followed by step(b) equals step(a+b).
 * tau in [1, n]; iters >= 0.  EINVAL otherwise.
 * The sampler: a 12-round balanced Feistel permutation pi_k of [0, 2^w) (w the
 * least even width with 2^w >= n, at least 2), walked back into [0, n) by
 * re-applying it; S_k = (pi_k(0) .. pi_k(tau-1)).  Its round keys K[0..11] are
 * the three Philox4x32-10 blocks (Salmon et al., SC'11) with counter
 * (c, 0, lo32 k, hi32 k), c = 0, 1, 2, and key (lo32 seed, hi32 seed); round r
 * maps (L, R) to (R, L xor (fmix32(R xor K[r]) & (2^(w/2) - 1))), fmix32 being
 * the MurmurHash3 finaliser.
 */
pcdm_status pcdm_step(pcdm_handle h, int64_t tau, int64_t iters, uint64_t seed);

/*
 * Asynchronous mode (the shared-memory implementation of Sec. 8.1, not
 * Algorithm 1's synchronous iteration): `threads` GPU threads (0: as many as
 * the device holds at once, at most n) take updates u = 0, 1, 2, ... of a
 * global sequence without any barrier.  Update u picks block i_u uniformly
 * (the INDEPENDENT pick with k = u, position 0), reads x_i and g as they are,
 * computes the step of eq. (h(x)) and applies it with atomic additions to x_i
 * and g.  beta is that of the tau-independent sampling with tau = threads
 * (Theorem ESO-DU).  With threads = 1 this is the serial method with iid
 * blocks: it equals `updates` iterations of the INDEPENDENT sampling with
 * tau = 1.  Results are not deterministic for threads > 1.  The update counter
 * continues across calls (pcdm_reset sets it to 0).
 */
pcdm_status pcdm_step_async(pcdm_handle h, int64_t updates, uint64_t seed, int32_t threads);

/* pcdm_step_async in chunks (first one epoch = n updates, then the adaptive
 * schedule of pcdm_next_check_interval) until gap / primal <= rel_gap_tol; the
 * gap check refreshes g.  PCDM_ENOTCONV when max_updates ran out first. */
pcdm_status pcdm_solve_async(pcdm_handle h, uint64_t seed, double rel_gap_tol, int64_t max_updates,
                             int32_t threads, int64_t *updates_done, double *rel_gap);

/*
 * Autotuner: choose the iteration kernel for tau by timing trial_iters
 * iterations of each candidate on this handle's matrix, from its current
 * state (which is restored afterwards; the counters of pcdm_get_stats are not
 * changed).  Candidates: the pipelined one-lane-per-column kernel with blocks
 * of 128 .. 448 threads (the tau positions per block; when tau fits one pass of
 * the grid), each with and without the column heads (and, in the FP64 form of LASSO,
 * with and without zero_cert), its rounds form with blocks of 128 or 256 threads (several
 * positions per thread and iteration), the fused kernel with 1 .. 32 lanes per
 * column (its scatter reloads the column), the two-kernel form with 1, 4 or
 * 16 lanes, and the streaming kernel (4) with blocks of 128, 256 or 448 threads:
 * one lane per column as the pipelined kernel, but the whole column reaches its
 * thread chunk by chunk through TMA bulk copies into shared memory, two chunks
 * ahead of the gathers (for long columns), and the warp-cooperative kernel (5) with
 * blocks of 128, 256 or 512 threads: the 32 lanes of a warp share each of its columns
 * (at most 32 positions per warp, so tau <= 32 * warps of the grid), one column after
 * another with the next column's entries loading and its gathers in flight while the
 * current column's products are taken; the partial sums of four (FP64) or eight
 * columns are reduced over the warp together and the owner lanes take their steps
 * side by side (for long columns; the FP64 form of LASSO certifies zero steps in FP32
 * as zero_cert describes).
 * The fastest is kept for later pcdm_step /
 * pcdm_solve calls (for any tau; tune again for a very different one).
 * Needs the tau-nice sampling and opts.fused = 1.
 */
typedef struct {
    int32_t kernel;             /* 0 pipelined, 1 fused with lanes_per_col lanes, 2 two-kernel form,
                                   3 pipelined rounds, 4 streaming, 5 warp-cooperative */
    int32_t lanes_per_col;
    int32_t threads_per_block;  /* pipelined, rounds, streaming and warp-cooperative kernels */
    int32_t heads;              /* pipelined kernels: 1 = fetch each sampled column's first E
                                   entries (16 row indices, 16 values, then E - 16 row indices
                                   and as many values) with one bulk copy from a per-column
                                   head array, n * E * (4 + sizeof(value)) bytes (E = 24 for
                                   FP64 values, 32 for FP32 and BF16) built on first use when
                                   free device memory holds four times that; 0 = two to four
                                   copies from the padded CSC arrays */
    int32_t zero_cert;          /* pipelined and warp-cooperative kernels, FP64 form, LASSO:
                                   1 = before the FP64 sum
                                   a_i^T g, bound it in FP32 from the high words of the operands
                                   and take the step as 0 when the bound shows |a_i^T g| <= lambda
                                   at x_i = 0 (the same step the FP64 sum gives: eq. (h(x)) with
                                   x_i = 0 is 0 exactly when |grad_i| <= lambda); a warp whose
                                   lanes are all certified issues no FP64 instruction;
                                   0 = the FP64 sum for every column; -1 (pcdm_set_tuning, and
                                   pcdm_autotune's report for kernel 5) =
                                   the built-in rule: for kernel 0 on when nnz <= 8 n; for
                                   kernel 5 (whose bound covers the warp's summation order)
                                   on while at most a quarter of the sampled coordinates
                                   move, which pcdm_solve measures between its gap checks
                                   (off after create and reset, when x = 0; on after
                                   set_x).  The FP32 and BF16
                                   forms always compare their FP32 gradient with lambda rounded
                                   down, an exact test, and ignore this field. */
    double us_per_iteration;    /* measured */
} pcdm_tuning;

pcdm_status pcdm_autotune(pcdm_handle h, int64_t tau, int64_t trial_iters, pcdm_tuning *best);

/* Choose the iteration kernel by hand (the fields of pcdm_tuning; us_per_iteration
 * is ignored; heads 0 or 1; zero_cert -1, 0 or 1; threads_per_block a multiple of 32,
 * up to 448 for kernels 0 and 4, 256 for kernel 3 and 512 for kernel 5), or return to
 * the built-in rule with t = NULL.  A pipelined, streaming or warp-cooperative kernel
 * that cannot hold tau at that block size falls back to the fused one. */
pcdm_status pcdm_set_tuning(pcdm_handle h, const pcdm_tuning *t);

/* Recompute g = A x - b in FP64 (stored in g's dtype). */
pcdm_status pcdm_refresh(pcdm_handle h);

/*
 * Refresh g, then evaluate in FP64 the LASSO duality gap at the dual point
 * theta = s g, s = min(1, lambda / ||A^T g||_inf):
 *   primal = 1/2 ||g||^2 + lambda ||x||_1,  dual = -1/2 s^2 ||g||^2 - s b^T g,
 *   gap = 1/2 (1-s)^2 ||g||^2 + lambda ||x||_1 + s x^T A^T g   (= primal - dual).
 * Any output pointer may be NULL.  Synchronises the stream.
 */
pcdm_status pcdm_gap(pcdm_handle h, double *primal, double *dual, double *gap);

/*
 * Iterate until gap / primal <= rel_gap_tol: check the gap first, then run
 * chunks of iterations, checking after each: opts.check_every iterations when
 * it is positive, else the adaptive schedule of pcdm_next_check_interval.  Its
 * first chunk is one epoch, ceil(n / tau) iterations, or, when the handle's
 * previous pcdm_solve ran K iterations since pcdm_create / pcdm_reset (a warm
 * start such as the next lambda of a path), max(epoch, K / 2).  The gap check is not part
 * of Algorithm 1; it is the stopping test.  iters_done and rel_gap (either may
 * be NULL) receive the iterations run and the last relative gap.  Returns
 * PCDM_ENOTCONV when max_iters ran out first.
 */
pcdm_status pcdm_solve(pcdm_handle h, int64_t tau, uint64_t seed, double rel_gap_tol, int64_t max_iters,
                       int64_t *iters_done, double *rel_gap);

/*
 * The adaptive gap-check schedule of pcdm_solve (host arithmetic only; needs no
 * handle and no device).  After checks at iterations k_prev and k_cur with
 * relative gaps rel_prev > rel_cur > rel_gap_tol, the rate of the last interval,
 * log(rel_prev / rel_cur) / (k_cur - k_prev), is extrapolated to the tolerance
 * with a 5% margin; the result is clamped to [ceil(epoch / 4), 64 epoch] and to
 * twice the last interval.  Without a decrease (or with a non-positive input) it
 * returns epoch.  A gap evaluation is a full FP64 pass over A, costing about as
 * much as 20 iterations at tau = 65536, so fewer checks near the end of a solve
 * save time; overshooting the tolerance costs at most the margin.
 */
int64_t pcdm_next_check_interval(int64_t epoch, int64_t k_prev, double rel_prev, int64_t k_cur, double rel_cur,
                                 double rel_gap_tol);

/* Copy x (n doubles) to host (on_device = 0) or device memory. */
pcdm_status pcdm_get_x(pcdm_handle h, void *x_out, int32_t on_device);

/* Replace x (n doubles, host or device) and recompute g = A x - b (warm start). */
pcdm_status pcdm_set_x(pcdm_handle h, const void *x_in, int32_t on_device);

/* Copy the maintained residual g (m entries of xg_dtype) to host or device memory. */
pcdm_status pcdm_get_residual(pcdm_handle h, void *g_out, int32_t on_device);

/* Copy L (n doubles, L_i = ||a_i||^2) to host or device memory. */
pcdm_status pcdm_get_L(pcdm_handle h, double *L_out, int32_t on_device);

/* Change lambda (finite, >= 0) for the following iterations; x and g are kept. */
pcdm_status pcdm_set_lambda(pcdm_handle h, double lambda);

/* omega, the degree of partial separability of f (largest row count of A). */
pcdm_status pcdm_omega(pcdm_handle h, int64_t *omega);

/* beta of the handle's sampling for tau (Theorem ESO-DU; for the tau-nice
 * sampling 1 + (omega-1)(tau-1)/max(1, n-1), Theorem ESO-nice); omega taken as >= 1. */
pcdm_status pcdm_beta(pcdm_handle h, int64_t tau, double *beta);

/* The iteration counter k (iterations run since create or reset), and its setter
 * (checkpoint/resume: restore x with pcdm_set_x and k with pcdm_set_iteration). */
pcdm_status pcdm_get_iteration(pcdm_handle h, int64_t *k);
pcdm_status pcdm_set_iteration(pcdm_handle h, int64_t k);

/* x = 0, g = -b, k = 0, and clear a failed state.  The counters of pcdm_get_stats
 * are kept (pcdm_reset_stats clears them). */
pcdm_status pcdm_reset(pcdm_handle h);

/* Counters (see pcdm_stats); synchronises the stream. */
pcdm_status pcdm_get_stats(pcdm_handle h, pcdm_stats *out);
pcdm_status pcdm_reset_stats(pcdm_handle h);

/*
 * The tau-nice sample of iteration k on its own: S_device[j] = pi_k(j) for
 * j < tau (see pcdm_step), written to device memory on cuda_stream.
 * 1 <= n < 2^31, 0 <= tau <= n, k >= 0.  No handle needed.
 */
pcdm_status pcdm_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S_device, void *cuda_stream);

/*
 * The list of iteration k of sampling `kind` on its own (no handle): for NICE
 * and BINOMIAL the tau-nice positions S_device[j] = pi_k(j), for INDEPENDENT
 * the tau picks (repeats included; which of them are idle is decided inside
 * the solver).  keep_device (tau bytes, may be NULL) receives 1 for the kept
 * positions of BINOMIAL (all 1 for NICE; not written for INDEPENDENT).
 */
pcdm_status pcdm_sample_kind(int32_t kind, uint64_t seed, int64_t k, int64_t n, int64_t tau, double p_b,
                             int32_t *S_device, uint8_t *keep_device, void *cuda_stream);

/*
 * Self-test of the bounded grid barrier used by the fused kernel: launches a
 * small cooperative kernel whose barrier waits for one arrival more than there
 * are blocks, so every wait must give up after timeout_ns.  Returns PCDM_ETIMEOUT
 * when the bound worked (the expected outcome), PCDM_OK if the wait was
 * satisfied (it cannot be), ECUDA on a CUDA error.  The device stays usable.
 */
pcdm_status pcdm_selftest_barrier_timeout(uint64_t timeout_ns, void *cuda_stream);

/*
 * Random-gather rate of the current GPU, a measurement helper with no
 * counterpart in the paper: the iteration kernels spend their time on gathers
 * of the residual at random rows, so this rate is their second ceiling beside
 * the HBM copy bandwidth.  A full grid (two blocks of 1024 threads per SM)
 * issues rounds of 16 independent coherent loads of elem_bytes (4 or 8) at
 * hashed positions of src (device memory, n elements, 1 <= n < 2^32; every
 * index is below n), twice untimed and five times between CUDA events on
 * cuda_stream; *gathers_per_s (host) receives loads per second.  src is only
 * read.  EINVAL for NULL pointers or bad sizes, ECUDA on a CUDA error.
 * Synchronises the stream.
 */
pcdm_status pcdm_gather_rate(const void *src, int64_t n, int32_t elem_bytes, double *gathers_per_s,
                             void *cuda_stream);

/*
 * omega = the largest number of nonzeros in one row of A (the omega of the
 * tau-nice ESO parameter beta, Theorem ESO-nice, Sec. 6.3) for a CSC matrix already in
 * device memory, with no handle and WITHOUT ALLOCATING ANY MEMORY.  The paper
 * has no counterpart: this is a library convenience.
 *
 * Who needs it: callers that cannot allocate device memory at the point where
 * they need omega (and so beta for a new tau), for instance a process that has
 * given all free device memory to its own pool or arena, where cudaMalloc would
 * fail, or a loop that must not pay cudaMalloc/cudaFree, which can synchronise
 * the whole device.  pcdm_create computes the same omega (pcdm_omega) but
 * allocates a handle and an m-entry row-count buffer to do it.
 *
 * The row counters live in a fixed device array of PCDM_NOALLOC_MAX_ROWS ints
 * (4 MiB) inside the library, so m may be at most PCDM_NOALLOC_MAX_ROWS; larger
 * m returns PCDM_EINVAL before any device work.  A: col_ptr, row_idx on the
 * device (A->on_device must be 1; host arrays would need a staging buffer), the
 * values are not read.  The matrix is checked as pcdm_create checks it (1 <= m,
 * n < 2^31, nnz >= 0, col_ptr monotone from 0 to nnz, rows in [0, m), strictly
 * increasing in a column); a violation returns PCDM_EINVAL.  The call clears the counters it uses, runs
 * on cuda_stream and synchronises it before writing *omega (host memory).
 *
 * The first call on a device looks up the array's device address (a one-time
 * set-up per device); make that first call before any stream capture begins.
 * Calls that overlap in time (two host threads, or two streams, at once) share
 * the one array and race: serialise them.
 */
#define PCDM_NOALLOC_MAX_ROWS 1048576
pcdm_status pcdm_omega_noalloc(const pcdm_csc *A, int64_t *omega, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Derivatives of the LASSO solution (implicit function theorem on the active
 * set).  With S = {i : x_i != 0} and s = sign(x_S), a solution satisfies
 *   A_S^T (A_S x_S - b) + lambda s = 0,
 * so for a loss L(x) with v = dL/dx restricted to S and u solving
 * (A_S^T A_S) u = v:  dL/db = A_S u  and  dL/dlambda = -s^T u.
 * Both solves below run the coordinate kernel of Algorithm 1 on the positions
 * of S (tau-nice sampling over S, beta of Theorem ESO-nice with omega_S = the
 * largest row count of A_S) without the prox, in FP64 for every precision
 * pair.  The paper has no derivatives; this is the differentiation layer
 * (torch.autograd) of the package.  Memory: O(n + m) beyond the handle.
 * ------------------------------------------------------------------------ */

/* Replace b (m entries of b_dtype, host or device) keeping x; g = A x - b.
 * EINVAL for a non-finite value (for an FP32 b the handle then needs
 * pcdm_set_b or pcdm_reset before further work). */
pcdm_status pcdm_set_b(pcdm_handle h, const void *b, int32_t b_dtype, int32_t on_device);

/* |S| = number of nonzero x_i. */
pcdm_status pcdm_support_size(pcdm_handle h, int64_t *count);

/* Polish x on its current support: solve A_S^T (A_S x_S - b) + lambda s = 0
 * for x_S (x fixed at 0 off S) from the current x, until
 * ||A_S^T (A_S x_S - b) + lambda s|| / ||lambda s|| <= tol, then recompute g.
 * Meant after pcdm_solve has settled the support and signs: it does not move
 * coordinates off S, and pcdm_gap tells whether the result is optimal.
 * tau = 0: all of S per iteration.  iters, rel_res may be NULL.
 * PCDM_ENOTCONV when max_iters ran out first. */
pcdm_status pcdm_polish(pcdm_handle h, int64_t tau, uint64_t seed, double tol, int64_t max_iters,
                        int64_t *iters, double *rel_res);

/* Backward pass at the current x: given dx = dL/dx (n doubles, host or device;
 * entries off S are ignored), solve (A_S^T A_S) u = dx_S to relative residual
 * tol and write db = A_S u (m doubles, host or device as db_on_device says;
 * may be NULL) and *dlambda = -sign(x_S)^T u (may be NULL).  tau = 0: all of S
 * per iteration.  PCDM_ENOTCONV when max_iters ran out first (outputs are
 * still written). */
pcdm_status pcdm_backward(pcdm_handle h, const double *dx, int32_t dx_on_device, double *db,
                          int32_t db_on_device, double *dlambda, int64_t tau, uint64_t seed, double tol,
                          int64_t max_iters, int64_t *iters, double *rel_res);

/* ------------------------------------------------------------------------
 * Batched solver: nrhs <= 32 LASSO problems that share A,
 *   min_x 1/2 ||A x - b_l||^2 + lambda_l ||x||_1,  l = 0 .. nrhs-1,
 * solved together.  Each problem runs Algorithm 1 exactly as pcdm_step would
 * (the same sampler, the same S_k for every problem, beta of Theorem ESO-nice),
 * so problem l follows the trajectory of a single-problem handle created with
 * b_l and lambda_l and stepped with the same seed.  What the batch shares is
 * the read of each sampled column of A: the residuals and iterates are stored
 * interleaved by problem, so one column's gathers read nrhs consecutive
 * residual entries of a row.  The paper's PCDM1 is one problem; the batch is
 * this library's data-parallel form of many (regularisation paths, multiple
 * right-hand sides).  Conventions as above: one stream (from opts/cuda_stream),
 * status returns, not thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct pcdm_batch_ctx *pcdm_batch_handle;

/*
 * A           as for pcdm_create (validated the same way)
 * nrhs        number of problems, 1 .. 32
 * B           nrhs right-hand sides, each m entries of b_dtype, stored one after
 *             the other (b_l at B + l*m); host or device as A->on_device says;
 *             copied and kept in FP64
 * lambdas     nrhs host doubles, finite and >= 0
 * opts        as for pcdm_create (xg_dtype, refresh_every, check_every,
 *             barrier_timeout_ns, profile are used; sampling must be NICE)
 * Errors: those of pcdm_create, EINVAL for nrhs out of range, a bad lambda or a
 * non-finite value in B.
 */
pcdm_status pcdm_batch_create(const pcdm_csc *A, int64_t nrhs, const void *B, int32_t b_dtype,
                              const double *lambdas, const pcdm_opts *opts, void *cuda_stream,
                              pcdm_batch_handle *out);

/* `iters` iterations of every active problem, continuing the batch's counter k. */
pcdm_status pcdm_batch_step(pcdm_batch_handle h, int64_t tau, int64_t iters, uint64_t seed);

/* Recompute every residual g_l = A x_l - b_l in FP64. */
pcdm_status pcdm_batch_refresh(pcdm_batch_handle h);

/* Refresh, then the duality gap of every problem as pcdm_gap defines it;
 * primal, dual, gap: nrhs host doubles each, any may be NULL. */
pcdm_status pcdm_batch_gap(pcdm_batch_handle h, double *primal, double *dual, double *gap);

/* Iterate until every problem has gap / primal <= rel_gap_tol.  A problem that
 * reaches the tolerance at a check is frozen (its x no longer changes) for the
 * rest of the call; the checks follow opts.check_every or, when 0, the schedule
 * of pcdm_next_check_interval applied to the largest relative gap among the
 * problems still running (first chunk as in pcdm_solve, from the batch's
 * previous solve).  rel_gaps: nrhs host doubles (may be NULL).
 * PCDM_ENOTCONV when max_iters ran out first. */
pcdm_status pcdm_batch_solve(pcdm_batch_handle h, int64_t tau, uint64_t seed, double rel_gap_tol,
                             int64_t max_iters, int64_t *iters_done, double *rel_gaps);

/* x of every problem, x_l at X + l*n (n x nrhs doubles), host or device. */
pcdm_status pcdm_batch_get_x(pcdm_batch_handle h, double *X_out, int32_t on_device);

/* Replace every x (same layout; warm start) and recompute the residuals. */
pcdm_status pcdm_batch_set_x(pcdm_batch_handle h, const double *X_in, int32_t on_device);

/* New lambdas (nrhs host doubles, finite and >= 0); x and the residuals are kept
 * (the next point of a regularisation path starts from the current x). */
pcdm_status pcdm_batch_set_lambda(pcdm_batch_handle h, const double *lambdas);

/* x = 0, g_l = -b_l, k = 0; clears a failed state. */
pcdm_status pcdm_batch_reset(pcdm_batch_handle h);

/* Counters as in pcdm_stats, with updates counted per problem (tau per active
 * problem per iteration) and gathered / scattered nonzeros counted per column
 * read. */
pcdm_status pcdm_batch_get_stats(pcdm_batch_handle h, pcdm_stats *out);
pcdm_status pcdm_batch_reset_stats(pcdm_batch_handle h);

void pcdm_batch_destroy(pcdm_batch_handle h);

/* Autotuner of the batched iteration kernel (NEXT row 1 of the build's scope:
 * the launch shape of k_batch_iter).  A group of bp lanes (one per right-hand
 * side) owns a sampled column at a time; the grid decides how many columns a
 * group takes per iteration (the tau-chunk) against how many groups share each
 * SM.  Times trial_iters iterations for every grid of 1, 2, ... blocks per SM
 * up to the co-resident limit (and the blocks tau needs), from the handle's
 * current state, which is restored after every trial (X, G, the iteration
 * counter and the statistics), and keeps the fastest for later steps and
 * solves.  *blocks_per_sm and *us_per_iteration (either may be NULL) receive
 * the choice and its time per iteration.  EINVAL for a bad tau or
 * trial_iters; ENOMEM when the state copy does not fit. */
pcdm_status pcdm_batch_autotune(pcdm_batch_handle h, int64_t tau, int64_t trial_iters, int32_t *blocks_per_sm,
                                double *us_per_iteration);

/* Last error of the batch handle; with NULL, that of a failed pcdm_batch_create
 * on this thread. */
const char *pcdm_batch_last_error(pcdm_batch_handle h);

/* ------------------------------------------------------------------------
 * Many independent problems: count LASSO problems, each with its own A_p, b_p
 * and lambda_p, all of the same dtype pair.  One thread block runs Algorithm 1
 * (tau-nice sampling with tau_p = min(tau, n_p), beta of Theorem ESO-nice for
 * (omega_p, tau_p, n_p)) for one problem with block barriers only, so small
 * problems of uneven size run side by side.  A check period (copy of the
 * active flags, iters_per_check iterations, FP64 refresh and duality gap of
 * every running problem, copy of the gap records) is captured once as a CUDA
 * graph and replayed; a problem stops at its first check with
 * gap / primal <= rel_gap_tol.  Meant for problems that fit one block's reach
 * (n up to about 1e5); each problem p follows a single-problem handle stepped
 * with the same seed and tau_p (with an FP64 refresh at every check).
 * ------------------------------------------------------------------------ */
typedef struct pcdm_multi_ctx *pcdm_multi_handle;

/* As[p], bs[p] (m_p entries of b_dtype), lambdas[p] for p < count (1 .. 65535),
 * host or device as As[p].on_device says; validated and copied as by
 * pcdm_create (opts likewise; sampling must be NICE).  The solves run on an
 * internal stream; cuda_stream is used for the copies of the set-up only. */
pcdm_status pcdm_multi_create(int64_t count, const pcdm_csc *As, const void *const *bs, int32_t b_dtype,
                              const double *lambdas, const pcdm_opts *opts, void *cuda_stream,
                              pcdm_multi_handle *out);

/* Iterate every problem from its current x until its relative gap is at most
 * rel_gap_tol (checks every iters_per_check iterations; 1 <= tau <= 256).
 * iters_done, rel_gaps: count entries each (may be NULL).  PCDM_ENOTCONV when a
 * problem ran max_iters iterations first. */
pcdm_status pcdm_multi_solve(pcdm_multi_handle h, int64_t tau, uint64_t seed, double rel_gap_tol,
                             int64_t max_iters, int64_t iters_per_check, int64_t *iters_done, double *rel_gaps);

/* x of problem p (n_p doubles, host memory). */
pcdm_status pcdm_multi_get_x(pcdm_multi_handle h, int64_t p, double *x_out);

/* x = 0 and g = -b for every problem, iteration counters to 0. */
pcdm_status pcdm_multi_reset(pcdm_multi_handle h);

/* Counters (updates = sum over problems of tau_p per iteration run). */
pcdm_status pcdm_multi_get_stats(pcdm_multi_handle h, pcdm_stats *out);

void pcdm_multi_destroy(pcdm_multi_handle h);
const char *pcdm_multi_last_error(pcdm_multi_handle h);

/* Free everything the handle owns.  NULL is ignored. */
void pcdm_destroy(pcdm_handle h);

/* Last error message of the handle ("" if none); valid until the next call on it.
 * With h == NULL: the last error of a failed pcdm_create, pcdm_sample or
 * pcdm_omega_noalloc on this thread. */
const char *pcdm_last_error(pcdm_handle h);

/* Static name of a status code. */
const char *pcdm_status_string(pcdm_status s);

#ifdef __cplusplus
}
#endif

#endif /* PCDM_H */

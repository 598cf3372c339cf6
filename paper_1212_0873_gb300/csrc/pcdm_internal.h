// Host-side declarations shared by the C-ABI implementation (pcdm_api.cu) and
// the kernel translation units (kernels_*.cu).  Not part of the public ABI.
//
// Device layout of A (built once by pcdm_create from the caller's CSC):
//   desc[i]   16-byte column descriptor {start of the padded segment / 4, nnz of
//             column i, 1/L_i (0 for an empty column)}: one vector load gives all a
//             kernel needs to walk column i and take its step.
//   prow[]    row indices, each column's segment starting at a multiple of G
//             entries (G = 4 for FP64/FP32 values, 8 for BF16) and padded to a
//             multiple of G with row 0 / value 0, so every segment is 16-byte
//             aligned and a whole number of 16-byte words (vector loads, bulk copies).
//   pval[]    values in the same layout.
// Both arrays carry kSlack trailing entries so that a lane may read a full run
// of E entries starting anywhere inside a segment.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pcdm_device.cuh"

namespace pcdm {

constexpr int kBlock = 256;          // threads per block of the grid-stride column kernels
constexpr int kFinishBlock = 256;    // threads of the single-block gap reduction
// Largest block of the persistent iteration kernel: 448 threads (up to 144
// registers each; 152 such blocks hold 65536 one-lane groups) for one lane per
// column, 256 (up to 255 registers) for wider groups, whose chunk loops need more.
__host__ __device__ constexpr int fused_max_block(int W) { return W == 1 ? 448 : 256; }
constexpr int kPipeMaxBlock = 448;   // block limit of the pipelined kernel (its chunk buffers fill shared memory)
constexpr int kPipeRoundsMaxBlock = 256;   // block limit of the pipelined rounds kernel (up to 255 registers)
constexpr int64_t kSlack = 1024;     // trailing entries of prow / pval
constexpr int kLaneRun = 16;         // entries a lane reads per chunk (16-byte vector loads)
// The warp-cooperative kernel (warp_kernels.cuh): the first warp_rounds<XT>()
// runs of 64 entries of a column are held in registers (longer columns loop
// over the rest: 256 entries with an FP32 residual, 192 with FP64, whose
// registers run out first); columns are prefetched into L2 kWarpAhead
// positions ahead of their loads; blocks of up to kWarpMaxBlock threads.
template <typename XT>
__host__ __device__ constexpr int warp_rounds()
{
    return sizeof(XT) == 8 ? 2 : 3;
}
constexpr int kWarpAhead = 4;
constexpr int kWarpMaxBlock = 512;

template <typename XT>
struct ColDesc;
template <>
struct alignas(16) ColDesc<double> {
    uint32_t pb4;      // segment start / 4
    int32_t cnt;       // nonzeros of the column
    double invL;       // 1 / ||a_i||^2, 0 for an empty column
};
template <>
struct alignas(16) ColDesc<float> {
    uint32_t pb4;
    int32_t cnt;
    float invL;
    float unused;
};

template <typename VT>
__host__ __device__ constexpr int pad_granule()
{
    return sizeof(VT) == 2 ? 8 : 4;
}

// Everything one PCDM1 iteration reads and writes.  XT is the dtype of g, h,
// 1/L and of the gradient accumulator; VT the dtype of the stored values.  x and
// the proximal step are FP64 in every precision pair (an FP32 x bounds the
// reachable relative duality gap at about 1e-6).
template <typename VT, typename XT>
struct IterArgs {
    const ColDesc<XT> *desc;
    const int32_t *prow;
    const VT *pval;
    double *x;
    XT *g;
    XT *g2;                     // second residual buffer of the pipelined kernel (equal to g at launch)
    XT *h;                      // h[j] = step of coordinate S_k[j]
    int32_t *S[2];              // S_k lives in S[k & 1]
    double inv_beta, lambda;
    int64_t n, tau;
    uint64_t seed;
    unsigned long long *counters;   // [0] gathered nnz, [1] scattered nnz, [2] nonzero updates
    unsigned long long *bar;        // grid-barrier counter of the fused kernel (0 at launch)
    int *status;                    // DEV_OK or DEV_TIMEOUT
    uint64_t timeout_ns;
    // Sampling (two-kernel form only for the non-nice kinds): 0 tau-nice,
    // 1 tau-independent (win[i] holds the key of the first pick of block i),
    // 2 (tau, p_b)-binomial (position kept iff its coin is below keep_T).
    int sampling;
    uint64_t keep_T;
    const unsigned long long *win;
    // Per-column heads for the pipelined kernels (NULL: copy rows and values
    // separately): column i's first kLaneRun row indices at head + i * stride,
    // its first kLaneRun values 64 bytes further.
    const unsigned char *head;
    // Objective: 0 LASSO, 1 SVM dual (Sec. 8.3), 2 logistic regression (Sec. 8.4);
    // kappa = lambda n for the SVM dual (the linear term in the scale of ||a_i||^2).
    // The rounds kernel, the asynchronous kernel and the batched kernels take problem 0 only.
    int problem;
    double kappa;
};

// Entries of a wide slot after its first chunk (the pipelined kernel): 8 for
// FP64 (32 cost the FP64 pipe more predicated products than the dependent loads
// they saved: 18.1 against 16.4 us per iteration at the bench workload), 16 for
// FP32 (11.8 against 12.3 us) and BF16 values.
template <typename VT>
__host__ __device__ constexpr int wide_tail()
{
    return sizeof(VT) == 8 ? kLaneRun / 2 : kLaneRun;
}

// Entries of one column head: kLaneRun (the first chunk), then wide_tail more,
// the pipelined kernel's wide slot.
template <typename VT>
__host__ __device__ constexpr int head_entries()
{
    return kLaneRun + wide_tail<VT>();
}

// Bytes of one column head: kLaneRun row indices, then kLaneRun values (the first
// chunk), then (wide heads) the next wide_tail row indices and values, so that
// the wide slot's entries come in one bulk copy.
template <typename VT>
__host__ __device__ constexpr int64_t head_stride()
{
    return int64_t(head_entries<VT>()) * (4 + int64_t(sizeof(VT)));
}

// Launch shape of the fused kernel.
struct FusedShape {
    int W = 1;          // lanes per column
    int blocks = 1;
    int threads = 32;
};

// Column kernels, instantiated for (double,double), (float,float), (bf16_t,float).
template <typename VT, typename XT>
struct Kernels {
    // Two-kernel form.  S_k must already be in S[k & 1].
    static cudaError_t gather(const IterArgs<VT, XT> &a, int W, int64_t k, cudaStream_t st);
    static cudaError_t scatter(const IterArgs<VT, XT> &a, int W, int64_t k, bool sample_next, cudaStream_t st);
    // Persistent cooperative kernel: iterations k0 .. k0+iters-1, S_{k0} already drawn;
    // leaves S_{k0+iters} drawn.
    static cudaError_t fused(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                             cudaStream_t st);
    // Largest co-resident grid of the fused kernel for W lanes per column and a block of `threads`.
    static int fused_max_blocks(int W, int threads);
    // Pipelined persistent kernel (one lane per column, tau <= blocks * threads).
    static cudaError_t fused_pipe(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                  bool zero_cert, cudaStream_t st);
    static int pipe_max_blocks(int threads);
    // Pipelined kernel for tau beyond the grid (several positions per thread per iteration).
    static cudaError_t fused_pipe_rounds(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                         cudaStream_t st);
    static int pipe_rounds_max_blocks(int threads);
    // Streaming persistent kernel for long columns (one lane per column, tau <= blocks * threads):
    // every chunk of a column reaches its thread by TMA bulk copies (stream_kernels.cuh).
    static cudaError_t fused_stream(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                    cudaStream_t st);
    static int stream_max_blocks(int threads);
    // Warp-cooperative persistent kernel for long columns (a warp shares each of its
    // columns, at most 32 positions per warp: tau <= 32 * warps of the grid; warp_kernels.cuh).
    static cudaError_t fused_warp(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                  bool zero_cert, cudaStream_t st);
    static int warp_max_blocks(int threads);
    // Asynchronous updates u0 .. u0+count-1 (no barrier; atomics on x and g).
    static cudaError_t async(const IterArgs<VT, XT> &a, int blocks, uint64_t nthreads, uint64_t u0, uint64_t count,
                             cudaStream_t st);
    static int async_max_blocks();
    // L_i = sum a_ri^2 (FP64), row counts and validation, on the caller's CSC layout.
    static cudaError_t setup_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                  int64_t n, double *L, int *rowcnt, int *flags, cudaStream_t st);
    // Padded layout: copy the columns into prow/pval at pbeg (entries) and write desc.
    // head + i * head_stride<VT>(): the first chunk of column i (rows, then values), then (wide
    // heads) its next wide_tail entries (rows, then values), zero-padded.
    static cudaError_t build_heads(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, int64_t n,
                                   unsigned char *head, cudaStream_t st);
    static cudaError_t build_layout(const int64_t *col_ptr, const int32_t *row_idx, const VT *val,
                                    const int64_t *pbeg, const double *L, int64_t n, ColDesc<XT> *desc,
                                    int32_t *prow, VT *pval, cudaStream_t st);
    // g64 += A x over the columns with x_i != 0.
    static cudaError_t refresh_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *x,
                                    int64_t n, double *g64, int W, cudaStream_t st);
    // Per-block partials (max |c_i|, sum |x_i|, sum x_i c_i), c = A^T r.
    static cudaError_t gap_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *r,
                                const double *x, int64_t n, double *part, int blocks, int W, cudaStream_t st);
    // The same for the SVM dual (problem 1) and logistic regression (problem 2):
    // three per-block sums each (see k_glm_gap_cols).
    static cudaError_t glm_gap_cols(int problem, const ColDesc<XT> *desc, const int32_t *prow, const VT *pval,
                                    const double *r, const double *x, int64_t n, double lambda, double kappa,
                                    double *part, int blocks, int W, cudaStream_t st);
    // Sign the stored values by the labels y (problem 1: y_i on column i; 2: y_r on row r).
    static cudaError_t apply_labels(int problem, const ColDesc<XT> *desc, const int32_t *prow, VT *pval, int64_t n,
                                    const double *y, cudaStream_t st);
};

// Deterministic two-kernel form (det_kernels.cuh; pcdm_opts.deterministic_scatter):
// fixed summation order and separately rounded products and sums.
template <typename VT, typename XT>
struct DetKernels {
    // Row-major copy of A: rcol / rval at rptr (the exclusive scan of the row
    // counts), each row sorted by column; cursor is m words of scratch.
    static cudaError_t build_rows(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                  int64_t n, const int64_t *rptr, unsigned long long *cursor, int32_t *rcol, VT *rval,
                                  cudaStream_t st);
    // Gradients and steps of S_k (in S[k & 1]); stamps mark[i] of the nonzero steps.
    static cudaError_t gather(const IterArgs<VT, XT> &a, const double *L64, double beta, unsigned long long *mark,
                              int64_t k, cudaStream_t st);
    // The nonzero steps of iteration k into g, row by row in increasing position.
    static cudaError_t scatter(const IterArgs<VT, XT> &a, const int64_t *rptr, const int32_t *rcol, const VT *rval,
                               const unsigned long long *mark, int64_t k, cudaStream_t st);
    // g64 = A x - b by rows in increasing column (and g = g64 rounded when g is FP32).
    static cudaError_t refresh(const int64_t *rptr, const int32_t *rcol, const VT *rval, const double *x,
                               const double *b, int64_t m, double *g64, XT *g, cudaStream_t st);
};
// out[0..m) = exclusive prefix sums of cnt, out[m] = the total (tile: scan_tile_count(m) + 1 int64).
cudaError_t launch_count_scan(const int *cnt, int64_t m, int64_t *out, int64_t *tile, cudaStream_t st);

template <typename VT, typename XT>
struct BatchArgs {
    const ColDesc<XT> *desc;
    const int32_t *prow;
    const VT *pval;
    double *X;                  // n x bp, FP64
    XT *G;                      // m x bp
    XT *H;                      // tau x bp: steps of the listed columns (list slot s at H[s * bp])
    int32_t *list;              // tau: the columns of the current iteration with a nonzero step
    unsigned *list_cnt;         // [2]: list length of iterations k with k & 1 = 0, 1 (0 at launch)
    const double *lambda;       // bp
    const int *active;          // bp: 0 = this problem is frozen (converged or padding)
    double inv_beta;
    int64_t n, tau;
    uint64_t seed;
    unsigned long long *counters;   // [0] gathered nnz (per column), [1] scattered nnz (per column), [2] nonzero steps
    unsigned long long *bar;
    int *status;
    uint64_t timeout_ns;
};

constexpr int kBatchBlock = 256;

// Batched kernels (batch_kernels.cuh), bp in {4, 8, 16, 32} right-hand sides.
template <typename VT, typename XT>
struct BatchKernels {
    // Persistent cooperative iterations k0 .. k0+iters-1 (two bounded grid barriers each).
    static cudaError_t iter(const BatchArgs<VT, XT> &a, int bp, int blocks, int64_t k0, int64_t iters,
                            cudaStream_t st);
    static int iter_max_blocks(int bp);
    // G64 (m x bp, holding -b) += A X over the columns with a nonzero x.
    static cudaError_t refresh(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *X,
                               int64_t n, int bp, double *G64, int blocks, cudaStream_t st);
    // Block partials of max|c|, sum|x|, sum x c per right-hand side, c = A^T R.
    static cudaError_t gap_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *R,
                                const double *X, int64_t n, int bp, double *part, int blocks, cudaStream_t st);
};
// Per right-hand side: block partials of ||r||^2, b^T r over the interleaved m x bp
// vectors, and the final gap records out[l * 9 + q] (q as in launch_gap_finish).
cudaError_t launch_batch_gap_rows(const double *R, const double *Bm, int64_t m, int bp, double *part, int blocks,
                                  cudaStream_t st);
// src[l * len + r] (FP64, or FP32 when src_is_f32) -> dst[r * bp + l] (FP64, 0 for l >= nsrc), and back.
cudaError_t launch_interleave(const void *src, int src_is_f32, int64_t len, int nsrc, int bp, double *dst,
                              cudaStream_t st);
cudaError_t launch_deinterleave(const double *src, int64_t len, int nout, int bp, double *dst, cudaStream_t st);
cudaError_t launch_batch_gap_finish(const double *pc, int nbc, const double *pr, int nbr, int bp,
                                    const double *lambda, double *out, cudaStream_t st);

// Many independent problems, one thread block each (multi_kernels.cuh).
constexpr int kMultiBlock = 256;   // threads per problem; tau <= kMultiBlock
constexpr int kMultiSplit = 16;    // blocks per problem in the refresh and gap kernels
template <typename VT, typename XT>
struct MultiInst {
    const ColDesc<XT> *desc;
    const int32_t *prow;
    const VT *pval;
    double *x;
    XT *g;
    double *g64;                // FP64 refresh target (aliases g in the FP64 form)
    const double *b;
    int64_t m, n, tau;
    double inv_beta, lambda;
};
template <typename VT, typename XT>
struct MultiKernels {
    // iters iterations of every active problem p, from its counter kcount[p]
    static cudaError_t iter(const MultiInst<VT, XT> *inst, const int *active, int64_t *kcount, int count,
                            int64_t iters, uint64_t seed, unsigned long long *counters, cudaStream_t st);
    // refresh and gap record (9 doubles) of every active problem; part: count x kMultiSplit x 5 doubles
    static cudaError_t gap(const MultiInst<VT, XT> *inst, const int *active, int count, double *part, double *rec,
                           cudaStream_t st);
};

// Active-set coordinate descent (active_set_kernels.cuh): FP64 u, q and sums for
// any stored value type; DT is the handle's iterate dtype (type of 1/L in desc).
template <typename VT, typename DT>
struct ActiveSetKernels {
    static cudaError_t gather(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval, const int32_t *sidx,
                              const double *c, int64_t nS, int64_t tau, uint64_t seed, int64_t k, double inv_beta,
                              const double *q, double *u, double *H, int32_t *Sbuf, cudaStream_t st);
    static cudaError_t scatter(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval, int64_t tau,
                               const double *H, const int32_t *Sbuf, double *q, cudaStream_t st);
    static cudaError_t refresh(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval, const int32_t *sidx,
                               int64_t nS, const double *u, double *q, cudaStream_t st);
    static cudaError_t resid(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval, const int32_t *sidx,
                             const double *c, int64_t nS, const double *q, const double *w, const double *u,
                             double *part, int blocks, cudaStream_t st);
    static cudaError_t rowcount(const ColDesc<DT> *desc, const int32_t *prow, const int32_t *sidx, int64_t nS,
                                int *rowcnt, cudaStream_t st);
};
// The support S = {i : x_i != 0} in increasing order (one block; *count = |S|).
cudaError_t launch_compact_support(const double *x, int64_t n, int32_t *sidx, int *count, cudaStream_t st);
// sgn[p] = sign(x[sidx[p]]); c[p] = src[sidx[p]] if src, else -lambda * sgn[p].
cudaError_t launch_as_linear(const double *x, const double *src, const int32_t *sidx, int64_t nS, double lambda,
                             double *c, double *sgn, cudaStream_t st);

// Type-independent kernels (kernels_common.cu).
cudaError_t launch_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S, cudaStream_t st);
// S_k of sampling `kind` (0, 2: tau-nice positions; 1: tau-independent picks,
// claiming win[pick] when win is not NULL); keep (may be NULL) receives the
// binomial keep flags for kind 2.
cudaError_t launch_sample_kind(int kind, uint64_t seed, int64_t k, int64_t n, int64_t tau, uint64_t keep_T,
                               int32_t *S, unsigned long long *win, uint8_t *keep, cudaStream_t st);
cudaError_t launch_check_colptr(const int64_t *col_ptr, int64_t n, int64_t nnz, int *flags, cudaStream_t st);
cudaError_t launch_check_finite(const double *v, int64_t count, int *flags, cudaStream_t st);
cudaError_t launch_max_int(const int *a, int64_t count, int *out, cudaStream_t st);
cudaError_t launch_convert_b(const void *b_in, int b_is_f32, int64_t m, double *b_out, cudaStream_t st);
template <typename XT>
cudaError_t launch_neg_store(XT *g, const double *b, int64_t m, cudaStream_t st);        // g = -b
template <typename XT>
cudaError_t launch_store_from_f64(XT *dst, const double *src, int64_t m, cudaStream_t st);
cudaError_t launch_f64_to_f32(float *dst, const double *src, int64_t count, cudaStream_t st);
cudaError_t launch_gap_rows(const double *r, const double *b, int64_t m, double *part, int blocks, cudaStream_t st);
cudaError_t launch_gap_finish(const double *pc, int nbc, const double *pr, int nbr, double *out, double lambda,
                              cudaStream_t st);
// SVM dual and logistic regression (problems 1 and 2): flag labels other than
// +-1; scale v by a constant; rows part of the gap (block partials of ||r||^2
// for the SVM dual, of sum_r log(1 + exp(-r_r)) for logistic regression); and
// the record out = {P, D, gap, t1, t2, t3, rows, 0, 0} from the column
// partials t of k_glm_gap_cols (n = number of columns).
cudaError_t launch_check_labels(const double *y, int64_t count, int *flags, cudaStream_t st);
cudaError_t launch_scale(double *v, int64_t count, double factor, cudaStream_t st);
cudaError_t launch_glm_gap_rows(int problem, const double *r, int64_t m, double *part, int blocks, cudaStream_t st);
cudaError_t launch_glm_gap_finish(int problem, const double *pc, int nbc, const double *pr, int nbr, double lambda,
                                  int64_t n, double *out, cudaStream_t st);
cudaError_t launch_barrier_selftest(unsigned long long *bar, int *status, uint64_t timeout_ns, int blocks,
                                    cudaStream_t st);
// Exclusive scan of the padded column lengths: pbeg[i] = sum_{q<i} roundup(cnt_q, granule),
// pbeg[n] = total.  `tile` is scratch of scan_tile_count(n) + 1 int64.
int64_t scan_tile_count(int64_t n);
cudaError_t launch_padded_scan(const int64_t *col_ptr, int64_t n, int granule, int64_t *pbeg, int64_t *tile,
                               cudaStream_t st);

// No-allocation row counts (kernels_common.cu): the static scratch of the
// current device (row counters, then flags and result words) and its kernel.
constexpr int kMaxNoAllocDevices = 64;
cudaError_t noalloc_rows_scratch(int device, int **rows, int **tail);
cudaError_t launch_rows_checked(const int64_t *col_ptr, const int32_t *row_idx, int64_t m, int64_t n, int64_t nnz,
                                int *cnt, int *flags, cudaStream_t st);

// Validation flag bits (setup kernels).
enum : int {
    FLAG_COLPTR = 1,      // col_ptr not monotone, not starting at 0 or not ending at nnz
    FLAG_ROW_RANGE = 2,   // a row index outside [0, m)
    FLAG_ROW_ORDER = 4,   // rows of a column not strictly increasing
    FLAG_NONFINITE = 8,   // a non-finite value in A
    FLAG_B_NONFINITE = 16,// a non-finite value in b
    FLAG_LABEL = 32       // a label other than -1 or +1
};

}  // namespace pcdm

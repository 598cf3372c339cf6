// Host-side declarations shared by the C-ABI implementation (pcdm_api.cu) and
// the kernel translation units (kernels_*.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pcdm_device.cuh"

namespace pcdm {

constexpr int kBlock = 256;          // threads per block of every column kernel
constexpr int kFinishBlock = 256;    // threads of the single-block gap reduction

// Everything one PCDM1 iteration reads and writes.  XT is the dtype of x, g, h,
// L and of the gradient accumulator; VT the dtype of the stored values.
template <typename VT, typename XT>
struct IterArgs {
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const VT *val;
    const XT *L;
    XT *x;
    XT *g;
    XT *h;                      // h[j] = step of coordinate S_k[j]
    int32_t *S[2];              // S_k lives in S[k & 1]
    XT beta, lambda;
    int64_t n, tau;
    uint64_t seed;
    unsigned long long *counters;   // [0] gathered nnz, [1] scattered nnz, [2] nonzero updates
    unsigned long long *bar;        // grid-barrier counter of the fused kernel (0 at launch)
    int *status;                    // DEV_OK or DEV_TIMEOUT
    uint64_t timeout_ns;
};

// Column kernels, instantiated for (double,double), (float,float), (bf16_t,float).
template <typename VT, typename XT>
struct Kernels {
    // S_{k} must already be in S[k & 1].  Gather + prox + x update for j < tau.
    static cudaError_t gather(const IterArgs<VT, XT> &a, int W, int64_t k, cudaStream_t st);
    // Scatter of the columns with h != 0; with sample_next, also S_{k+1} -> S[(k+1) & 1].
    static cudaError_t scatter(const IterArgs<VT, XT> &a, int W, int64_t k, bool sample_next, cudaStream_t st);
    // Persistent cooperative kernel: iterations k0 .. k0+iters-1, S_{k0} already drawn;
    // leaves S_{k0+iters} drawn.  `blocks` must not exceed fused_max_blocks(W).
    static cudaError_t fused(const IterArgs<VT, XT> &a, int W, int64_t k0, int64_t iters, int blocks,
                             cudaStream_t st);
    static int fused_max_blocks(int W);
    // L_i = sum a_ri^2 (FP64), row counts and validation of rows/values.
    static cudaError_t setup_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                  int64_t n, double *L, int *rowcnt, int *flags, cudaStream_t st);
    // g64 += A x over the columns with x_i != 0.
    static cudaError_t refresh_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, const XT *x,
                                    int64_t n, double *g64, int W, cudaStream_t st);
    // Per-block partials (max |c_i|, sum |x_i|, sum x_i c_i), c = A^T r.
    static cudaError_t gap_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, const double *r,
                                const XT *x, int64_t n, double *part, int blocks, int W, cudaStream_t st);
};

// Type-independent kernels (kernels_common.cu).
cudaError_t launch_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S, cudaStream_t st);
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
cudaError_t launch_barrier_selftest(unsigned long long *bar, int *status, uint64_t timeout_ns, int blocks,
                                    cudaStream_t st);

// Validation flag bits (setup kernels).
enum : int {
    FLAG_COLPTR = 1,      // col_ptr not monotone, not starting at 0 or not ending at nnz
    FLAG_ROW_RANGE = 2,   // a row index outside [0, m)
    FLAG_ROW_ORDER = 4,   // rows of a column not strictly increasing
    FLAG_NONFINITE = 8,   // a non-finite value in A
    FLAG_B_NONFINITE = 16 // a non-finite value in b
};

}  // namespace pcdm

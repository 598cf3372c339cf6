/*
 * libpcdm_gen: seeded synthetic LASSO instances generated on the GPU.
 *
 * Input generation only (no step of the method): it serves the solver and the
 * tests alike, for sizes that host generation cannot reach (billions of
 * nonzeros).  Every number is a function of (seed, index) through
 * Philox4x32-10 (Salmon et al., SC'11), key = (lo32(seed), hi32(seed)), so a
 * column, an x* entry or a noise term can be regenerated alone.
 *
 * pcdm_gen_per_col writes, into caller-allocated device memory:
 *   col_ptr[i] = i * per_col                      (n + 1 int64)
 *   row_idx    column i: per_col distinct rows in [0, m), ascending.  Slot s
 *              draws W = words 0,1 of Philox(counter (lo32 i, hi32 i, t, 0x636f6c31))
 *              for t = 0, 1, 2, ... until floor(W * m / 2^64) differs from the
 *              rows of the earlier slots (t continues across slots); the slots
 *              are then sorted.                   (n * per_col int32)
 *   val        entry e of column i: the Irwin-Hall(12) approximation of N(0,1),
 *              ((u_0 + u_1) + ... + u_11) - 6 in FP32 left to right, u_j =
 *              (w_j >> 8) * 2^-24 from the 12 words of Philox(counter
 *              (lo32 i, hi32 i, e, 0x76616c31 + c)), c = 0, 1, 2; stored as
 *              val_dtype (0 FP64, 1 FP32, 2 BF16 rounded to nearest even)
 *   x_star     x*_i != 0 iff word 0 of Philox(counter (lo32 i, hi32 i, 0,
 *              0x78737431)) < x_density * 2^32; then x*_i = +-(1 + w1 * 2^-32),
 *              sign - iff w2 is odd                (n doubles)
 *   b          b_r = (A x*)_r + noise_sd * (IH_r - 6), IH_r the sum of 12
 *              doubles w * 2^-32 of the words of Philox(counter (lo32 r, hi32 r, c,
 *              0x6e6f6931)), c = 0, 1, 2; (A x*)_r summed in FP64 (atomic
 *              order); stored as b_dtype (0 FP64, 1 FP32)  (m entries)
 *   *lambda_max (host) = max_i |a_i^T b| in FP64, with b as stored
 * scratch: m doubles of device memory.  1 <= per_col <= 32, per_col <= m,
 * m < 2^32.  Returns 0, or a cudaError_t value.
 */
#ifndef PCDM_GEN_H
#define PCDM_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int pcdm_gen_per_col(int64_t m, int64_t n, int32_t per_col, uint64_t seed, int32_t val_dtype,
                     double x_density, double noise_sd, int32_t b_dtype, int64_t *col_ptr, int32_t *row_idx,
                     void *val, void *b, double *x_star, double *scratch, double *lambda_max,
                     void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif

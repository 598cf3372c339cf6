// Coordinate descent on an active set S (the support of x), without the prox.
//
// On a fixed sign pattern s_S the LASSO optimality condition is linear,
//     A_S^T (A_S x_S - b) + lambda s_S = 0,
// and the implicit-function derivatives of x_S(b, lambda) solve the same normal
// equations (A_S^T A_S) u = v.  Both are minimisers of a quadratic
//     Q(u) = 1/2 ||A_S u - y||^2 - c^T u   (gradient a_i^T (A_S u - y) - c_i),
// solved here by the coordinate kernel of PCDM1 (Algorithm 1) with the
// tau-nice sampling over the positions of S and the step of eq. (h(x)) with
// Omega = 0 (no prox): h_i = -(a_i^T q - c_i) / (beta L_i), q = A_S u - y
// maintained by red.global.add.  Everything is FP64 (u, q, c, the sums), for
// any stored value type, since these solves serve finite-difference-accurate
// derivatives.  Gather and scatter are separate kernels (the sets are small).
#pragma once

#include "pcdm_kernels.cuh"

namespace pcdm {

// Gather phase of one iteration: position j of the sample picks p = pi_k(j) in
// [0, nS), column i = sidx[p]; h = -(a_i^T q - c_p) (1/L_i)(1/beta); u_i += h.
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock) k_as_gather(const ColDesc<DT> *__restrict__ desc,
                                                      const int32_t *__restrict__ prow, const VT *__restrict__ pval,
                                                      const int32_t *__restrict__ sidx, const double *__restrict__ c,
                                                      int64_t nS, int64_t tau, uint64_t seed, int64_t k,
                                                      double inv_beta, const double *__restrict__ q,
                                                      double *__restrict__ u, double *__restrict__ H,
                                                      int32_t *__restrict__ Sbuf)
{
    const SampleKey key = make_sample_key(seed, k, nS);
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t j = int64_t(blockIdx.x) * kBlock + threadIdx.x; j < tau; j += stride) {
        const int32_t p = sample_index(uint32_t(j), key);
        const int32_t i = sidx[p];
        const Col<DT> col = load_col(desc, i);
        double acc = 0.0;
        for (int cs = 0; cs < col.cnt; cs += kE) {
            Chunk<kE, DT> t;
            ld_chunk<kE>(t, prow, pval, col.pbeg + cs);
            const int valid = col.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) acc = fma(double(t.val[e]), ldcg(q + t.row[e]), acc);
        }
        const double h = col.invL == DT(0) ? 0.0 : -(acc - c[p]) * (double(col.invL) * inv_beta);
        u[i] += h;
        H[j] = h;
        Sbuf[j] = i;
    }
}

// Scatter phase: q_r += a_ri h for the iteration's columns.
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock) k_as_scatter(const ColDesc<DT> *__restrict__ desc,
                                                       const int32_t *__restrict__ prow, const VT *__restrict__ pval,
                                                       int64_t tau, const double *__restrict__ H,
                                                       const int32_t *__restrict__ Sbuf, double *__restrict__ q)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t j = int64_t(blockIdx.x) * kBlock + threadIdx.x; j < tau; j += stride) {
        const double h = H[j];
        if (h == 0.0) continue;
        const Col<DT> col = load_col(desc, Sbuf[j]);
        for (int cs = 0; cs < col.cnt; cs += kE) {
            Chunk<kE, DT> t;
            ld_chunk<kE>(t, prow, pval, col.pbeg + cs);
            const int valid = col.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) red_add(q + t.row[e], double(t.val[e]) * h);
        }
    }
}

// q (holding -y, or 0) += A_S u_S.
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock) k_as_refresh(const ColDesc<DT> *__restrict__ desc,
                                                       const int32_t *__restrict__ prow, const VT *__restrict__ pval,
                                                       const int32_t *__restrict__ sidx, int64_t nS,
                                                       const double *__restrict__ u, double *__restrict__ q)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t p = int64_t(blockIdx.x) * kBlock + threadIdx.x; p < nS; p += stride) {
        const int32_t i = sidx[p];
        const double ui = u[i];
        if (ui == 0.0) continue;
        const Col<DT> col = load_col(desc, i);
        for (int cs = 0; cs < col.cnt; cs += kE) {
            Chunk<kE, DT> t;
            ld_chunk<kE>(t, prow, pval, col.pbeg + cs);
            const int valid = col.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) red_add(q + t.row[e], double(t.val[e]) * ui);
        }
    }
}

// Block partials of sum_p (a_i^T q - c_p)^2 and sum_p c_p^2 (relative residual
// of the normal equations), and of sum_p w_p u_{i_p} (w may be NULL).
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock) k_as_resid(const ColDesc<DT> *__restrict__ desc,
                                                     const int32_t *__restrict__ prow, const VT *__restrict__ pval,
                                                     const int32_t *__restrict__ sidx, const double *__restrict__ c,
                                                     int64_t nS, const double *__restrict__ q,
                                                     const double *__restrict__ w, const double *__restrict__ u,
                                                     double *__restrict__ part)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    double rr = 0.0, cc = 0.0, wu = 0.0;
    for (int64_t p = int64_t(blockIdx.x) * kBlock + threadIdx.x; p < nS; p += stride) {
        const int32_t i = sidx[p];
        const Col<DT> col = load_col(desc, i);
        double acc = 0.0;
        for (int cs = 0; cs < col.cnt; cs += kE) {
            Chunk<kE, DT> t;
            ld_chunk<kE>(t, prow, pval, col.pbeg + cs);
            const int valid = col.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) acc = fma(double(t.val[e]), q[t.row[e]], acc);
        }
        const double r = acc - c[p];
        rr += r * r;
        cc += c[p] * c[p];
        if (w) wu += w[p] * u[i];
    }
    __shared__ double sm[3][kBlock / 32];
    rr = warp_sum(rr);
    cc = warp_sum(cc);
    wu = warp_sum(wu);
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = rr;
        sm[1][threadIdx.x >> 5] = cc;
        sm[2][threadIdx.x >> 5] = wu;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int t = 0; t < kBlock / 32; ++t) {
            a0 += sm[0][t];
            a1 += sm[1][t];
            a2 += sm[2][t];
        }
        part[3 * blockIdx.x + 0] = a0;
        part[3 * blockIdx.x + 1] = a1;
        part[3 * blockIdx.x + 2] = a2;
    }
}

// Row counts of A_S (for omega_S).
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock) k_as_rowcount(const ColDesc<DT> *__restrict__ desc,
                                                        const int32_t *__restrict__ prow,
                                                        const int32_t *__restrict__ sidx, int64_t nS,
                                                        int *__restrict__ rowcnt)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t p = int64_t(blockIdx.x) * kBlock + threadIdx.x; p < nS; p += stride) {
        const Col<DT> col = load_col(desc, sidx[p]);
        for (int e = 0; e < col.cnt; ++e) atomicAdd(rowcnt + prow[col.pbeg + e], 1);
    }
}

template <typename VT, typename DT>
cudaError_t ActiveSetKernels<VT, DT>::gather(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval,
                                             const int32_t *sidx, const double *c, int64_t nS, int64_t tau,
                                             uint64_t seed, int64_t k, double inv_beta, const double *q, double *u,
                                             double *H, int32_t *Sbuf, cudaStream_t st)
{
    const int64_t blocks = (tau + kBlock - 1) / kBlock;
    k_as_gather<VT, DT><<<unsigned(blocks < 1 ? 1 : (blocks > 4864 ? 4864 : blocks)), kBlock, 0, st>>>(
        desc, prow, pval, sidx, c, nS, tau, seed, k, inv_beta, q, u, H, Sbuf);
    return cudaGetLastError();
}

template <typename VT, typename DT>
cudaError_t ActiveSetKernels<VT, DT>::scatter(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval,
                                              int64_t tau, const double *H, const int32_t *Sbuf, double *q,
                                              cudaStream_t st)
{
    const int64_t blocks = (tau + kBlock - 1) / kBlock;
    k_as_scatter<VT, DT><<<unsigned(blocks < 1 ? 1 : (blocks > 4864 ? 4864 : blocks)), kBlock, 0, st>>>(
        desc, prow, pval, tau, H, Sbuf, q);
    return cudaGetLastError();
}

template <typename VT, typename DT>
cudaError_t ActiveSetKernels<VT, DT>::refresh(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval,
                                              const int32_t *sidx, int64_t nS, const double *u, double *q,
                                              cudaStream_t st)
{
    if (nS <= 0) return cudaSuccess;
    const int64_t blocks = (nS + kBlock - 1) / kBlock;
    k_as_refresh<VT, DT><<<unsigned(blocks > 4864 ? 4864 : blocks), kBlock, 0, st>>>(desc, prow, pval, sidx, nS,
                                                                                      u, q);
    return cudaGetLastError();
}

template <typename VT, typename DT>
cudaError_t ActiveSetKernels<VT, DT>::resid(const ColDesc<DT> *desc, const int32_t *prow, const VT *pval,
                                            const int32_t *sidx, const double *c, int64_t nS, const double *q,
                                            const double *w, const double *u, double *part, int blocks,
                                            cudaStream_t st)
{
    k_as_resid<VT, DT><<<unsigned(blocks), kBlock, 0, st>>>(desc, prow, pval, sidx, c, nS, q, w, u, part);
    return cudaGetLastError();
}

template <typename VT, typename DT>
cudaError_t ActiveSetKernels<VT, DT>::rowcount(const ColDesc<DT> *desc, const int32_t *prow, const int32_t *sidx,
                                               int64_t nS, int *rowcnt, cudaStream_t st)
{
    if (nS <= 0) return cudaSuccess;
    const int64_t blocks = (nS + kBlock - 1) / kBlock;
    k_as_rowcount<VT, DT><<<unsigned(blocks > 4864 ? 4864 : blocks), kBlock, 0, st>>>(desc, prow, sidx, nS, rowcnt);
    return cudaGetLastError();
}

}  // namespace pcdm

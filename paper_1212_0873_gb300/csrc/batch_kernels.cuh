// Batched PCDM1: one matrix A, BP right-hand sides b_0 .. b_{BP-1}, each with
// its own lambda, solved together.  Every problem runs Algorithm 1 with the
// same sample S_k (the sampler of pcdm_step), so each right-hand side follows
// exactly the trajectory of a single-problem run with the same seed; what the
// batch shares is the read of each sampled column of A.
//
// Layout: the residuals and iterates are interleaved by right-hand side,
// G[r * BP + l] (m x BP, the iterate dtype XT), X[i * BP + l] (n x BP, FP64),
// so that the BP lanes working on one column read BP consecutive residual
// entries of a row: one or two 32-byte sectors instead of BP scattered ones.
//
// Work mapping: a group of BP lanes owns one sampled column at a time, lane l
// the right-hand side l.  The column's rows and values are read by every lane
// of the group at the same addresses (broadcast loads).  Phase 1 computes the
// BP gradients, steps and x updates; phase 2 (after a bounded grid barrier)
// scatters the nonzero steps with red.global.add into the interleaved rows.
#pragma once

#include "pcdm_kernels.cuh"

namespace pcdm {

// The step of eq. (h(x)) for one coordinate of one problem, returning h and
// the new x.  FP64 iterates: the FP64 step of prox_step.  FP32 iterates: the
// step is formed in FP32 from the gradient, without rounding x: with
// d = -grad/(beta L) and t = lambda/(beta L),
//   x + d >  t  ->  h = d - t,   x + d < -t  ->  h = d + t,   else h = -x,
// which is soft(x + d, t) - x; only the comparison sees x in FP32.  x + h is
// formed in FP64.  The fixed point (h = 0 exactly when d = -/+ t, i.e.
// grad = -/+ lambda) does not depend on the precision of x.
template <typename XT>
__device__ __forceinline__ double step_delta(double xi, XT grad, XT invL, double inv_beta, double lambda, double &xn)
{
    if constexpr (sizeof(XT) == 8) {
        xn = prox_step(xi, grad, invL, inv_beta, lambda);
        return xn - xi;
    } else {
        if (invL == 0.f) {
            xn = 0.0;
            return -xi;
        }
        const float ibl = invL * float(inv_beta);
        const float t = float(lambda) * ibl;
        const float d = -grad * ibl;
        const float u = float(xi) + d;
        double h;
        if (u > t) {
            h = double(d - t);
            xn = xi + h;
        } else if (u < -t) {
            h = double(d + t);
            xn = xi + h;
        } else {
            h = -xi;
            xn = 0.0;
        }
        return h;
    }
}


template <typename VT, typename XT, int BP>
__global__ void __launch_bounds__(kBatchBlock) k_batch_iter(const BatchArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    const int lane = threadIdx.x & (BP - 1);
    const unsigned gmask = group_mask<BP>(threadIdx.x & 31);
    const int64_t grp = (int64_t(blockIdx.x) * kBatchBlock + threadIdx.x) / BP;
    const int64_t ngrp = int64_t(gridDim.x) * kBatchBlock / BP;
    const double lam = a.lambda[lane];
    const bool act = a.active[lane] != 0;
    unsigned long long target = 0;
    Counters cnt;

    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const SampleKey key = make_sample_key(a.seed, k, a.n);
        // ---------------- phase 1: gradients, steps, x
        // Round r of this group covers positions grp + (r*BP + q)*ngrp, q < BP;
        // lane q draws the sample of the q-th one.
        for (int64_t base = grp; base < a.tau; base += ngrp * BP) {
            const int64_t jq = base + int64_t(lane) * ngrp;
            int32_t iq = 0;
            if (jq < a.tau) {
                iq = sample_index(uint32_t(jq), key);
                a.S[jq] = iq;
            }
            for (int q = 0; q < BP; ++q) {
                const int64_t j = base + int64_t(q) * ngrp;
                if (j >= a.tau) break;   // the same for every lane of the group
                const int32_t i = __shfl_sync(gmask, iq, q, BP);
                const Col<XT> c = load_col(a.desc, i);
                const double xi = ldcg(a.X + int64_t(i) * BP + lane);
                XT acc = XT(0);
                for (int cs = 0; cs < c.cnt; cs += kE) {
                    Chunk<kE, XT> t;
                    ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + cs);
                    const int valid = c.cnt - cs;
                    XT gv[kE];
#pragma unroll
                    for (int e = 0; e < kE; ++e)
                        gv[e] = (e < valid) ? ldcg(a.G + int64_t(t.row[e]) * BP + lane) : XT(0);
#pragma unroll
                    for (int e = 0; e < kE; ++e)
                        if (e < valid) acc = fma(t.val[e], gv[e], acc);
                }
                double h = 0.0;
                if (act) {
                    double xn;
                    h = step_delta<XT>(xi, acc, c.invL, a.inv_beta, lam, xn);
                    if (h != 0.0) a.X[int64_t(i) * BP + lane] = xn;
                }
                a.H[j * BP + lane] = XT(h);
                if (lane == 0) cnt.gathered += (unsigned long long)c.cnt;
                if (h != 0.0) cnt.nonzero += 1;
            }
        }
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;

        // ---------------- phase 2: scatter of the nonzero steps
        for (int64_t j = grp; j < a.tau; j += ngrp) {
            const XT h = ldcg(a.H + j * BP + lane);
            if (!__any_sync(gmask, h != XT(0))) continue;
            const int32_t i = ldcg(a.S + j);
            const Col<XT> c = load_col(a.desc, i);
            for (int cs = 0; cs < c.cnt; cs += kE) {
                Chunk<kE, XT> t;
                ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + cs);
                const int valid = c.cnt - cs;
                if (h != XT(0)) {
#pragma unroll
                    for (int e = 0; e < kE; ++e)
                        if (e < valid) red_add(a.G + int64_t(t.row[e]) * BP + lane, t.val[e] * h);
                }
            }
            if (lane == 0) cnt.scattered += (unsigned long long)c.cnt;
        }
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;
    }
    flush_counters(cnt, a.counters);
}

// Refresh: G64 (m x BP, FP64, holding -b) += A X over the columns with a nonzero x.
template <typename VT, typename XT, int BP>
__global__ void __launch_bounds__(kBatchBlock) k_batch_refresh(const ColDesc<XT> *__restrict__ desc,
                                                               const int32_t *__restrict__ prow,
                                                               const VT *__restrict__ pval,
                                                               const double *__restrict__ X, int64_t n,
                                                               double *__restrict__ G64)
{
    const int lane = threadIdx.x & (BP - 1);
    const unsigned gmask = group_mask<BP>(threadIdx.x & 31);
    const int64_t ngrp = int64_t(gridDim.x) * kBatchBlock / BP;
    for (int64_t i = (int64_t(blockIdx.x) * kBatchBlock + threadIdx.x) / BP; i < n; i += ngrp) {
        const double xi = __ldg(X + i * BP + lane);
        if (!__any_sync(gmask, xi != 0.0)) continue;
        const Col<XT> c = load_col(desc, int32_t(i));
        for (int cs = 0; cs < c.cnt; cs += kE) {
            Chunk<kE, XT> t;
            ld_chunk<kE>(t, prow, pval, c.pbeg + cs);
            const int valid = c.cnt - cs;
            if (xi != 0.0) {
#pragma unroll
                for (int e = 0; e < kE; ++e)
                    if (e < valid) red_add(G64 + int64_t(t.row[e]) * BP + lane, double(t.val[e]) * xi);
            }
        }
    }
}

// Gap, column part, per right-hand side l: c_il = a_i^T r_l in FP64; block
// partials part[(block * BP + l) * 3 + {0,1,2}] = max|c_il|, sum|x_il|, sum x_il c_il.
template <typename VT, typename XT, int BP>
__global__ void __launch_bounds__(kBatchBlock) k_batch_gap_cols(const ColDesc<XT> *__restrict__ desc,
                                                                const int32_t *__restrict__ prow,
                                                                const VT *__restrict__ pval,
                                                                const double *__restrict__ R,
                                                                const double *__restrict__ X, int64_t n,
                                                                double *__restrict__ part)
{
    const int lane = threadIdx.x & (BP - 1);
    const int64_t ngrp = int64_t(gridDim.x) * kBatchBlock / BP;
    double cmax = 0.0, l1 = 0.0, xc = 0.0;
    for (int64_t i = (int64_t(blockIdx.x) * kBatchBlock + threadIdx.x) / BP; i < n; i += ngrp) {
        const Col<XT> c = load_col(desc, int32_t(i));
        double acc = 0.0;
        for (int cs = 0; cs < c.cnt; cs += kE) {
            Chunk<kE, XT> t;
            ld_chunk<kE>(t, prow, pval, c.pbeg + cs);
            const int valid = c.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) acc = fma(double(t.val[e]), __ldg(R + int64_t(t.row[e]) * BP + lane), acc);
        }
        const double xi = __ldg(X + i * BP + lane);
        cmax = fmax(cmax, fabs(acc));
        l1 += fabs(xi);
        xc += xi * acc;
    }
    __shared__ double sm[3][kBatchBlock];
    sm[0][threadIdx.x] = cmax;
    sm[1][threadIdx.x] = l1;
    sm[2][threadIdx.x] = xc;
    __syncthreads();
    if (threadIdx.x < BP) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int q = threadIdx.x; q < kBatchBlock; q += BP) {
            a0 = fmax(a0, sm[0][q]);
            a1 += sm[1][q];
            a2 += sm[2][q];
        }
        double *o = part + (int64_t(blockIdx.x) * BP + threadIdx.x) * 3;
        o[0] = a0;
        o[1] = a1;
        o[2] = a2;
    }
}

// ---------------------------------------------------------------------------
// Launchers (instantiated per dtype pair in kernels_batch_*.cu).
#define PCDM_DISPATCH_BP(BPV, ...)                       \
    switch (BPV) {                                       \
    case 4: { constexpr int BP_ = 4; __VA_ARGS__ } break;   \
    case 8: { constexpr int BP_ = 8; __VA_ARGS__ } break;   \
    case 16: { constexpr int BP_ = 16; __VA_ARGS__ } break; \
    case 32: { constexpr int BP_ = 32; __VA_ARGS__ } break; \
    default: return cudaErrorInvalidValue;               \
    }

template <typename VT, typename XT>
int BatchKernels<VT, XT>::iter_max_blocks(int bp)
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (bp) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_iter<VT, XT, 4>, kBatchBlock, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_iter<VT, XT, 8>, kBatchBlock, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_iter<VT, XT, 16>, kBatchBlock, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_iter<VT, XT, 32>, kBatchBlock, 0); break;
    default: return 0;
    }
    if (e != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <typename VT, typename XT>
cudaError_t BatchKernels<VT, XT>::iter(const BatchArgs<VT, XT> &a, int bp, int blocks, int64_t k0, int64_t iters,
                                       cudaStream_t st)
{
    BatchArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    PCDM_DISPATCH_BP(bp, {
        return cudaLaunchCooperativeKernel((const void *)k_batch_iter<VT, XT, BP_>, dim3(unsigned(blocks)),
                                           dim3(kBatchBlock), params, 0, st);
    });
    return cudaSuccess;
}

template <typename VT, typename XT>
cudaError_t BatchKernels<VT, XT>::refresh(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval,
                                          const double *X, int64_t n, int bp, double *G64, int blocks,
                                          cudaStream_t st)
{
    PCDM_DISPATCH_BP(bp, {
        k_batch_refresh<VT, XT, BP_><<<dim3(unsigned(blocks)), kBatchBlock, 0, st>>>(desc, prow, pval, X, n, G64);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t BatchKernels<VT, XT>::gap_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval,
                                           const double *R, const double *X, int64_t n, int bp, double *part,
                                           int blocks, cudaStream_t st)
{
    PCDM_DISPATCH_BP(bp, {
        k_batch_gap_cols<VT, XT, BP_><<<dim3(unsigned(blocks)), kBatchBlock, 0, st>>>(desc, prow, pval, R, X, n,
                                                                                       part);
    });
    return cudaGetLastError();
}

}  // namespace pcdm

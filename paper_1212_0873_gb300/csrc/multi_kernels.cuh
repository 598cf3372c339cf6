// Many independent small LASSO problems (each its own A, b, lambda) solved at
// once: one thread block per problem runs Algorithm 1 (tau-nice sampling, the
// step of eq. (h(x)), beta of Theorem ESO-nice) with block barriers only, so a
// problem's iteration costs a few block-level synchronisations instead of grid
// barriers.  The blocks of converged problems return at once.  A second kernel,
// again one block per problem, refreshes the residual and evaluates the duality
// gap in FP64.
#pragma once

#include "pcdm_kernels.cuh"

namespace pcdm {

// One iteration-block's problem: iterations k .. k+iters-1 while active.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kMultiBlock) k_multi_iter(const MultiInst<VT, XT> *__restrict__ inst,
                                                            const int *__restrict__ active,
                                                            int64_t *__restrict__ kcount, int64_t iters,
                                                            uint64_t seed, unsigned long long *__restrict__ counters)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    const MultiInst<VT, XT> P = inst[p];
    __shared__ SampleKey skey;
    const int t = threadIdx.x;
    const int64_t k0 = kcount[p];
    Counters cnt;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        if (t == 0) skey = make_sample_key(seed, k, P.n);
        __syncthreads();
        XT h = XT(0);
        int32_t i = 0;
        if (t < P.tau) {
            i = sample_index(uint32_t(t), skey);
            const Col<XT> c = load_col(P.desc, i);
            const double xi = P.x[i];
            XT acc = XT(0);
            for (int cs = 0; cs < c.cnt; cs += kE) {
                Chunk<kE, XT> ch;
                ld_chunk<kE>(ch, P.prow, P.pval, c.pbeg + cs);
                acc += chunk_dot<kE, XT, XT, XT>(ch, P.g, c.cnt - cs);
            }
            const double xn = prox_step(xi, double(acc), double(c.invL), P.inv_beta, P.lambda);
            const double h64 = xn - xi;
            if (h64 != 0.0) P.x[i] = xn;
            h = XT(h64);
            cnt.gathered += (unsigned long long)c.cnt;
            if (h64 != 0.0) {
                cnt.nonzero += 1;
                cnt.scattered += (unsigned long long)c.cnt;
            }
        }
        __syncthreads();   // every gradient of iteration k read g_k
        if (t < P.tau && h != XT(0)) {
            const Col<XT> c = load_col(P.desc, i);
            for (int cs = 0; cs < c.cnt; cs += kE) {
                Chunk<kE, XT> ch;
                ld_chunk<kE>(ch, P.prow, P.pval, c.pbeg + cs);
                chunk_scatter<kE>(ch, P.g, h, c.cnt - cs);
            }
        }
        __threadfence_block();
        __syncthreads();   // g_{k+1} complete before the next gathers
    }
    if (t == 0) kcount[p] = k0 + iters;
    flush_counters(cnt, counters);
}

// Block reductions of the gap kernel.
__device__ __forceinline__ double block_sum(double v, double *sm)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kMultiBlock / 32; ++w) s += sm[w];
    return s;
}

__device__ __forceinline__ double block_max(double v, double *sm)
{
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kMultiBlock / 32; ++w) s = fmax(s, sm[w]);
    return s;
}

// Refresh (g64 = A x - b in FP64, then g = g64 in XT) and the gap record
// rec[p*9 + q] = {P, D, gap, ||c||_inf, s, ||r||^2, b^T r, ||x||_1, x^T c}.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kMultiBlock) k_multi_gap(const MultiInst<VT, XT> *__restrict__ inst,
                                                           const int *__restrict__ active, double *__restrict__ rec)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    const MultiInst<VT, XT> P = inst[p];
    const int t = threadIdx.x;
    __shared__ double sm[kMultiBlock / 32];
    for (int64_t r = t; r < P.m; r += kMultiBlock) P.g64[r] = -P.b[r];
    __syncthreads();
    for (int64_t i = t; i < P.n; i += kMultiBlock) {
        const double xi = P.x[i];
        if (xi == 0.0) continue;
        const Col<XT> c = load_col(P.desc, int32_t(i));
        for (int cs = 0; cs < c.cnt; cs += kE) {
            Chunk<kE, XT> ch;
            ld_chunk<kE>(ch, P.prow, P.pval, c.pbeg + cs);
            const int valid = c.cnt - cs;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) red_add(P.g64 + ch.row[e], double(ch.val[e]) * xi);
        }
    }
    __threadfence_block();
    __syncthreads();
    double cmax = 0.0, l1 = 0.0, xc = 0.0, rr = 0.0, br = 0.0;
    for (int64_t i = t; i < P.n; i += kMultiBlock) {
        const Col<XT> c = load_col(P.desc, int32_t(i));
        double acc = 0.0;
        for (int cs = 0; cs < c.cnt; cs += kE) {
            Chunk<kE, XT> ch;
            ld_chunk<kE>(ch, P.prow, P.pval, c.pbeg + cs);
            acc += chunk_dot<kE, XT, double, double>(ch, P.g64, c.cnt - cs);
        }
        const double xi = P.x[i];
        cmax = fmax(cmax, fabs(acc));
        l1 += fabs(xi);
        xc += xi * acc;
    }
    for (int64_t r = t; r < P.m; r += kMultiBlock) {
        const double v = P.g64[r];
        rr += v * v;
        br += P.b[r] * v;
        if constexpr (sizeof(XT) == 4) P.g[r] = float(v);
    }
    cmax = block_max(cmax, sm);
    l1 = block_sum(l1, sm);
    xc = block_sum(xc, sm);
    rr = block_sum(rr, sm);
    br = block_sum(br, sm);
    if (t == 0) {
        const double lam = P.lambda;
        double s = 1.0;
        if (cmax > 0.0 && lam / cmax < 1.0) s = lam / cmax;
        double *o = rec + int64_t(p) * 9;
        o[0] = 0.5 * rr + lam * l1;
        o[1] = -0.5 * s * s * rr - s * br;
        o[2] = 0.5 * (1.0 - s) * (1.0 - s) * rr + (lam * l1 + s * xc);
        o[3] = cmax;
        o[4] = s;
        o[5] = rr;
        o[6] = br;
        o[7] = l1;
        o[8] = xc;
    }
}

template <typename VT, typename XT>
cudaError_t MultiKernels<VT, XT>::iter(const MultiInst<VT, XT> *inst, const int *active, int64_t *kcount,
                                       int count, int64_t iters, uint64_t seed, unsigned long long *counters,
                                       cudaStream_t st)
{
    k_multi_iter<VT, XT><<<dim3(unsigned(count)), kMultiBlock, 0, st>>>(inst, active, kcount, iters, seed, counters);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t MultiKernels<VT, XT>::gap(const MultiInst<VT, XT> *inst, const int *active, int count, double *rec,
                                      cudaStream_t st)
{
    k_multi_gap<VT, XT><<<dim3(unsigned(count)), kMultiBlock, 0, st>>>(inst, active, rec);
    return cudaGetLastError();
}

}  // namespace pcdm

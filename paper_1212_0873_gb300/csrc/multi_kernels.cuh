// Many independent small LASSO problems (each its own A, b, lambda) solved at
// once: one thread block per problem runs Algorithm 1 (tau-nice sampling, the
// step of eq. (h(x)), beta of Theorem ESO-nice) with block barriers only, so a
// problem's iteration costs a few block-level synchronisations instead of grid
// barriers.  The blocks of converged problems return at once.  The FP64 refresh
// and duality gap spread each problem over kMultiSplit blocks.
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

// Refresh and duality gap of every running problem, spread over kMultiSplit
// blocks per problem (blockIdx.x = problem, blockIdx.y = part): g64 = -b; then
// g64 += a_i x_i over the columns with x_i != 0 (FP64); then per-part partials
// of max|c_i|, sum|x_i|, sum x_i c_i (c = A^T g64) and of ||g64||^2, b^T g64, with
// g = g64 stored in the iterate dtype; then one block per problem turns the
// partials into the record rec[p*9 + q] = {P, D, gap, ||c||_inf, s, ||r||^2,
// b^T r, ||x||_1, x^T c}.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kMultiBlock) k_multi_negb(const MultiInst<VT, XT> *__restrict__ inst,
                                                            const int *__restrict__ active)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    const MultiInst<VT, XT> P = inst[p];
    const int64_t stride = int64_t(gridDim.y) * kMultiBlock;
    for (int64_t r = int64_t(blockIdx.y) * kMultiBlock + threadIdx.x; r < P.m; r += stride) P.g64[r] = -P.b[r];
}

template <typename VT, typename XT>
__global__ void __launch_bounds__(kMultiBlock) k_multi_refresh(const MultiInst<VT, XT> *__restrict__ inst,
                                                               const int *__restrict__ active)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    const MultiInst<VT, XT> P = inst[p];
    const int64_t stride = int64_t(gridDim.y) * kMultiBlock;
    for (int64_t i = int64_t(blockIdx.y) * kMultiBlock + threadIdx.x; i < P.n; i += stride) {
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
}

template <typename VT, typename XT>
__global__ void __launch_bounds__(kMultiBlock) k_multi_gap_part(const MultiInst<VT, XT> *__restrict__ inst,
                                                                const int *__restrict__ active,
                                                                double *__restrict__ part)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    const MultiInst<VT, XT> P = inst[p];
    const int64_t stride = int64_t(gridDim.y) * kMultiBlock;
    const int64_t t0 = int64_t(blockIdx.y) * kMultiBlock + threadIdx.x;
    double cmax = 0.0, l1 = 0.0, xc = 0.0, rr = 0.0, br = 0.0;
    for (int64_t i = t0; i < P.n; i += stride) {
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
    for (int64_t r = t0; r < P.m; r += stride) {
        const double v = P.g64[r];
        rr += v * v;
        br += P.b[r] * v;
        if constexpr (sizeof(XT) == 4) P.g[r] = float(v);
    }
    __shared__ double sm[5][kMultiBlock / 32];
    cmax = warp_max(cmax);
    l1 = warp_sum(l1);
    xc = warp_sum(xc);
    rr = warp_sum(rr);
    br = warp_sum(br);
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        sm[0][w] = cmax;
        sm[1][w] = l1;
        sm[2][w] = xc;
        sm[3][w] = rr;
        sm[4][w] = br;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kMultiBlock / 32; ++w) {
            a[0] = fmax(a[0], sm[0][w]);
            for (int q = 1; q < 5; ++q) a[q] += sm[q][w];
        }
        double *o = part + (int64_t(p) * gridDim.y + blockIdx.y) * 5;
        for (int q = 0; q < 5; ++q) o[q] = a[q];
    }
}

template <typename VT, typename XT>
__global__ void k_multi_gap_finish(const MultiInst<VT, XT> *__restrict__ inst, const int *__restrict__ active,
                                   const double *__restrict__ part, int parts, double *__restrict__ rec)
{
    const int p = blockIdx.x;
    if (!active[p] || threadIdx.x != 0) return;
    double cmax = 0.0, l1 = 0.0, xc = 0.0, rr = 0.0, br = 0.0;
    for (int y = 0; y < parts; ++y) {
        const double *o = part + (int64_t(p) * parts + y) * 5;
        cmax = fmax(cmax, o[0]);
        l1 += o[1];
        xc += o[2];
        rr += o[3];
        br += o[4];
    }
    const double lam = inst[p].lambda;
    double s = 1.0;
    if (cmax > 0.0 && lam / cmax < 1.0) s = lam / cmax;
    double *r = rec + int64_t(p) * 9;
    r[0] = 0.5 * rr + lam * l1;
    r[1] = -0.5 * s * s * rr - s * br;
    r[2] = 0.5 * (1.0 - s) * (1.0 - s) * rr + (lam * l1 + s * xc);
    r[3] = cmax;
    r[4] = s;
    r[5] = rr;
    r[6] = br;
    r[7] = l1;
    r[8] = xc;
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
cudaError_t MultiKernels<VT, XT>::gap(const MultiInst<VT, XT> *inst, const int *active, int count, double *part,
                                      double *rec, cudaStream_t st)
{
    const dim3 grid{unsigned(count), unsigned(kMultiSplit), 1u};
    k_multi_negb<VT, XT><<<grid, kMultiBlock, 0, st>>>(inst, active);
    k_multi_refresh<VT, XT><<<grid, kMultiBlock, 0, st>>>(inst, active);
    k_multi_gap_part<VT, XT><<<grid, kMultiBlock, 0, st>>>(inst, active, part);
    k_multi_gap_finish<VT, XT><<<dim3(unsigned(count)), 32, 0, st>>>(inst, active, part, kMultiSplit, rec);
    return cudaGetLastError();
}

}  // namespace pcdm

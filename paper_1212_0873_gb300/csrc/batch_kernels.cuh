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

// The step of eq. (h(x)) for one coordinate of one problem: returns h in the
// iterate dtype and sets the new x.  FP64 iterates: prox_step.  FP32 iterates:
// the step is formed in FP32 from the gradient, without rounding x: with
// d = -grad/(beta L) and t = lambda/(beta L),
//   x + d >  t  ->  h = d - t,   x + d < -t  ->  h = d + t,   else x -> 0,
// which is soft(x + d, t) - x; only the comparison sees x in FP32, and x + h is
// formed in FP64.  The fixed point (h = 0 exactly when d = -/+ t, i.e.
// grad = -/+ lambda) does not depend on the precision of x.  Apart from the
// conversion of x, FP64 work happens only when x moves (GB300 issues about 2
// FP64 operations per clock per SM).
template <typename XT>
__device__ __forceinline__ XT step_delta(double xi, XT grad, XT invL, XT inv_beta, XT lambda, double &xn)
{
    if constexpr (sizeof(XT) == 8) {
        xn = prox_step(xi, grad, invL, inv_beta, lambda);
        return xn - xi;
    } else {
        const float xf = float(xi);
        if (invL == 0.f) {
            xn = 0.0;
            return -xf;
        }
        const float ibl = invL * inv_beta;
        const float t = lambda * ibl;
        const float d = -grad * ibl;
        const float u = xf + d;
        if (u > t || u < -t) {
            const float h = u > t ? d - t : d + t;
            xn = xi + double(h);
            return h;
        }
        xn = 0.0;
        return -xf;
    }
}

// Shared-memory slot of one column of a round: the raw 16-byte descriptor,
// then the first kE row indices, then the first kE values.
template <typename VT>
__host__ __device__ constexpr int batch_slot_bytes()
{
    return 16 + 4 * kE + kE * int(sizeof(VT));
}

template <typename VT>
__host__ __device__ constexpr size_t batch_smem_bytes()
{
    return size_t(kBatchBlock) * size_t(batch_slot_bytes<VT>());
}

// The gradients of one column for the group's BP problems, from its slot
// (rows and values broadcast to every lane) and, past kE entries, from memory.
template <typename VT, typename XT, int BP>
__device__ __forceinline__ XT batch_column_dot(const BatchArgs<VT, XT> &a, const unsigned char *slot,
                                               const Col<XT> &c, int lane)
{
    constexpr int EPW = 16 / int(sizeof(VT));
    const int valid = c.cnt < kE ? c.cnt : kE;
    XT gv[kE];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 r4 = reinterpret_cast<const uint4 *>(slot + 16)[q];
        const int32_t r[4] = {int32_t(r4.x), int32_t(r4.y), int32_t(r4.z), int32_t(r4.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            gv[4 * q + t] = (4 * q + t < valid) ? ldcg(a.G + int64_t(r[t]) * BP + lane) : XT(0);
    }
    XT acc = XT(0);
#pragma unroll
    for (int w = 0; w < kE / EPW; ++w) {
        XT vw[EPW];
        decode_word<VT, XT>(reinterpret_cast<const uint4 *>(slot + 16 + 4 * kE)[w], vw);
#pragma unroll
        for (int q = 0; q < EPW; ++q)
            if (w * EPW + q < valid) acc = fma(vw[q], gv[w * EPW + q], acc);
    }
    for (int cs = kE; cs < c.cnt; cs += kE) {   // long columns: the rest from memory
        Chunk<kE, XT> t;
        ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + cs);
        const int v = c.cnt - cs;
#pragma unroll
        for (int e = 0; e < kE; ++e) gv[e] = (e < v) ? ldcg(a.G + int64_t(t.row[e]) * BP + lane) : XT(0);
#pragma unroll
        for (int e = 0; e < kE; ++e)
            if (e < v) acc = fma(t.val[e], gv[e], acc);
    }
    return acc;
}

// Persistent iterations k0 .. k0+iters-1.  A group of BP lanes takes the
// positions grp + (r*BP + q)*ngrp (q < BP) in rounds r.  In a round, lane q
// draws the q-th sample, loads its descriptor and copies the column's first
// chunk into the group's slot q (cp.async), so that the round's columns
// arrive with one memory latency; then the group walks the slots, every lane
// computing its own problem's gradient, step and x.  Phase 2 scatters the
// nonzero steps after a bounded grid barrier; a second barrier ends the
// iteration.
template <typename VT, typename XT, int BP>
__global__ void __launch_bounds__(kBatchBlock) k_batch_iter(const BatchArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    constexpr int SB = batch_slot_bytes<VT>();
    constexpr int G = pad_granule<VT>();
    const int lane = threadIdx.x & (BP - 1);
    const unsigned gmask = group_mask<BP>(threadIdx.x & 31);
    const int64_t grp = (int64_t(blockIdx.x) * kBatchBlock + threadIdx.x) / BP;
    const int64_t ngrp = int64_t(gridDim.x) * kBatchBlock / BP;
    unsigned char *gslots = bsm + size_t(threadIdx.x - lane) * SB;   // the group's BP slots
    unsigned char *myslot = bsm + size_t(threadIdx.x) * SB;           // slot `lane` of the group
    const XT lam = XT(a.lambda[lane]);
    const XT ib = XT(a.inv_beta);
    const bool act = a.active[lane] != 0;
    unsigned long long target = 0;
    Counters cnt;

    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const SampleKey key = make_sample_key(a.seed, k, a.n);
        unsigned *cnt_k = a.list_cnt + (k & 1);
        // the other counter was last read in phase 2 of iteration k-1 (before
        // its second barrier) and is next appended to in iteration k+1
        if (blockIdx.x == 0 && threadIdx.x == 0) a.list_cnt[(k + 1) & 1] = 0u;
        // ---------------- phase 1: gradients, steps, x
        for (int64_t base = grp; base < a.tau; base += ngrp * BP) {
            const int64_t jq = base + int64_t(lane) * ngrp;
            int32_t iq = 0;
            if (jq < a.tau) {
                iq = sample_index(uint32_t(jq), key);
                const int4 w = __ldg(reinterpret_cast<const int4 *>(a.desc + iq));
                *reinterpret_cast<int4 *>(myslot) = w;
                const Col<XT> c = col_from_word<XT>(w);
                if (c.cnt > 0) {
                    const int64_t pc = (int64_t(c.cnt) + G - 1) / G * G;
                    const int e = int(pc < kE ? pc : kE);
                    for (int q = 0; q < e / 4; ++q) cp_async16(myslot + 16 + 16 * q, a.prow + c.pbeg + 4 * q);
                    for (int q = 0; q < e * int(sizeof(VT)) / 16; ++q)
                        cp_async16(myslot + 16 + 4 * kE + 16 * q,
                                   reinterpret_cast<const unsigned char *>(a.pval + c.pbeg) + 16 * q);
                }
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp(gmask);
            for (int q = 0; q < BP; ++q) {
                const int64_t j = base + int64_t(q) * ngrp;
                if (j >= a.tau) break;   // the same for every lane of the group
                const int32_t i = __shfl_sync(gmask, iq, q, BP);
                const unsigned char *slot = gslots + size_t(q) * SB;
                const Col<XT> c = col_from_word<XT>(*reinterpret_cast<const int4 *>(slot));
                const double xi = ldcg(a.X + int64_t(i) * BP + lane);
                const XT acc = batch_column_dot<VT, XT, BP>(a, slot, c, lane);
                XT h = XT(0);
                if (act) {
                    double xn;
                    h = step_delta<XT>(xi, acc, c.invL, ib, lam, xn);
                    if (h != XT(0)) a.X[int64_t(i) * BP + lane] = xn;
                }
                // columns with a nonzero step go on the iteration's list
                if (__any_sync(gmask, h != XT(0))) {
                    unsigned sl = 0;
                    if (lane == 0) {
                        sl = atomicAdd(cnt_k, 1u);
                        a.list[sl] = i;
                    }
                    sl = __shfl_sync(gmask, sl, 0, BP);
                    a.H[int64_t(sl) * BP + lane] = h;
                }
                if (lane == 0) cnt.gathered += (unsigned long long)c.cnt;
                if (h != XT(0)) cnt.nonzero += 1;
            }
            __syncwarp(gmask);   // the slots are refilled by the next round
        }
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;

        // ---------------- phase 2: scatter of the listed columns' steps
        // FP32 residuals: lane 4q adds the steps of problems 4q .. 4q+3 into the
        // four consecutive entries of row r with one vector reduction (16-byte
        // aligned: bp is a multiple of 4); FP64 residuals: one reduction per lane.
        const int64_t total = int64_t(ld_volatile_u32(cnt_k));
        const uint64_t pl = l2_evict_last();
        for (int64_t sl = grp; sl < total; sl += ngrp) {
            const int32_t i = ldcg(a.list + sl);
            const XT h = ldcg(a.H + sl * BP + lane);
            const Col<XT> c = load_col(a.desc, i);
            if constexpr (sizeof(XT) == 4) {
                const int q0 = lane & ~3;
                const float h0 = __shfl_sync(gmask, h, q0 + 0, BP), h1 = __shfl_sync(gmask, h, q0 + 1, BP);
                const float h2 = __shfl_sync(gmask, h, q0 + 2, BP), h3 = __shfl_sync(gmask, h, q0 + 3, BP);
                const bool mine = (lane & 3) == 0 && (h0 != 0.f || h1 != 0.f || h2 != 0.f || h3 != 0.f);
                for (int cs = 0; cs < c.cnt; cs += kE) {
                    Chunk<kE, XT> t;
                    ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + cs);
                    const int valid = c.cnt - cs;
                    if (mine) {
#pragma unroll
                        for (int e = 0; e < kE; ++e)
                            if (e < valid)
                                red_add_v4(reinterpret_cast<float *>(a.G) + int64_t(t.row[e]) * BP + lane,
                                           t.val[e] * h0, t.val[e] * h1, t.val[e] * h2, t.val[e] * h3, pl);
                    }
                }
            } else {
                for (int cs = 0; cs < c.cnt; cs += kE) {
                    Chunk<kE, XT> t;
                    ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + cs);
                    const int valid = c.cnt - cs;
                    if (h != XT(0)) {
#pragma unroll
                        for (int e = 0; e < kE; ++e)
                            if (e < valid) red_add(a.G + int64_t(t.row[e]) * BP + lane, t.val[e] * h, pl);
                    }
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

template <typename K>
cudaError_t batch_occupancy(int *per_sm, K kernel, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, kBatchBlock, smem);
}

template <typename VT, typename XT>
int BatchKernels<VT, XT>::iter_max_blocks(int bp)
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (bp) {
    case 4: e = batch_occupancy(&per_sm, k_batch_iter<VT, XT, 4>, batch_smem_bytes<VT>()); break;
    case 8: e = batch_occupancy(&per_sm, k_batch_iter<VT, XT, 8>, batch_smem_bytes<VT>()); break;
    case 16: e = batch_occupancy(&per_sm, k_batch_iter<VT, XT, 16>, batch_smem_bytes<VT>()); break;
    case 32: e = batch_occupancy(&per_sm, k_batch_iter<VT, XT, 32>, batch_smem_bytes<VT>()); break;
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
                                           dim3(kBatchBlock), params, batch_smem_bytes<VT>(), st);
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

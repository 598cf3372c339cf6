// Column kernels of libpcdm, templated on the stored value type VT and the
// iterate type XT (x, g, h, L and the gradient accumulator).  Included by one
// translation unit per (VT, XT) pair, which instantiates Kernels<VT, XT>.
//
// Work mapping: a group of W lanes of one warp (W in {4, 8, 16, 32}) owns one
// sampled column at a time; lane l reads entries beg+l, beg+l+W, ... so the
// group's loads of row_idx and val are contiguous, and the partial sums meet in
// a shuffle tree inside the group.
//
// One PCDM1 iteration (Algorithm 1, step 4, with h(x) of eq. (h(x)), w = L):
//   phase 1 (gather):  grad_i = a_i^T g for i = S_k[j], all from the same g;
//                      x_new = soft(x_i - grad_i/(beta L_i), lambda/(beta L_i));
//                      h[j] = x_new - x_i; x_i = x_new
//   phase 2 (scatter): g_r += a_ri h[j] for the columns with h[j] != 0 (red.global.add),
//                      and S_{k+1} is drawn into the other sample buffer.
// The two phases are separated by a kernel boundary (two-kernel form) or by a
// bounded grid barrier (fused persistent form), which keeps the update Jacobi.
#pragma once

#include <cmath>

#include "pcdm_internal.h"

namespace pcdm {

template <typename VT, typename XT>
__device__ __forceinline__ int32_t *sample_buf(const IterArgs<VT, XT> &a, int64_t k)
{
    return (k & 1) ? a.S[1] : a.S[0];
}

struct Counters {
    unsigned long long gathered = 0, scattered = 0, nonzero = 0;
};

__device__ __forceinline__ void flush_counters(const Counters &c, unsigned long long *out)
{
    const unsigned long long a = warp_sum(c.gathered);
    const unsigned long long b = warp_sum(c.scattered);
    const unsigned long long d = warp_sum(c.nonzero);
    if ((threadIdx.x & 31) == 0 && (a | b | d)) {
        atomicAdd(out + 0, a);
        atomicAdd(out + 1, b);
        atomicAdd(out + 2, d);
    }
}

// Phase 1 for sampled position j (all W lanes of the group call it together).
template <int W, typename VT, typename XT>
__device__ __forceinline__ void gather_prox_one(const IterArgs<VT, XT> &a, const int32_t *S, int64_t j, int lane,
                                                unsigned gmask, Counters &cnt)
{
    const int32_t i = ldcg(S + j);
    const int64_t beg = __ldg(a.col_ptr + i);
    const int64_t end = __ldg(a.col_ptr + i + 1);
    XT acc = XT(0);
    for (int64_t p = beg + lane; p < end; p += W) acc += XT(ldv(a.val + p)) * ldcg(a.g + __ldg(a.row_idx + p));
    acc = group_sum<W>(acc, gmask);
    if (lane == 0) {
        const XT xi = ldcg(a.x + i);
        const XT Li = __ldg(a.L + i);
        XT xn = XT(0);
        if (Li > XT(0)) {
            const XT bl = a.beta * Li;
            xn = soft_threshold<XT>(xi - acc / bl, a.lambda / bl);
        }
        const XT h = xn - xi;
        a.x[i] = xn;
        a.h[j] = h;
        cnt.gathered += (unsigned long long)(end - beg);
        if (h != XT(0)) {
            cnt.nonzero += 1;
            cnt.scattered += (unsigned long long)(end - beg);
        }
    }
}

// Phase 2 for sampled position j.
template <int W, typename VT, typename XT>
__device__ __forceinline__ void scatter_one(const IterArgs<VT, XT> &a, const int32_t *S, int64_t j, int lane)
{
    const XT h = ldcg(a.h + j);
    if (h == XT(0)) return;
    const int32_t i = ldcg(S + j);
    const int64_t beg = __ldg(a.col_ptr + i);
    const int64_t end = __ldg(a.col_ptr + i + 1);
    for (int64_t p = beg + lane; p < end; p += W) red_add(a.g + __ldg(a.row_idx + p), XT(ldv(a.val + p)) * h);
}

// ---------------------------------------------------------------------------
// Two-kernel form.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_gather(const IterArgs<VT, XT> a, int64_t k)
{
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t grp = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W;
    Counters cnt;
    if (grp < a.tau) gather_prox_one<W>(a, sample_buf(a, k), grp, lane, gmask, cnt);
    flush_counters(cnt, a.counters);
}

template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_scatter(const IterArgs<VT, XT> a, int64_t k, int sample_next)
{
    const int lane = threadIdx.x & (W - 1);
    const int64_t gid = int64_t(blockIdx.x) * kBlock + threadIdx.x;
    const int64_t grp = gid / W;
    if (grp < a.tau) scatter_one<W>(a, sample_buf(a, k), grp, lane);
    if (sample_next && gid < a.tau) {
        const SampleKey key = make_sample_key(a.seed, k + 1, a.n);
        sample_buf(a, k + 1)[gid] = sample_index(uint32_t(gid), key);
    }
}

// ---------------------------------------------------------------------------
// Fused persistent form: one cooperative launch runs `iters` iterations.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_fused(const IterArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t nthreads = int64_t(gridDim.x) * kBlock;
    const int64_t gid = int64_t(blockIdx.x) * kBlock + threadIdx.x;
    const int64_t grp = gid / W;
    const int64_t ngrp = nthreads / W;
    unsigned long long target = 0;
    Counters cnt;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const int32_t *S = sample_buf(a, k);
        for (int64_t j = grp; j < a.tau; j += ngrp) gather_prox_one<W>(a, S, j, lane, gmask, cnt);
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;
        for (int64_t j = grp; j < a.tau; j += ngrp) scatter_one<W>(a, S, j, lane);
        {
            const SampleKey key = make_sample_key(a.seed, k + 1, a.n);
            int32_t *Snext = sample_buf(a, k + 1);
            for (int64_t j = gid; j < a.tau; j += nthreads) Snext[j] = sample_index(uint32_t(j), key);
        }
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;
    }
    flush_counters(cnt, a.counters);
}

// ---------------------------------------------------------------------------
// Set-up: one thread per column (runs once per matrix).
template <typename VT>
__global__ void k_setup_cols(const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
                             const VT *__restrict__ val, int64_t m, int64_t n, double *__restrict__ L,
                             int *__restrict__ rowcnt, int *__restrict__ flags)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int f = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        double s = 0.0;
        int64_t prev = -1;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) {
            const int64_t r = row_idx[p];
            if (r < 0 || r >= m) {
                f |= FLAG_ROW_RANGE;
                continue;
            }
            if (r <= prev) f |= FLAG_ROW_ORDER;
            prev = r;
            const double v = double(ldv(val + p));
            if (!isfinite(v)) f |= FLAG_NONFINITE;
            s = __dadd_rn(s, __dmul_rn(v, v));   // no contraction: the same bits as a plain sum of squares
            atomicAdd(rowcnt + r, 1);
        }
        L[i] = s;
    }
    if (f) atomicOr(flags, f);
}

// Refresh: g64 += a_i x_i over the columns with x_i != 0, in FP64.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_refresh_cols(const int64_t *__restrict__ col_ptr,
                                                         const int32_t *__restrict__ row_idx,
                                                         const VT *__restrict__ val, const XT *__restrict__ x,
                                                         int64_t n, double *__restrict__ g64)
{
    const int lane = threadIdx.x & (W - 1);
    const int64_t ngrp = int64_t(gridDim.x) * kBlock / W;
    for (int64_t i = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W; i < n; i += ngrp) {
        const double xi = double(__ldg(x + i));
        if (xi == 0.0) continue;
        const int64_t beg = __ldg(col_ptr + i), end = __ldg(col_ptr + i + 1);
        for (int64_t p = beg + lane; p < end; p += W) red_add(g64 + __ldg(row_idx + p), double(ldv(val + p)) * xi);
    }
}

// Gap, column part: c_i = a_i^T r in FP64; block partials of max|c_i|, sum|x_i|, sum x_i c_i.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_gap_cols(const int64_t *__restrict__ col_ptr,
                                                     const int32_t *__restrict__ row_idx,
                                                     const VT *__restrict__ val, const double *__restrict__ r,
                                                     const XT *__restrict__ x, int64_t n, double *__restrict__ part)
{
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t ngrp = int64_t(gridDim.x) * kBlock / W;
    double cmax = 0.0, l1 = 0.0, xc = 0.0;
    for (int64_t i = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W; i < n; i += ngrp) {
        const int64_t beg = __ldg(col_ptr + i), end = __ldg(col_ptr + i + 1);
        double c = 0.0;
        for (int64_t p = beg + lane; p < end; p += W) c += double(ldv(val + p)) * __ldg(r + __ldg(row_idx + p));
        c = group_sum<W>(c, gmask);
        if (lane == 0) {
            const double xi = double(__ldg(x + i));
            cmax = fmax(cmax, fabs(c));
            l1 += fabs(xi);
            xc += xi * c;
        }
    }
    __shared__ double sm[3][kBlock / 32];
    cmax = warp_max(cmax);
    l1 = warp_sum(l1);
    xc = warp_sum(xc);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sm[0][w] = cmax;
        sm[1][w] = l1;
        sm[2][w] = xc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) {
            a0 = fmax(a0, sm[0][q]);
            a1 += sm[1][q];
            a2 += sm[2][q];
        }
        part[3 * blockIdx.x + 0] = a0;
        part[3 * blockIdx.x + 1] = a1;
        part[3 * blockIdx.x + 2] = a2;
    }
}

// ---------------------------------------------------------------------------
// Launchers.
template <int W>
static inline int64_t blocks_for_groups(int64_t groups)
{
    return (groups * W + kBlock - 1) / kBlock;
}

#define PCDM_DISPATCH_W(W, ...)                                    \
    switch (W) {                                                   \
    case 4: { constexpr int W_ = 4; __VA_ARGS__; } break;          \
    case 8: { constexpr int W_ = 8; __VA_ARGS__; } break;          \
    case 16: { constexpr int W_ = 16; __VA_ARGS__; } break;        \
    case 32: { constexpr int W_ = 32; __VA_ARGS__; } break;        \
    default: return cudaErrorInvalidValue;                         \
    }

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::gather(const IterArgs<VT, XT> &a, int W, int64_t k, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    PCDM_DISPATCH_W(W, {
        const int64_t blocks = blocks_for_groups<W_>(a.tau);
        k_gather<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(a, k);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::scatter(const IterArgs<VT, XT> &a, int W, int64_t k, bool sample_next, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    PCDM_DISPATCH_W(W, {
        const int64_t blocks = blocks_for_groups<W_>(a.tau);
        k_scatter<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(a, k, sample_next ? 1 : 0);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
int Kernels<VT, XT>::fused_max_blocks(int W)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (W) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<4, VT, XT>, kBlock, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<8, VT, XT>, kBlock, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<16, VT, XT>, kBlock, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<32, VT, XT>, kBlock, 0); break;
    default: return 0;
    }
    if (e != cudaSuccess) return 0;
    return per_sm * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused(const IterArgs<VT, XT> &a, int W, int64_t k0, int64_t iters, int blocks,
                                   cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    PCDM_DISPATCH_W(W, {
        return cudaLaunchCooperativeKernel((const void *)k_fused<W_, VT, XT>, dim3(unsigned(blocks)), dim3(kBlock),
                                           params, 0, st);
    });
    return cudaErrorInvalidValue;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::setup_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                        int64_t n, double *L, int *rowcnt, int *flags, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    k_setup_cols<VT><<<dim3(unsigned(blocks)), 256, 0, st>>>(col_ptr, row_idx, val, m, n, L, rowcnt, flags);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::refresh_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, const XT *x,
                                          int64_t n, double *g64, int W, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    PCDM_DISPATCH_W(W, {
        int64_t blocks = blocks_for_groups<W_>(n);
        if (blocks > 152 * 64) blocks = 152 * 64;
        k_refresh_cols<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(col_ptr, row_idx, val, x, n, g64);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::gap_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, const double *r,
                                      const XT *x, int64_t n, double *part, int blocks, int W, cudaStream_t st)
{
    PCDM_DISPATCH_W(W, {
        k_gap_cols<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(col_ptr, row_idx, val, r, x, n, part);
    });
    return cudaGetLastError();
}

}  // namespace pcdm

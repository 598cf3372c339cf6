// Type-independent kernels of libpcdm: the standalone tau-nice sampler, input
// validation, conversions, the row part and the final reduction of the duality
// gap, the self-test of the bounded grid barrier, and the row counts of
// pcdm_omega_noalloc.
#include <cmath>
#include <mutex>

#include "pcdm.h"
#include "pcdm_internal.h"

namespace pcdm {

static inline unsigned grid_for(int64_t count, int per_block = 256, int64_t cap = 152 * 64)
{
    int64_t b = (count + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return unsigned(b);
}

__global__ void k_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S)
{
    const SampleKey key = warp_sample_key(seed, k, n);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < tau; j += stride)
        S[j] = sample_index(uint32_t(j), key);
}

cudaError_t launch_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S, cudaStream_t st)
{
    if (tau <= 0) return cudaSuccess;
    k_sample<<<grid_for(tau), 256, 0, st>>>(seed, k, n, tau, S);
    return cudaGetLastError();
}

__global__ void k_check_colptr(const int64_t *col_ptr, int64_t n, int64_t nnz, int *flags)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int f = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += stride) {
        const int64_t c = col_ptr[i];
        if (c < 0 || c > nnz) f = FLAG_COLPTR;
        if (i == 0 && c != 0) f = FLAG_COLPTR;
        if (i == n && c != nnz) f = FLAG_COLPTR;
        if (i < n && col_ptr[i + 1] < c) f = FLAG_COLPTR;
    }
    if (f) atomicOr(flags, f);
}

// S_k of the other samplings (see launch_sample_kind in pcdm_internal.h).
__global__ void k_sample_kind(int kind, uint64_t seed, int64_t k, int64_t n, int64_t tau, uint64_t keep_T,
                              int32_t *S, unsigned long long *win, uint8_t *keep)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (kind == 1) {
        for (; j < tau; j += stride) {
            const int32_t i = independent_pick(seed, k, uint32_t(j), n);
            S[j] = i;
            if (win) atomicMax(win + i, independent_key(k, uint32_t(j)));
        }
        return;
    }
    const SampleKey key = warp_sample_key(seed, k, n);
    for (; j < tau; j += stride) {
        S[j] = sample_index(uint32_t(j), key);
        if (keep) keep[j] = (kind == 2 && !binomial_keep(seed, k, uint32_t(j), keep_T)) ? 0 : 1;
    }
}

cudaError_t launch_sample_kind(int kind, uint64_t seed, int64_t k, int64_t n, int64_t tau, uint64_t keep_T,
                               int32_t *S, unsigned long long *win, uint8_t *keep, cudaStream_t st)
{
    if (tau <= 0) return cudaSuccess;
    k_sample_kind<<<grid_for(tau), 256, 0, st>>>(kind, seed, k, n, tau, keep_T, S, win, keep);
    return cudaGetLastError();
}

cudaError_t launch_check_colptr(const int64_t *col_ptr, int64_t n, int64_t nnz, int *flags, cudaStream_t st)
{
    k_check_colptr<<<grid_for(n + 1), 256, 0, st>>>(col_ptr, n, nnz, flags);
    return cudaGetLastError();
}

__global__ void k_check_finite(const double *v, int64_t count, int *flags)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int f = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        if (!isfinite(v[i])) f = FLAG_B_NONFINITE;
    if (f) atomicOr(flags, f);
}

cudaError_t launch_check_finite(const double *v, int64_t count, int *flags, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_check_finite<<<grid_for(count), 256, 0, st>>>(v, count, flags);
    return cudaGetLastError();
}

__global__ void k_max_int(const int *a, int64_t count, int *out)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int best = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) best = max(best, a[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, off));
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, best);
}

cudaError_t launch_max_int(const int *a, int64_t count, int *out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_max_int<<<grid_for(count), 256, 0, st>>>(a, count, out);
    return cudaGetLastError();
}

__global__ void k_convert_b(const void *b_in, int b_is_f32, int64_t m, double *b_out)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride)
        b_out[i] = b_is_f32 ? double(static_cast<const float *>(b_in)[i]) : static_cast<const double *>(b_in)[i];
}

cudaError_t launch_convert_b(const void *b_in, int b_is_f32, int64_t m, double *b_out, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_convert_b<<<grid_for(m), 256, 0, st>>>(b_in, b_is_f32, m, b_out);
    return cudaGetLastError();
}

template <typename XT>
__global__ void k_neg_store(XT *g, const double *b, int64_t m)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) g[i] = XT(-b[i]);
}

template <typename XT>
cudaError_t launch_neg_store(XT *g, const double *b, int64_t m, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_neg_store<XT><<<grid_for(m), 256, 0, st>>>(g, b, m);
    return cudaGetLastError();
}
template cudaError_t launch_neg_store<double>(double *, const double *, int64_t, cudaStream_t);
template cudaError_t launch_neg_store<float>(float *, const double *, int64_t, cudaStream_t);

template <typename XT>
__global__ void k_store_from_f64(XT *dst, const double *src, int64_t m)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) dst[i] = XT(src[i]);
}

template <typename XT>
cudaError_t launch_store_from_f64(XT *dst, const double *src, int64_t m, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_store_from_f64<XT><<<grid_for(m), 256, 0, st>>>(dst, src, m);
    return cudaGetLastError();
}
template cudaError_t launch_store_from_f64<double>(double *, const double *, int64_t, cudaStream_t);
template cudaError_t launch_store_from_f64<float>(float *, const double *, int64_t, cudaStream_t);

cudaError_t launch_f64_to_f32(float *dst, const double *src, int64_t count, cudaStream_t st)
{
    return launch_store_from_f64<float>(dst, src, count, st);
}

// Row part of the gap: block partials of ||r||^2 and b^T r.
__global__ void __launch_bounds__(kBlock) k_gap_rows(const double *__restrict__ r, const double *__restrict__ b,
                                                     int64_t m, double *__restrict__ part)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    double rr = 0.0, br = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < m; i += stride) {
        const double ri = r[i];
        rr += ri * ri;
        br += b[i] * ri;
    }
    __shared__ double sm[2][kBlock / 32];
    rr = warp_sum(rr);
    br = warp_sum(br);
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = rr;
        sm[1][threadIdx.x >> 5] = br;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) {
            a0 += sm[0][q];
            a1 += sm[1][q];
        }
        part[2 * blockIdx.x + 0] = a0;
        part[2 * blockIdx.x + 1] = a1;
    }
}

cudaError_t launch_gap_rows(const double *r, const double *b, int64_t m, double *part, int blocks, cudaStream_t st)
{
    k_gap_rows<<<blocks, kBlock, 0, st>>>(r, b, m, part);
    return cudaGetLastError();
}

// Final fixed-order reduction and the gap record (all in FP64):
//   out = {P, D, gap, ||c||_inf, s, ||r||^2, b^T r, ||x||_1, x^T c}
//   s = min(1, lambda/||c||_inf) (1 when c = 0), P = ||r||^2/2 + lambda ||x||_1,
//   D = -s^2 ||r||^2/2 - s b^T r, gap = (1-s)^2 ||r||^2/2 + lambda ||x||_1 + s x^T c.
__global__ void __launch_bounds__(kFinishBlock) k_gap_finish(const double *pc, int nbc, const double *pr, int nbr,
                                                             double lambda, double *out)
{
    double cmax = 0.0, l1 = 0.0, xc = 0.0, rr = 0.0, br = 0.0;
    for (int q = threadIdx.x; q < nbc; q += kFinishBlock) {
        cmax = fmax(cmax, pc[3 * q + 0]);
        l1 += pc[3 * q + 1];
        xc += pc[3 * q + 2];
    }
    for (int q = threadIdx.x; q < nbr; q += kFinishBlock) {
        rr += pr[2 * q + 0];
        br += pr[2 * q + 1];
    }
    __shared__ double sm[5][kFinishBlock / 32];
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
        for (int w = 0; w < kFinishBlock / 32; ++w) {
            a[0] = fmax(a[0], sm[0][w]);
            for (int q = 1; q < 5; ++q) a[q] += sm[q][w];
        }
        const double cinf = a[0], l1s = a[1], xcs = a[2], rrs = a[3], brs = a[4];
        double s = 1.0;
        if (cinf > 0.0 && lambda / cinf < 1.0) s = lambda / cinf;
        out[0] = 0.5 * rrs + lambda * l1s;
        out[1] = -0.5 * s * s * rrs - s * brs;
        out[2] = 0.5 * (1.0 - s) * (1.0 - s) * rrs + (lambda * l1s + s * xcs);
        out[3] = cinf;
        out[4] = s;
        out[5] = rrs;
        out[6] = brs;
        out[7] = l1s;
        out[8] = xcs;
    }
}

cudaError_t launch_gap_finish(const double *pc, int nbc, const double *pr, int nbr, double *out, double lambda,
                              cudaStream_t st)
{
    k_gap_finish<<<1, kFinishBlock, 0, st>>>(pc, nbc, pr, nbr, lambda, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SVM dual and logistic regression.
__global__ void k_check_labels(const double *y, int64_t count, int *flags)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int f = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        if (!(y[i] == 1.0 || y[i] == -1.0)) f = FLAG_LABEL;
    if (f) atomicOr(flags, f);
}

cudaError_t launch_check_labels(const double *y, int64_t count, int *flags, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_check_labels<<<grid_for(count), 256, 0, st>>>(y, count, flags);
    return cudaGetLastError();
}

__global__ void k_scale(double *v, int64_t count, double factor)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) v[i] *= factor;
}

cudaError_t launch_scale(double *v, int64_t count, double factor, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_scale<<<grid_for(count), 256, 0, st>>>(v, count, factor);
    return cudaGetLastError();
}

// log(1 + e^t) without overflow.
__device__ __forceinline__ double softplus(double t)
{
    return t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t));
}

__global__ void __launch_bounds__(kBlock) k_glm_gap_rows(int problem, const double *__restrict__ r, int64_t m,
                                                         double *__restrict__ part)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < m; i += stride) {
        const double ri = r[i];
        s += problem == 1 ? ri * ri : softplus(-ri);
    }
    __shared__ double sm[kBlock / 32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) a += sm[q];
        part[2 * blockIdx.x + 0] = a;
        part[2 * blockIdx.x + 1] = 0.0;
    }
}

cudaError_t launch_glm_gap_rows(int problem, const double *r, int64_t m, double *part, int blocks, cudaStream_t st)
{
    k_glm_gap_rows<<<blocks, kBlock, 0, st>>>(problem, r, m, part);
    return cudaGetLastError();
}

// SVM dual (Sec. 8.3), rows = ||r||^2 = ||u||^2, w = u/(lambda n):
//   P = t2/n + ||u||^2/(2 lambda n^2)  (hinge loss + lambda/2 ||w||^2),
//   D = t3/n - ||u||^2/(2 lambda n^2)  (= -f(x)),   gap = t1/n.
// Logistic (Sec. 8.4), rows = sum_r log(1 + exp(-margin_r)):
//   P = rows + lambda t2,  gap = t1/(4 lambda) (the Fenchel gap at
//   alpha_r = 1/(1 + exp(margin_r)) equals ||grad F||^2/(4 lambda)),  D = P - gap.
__global__ void __launch_bounds__(kFinishBlock) k_glm_gap_finish(int problem, const double *pc, int nbc,
                                                                 const double *pr, int nbr, double lambda, int64_t n,
                                                                 double *out)
{
    double t1 = 0.0, t2 = 0.0, t3 = 0.0, rows = 0.0;
    for (int q = threadIdx.x; q < nbc; q += kFinishBlock) {
        t1 += pc[3 * q + 0];
        t2 += pc[3 * q + 1];
        t3 += pc[3 * q + 2];
    }
    for (int q = threadIdx.x; q < nbr; q += kFinishBlock) rows += pr[2 * q + 0];
    __shared__ double sm[4][kFinishBlock / 32];
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    t3 = warp_sum(t3);
    rows = warp_sum(rows);
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        sm[0][w] = t1;
        sm[1][w] = t2;
        sm[2][w] = t3;
        sm[3][w] = rows;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kFinishBlock / 32; ++w)
            for (int q = 0; q < 4; ++q) a[q] += sm[q][w];
        const double nn = double(n);
        if (problem == 1) {
            const double quad = a[3] / (2.0 * lambda * nn * nn);
            out[0] = a[1] / nn + quad;
            out[1] = a[2] / nn - quad;
            out[2] = a[0] / nn;
        } else {
            out[0] = a[3] + lambda * a[1];
            out[2] = a[0] / (4.0 * lambda);
            out[1] = out[0] - out[2];
        }
        out[3] = a[0];
        out[4] = a[1];
        out[5] = a[2];
        out[6] = a[3];
        out[7] = 0.0;
        out[8] = 0.0;
    }
}

cudaError_t launch_glm_gap_finish(int problem, const double *pc, int nbc, const double *pr, int nbr, double lambda,
                                  int64_t n, double *out, cudaStream_t st)
{
    k_glm_gap_finish<<<1, kFinishBlock, 0, st>>>(problem, pc, nbc, pr, nbr, lambda, n, out);
    return cudaGetLastError();
}

// Support of x in increasing index order, by one block: each pass takes
// kBlock entries, the block's ballots give every nonzero its rank.
__global__ void __launch_bounds__(kBlock) k_compact_support(const double *__restrict__ x, int64_t n,
                                                            int32_t *__restrict__ sidx, int *__restrict__ count)
{
    __shared__ int wsum[kBlock / 32];
    __shared__ int base_s;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t0 = 0; t0 < n; t0 += kBlock) {
        const int64_t i = t0 + threadIdx.x;
        const bool nz = i < n && x[i] != 0.0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, nz);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        int off = base_s;
        for (int q = 0; q < w; ++q) off += wsum[q];
        if (nz) sidx[off + __popc(bal & ((1u << lane) - 1u))] = int32_t(i);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < kBlock / 32; ++q) tot += wsum[q];
            base_s += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base_s;
}

cudaError_t launch_compact_support(const double *x, int64_t n, int32_t *sidx, int *count, cudaStream_t st)
{
    k_compact_support<<<1, kBlock, 0, st>>>(x, n, sidx, count);
    return cudaGetLastError();
}

__global__ void k_as_linear(const double *__restrict__ x, const double *__restrict__ src,
                            const int32_t *__restrict__ sidx, int64_t nS, double lambda, double *__restrict__ c,
                            double *__restrict__ sgn)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nS; p += stride) {
        const int32_t i = sidx[p];
        const double xi = x[i];
        const double s = xi > 0.0 ? 1.0 : (xi < 0.0 ? -1.0 : 0.0);
        sgn[p] = s;
        c[p] = src ? src[i] : -lambda * s;
    }
}

cudaError_t launch_as_linear(const double *x, const double *src, const int32_t *sidx, int64_t nS, double lambda,
                             double *c, double *sgn, cudaStream_t st)
{
    if (nS <= 0) return cudaSuccess;
    k_as_linear<<<grid_for(nS), 256, 0, st>>>(x, src, sidx, nS, lambda, c, sgn);
    return cudaGetLastError();
}

// Interleaving of nsrc vectors of length len (src[l * len + r], FP64 or FP32)
// into dst[r * bp + l] (FP64); the padding lanes l >= nsrc get 0.
__global__ void k_interleave(const void *src, int src_is_f32, int64_t len, int nsrc, int bp, double *dst)
{
    const int64_t total = len * bp;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t r = e / bp;
        const int l = int(e - r * bp);
        double v = 0.0;
        if (l < nsrc) {
            const int64_t q = int64_t(l) * len + r;
            v = src_is_f32 ? double(static_cast<const float *>(src)[q]) : static_cast<const double *>(src)[q];
        }
        dst[e] = v;
    }
}

cudaError_t launch_interleave(const void *src, int src_is_f32, int64_t len, int nsrc, int bp, double *dst,
                              cudaStream_t st)
{
    if (len <= 0) return cudaSuccess;
    k_interleave<<<grid_for(len * bp), 256, 0, st>>>(src, src_is_f32, len, nsrc, bp, dst);
    return cudaGetLastError();
}

// The inverse for the first nout lanes: dst[l * len + r] = src[r * bp + l].
__global__ void k_deinterleave(const double *src, int64_t len, int nout, int bp, double *dst)
{
    const int64_t total = len * nout;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t r = e / nout;
        const int l = int(e - r * nout);
        dst[int64_t(l) * len + r] = src[r * bp + l];
    }
}

cudaError_t launch_deinterleave(const double *src, int64_t len, int nout, int bp, double *dst, cudaStream_t st)
{
    if (len <= 0) return cudaSuccess;
    k_deinterleave<<<grid_for(len * nout), 256, 0, st>>>(src, len, nout, bp, dst);
    return cudaGetLastError();
}

// Batched gap, row part: for right-hand side l (element e = r * bp + l of the
// interleaved vectors) block partials part[(block * bp + l) * 2 + {0,1}] of
// ||r_l||^2 and b_l^T r_l.  The grid stride is a multiple of bp, so each thread
// keeps one l.
__global__ void __launch_bounds__(kBlock) k_batch_gap_rows(const double *__restrict__ R,
                                                           const double *__restrict__ Bm, int64_t total, int bp,
                                                           double *__restrict__ part)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    double rr = 0.0, br = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * kBlock + threadIdx.x; e < total; e += stride) {
        const double r = R[e];
        rr += r * r;
        br += Bm[e] * r;
    }
    __shared__ double sm[2][kBlock];
    sm[0][threadIdx.x] = rr;
    sm[1][threadIdx.x] = br;
    __syncthreads();
    if (threadIdx.x < bp) {
        double a0 = 0.0, a1 = 0.0;
        for (int q = threadIdx.x; q < kBlock; q += bp) {
            a0 += sm[0][q];
            a1 += sm[1][q];
        }
        part[(int64_t(blockIdx.x) * bp + threadIdx.x) * 2 + 0] = a0;
        part[(int64_t(blockIdx.x) * bp + threadIdx.x) * 2 + 1] = a1;
    }
}

cudaError_t launch_batch_gap_rows(const double *R, const double *Bm, int64_t m, int bp, double *part, int blocks,
                                  cudaStream_t st)
{
    if (bp < 1 || kBlock % bp != 0) return cudaErrorInvalidValue;
    k_batch_gap_rows<<<blocks, kBlock, 0, st>>>(R, Bm, m * bp, bp, part);
    return cudaGetLastError();
}

// Batched gap records: block l of the grid reduces right-hand side l's partials
// and writes out[l * 9 + q] with the formulas of k_gap_finish.
__global__ void __launch_bounds__(kFinishBlock) k_batch_gap_finish(const double *pc, int nbc, const double *pr,
                                                                   int nbr, int bp, const double *lambda,
                                                                   double *out)
{
    const int l = blockIdx.x;
    double cmax = 0.0, l1 = 0.0, xc = 0.0, rr = 0.0, br = 0.0;
    for (int q = threadIdx.x; q < nbc; q += kFinishBlock) {
        const double *p = pc + (int64_t(q) * bp + l) * 3;
        cmax = fmax(cmax, p[0]);
        l1 += p[1];
        xc += p[2];
    }
    for (int q = threadIdx.x; q < nbr; q += kFinishBlock) {
        const double *p = pr + (int64_t(q) * bp + l) * 2;
        rr += p[0];
        br += p[1];
    }
    __shared__ double sm[5][kFinishBlock / 32];
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
        for (int w = 0; w < kFinishBlock / 32; ++w) {
            a[0] = fmax(a[0], sm[0][w]);
            for (int q = 1; q < 5; ++q) a[q] += sm[q][w];
        }
        const double lam = lambda[l];
        const double cinf = a[0], l1s = a[1], xcs = a[2], rrs = a[3], brs = a[4];
        double s = 1.0;
        if (cinf > 0.0 && lam / cinf < 1.0) s = lam / cinf;
        double *o = out + int64_t(l) * 9;
        o[0] = 0.5 * rrs + lam * l1s;
        o[1] = -0.5 * s * s * rrs - s * brs;
        o[2] = 0.5 * (1.0 - s) * (1.0 - s) * rrs + (lam * l1s + s * xcs);
        o[3] = cinf;
        o[4] = s;
        o[5] = rrs;
        o[6] = brs;
        o[7] = l1s;
        o[8] = xcs;
    }
}

cudaError_t launch_batch_gap_finish(const double *pc, int nbc, const double *pr, int nbr, int bp,
                                    const double *lambda, double *out, cudaStream_t st)
{
    k_batch_gap_finish<<<bp, kFinishBlock, 0, st>>>(pc, nbc, pr, nbr, bp, lambda, out);
    return cudaGetLastError();
}

// Barrier self-test: the wait target is one arrival more than the grid has, so
// every block's wait must end by its time budget.
__global__ void k_barrier_selftest(unsigned long long *bar, int *status, uint64_t timeout_ns)
{
    grid_sync(bar, (unsigned long long)gridDim.x + 1ull, status, timeout_ns);
}

cudaError_t launch_barrier_selftest(unsigned long long *bar, int *status, uint64_t timeout_ns, int blocks,
                                    cudaStream_t st)
{
    void *params[] = {(void *)&bar, (void *)&status, (void *)&timeout_ns};
    return cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(unsigned(blocks)), dim3(64), params, 0,
                                       st);
}


// ---------------------------------------------------------------------------
// Exclusive scan of padded column lengths (set-up of the padded layout).
// Tiles of kScanTile columns: tile sums, a single-block scan of the tile sums,
// then a block-local scan of each tile plus its offset.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

int64_t scan_tile_count(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ int64_t padded_len(const int64_t *col_ptr, int64_t i, int64_t n, int granule)
{
    if (i >= n) return 0;
    const int64_t c = col_ptr[i + 1] - col_ptr[i];
    return (c + granule - 1) / granule * granule;
}

// Block-wide exclusive scan of one int64 per thread; returns the block total in *total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t o = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t o = __shfl_up_sync(0xFFFFFFFFu, ti, off);
            if (lane >= off) ti += o;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;   // exclusive prefix of warp totals
        if (lane == 31) *total = ti;
    }
    __syncthreads();
    const int64_t out = warp_tot[w] + incl - v;
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int64_t *col_ptr, int64_t n, int granule,
                                                             int64_t *tile)
{
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q) s += padded_len(col_ptr, base + q, n, granule);
    __shared__ int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile[blockIdx.x] = tot;
}

// Single block: tile[0..ntiles) -> exclusive prefixes, tile[ntiles] = total.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_prefix(int64_t *tile, int64_t ntiles)
{
    const int64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
    const int64_t beg = int64_t(threadIdx.x) * per;
    const int64_t end = beg + per < ntiles ? beg + per : ntiles;
    int64_t s = 0;
    for (int64_t q = beg; q < end; ++q) s += tile[q];
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot);
    for (int64_t q = beg; q < end; ++q) {
        const int64_t v = tile[q];
        tile[q] = run;
        run += v;
    }
    if (threadIdx.x == 0) tile[ntiles] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int64_t *col_ptr, int64_t n, int granule,
                                                             const int64_t *tile, int64_t ntiles, int64_t *pbeg)
{
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int64_t len[kScanPer];
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q) {
        len[q] = padded_len(col_ptr, base + q, n, granule);
        s += len[q];
    }
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot) + tile[blockIdx.x];
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) pbeg[base + q] = run;
        run += len[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) pbeg[n] = tile[ntiles];
}

// The same three passes over plain int counts (the row counts of the row-major copy).
__global__ void __launch_bounds__(kScanThreads) k_count_scan_tiles(const int *cnt, int64_t m, int64_t *tile)
{
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q)
        if (base + q < m) s += cnt[base + q];
    __shared__ int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_count_scan_apply(const int *cnt, int64_t m, const int64_t *tile,
                                                                   int64_t ntiles, int64_t *out)
{
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int64_t len[kScanPer];
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q) {
        len[q] = base + q < m ? cnt[base + q] : 0;
        s += len[q];
    }
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot) + tile[blockIdx.x];
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < m) out[base + q] = run;
        run += len[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = tile[ntiles];
}

cudaError_t launch_count_scan(const int *cnt, int64_t m, int64_t *out, int64_t *tile, cudaStream_t st)
{
    const int64_t nt = scan_tile_count(m);
    if (nt <= 0) return cudaSuccess;
    k_count_scan_tiles<<<unsigned(nt), kScanThreads, 0, st>>>(cnt, m, tile);
    k_scan_tile_prefix<<<1, kScanThreads, 0, st>>>(tile, nt);
    k_count_scan_apply<<<unsigned(nt), kScanThreads, 0, st>>>(cnt, m, tile, nt, out);
    return cudaGetLastError();
}

cudaError_t launch_padded_scan(const int64_t *col_ptr, int64_t n, int granule, int64_t *pbeg, int64_t *tile,
                               cudaStream_t st)
{
    const int64_t nt = scan_tile_count(n);
    if (nt <= 0) return cudaSuccess;
    k_scan_tiles<<<unsigned(nt), kScanThreads, 0, st>>>(col_ptr, n, granule, tile);
    k_scan_tile_prefix<<<1, kScanThreads, 0, st>>>(tile, nt);
    k_scan_apply<<<unsigned(nt), kScanThreads, 0, st>>>(col_ptr, n, granule, tile, nt, pbeg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row counts and omega with no allocation (pcdm_omega_noalloc).  The scratch is
// this file-scope array: PCDM_NOALLOC_MAX_ROWS row counters, then a flags word
// and the result word.  One array per device context, shared by every caller:
// calls that overlap in time race on it.
constexpr int64_t kNoAllocTail = 64;
static __device__ __align__(256) int g_noalloc_rows[PCDM_NOALLOC_MAX_ROWS + kNoAllocTail];

// One thread per column: the same checks as the set-up (col_ptr monotone and in
// range, rows in [0, m) and strictly increasing within a column), then one count
// per valid entry.
__global__ void k_rows_checked(const int64_t *col_ptr, const int32_t *row_idx, int64_t m, int64_t n, int64_t nnz,
                               int *cnt, int *flags)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int f = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += stride) {
        const int64_t s = col_ptr[i];
        if ((i == 0 && s != 0) || (i == n && s != nnz)) f |= FLAG_COLPTR;
        if (i == n) continue;
        const int64_t e = col_ptr[i + 1];
        if (s < 0 || e < s || e > nnz) {
            f |= FLAG_COLPTR;
            continue;
        }
        int64_t prev = -1;
        for (int64_t p = s; p < e; ++p) {
            const int64_t r = row_idx[p];
            if (r < 0 || r >= m) {
                f |= FLAG_ROW_RANGE;
                continue;
            }
            if (r <= prev) f |= FLAG_ROW_ORDER;
            prev = r;
            atomicAdd(cnt + r, 1);
        }
    }
    if (f) atomicOr(flags, f);
}

cudaError_t noalloc_rows_scratch(int device, int **rows, int **tail)
{
    // cudaGetSymbolAddress once per device; later calls reuse the address.
    static std::mutex mu;
    static int *base[kMaxNoAllocDevices] = {};
    if (device < 0 || device >= kMaxNoAllocDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!base[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_rows);
        if (e != cudaSuccess) return e;
        base[device] = static_cast<int *>(p);
    }
    *rows = base[device];
    *tail = base[device] + PCDM_NOALLOC_MAX_ROWS;
    return cudaSuccess;
}

cudaError_t launch_rows_checked(const int64_t *col_ptr, const int32_t *row_idx, int64_t m, int64_t n, int64_t nnz,
                                int *cnt, int *flags, cudaStream_t st)
{
    k_rows_checked<<<grid_for(n + 1), 256, 0, st>>>(col_ptr, row_idx, m, n, nnz, cnt, flags);
    return cudaGetLastError();
}

}  // namespace pcdm

// Deterministic two-kernel form of PCDM1 (pcdm_opts.deterministic_scatter).
//
// The iteration is Algorithm 1, step 4, with h(x) of eq. (h(x)), w = L, exactly
// as in the other forms; what is fixed here is the order and the rounding of
// every floating-point operation, so that a run is bitwise reproducible:
//   gather   grad_i = sum over column i in storage order, each product and each
//            addition rounded on its own (no FMA), starting from 0;
//            beta L_i one rounded product; u = x_i - grad_i / (beta L_i) and
//            t = lambda / (beta L_i) with correctly rounded divisions;
//            x_new = soft(u, t) (u - t, u + t or 0); h = x_new - x_i; x_i = x_new
//   scatter  every residual entry g_r receives the nonzero steps of the
//            iteration in increasing sampled position j: g_r = g_r + a_ri h_j,
//            product and sum rounded on their own.  The thread of the smallest
//            active position on row r applies all of them, so each g_r has one
//            writer and a fixed order; no atomics.
//   refresh  g_r = -b_r, then + a_ri x_i over the columns of row r in increasing
//            column index (only x_i != 0), in FP64.
// In the FP64 form these are the operations, in the order, of a plain
// sequential FP64 run of Algorithm 1 that visits S_k[0], S_k[1], ... in turn.
//
// The scatter reads A by rows: rptr / rcol / rval, a row-major copy of the
// pattern and values, each row sorted by column, built once at create.  The
// stamp array mark[i] = (lo32(k+1) << 32) | j records that column i took a
// nonzero step at position j of iteration k; the host clears it before each run
// of iterations, so stamps of one run never repeat.
#pragma once

#include "pcdm_kernels.cuh"

namespace pcdm {

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Phase 1 for position j = the thread's global index.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_det_gather(const IterArgs<VT, XT> a, const double *__restrict__ L64,
                                                       double beta, unsigned long long *__restrict__ mark, int64_t k)
{
    const int64_t j = int64_t(blockIdx.x) * kBlock + threadIdx.x;
    Counters cnt;
    if (j < a.tau) {
        const int32_t i = ldcg(sample_buf(a, k) + j);
        const Col<XT> c = load_col(a.desc, i);
        XT grad = XT(0);
        for (int e = 0; e < c.cnt; ++e) {
            const int64_t p = c.pbeg + e;
            grad = add_rn(grad, mul_rn(XT(ldv(a.pval + p)), ldcg(a.g + a.prow[p])));
        }
        const double xi = ldcg(a.x + i);
        const double Li = L64[i];
        double xn = 0.0;   // an empty column: the minimiser of lambda |x_i + t| is x_i + t = 0
        if (Li > 0.0) {
            const double bl = __dmul_rn(beta, Li);
            const double u = __dsub_rn(xi, __ddiv_rn(double(grad), bl));
            const double t = __ddiv_rn(a.lambda, bl);
            xn = u > t ? __dsub_rn(u, t) : (u < -t ? __dadd_rn(u, t) : 0.0);
        }
        const XT h = XT(__dsub_rn(xn, xi));
        a.x[i] = xn;
        a.h[j] = h;
        cnt.gathered += (unsigned long long)c.cnt;
        if (h != XT(0)) {
            mark[i] = ((unsigned long long)uint32_t(uint64_t(k) + 1u) << 32) | (unsigned long long)uint32_t(j);
            cnt.nonzero += 1;
            cnt.scattered += (unsigned long long)c.cnt;
        }
    }
    flush_counters(cnt, a.counters);
}

// Phase 2: the thread of position j visits the rows of its column when h_j != 0
// and applies the row's steps when j is the row's smallest active position.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_det_scatter(const IterArgs<VT, XT> a, const int64_t *__restrict__ rptr,
                                                        const int32_t *__restrict__ rcol, const VT *__restrict__ rval,
                                                        const unsigned long long *__restrict__ mark, int64_t k)
{
    const int64_t j = int64_t(blockIdx.x) * kBlock + threadIdx.x;
    if (j >= a.tau) return;
    const XT hj = a.h[j];
    if (hj == XT(0)) return;
    const int32_t i = sample_buf(a, k)[j];
    const Col<XT> c = load_col(a.desc, i);
    const uint32_t stamp = uint32_t(uint64_t(k) + 1u);
    for (int e = 0; e < c.cnt; ++e) {
        const int32_t r = a.prow[c.pbeg + e];
        const int64_t rb = rptr[r], re = rptr[r + 1];
        bool owner = true;
        for (int64_t q = rb; q < re; ++q) {
            const unsigned long long mk = mark[rcol[q]];
            if (uint32_t(mk >> 32) == stamp && uint32_t(mk) < uint32_t(j)) {
                owner = false;
                break;
            }
        }
        if (!owner) continue;
        // the row's active positions in increasing order, from j on
        XT gr = a.g[r];
        uint32_t next = uint32_t(j);
        for (;;) {
            uint32_t best = 0xFFFFFFFFu;
            XT bv = XT(0);
            for (int64_t q = rb; q < re; ++q) {
                const unsigned long long mk = mark[rcol[q]];
                const uint32_t pos = uint32_t(mk);
                if (uint32_t(mk >> 32) == stamp && pos >= next && pos < best) {
                    best = pos;
                    bv = XT(ldv(rval + q));
                }
            }
            if (best == 0xFFFFFFFFu) break;
            gr = add_rn(gr, mul_rn(bv, a.h[best]));
            next = best + 1u;
        }
        a.g[r] = gr;
    }
}

// g64_r = -b_r + sum over row r in increasing column of a_ri x_i (x_i != 0), and
// g_r = g64_r rounded to XT when g is FP32.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_det_refresh(const int64_t *__restrict__ rptr,
                                                        const int32_t *__restrict__ rcol, const VT *__restrict__ rval,
                                                        const double *__restrict__ x, const double *__restrict__ b,
                                                        int64_t m, double *g64, XT *g)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t r = int64_t(blockIdx.x) * kBlock + threadIdx.x; r < m; r += stride) {
        double acc = -b[r];
        for (int64_t q = rptr[r]; q < rptr[r + 1]; ++q) {
            const double xi = x[rcol[q]];
            if (xi != 0.0) acc = __dadd_rn(acc, __dmul_rn(double(ldv(rval + q)), xi));
        }
        g64[r] = acc;
        if constexpr (sizeof(XT) == 4) g[r] = float(acc);
    }
}

// Row-major copy: entry p of column i goes to the next free slot of its row
// (cursor[r] starts at rptr[r]); k_det_sort_rows then orders each row by column.
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_det_fill_rows(const int64_t *__restrict__ col_ptr,
                                                          const int32_t *__restrict__ row_idx,
                                                          const VT *__restrict__ val, int64_t n,
                                                          unsigned long long *cursor, int32_t *__restrict__ rcol,
                                                          VT *__restrict__ rval)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < n; i += stride) {
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) {
            const unsigned long long q = atomicAdd(cursor + row_idx[p], 1ull);
            rcol[q] = int32_t(i);
            rval[q] = val[p];
        }
    }
}

// Sorts (rcol, rval)[lo, hi) by rcol: insertion sort for short rows, heapsort
// otherwise (column indices within a row are distinct).
template <typename VT>
__device__ void sort_row(int32_t *c, VT *v, int64_t len)
{
    if (len <= 32) {
        for (int64_t a = 1; a < len; ++a) {
            const int32_t kc = c[a];
            const VT kv = v[a];
            int64_t b = a - 1;
            while (b >= 0 && c[b] > kc) {
                c[b + 1] = c[b];
                v[b + 1] = v[b];
                --b;
            }
            c[b + 1] = kc;
            v[b + 1] = kv;
        }
        return;
    }
    auto sift = [&](int64_t root, int64_t end) {
        while (2 * root + 1 < end) {
            int64_t child = 2 * root + 1;
            if (child + 1 < end && c[child] < c[child + 1]) ++child;
            if (c[root] >= c[child]) return;
            const int32_t tc = c[root];
            c[root] = c[child];
            c[child] = tc;
            const VT tv = v[root];
            v[root] = v[child];
            v[child] = tv;
            root = child;
        }
    };
    for (int64_t s = len / 2 - 1; s >= 0; --s) sift(s, len);
    for (int64_t end = len - 1; end > 0; --end) {
        const int32_t tc = c[0];
        c[0] = c[end];
        c[end] = tc;
        const VT tv = v[0];
        v[0] = v[end];
        v[end] = tv;
        sift(0, end);
    }
}

template <typename VT>
__global__ void __launch_bounds__(kBlock) k_det_sort_rows(const int64_t *__restrict__ rptr, int64_t m,
                                                          int32_t *__restrict__ rcol, VT *__restrict__ rval)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t r = int64_t(blockIdx.x) * kBlock + threadIdx.x; r < m; r += stride)
        sort_row<VT>(rcol + rptr[r], rval + rptr[r], rptr[r + 1] - rptr[r]);
}

template <typename VT, typename XT>
cudaError_t DetKernels<VT, XT>::build_rows(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                           int64_t n, const int64_t *rptr, unsigned long long *cursor, int32_t *rcol,
                                           VT *rval, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(cursor, rptr, size_t(m) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_det_fill_rows<VT><<<blocks_for_threads(n, 152 * 64), kBlock, 0, st>>>(col_ptr, row_idx, val, n, cursor, rcol,
                                                                             rval);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_det_sort_rows<VT><<<blocks_for_threads(m, 152 * 64), kBlock, 0, st>>>(rptr, m, rcol, rval);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t DetKernels<VT, XT>::gather(const IterArgs<VT, XT> &a, const double *L64, double beta,
                                       unsigned long long *mark, int64_t k, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    k_det_gather<VT, XT><<<blocks_for_threads(a.tau, 0), kBlock, 0, st>>>(a, L64, beta, mark, k);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t DetKernels<VT, XT>::scatter(const IterArgs<VT, XT> &a, const int64_t *rptr, const int32_t *rcol,
                                        const VT *rval, const unsigned long long *mark, int64_t k, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    k_det_scatter<VT, XT><<<blocks_for_threads(a.tau, 0), kBlock, 0, st>>>(a, rptr, rcol, rval, mark, k);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t DetKernels<VT, XT>::refresh(const int64_t *rptr, const int32_t *rcol, const VT *rval, const double *x,
                                        const double *b, int64_t m, double *g64, XT *g, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_det_refresh<VT, XT><<<blocks_for_threads(m, 152 * 16), kBlock, 0, st>>>(rptr, rcol, rval, x, b, m, g64, g);
    return cudaGetLastError();
}

}  // namespace pcdm

// libpcdm_gen: the device instance generator declared in include/pcdm_gen.h.
// Input generation only; it shares no code with the solver.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pcdm_gen.h"

namespace {

__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                                       uint32_t out[4])
{
    uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = uint32_t(p1);
        c2 = n2;
        c3 = uint32_t(p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

constexpr int kMaxPerCol = 32;

__global__ void k_colptr(int64_t n, int32_t per_col, int64_t *col_ptr)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += stride) col_ptr[i] = i * per_col;
}

__global__ void k_columns(int64_t m, int64_t n, int32_t per_col, uint64_t seed, int32_t val_dtype,
                          int32_t *row_idx, void *val)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t rows[kMaxPerCol];
        uint32_t t = 0;
        for (int s = 0; s < per_col; ++s) {
            for (;;) {
                uint32_t w[4];
                philox(uint32_t(i), uint32_t(uint64_t(i) >> 32), t++, 0x636f6c31u, seed, w);
                const uint64_t W = uint64_t(w[0]) | (uint64_t(w[1]) << 32);
                const uint32_t r = uint32_t(__umul64hi(W, uint64_t(m)));
                bool dup = false;
                for (int q = 0; q < s; ++q) dup |= rows[q] == r;
                if (!dup) {
                    rows[s] = r;
                    break;
                }
            }
        }
        for (int s = 1; s < per_col; ++s) {   // insertion sort
            const uint32_t v = rows[s];
            int q = s - 1;
            while (q >= 0 && rows[q] > v) {
                rows[q + 1] = rows[q];
                --q;
            }
            rows[q + 1] = v;
        }
        const int64_t base = i * per_col;
        for (int e = 0; e < per_col; ++e) {
            row_idx[base + e] = int32_t(rows[e]);
            float acc = 0.f;
            for (uint32_t c = 0; c < 3; ++c) {
                uint32_t w[4];
                philox(uint32_t(i), uint32_t(uint64_t(i) >> 32), uint32_t(e), 0x76616c31u + c, seed, w);
                for (int q = 0; q < 4; ++q) acc = acc + float(w[q] >> 8) * 5.9604644775390625e-8f;
            }
            const float v = acc - 6.0f;
            if (val_dtype == 0)
                static_cast<double *>(val)[base + e] = double(v);
            else if (val_dtype == 1)
                static_cast<float *>(val)[base + e] = v;
            else
                static_cast<__nv_bfloat16 *>(val)[base + e] = __float2bfloat16_rn(v);
        }
    }
}

__global__ void k_xstar(int64_t n, uint64_t seed, double density, double *x)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const double thr = density * 4294967296.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t w[4];
        philox(uint32_t(i), uint32_t(uint64_t(i) >> 32), 0u, 0x78737431u, seed, w);
        double v = 0.0;
        if (double(w[0]) < thr) {
            v = 1.0 + double(w[1]) * 0x1p-32;
            v = (w[2] & 1u) ? -v : v;
        }
        x[i] = v;
    }
}

template <typename VT>
__device__ __forceinline__ double vload(const void *val, int64_t p)
{
    if constexpr (sizeof(VT) == 8)
        return static_cast<const double *>(val)[p];
    else if constexpr (sizeof(VT) == 4)
        return double(static_cast<const float *>(val)[p]);
    else
        return double(__bfloat162float(static_cast<const __nv_bfloat16 *>(val)[p]));
}

template <typename VT>
__global__ void k_ax(int64_t n, int32_t per_col, const int32_t *row_idx, const void *val, const double *x,
                     double *acc)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double xi = x[i];
        if (xi == 0.0) continue;
        for (int e = 0; e < per_col; ++e) {
            const int64_t p = i * per_col + e;
            atomicAdd(acc + row_idx[p], vload<VT>(val, p) * xi);
        }
    }
}

__global__ void k_b(int64_t m, uint64_t seed, double noise_sd, const double *ax, int32_t b_dtype, void *b)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < m; r += stride) {
        double ih = 0.0;
        for (uint32_t c = 0; c < 3; ++c) {
            uint32_t w[4];
            philox(uint32_t(r), uint32_t(uint64_t(r) >> 32), c, 0x6e6f6931u, seed, w);
            for (int q = 0; q < 4; ++q) ih += double(w[q]) * 0x1p-32;
        }
        const double v = ax[r] + noise_sd * (ih - 6.0);
        if (b_dtype == 0)
            static_cast<double *>(b)[r] = v;
        else
            static_cast<float *>(b)[r] = float(v);
    }
}

template <typename VT>
__global__ void k_atb_max(int64_t n, int32_t per_col, const int32_t *row_idx, const void *val, const void *b,
                          int32_t b_dtype, unsigned long long *best)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    double mx = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = 0.0;
        for (int e = 0; e < per_col; ++e) {
            const int64_t p = i * per_col + e;
            const int32_t r = row_idx[p];
            const double br = b_dtype == 0 ? static_cast<const double *>(b)[r] : double(static_cast<const float *>(b)[r]);
            acc += vload<VT>(val, p) * br;
        }
        mx = fmax(mx, fabs(acc));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(best, (unsigned long long)__double_as_longlong(mx));
}

unsigned grid(int64_t count)
{
    int64_t g = (count + 255) / 256;
    return unsigned(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

extern "C" int pcdm_gen_per_col(int64_t m, int64_t n, int32_t per_col, uint64_t seed, int32_t val_dtype,
                                double x_density, double noise_sd, int32_t b_dtype, int64_t *col_ptr,
                                int32_t *row_idx, void *val, void *b, double *x_star, double *scratch,
                                double *lambda_max, void *cuda_stream)
{
    if (m < 1 || m >= (int64_t(1) << 32) || n < 1 || per_col < 1 || per_col > kMaxPerCol || per_col > m ||
        val_dtype < 0 || val_dtype > 2 || b_dtype < 0 || b_dtype > 1 || !col_ptr || !row_idx || !val || !b ||
        !x_star || !scratch || !lambda_max)
        return int(cudaErrorInvalidValue);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long *best = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&best), sizeof(unsigned long long));
    if (e != cudaSuccess) return int(e);
    k_colptr<<<grid(n + 1), 256, 0, st>>>(n, per_col, col_ptr);
    k_columns<<<grid(n), 256, 0, st>>>(m, n, per_col, seed, val_dtype, row_idx, val);
    k_xstar<<<grid(n), 256, 0, st>>>(n, seed, x_density, x_star);
    e = cudaMemsetAsync(scratch, 0, sizeof(double) * size_t(m), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(best, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        if (val_dtype == 0) {
            k_ax<double><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, x_star, scratch);
        } else if (val_dtype == 1) {
            k_ax<float><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, x_star, scratch);
        } else {
            k_ax<__nv_bfloat16><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, x_star, scratch);
        }
        k_b<<<grid(m), 256, 0, st>>>(m, seed, noise_sd, scratch, b_dtype, b);
        if (val_dtype == 0)
            k_atb_max<double><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, b, b_dtype, best);
        else if (val_dtype == 1)
            k_atb_max<float><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, b, b_dtype, best);
        else
            k_atb_max<__nv_bfloat16><<<grid(n), 256, 0, st>>>(n, per_col, row_idx, val, b, b_dtype, best);
        e = cudaGetLastError();
    }
    unsigned long long hb = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, best, sizeof(hb), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(best);
    if (e != cudaSuccess) return int(e);
    double v;
    static_assert(sizeof(v) == sizeof(hb), "64-bit double");
    __builtin_memcpy(&v, &hb, sizeof(v));
    *lambda_max = v;
    return 0;
}

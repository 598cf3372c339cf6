// Random-gather rate of the current GPU: the second ceiling (beside the HBM
// copy bandwidth) against which the iteration kernels are measured, because
// their time goes to gathers of the residual at random rows.  No counterpart in
// the paper: a measurement helper of the C ABI (pcdm_gather_rate).
//
// Every thread of a full grid (two blocks of 1024 threads per SM) issues rounds
// of 16 independent coherent (L2) loads at hashed positions of src, each
// index mulhi(hash, n) < n, so every load stays inside the vector.
#include <cstdint>
#include <cuda_runtime.h>

#include "pcdm.h"
#include "pcdm_host.h"

namespace {

constexpr int kRateThreads = 1024;
constexpr int kRateLoads = 16;
constexpr int kRateRounds = 32;

__device__ unsigned long long g_rate_sink;   // keeps the loads alive

__device__ __forceinline__ uint32_t rate_hash(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }

template <typename T>
__global__ void __launch_bounds__(kRateThreads) k_gather_rate(const T *__restrict__ src, uint32_t n, uint32_t salt)
{
    const uint32_t tid = blockIdx.x * kRateThreads + threadIdx.x;
    T acc = T(0);
    for (int r = 0; r < kRateRounds; ++r) {
        T v[kRateLoads];
#pragma unroll
        for (int q = 0; q < kRateLoads; ++q) {
            const uint32_t h = rate_hash((tid * kRateLoads + q) ^ (uint32_t(r) * 0x9E3779B9u) ^ salt);
            v[q] = ld_cg(src + __umulhi(h, n));
        }
#pragma unroll
        for (int q = 0; q < kRateLoads; ++q) acc += v[q];
    }
    if (acc == T(12345.678)) atomicXor(&g_rate_sink, 1ull);   // practically never: the loads must not be dropped
}

template <typename T>
cudaError_t time_rate(const T *src, uint32_t n, int blocks, cudaStream_t st, double *rate)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int w = 0; e == cudaSuccess && w < 2; ++w) {
        k_gather_rate<T><<<blocks, kRateThreads, 0, st>>>(src, n, 0x5A5A5A5Au + uint32_t(w));
        e = cudaGetLastError();
    }
    const int reps = 5;
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int w = 0; e == cudaSuccess && w < reps; ++w) {
        k_gather_rate<T><<<blocks, kRateThreads, 0, st>>>(src, n, 0x1234567u * uint32_t(w + 1));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        *rate = double(blocks) * kRateThreads * kRateRounds * kRateLoads * reps / (double(ms) * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" pcdm_status pcdm_gather_rate(const void *src, int64_t n, int32_t elem_bytes, double *gathers_per_s,
                                        void *cuda_stream)
{
    using namespace pcdm_host;
    if (!src || !gathers_per_s) return set_err(nullptr, PCDM_EINVAL, "src or gathers_per_s is NULL");
    if (n < 1 || n > int64_t(0xFFFFFFFFu)) return set_err(nullptr, PCDM_EINVAL, "need 1 <= n < 2^32");
    if (elem_bytes != 4 && elem_bytes != 8) return set_err(nullptr, PCDM_EINVAL, "elem_bytes must be 4 or 8");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = 2 * sms;
    if (elem_bytes == 8)
        e = time_rate(static_cast<const double *>(src), uint32_t(n), blocks, st, gathers_per_s);
    else
        e = time_rate(static_cast<const float *>(src), uint32_t(n), blocks, st, gathers_per_s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pcdm_gather_rate");
    return PCDM_OK;
}

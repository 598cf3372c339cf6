// Device building blocks of libpcdm (sm_103a).
//
// - philox_w0 / feistel_pi / sample_index: the tau-nice sampler of pcdm_step
//   (Sec. 4.1 item 3: every tau-subset equally likely), a 12-round Feistel
//   permutation of [0, 2^w) whose round function is Philox4x32-10 (Salmon et al.,
//   SC'11), walked back into [0, n).
// - ldv: value loads for FP64 / FP32 / BF16 storage.
// - red_add: fire-and-forget global atomic adds (red.global.add.{f32,f64}).
// - group_sum / group_max: reductions inside a group of W lanes of one warp.
// - grid_sync: grid-wide barrier for cooperative launches; every wait is bounded
//   by a %globaltimer budget, after which the block records a timeout in the
//   status word and the kernel returns.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcdm {

// ---------------------------------------------------------------------------
// Status word written by kernels (host maps it to pcdm_status).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };

// BF16 storage tag: the upper 16 bits of an IEEE binary32.
struct bf16_t {
    uint16_t bits;
};

// ---------------------------------------------------------------------------
// Philox4x32-10, word 0 of the output block.
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// Key of the permutation of iteration k.
struct SampleKey {
    uint32_t key0, key1;   // lo32(seed), hi32(seed)
    uint32_t klo, khi;     // lo32(k), hi32(k)
    uint32_t hb;           // half width of the Feistel domain
    uint32_t mask;         // 2^hb - 1
    uint32_t n;            // ground set size
};

__host__ __device__ inline uint32_t feistel_half_bits(int64_t n)
{
    uint32_t w = 2;
    while ((int64_t(1) << w) < n) w += 2;
    return w / 2;
}

__host__ __device__ inline SampleKey make_sample_key(uint64_t seed, int64_t k, int64_t n)
{
    SampleKey s;
    s.key0 = uint32_t(seed);
    s.key1 = uint32_t(seed >> 32);
    s.klo = uint32_t(uint64_t(k));
    s.khi = uint32_t(uint64_t(k) >> 32);
    s.hb = feistel_half_bits(n);
    s.mask = (s.hb >= 32) ? 0xFFFFFFFFu : ((1u << s.hb) - 1u);
    s.n = uint32_t(n);
    return s;
}

constexpr int kFeistelRounds = 12;

__device__ __forceinline__ uint32_t feistel_pi(uint32_t v, const SampleKey &s)
{
    uint32_t left = v >> s.hb, right = v & s.mask;
#pragma unroll 1
    for (uint32_t r = 0; r < kFeistelRounds; ++r) {
        const uint32_t f = philox_w0(right, r, s.klo, s.khi, s.key0, s.key1) & s.mask;
        const uint32_t nr = left ^ f;
        left = right;
        right = nr;
    }
    return (left << s.hb) | right;
}

// j-th coordinate of S_k (cycle walking keeps the map a bijection of [0, n)).
__device__ __forceinline__ int32_t sample_index(uint32_t j, const SampleKey &s)
{
    uint32_t v = feistel_pi(j, s);
    while (v >= s.n) v = feistel_pi(v, s);
    return int32_t(v);
}

// ---------------------------------------------------------------------------
// Value loads (read-only data: non-coherent path is safe).
__device__ __forceinline__ double ldv(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const bf16_t *p)
{
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(uint32_t(b) << 16);
}

// Loads of data that other blocks write during the same kernel: L2 only.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ void red_add(double *p, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T soft_threshold(T u, T t)
{
    return u > t ? u - t : (u < -t ? u + t : T(0));
}

// Mask of the W-lane group that lane `lane_w` (0..31) belongs to.
template <int W>
__device__ __forceinline__ unsigned group_mask(unsigned lane_w)
{
    if (W == 32) return 0xFFFFFFFFu;
    return ((1u << W) - 1u) << (lane_w & ~unsigned(W - 1));
}

template <int W, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, W);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, off));
    return v;
}

// ---------------------------------------------------------------------------
// Grid barrier for cooperative launches (all blocks co-resident).
// `counter` starts at 0 for the launch; the b-th barrier (b = 1, 2, ...) waits
// until counter >= b * gridDim.x.  Returns false when the wait ran out of its
// time budget or another block reported a failure; the caller must then return.
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

__device__ __forceinline__ bool grid_sync(unsigned long long *counter, unsigned long long target, int *status,
                                          uint64_t timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        red_release_add_u64(counter, 1ull);
        const uint64_t t0 = global_ns();
        uint32_t spins = 0;
        while (ld_acquire_u64(counter) < target) {
            if (ld_volatile_int(status) != DEV_OK) {
                ok = 0;
                break;
            }
            if ((++spins & 31u) == 0u && global_ns() - t0 > timeout_ns) {
                atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace pcdm

// Device building blocks of libpcdm (sm_103a).
//
// - philox4x32_10 / feistel_pi / sample_index: the tau-nice sampler of pcdm_step
//   (Sec. 4.1 item 3: every tau-subset equally likely), a 12-round Feistel
//   permutation of [0, 2^w) keyed by Philox4x32-10 (Salmon et al., SC'11) round
//   keys, walked back into [0, n).
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
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies,
// a word permutation and xor with a Weyl-sequence key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4])
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
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// The other doubly uniform samplings (Sec. 4.1 items 4 and 5).
// tau-independent: pick j = floor(W * n / 2^64), W the low 64 bits of the Philox
// block with counter (j, 1, lo32(k), hi32(k)); a block picked more than once is
// updated by its first pick only, decided through the key below (larger for
// earlier picks of the same iteration, and for later iterations).
__device__ __forceinline__ int32_t independent_pick(uint64_t seed, int64_t k, uint32_t j, int64_t n)
{
    uint32_t w[4];
    philox4x32_10(j, 1u, uint32_t(uint64_t(k)), uint32_t(uint64_t(k) >> 32), uint32_t(seed), uint32_t(seed >> 32), w);
    const uint64_t W = uint64_t(w[0]) | (uint64_t(w[1]) << 32);
    return int32_t(__umul64hi(W, uint64_t(n)));
}

__device__ __forceinline__ unsigned long long independent_key(int64_t k, uint32_t j)
{
    return ((unsigned long long)(k + 1) << 32) | (unsigned long long)(0xFFFFFFFFu - j);
}

// (tau, p_b)-binomial: position j of the tau-nice sample is kept iff word 0 of
// the Philox block with counter (j, 2, lo32(k), hi32(k)) is below T.
__device__ __forceinline__ bool binomial_keep(uint64_t seed, int64_t k, uint32_t j, uint64_t T)
{
    uint32_t w[4];
    philox4x32_10(j, 2u, uint32_t(uint64_t(k)), uint32_t(uint64_t(k) >> 32), uint32_t(seed), uint32_t(seed >> 32), w);
    return uint64_t(w[0]) < T;
}

constexpr int kFeistelRounds = 12;

// Permutation key of iteration k: 12 round keys (three Philox blocks with
// counters (c, 0, lo32(k), hi32(k)), c = 0, 1, 2, keyed by the seed) and the
// Feistel domain of [0, n).
struct SampleKey {
    uint32_t K[kFeistelRounds];
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

__device__ __forceinline__ void sample_key_domain(SampleKey &s, int64_t n)
{
    s.hb = feistel_half_bits(n);
    s.mask = (s.hb >= 32) ? 0xFFFFFFFFu : ((1u << s.hb) - 1u);
    s.n = uint32_t(n);
}

// Every thread computes the three blocks itself.
__device__ __forceinline__ SampleKey make_sample_key(uint64_t seed, int64_t k, int64_t n)
{
    SampleKey s;
#pragma unroll
    for (uint32_t c = 0; c < 3; ++c)
        philox4x32_10(c, 0u, uint32_t(uint64_t(k)), uint32_t(uint64_t(k) >> 32), uint32_t(seed), uint32_t(seed >> 32),
                      s.K + 4 * c);
    sample_key_domain(s, n);
    return s;
}

// The same key, computed once per warp (lanes 0..2 one block each) and
// broadcast; every lane of the warp must call it.
__device__ __forceinline__ SampleKey warp_sample_key(uint64_t seed, int64_t k, int64_t n)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (lane < 3)
        philox4x32_10(lane, 0u, uint32_t(uint64_t(k)), uint32_t(uint64_t(k) >> 32), uint32_t(seed),
                      uint32_t(seed >> 32), w);
    SampleKey s;
#pragma unroll
    for (int r = 0; r < kFeistelRounds; ++r) s.K[r] = __shfl_sync(0xFFFFFFFFu, w[r & 3], r >> 2);
    sample_key_domain(s, n);
    return s;
}

// MurmurHash3's 32-bit finalizer (Appleby): the Feistel round function mixes
// R with the round key.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t feistel_pi(uint32_t v, const SampleKey &s)
{
    uint32_t left = v >> s.hb, right = v & s.mask;
#pragma unroll
    for (int r = 0; r < kFeistelRounds; ++r) {
        const uint32_t f = fmix32(right ^ s.K[r]) & s.mask;
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
// Asynchronous global -> shared copies of 16 bytes (L2 only), per-thread groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = uint32_t(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// TMA bulk copies global -> shared with mbarrier completion (sm_90+).  Source
// and destination 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

// Makes mbarrier initialisations visible to the async proxy (TMA completions).
__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the given phase of an mbarrier, bounded by timeout_ns; on expiry the
// status word records a timeout and false is returned.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, int *status, uint64_t timeout_ns);

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar)), "l"(pol)
        : "memory");
}

// ---------------------------------------------------------------------------
// L2 eviction priorities.  Every iteration reads the residual at random rows
// (the whole vector is hot) while the columns of A, their descriptors and x are
// touched once: the residual is marked evict-last and the streamed data
// evict-first, so that streaming A through L2 does not push the residual out.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Coherent (L2) loads and stores with an L2 policy.
__device__ __forceinline__ double ldcg_hint(const double *p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
// The high 32-bit word of the double at p (sign, exponent, 20 mantissa bits).
__device__ __forceinline__ uint32_t ldcg_hi_hint(const double *p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(reinterpret_cast<const char *>(p) + 4), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldcg_hint(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(double *p, double v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(float *p, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
// Read-only 16-byte load with an L2 policy.
__device__ __forceinline__ int4 ldnc_v4_hint(const void *p, uint64_t pol)
{
    int4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
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
__device__ __forceinline__ void red_add(double *p, double v, uint64_t pol)
{
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add(float *p, float v, uint64_t pol)
{
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

// g[0..3] += v[0..3] in one vector reduction (sm_90+); g 16-byte aligned.
__device__ __forceinline__ void red_add_v4(float *p, float v0, float v1, float v2, float v3, uint64_t pol)
{
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v0), "f"(v1),
                 "f"(v2), "f"(v3), "l"(pol)
                 : "memory");
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
    if constexpr (W == 32)
        return 0xFFFFFFFFu;
    else
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
__device__ __forceinline__ double ld_volatile_f64(const double *p) { return *reinterpret_cast<const volatile double *>(p); }
__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *reinterpret_cast<const volatile unsigned *>(p);
}

__device__ __forceinline__ bool wait_counter(unsigned long long *counter, unsigned long long target, int *status,
                                             uint64_t timeout_ns)
{
    // The acquire load that sees the target orders every later access of this
    // thread (and, through the block barrier that follows, of its block).
    int ok = 1;
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (ld_acquire_u64(counter) < target) {
        // every 16th spin: another block's failure, then the time limit
        if ((++spins & 15u) == 0u) {
            if (ld_volatile_int(status) != DEV_OK) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    return ok != 0;
}

__device__ __forceinline__ bool grid_sync(unsigned long long *counter, unsigned long long target, int *status,
                                          uint64_t timeout_ns)
{
    if (gridDim.x == 1) {
        __threadfence();
        __syncthreads();
        return true;
    }
    // The block barrier orders the block's accesses before thread 0's release
    // add, which publishes them at GPU scope.
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add_u64(counter, 1ull);
        s_ok = wait_counter(counter, target, status, timeout_ns) ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// Split form of grid_sync: arrive, do independent work, then wait.
__device__ __forceinline__ void grid_arrive(unsigned long long *counter)
{
    if (gridDim.x == 1) {
        __threadfence();
        __syncthreads();
        return;
    }
    __syncthreads();
    if (threadIdx.x == 0) red_release_add_u64(counter, 1ull);
}

__device__ __forceinline__ bool grid_wait(unsigned long long *counter, unsigned long long target, int *status,
                                          uint64_t timeout_ns)
{
    if (gridDim.x == 1) return true;
    __shared__ int s_ok2;
    if (threadIdx.x == 0) s_ok2 = wait_counter(counter, target, status, timeout_ns) ? 1 : 0;
    __syncthreads();
    return s_ok2 != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, int *status, uint64_t timeout_ns)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (!mbar_try_wait(mbar, parity)) {
        if ((++spins & 15u) == 0u) {
            if (ld_volatile_int(status) != DEV_OK) return false;
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// Asynchronous prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

}  // namespace pcdm

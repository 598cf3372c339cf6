// Column kernels of libpcdm, templated on the stored value type VT and the
// iterate type XT (x, g, h, 1/L and the gradient accumulator).  Included by one
// translation unit per (VT, XT) pair, which instantiates Kernels<VT, XT>.
//
// Work mapping.  A group of W lanes of one warp (W in {1, 2, 4, 8, 16, 32}) owns
// one column at a time; lane l owns the contiguous run of kE entries starting at
// l*kE inside each chunk of W*kE entries, read with 16-byte vector loads from the
// padded layout (see pcdm_internal.h).  Short columns (the common case) use
// W = 1: no cross-lane reduction, and the proximal step runs on all 32 lanes of
// a warp at once, which matters on GB300 where FP64 issues at about 2 DFMA per
// clock per SM.
//
// One PCDM1 iteration (Algorithm 1, step 4, with h(x) of eq. (h(x)), w = L):
//   phase 1 (gather):  grad_i = a_i^T g for i = S_k[j], all from the same g;
//                      x_new = soft(x_i - grad_i/(beta L_i), lambda/(beta L_i));
//                      h_j = x_new - x_i; x_i = x_new
//   phase 2 (scatter): g_r += a_ri h_j for the columns with h_j != 0 (red.global.add),
//                      and S_{k+1} is drawn.
// The phases are separated by a kernel boundary (two-kernel form) or by a
// bounded grid barrier (fused persistent form).  The fused form keeps each
// group's next column in registers across the barrier: during phase 2 of
// iteration k it already draws its sample of iteration k+1 and loads that
// column's descriptor and first chunk, so that after the barrier only the
// gathers of g and x remain on the critical path.
#pragma once

#include <cmath>

#include "pcdm_internal.h"

namespace pcdm {

constexpr int kE = kLaneRun;   // entries per lane and chunk

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

// ---------------------------------------------------------------------------
// Column descriptor and chunk loads.
template <typename XT>
struct Col {
    int64_t pbeg;
    int cnt;
    XT invL;
};

template <typename XT>
__device__ __forceinline__ Col<XT> col_from_word(const int4 v)
{
    Col<XT> c;
    c.pbeg = int64_t(uint32_t(v.x)) * 4;
    c.cnt = v.y;
    if constexpr (sizeof(XT) == 8)
        c.invL = __hiloint2double(v.w, v.z);
    else
        c.invL = __int_as_float(v.z);
    return c;
}

template <typename XT>
__device__ __forceinline__ Col<XT> load_col(const ColDesc<XT> *d, int32_t i, uint64_t pol)
{
    return col_from_word<XT>(ldnc_v4_hint(d + i, pol));
}

template <typename XT>
__device__ __forceinline__ Col<XT> load_col(const ColDesc<XT> *d, int32_t i)
{
    const int4 v = __ldg(reinterpret_cast<const int4 *>(d + i));
    Col<XT> c;
    c.pbeg = int64_t(uint32_t(v.x)) * 4;
    c.cnt = v.y;
    if constexpr (sizeof(XT) == 8)
        c.invL = __hiloint2double(v.w, v.z);
    else
        c.invL = __int_as_float(v.z);
    return c;
}

template <int E, typename XT>
struct Chunk {
    int32_t row[E];
    XT val[E];
};

template <int E>
__device__ __forceinline__ void ld_rows(int32_t (&r)[E], const int32_t *p)
{
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const int4 v = __ldg(reinterpret_cast<const int4 *>(p) + q);
        r[4 * q + 0] = v.x;
        r[4 * q + 1] = v.y;
        r[4 * q + 2] = v.z;
        r[4 * q + 3] = v.w;
    }
}

template <int E>
__device__ __forceinline__ void ld_vals(double (&v)[E], const double *p)
{
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
        const double2 d = __ldg(reinterpret_cast<const double2 *>(p) + q);
        v[2 * q + 0] = d.x;
        v[2 * q + 1] = d.y;
    }
}

template <int E>
__device__ __forceinline__ void ld_vals(float (&v)[E], const float *p)
{
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const float4 d = __ldg(reinterpret_cast<const float4 *>(p) + q);
        v[4 * q + 0] = d.x;
        v[4 * q + 1] = d.y;
        v[4 * q + 2] = d.z;
        v[4 * q + 3] = d.w;
    }
}

template <int E>
__device__ __forceinline__ void ld_vals(float (&v)[E], const bf16_t *p)
{
#pragma unroll
    for (int q = 0; q < E / 8; ++q) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + q);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[8 * q + 2 * t + 0] = __uint_as_float(w[t] << 16);
            v[8 * q + 2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
        }
    }
}

// Chunk load with an L2 policy (the pipelined kernel marks A evict-first).
template <int E, typename XT>
__device__ __forceinline__ void ld_chunk_hint(Chunk<E, XT> &c, const int32_t *prow, const double *pval, int64_t p,
                                              uint64_t pol)
{
    static_assert(sizeof(XT) == 8, "FP64 values go with FP64 iterates");
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const int4 v = ldnc_v4_hint(prow + p + 4 * q, pol);
        c.row[4 * q + 0] = v.x;
        c.row[4 * q + 1] = v.y;
        c.row[4 * q + 2] = v.z;
        c.row[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
        const int4 v = ldnc_v4_hint(pval + p + 2 * q, pol);
        c.val[2 * q + 0] = __hiloint2double(v.y, v.x);
        c.val[2 * q + 1] = __hiloint2double(v.w, v.z);
    }
}
template <int E, typename XT>
__device__ __forceinline__ void ld_chunk_hint(Chunk<E, XT> &c, const int32_t *prow, const float *pval, int64_t p,
                                              uint64_t pol)
{
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const int4 v = ldnc_v4_hint(prow + p + 4 * q, pol);
        c.row[4 * q + 0] = v.x;
        c.row[4 * q + 1] = v.y;
        c.row[4 * q + 2] = v.z;
        c.row[4 * q + 3] = v.w;
        const int4 u = ldnc_v4_hint(pval + p + 4 * q, pol);
        c.val[4 * q + 0] = __int_as_float(u.x);
        c.val[4 * q + 1] = __int_as_float(u.y);
        c.val[4 * q + 2] = __int_as_float(u.z);
        c.val[4 * q + 3] = __int_as_float(u.w);
    }
}
template <int E, typename XT>
__device__ __forceinline__ void ld_chunk_hint(Chunk<E, XT> &c, const int32_t *prow, const bf16_t *pval, int64_t p,
                                              uint64_t pol)
{
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const int4 v = ldnc_v4_hint(prow + p + 4 * q, pol);
        c.row[4 * q + 0] = v.x;
        c.row[4 * q + 1] = v.y;
        c.row[4 * q + 2] = v.z;
        c.row[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < E / 8; ++q) {
        const int4 u = ldnc_v4_hint(pval + p + 8 * q, pol);
        const uint32_t w[4] = {uint32_t(u.x), uint32_t(u.y), uint32_t(u.z), uint32_t(u.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            c.val[8 * q + 2 * t + 0] = __uint_as_float(w[t] << 16);
            c.val[8 * q + 2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
        }
    }
}

// Chunk load of the column kernels: A is read once per use, so it is marked
// evict-first in L2, where it would otherwise push out the residual that every
// gather reads (long columns stream about as many bytes of A per iteration as
// L2 holds).
template <int E, typename VT, typename XT>
__device__ __forceinline__ void ld_chunk(Chunk<E, XT> &c, const int32_t *prow, const VT *pval, int64_t p)
{
    ld_chunk_hint<E>(c, prow, pval, p, l2_evict_first());
}

// The coordinate gradient of the smooth part is grad_i = sum_r a_ri phi(g_r).
// GM = 0: phi is the identity (the square losses: LASSO with g = A x - b, the
// SVM dual with g = A x for the label-signed examples).  GM = 1: the logistic
// loss (Sec. 8.4), g holds the margins y_r A_r^T x (labels folded into the
// rows) and phi(t) = d/dt log(1 + e^-t) = -1/(1 + e^t).
template <int GM, typename T>
__device__ __forceinline__ T grad_map(T v)
{
    if constexpr (GM == 0)
        return v;
    else if constexpr (sizeof(T) == 8)
        return -1.0 / (1.0 + exp(v));
    else
        return -1.0f / (1.0f + expf(v));
}

// sum_e val[e] * phi(v[row[e]]) over the first `valid` entries of the lane's run
// (the gathered vector marked evict-last in L2).
template <int E, typename XT, typename GT, typename AT, int GM = 0>
__device__ __forceinline__ AT chunk_dot(const Chunk<E, XT> &c, const GT *v, int valid)
{
    const uint64_t pl = l2_evict_last();
    GT gv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) gv[e] = (e < valid) ? ldcg_hint(v + c.row[e], pl) : GT(0);
    AT acc = AT(0);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e < valid) acc = fma(AT(c.val[e]), AT(grad_map<GM>(gv[e])), acc);
    return acc;
}

template <int E, typename XT>
__device__ __forceinline__ void chunk_scatter(const Chunk<E, XT> &c, XT *g, XT h, int valid)
{
    const uint64_t pl = l2_evict_last();
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e < valid) red_add(g + c.row[e], c.val[e] * h, pl);
}

template <int E, typename XT>
__device__ __forceinline__ void chunk_scatter_hint(const Chunk<E, XT> &c, XT *g, XT h, int valid, uint64_t pol)
{
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e < valid) red_add(g + c.row[e], c.val[e] * h, pol);
}

template <int E, typename XT, typename GT = XT, int GM = 0>
__device__ __forceinline__ GT chunk_dot_hint(const Chunk<E, XT> &c, const GT *v, int valid, uint64_t pol)
{
    GT gv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) gv[e] = (e < valid) ? ldcg_hint(v + c.row[e], pol) : GT(0);
    GT acc = GT(0);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e < valid) acc = fma(GT(c.val[e]), grad_map<GM>(gv[e]), acc);
    return acc;
}

// a_i^T phi(g) over a whole column, chunk by chunk (all W lanes of the group together).
template <int W, typename VT, typename XT, int GM = 0>
__device__ __forceinline__ XT column_dot(const IterArgs<VT, XT> &a, const Col<XT> &c, int lane, unsigned gmask)
{
    constexpr int CH = W * kE;
    XT acc = XT(0);
    for (int cs = 0; cs < c.cnt; cs += CH) {
        Chunk<kE, XT> t;
        const int st = cs + lane * kE;
        if (st < c.cnt) ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + st);
        acc += chunk_dot<kE, XT, XT, XT, GM>(t, a.g, c.cnt - st);
    }
    return group_sum<W>(acc, gmask);
}

template <int W, typename VT, typename XT>
__device__ __forceinline__ void column_scatter(const IterArgs<VT, XT> &a, const Col<XT> &c, int lane, XT h,
                                               int from)
{
    constexpr int CH = W * kE;
    for (int cs = from; cs < c.cnt; cs += CH) {
        Chunk<kE, XT> t;
        const int st = cs + lane * kE;
        if (st < c.cnt) {
            ld_chunk<kE>(t, a.prow, a.pval, c.pbeg + st);
            chunk_scatter<kE>(t, a.g, h, c.cnt - st);
        }
    }
}

// The step of eq. (h(x)) for one coordinate: soft(x - grad/(beta L), lambda/(beta L)),
// with 1/(beta L) = (1/L)(1/beta); an empty column (1/L stored as 0) goes to 0.
// FP64 in every precision pair: the fixed point of the step (the optimality
// condition -grad in lambda d|x|) does not depend on the step length, so an FP32
// 1/L costs no accuracy, but x itself must not be rounded to FP32.
__device__ __forceinline__ double prox_step(double xi, double grad, double invL, double inv_beta, double lambda)
{
    if (invL == 0.0) return 0.0;
    const double ibl = invL * inv_beta;
    return soft_threshold<double>(fma(-grad, ibl, xi), lambda * ibl);
}

// ---------------------------------------------------------------------------
// FP32 certificate of a zero LASSO step.
//
// With x_i = 0 (either sign), prox_step returns exactly 0 whenever |grad| <=
// lambda: grad*ibl and lambda*ibl are rounded monotonically, so |u| <= t.  On
// GB300 an FP64 instruction (FMA, compare, or conversion to or from FP32)
// occupies a sub-partition's FP64 unit for about 76 cycles per warp, masked
// lanes included, while most sampled coordinates of a LASSO solve sit at
// x_i = 0 with |grad_i| < lambda.  The FP64 form therefore first sums
// grad_i = sum_e v_e g_e in FP32 over images of the FP64 operands made with
// integer operations, with a bound on the distance to the FP64 sum.  When the
// bound shows |grad_i| <= lambda the step is 0, the value the FP64 path would
// return, and the lane needs no FP64 instruction; a warp skips the FP64 block
// when all its lanes are certified.
//
// Image of a double y with high word hi: the FP32 number with y's sign,
// exponent and 20 leading mantissa bits, its magnitude clamped to [2^-126, inf]:
// |y| - |image| < 2^-20 |image| for 2^-126 <= |y| < 2^128, |y - image| <= 2^-126
// below that, and inf (no certificate) above.
__device__ __forceinline__ float f32_image(uint32_t hi)
{
    const uint32_t m = min(max(hi & 0x7FFFFFFFu, 0x38100000u), 0x47F00000u);
    return __uint_as_float(((m - 0x38000000u) << 3) | (hi & 0x80000000u));
}

__device__ __forceinline__ uint32_t hi_word(double y)
{
    return uint32_t(__double2hiint(y));
}

// |v| <= lam for a finite lam >= 0, by integer compare of the bit patterns
// (non-negative doubles order as their bits; a NaN v compares above any finite lam).
__device__ __forceinline__ bool abs_le_bits(double v, double lam)
{
    return (uint64_t(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull) <= uint64_t(__double_as_longlong(lam));
}

// Either zero (the sign bit ignored), by integer compare.
__device__ __forceinline__ bool is_zero_bits(double y)
{
    return (uint64_t(__double_as_longlong(y)) << 1) == 0;
}
__device__ __forceinline__ bool is_zero_bits(float y)
{
    return (__float_as_uint(y) << 1) == 0;
}

// Running FP32 sums of one column's products v_e g_e (operands as high words).
// Error analysis, u = 2^-24, c products, vi, gi the images, M = max |image|,
// S = sum |vi gi|, D = sum v g exactly, a32 / s32 the FP32 FMA sums:
//   |D - sum vi gi| <= (2^-19 + 2^-40) S + c 2^-125 M      (images)
//   |a32 - sum vi gi| <= gamma_c S + c 2^-149,  S <= (s32 + c 2^-149)/(1 - gamma_c)
//   the FP64 sum differs from D by at most gamma64_2c sum |v g| <= 2^-38 S (c <= 1024)
// so for c <= 1024, |FP64 sum| <= |a32| + (c + 40) u s32 + c 2^-123 M + 2^-120,
// the left side of the test below, evaluated rounding upwards.
struct ZeroCert {
    float acc = 0.f, sabs = 0.f, mx = 0.f;
    __device__ __forceinline__ void add(uint32_t hv, uint32_t hg)
    {
        const float v = f32_image(hv), g = f32_image(hg);
        acc = fmaf(v, g, acc);
        sabs = fmaf(fabsf(v), fabsf(g), sabs);
        mx = fmaxf(mx, fmaxf(fabsf(v), fabsf(g)));
    }
    // true only if the FP64 sum of the c products added is at most lamf <= lambda
    // in magnitude (inf or NaN operands never certify)
    __device__ __forceinline__ bool below(int c, float lamf) const
    {
        if (c > 1024) return false;
        float lhs = __fadd_ru(fabsf(acc), 0x1p-120f);
        lhs = __fmaf_ru(mx, float(c) * 0x1p-123f, lhs);
        lhs = __fmaf_ru(sabs, float(c + 40) * 0x1p-24f, lhs);
        return lhs <= lamf;
    }
};

// The new coordinate for each objective (argmin over t of the model of eq.
// (h(x)): grad_i t + (beta L_i / 2) t^2 + Psi_i(x_i + t)), from grad = a_i^T phi(g):
//   problem 0, LASSO: prox_step above.
//   problem 1, SVM dual (Sec. 8.3), Psi the indicator of [0, 1]: with the examples
//     signed by their labels and 1/L stored as 1/||a_i||^2, the paper's
//     grad_i/(beta L_i) = (a_i^T g - kappa)/(beta ||a_i||^2), kappa = lambda n;
//     the step is clip(x_i - that, 0, 1); an all-zero example goes to 1.
//   problem 2, logistic (Sec. 8.4), Psi_i = lambda x_i^2, 1/L stored as 4/||a_i||^2:
//     x_i - (grad + 2 lambda x_i)/(beta L_i + 2 lambda).
__device__ __forceinline__ double coord_step(int problem, double xi, double grad, double invL, double inv_beta,
                                             double lambda, double kappa)
{
    if (problem == 0) return prox_step(xi, grad, invL, inv_beta, lambda);
    if (problem == 1) {
        if (invL == 0.0) return 1.0;
        const double u = fma(-(grad - kappa), invL * inv_beta, xi);
        return fmin(fmax(u, 0.0), 1.0);
    }
    const double bl = invL == 0.0 ? 0.0 : 1.0 / (invL * inv_beta);
    return xi - fma(2.0 * lambda, xi, grad) / (bl + 2.0 * lambda);
}

// Phase 1 for sampled position j, columns read from memory (no prefetch).
template <int W, typename VT, typename XT, int GM = 0>
__device__ __forceinline__ void gather_generic(const IterArgs<VT, XT> &a, const int32_t *S, int64_t j, int lane,
                                               unsigned gmask, Counters &cnt, int64_t k = -1)
{
    const int32_t i = ldcg(S + j);
    // positions idle under the tau-independent (a repeated pick) or binomial
    // (a dropped position) samplings take no step
    if (k >= 0 && a.sampling != 0) {
        const bool idle = a.sampling == 1 ? (ldcg(a.win + i) != independent_key(k, uint32_t(j)))
                                          : !binomial_keep(a.seed, k, uint32_t(j), a.keep_T);
        if (idle) {
            if (lane == 0) a.h[j] = XT(0);
            return;
        }
    }
    const Col<XT> c = load_col(a.desc, i);
    const double xi = ldcg(a.x + i);
    const XT grad = column_dot<W, VT, XT, GM>(a, c, lane, gmask);
    const double xn = coord_step(a.problem, xi, double(grad), double(c.invL), a.inv_beta, a.lambda, a.kappa);
    const double h64 = xn - xi;
    if (lane == 0) {
        if (h64 != 0.0) a.x[i] = xn;
        a.h[j] = XT(h64);
        cnt.gathered += (unsigned long long)c.cnt;
        if (h64 != 0.0) {
            cnt.nonzero += 1;
            cnt.scattered += (unsigned long long)c.cnt;
        }
    }
}

// Phase 2 for sampled position j.
template <int W, typename VT, typename XT>
__device__ __forceinline__ void scatter_generic(const IterArgs<VT, XT> &a, const int32_t *S, int64_t j, int lane)
{
    const XT h = ldcg(a.h + j);
    if (h == XT(0)) return;
    const int32_t i = ldcg(S + j);
    column_scatter<W>(a, load_col(a.desc, i), lane, h, 0);
}

// ---------------------------------------------------------------------------
// Two-kernel form.
template <int W, typename VT, typename XT, int GM = 0>
__global__ void __launch_bounds__(kBlock) k_gather(const IterArgs<VT, XT> a, int64_t k)
{
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t grp = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W;
    Counters cnt;
    if (grp < a.tau) gather_generic<W, VT, XT, GM>(a, sample_buf(a, k), grp, lane, gmask, cnt, k);
    flush_counters(cnt, a.counters);
}

template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_scatter(const IterArgs<VT, XT> a, int64_t k, int sample_next)
{
    const int lane = threadIdx.x & (W - 1);
    const int64_t gid = int64_t(blockIdx.x) * kBlock + threadIdx.x;
    const int64_t grp = gid / W;
    if (grp < a.tau) scatter_generic<W>(a, sample_buf(a, k), grp, lane);
    if (sample_next) {
        const SampleKey key = warp_sample_key(a.seed, k + 1, a.n);
        if (gid < a.tau) sample_buf(a, k + 1)[gid] = sample_index(uint32_t(gid), key);
    }
}

// ---------------------------------------------------------------------------
// Fused persistent form: one cooperative launch runs `iters` iterations.
// Position j0 = (global thread index) / W is this group's register-resident
// column; positions j0 + ngrp, j0 + 2 ngrp, ... (only when tau exceeds the
// number of groups) go through the generic path.
template <int W, typename VT, typename XT, int GM = 0>
__global__ void __launch_bounds__(fused_max_block(W), 1) k_fused(const IterArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    constexpr int CH = W * kE;
    constexpr int G = pad_granule<VT>();
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t j0 = gid / W;
    const int64_t ngrp = nthreads / W;
    const bool own = j0 < a.tau;
    unsigned long long target = 0;
    Counters cnt;
    const float lamf = __double2float_rd(a.lambda);   // the largest float <= lambda

    // Prologue: the column of iteration k0 into registers.
    int32_t i0 = 0;
    Col<XT> c0;
    c0.pbeg = 0;
    c0.cnt = 0;
    c0.invL = XT(0);
    Chunk<kE, XT> ch;
    if (own) {
        i0 = ldcg(sample_buf(a, k0) + j0);
        c0 = load_col(a.desc, i0);
        if (lane * kE < c0.cnt) ld_chunk<kE>(ch, a.prow, a.pval, c0.pbeg + lane * kE);
    }

    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        const int32_t *S = sample_buf(a, k);
        XT h0 = XT(0);
        // ---------------- phase 1: gradient, step, x update
        // Issue the loads of x_i and of g at the chunk's rows first, draw this
        // group's sample of iteration k+1 (integer work) while they are in
        // flight, then consume them on the FP pipe.
        const SampleKey key = warp_sample_key(a.seed, k + 1, a.n);
        int32_t i_next = 0;
        Col<XT> c_next = c0;
        if (own) {
            const double xi = ldcg(a.x + i0);
            XT gv[kE];
            const int valid0 = c0.cnt - lane * kE;
            const uint64_t pl = l2_evict_last();
#pragma unroll
            for (int e = 0; e < kE; ++e) gv[e] = (e < valid0) ? ldcg_hint(a.g + ch.row[e], pl) : XT(0);
            i_next = sample_index(uint32_t(j0), key);
            c_next = load_col(a.desc, i_next);
            XT acc = XT(0);
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid0) acc = fma(ch.val[e], grad_map<GM>(gv[e]), acc);
            for (int cs = CH; cs < c0.cnt; cs += CH) {
                Chunk<kE, XT> t;
                const int st = cs + lane * kE;
                if (st < c0.cnt) ld_chunk<kE>(t, a.prow, a.pval, c0.pbeg + st);
                acc += chunk_dot<kE, XT, XT, XT, GM>(t, a.g, c0.cnt - st);
            }
            acc = group_sum<W>(acc, gmask);
            // At x_i = 0 the LASSO step is 0 when |grad| <= lambda: tested in FP32
            // against lambda rounded down, or on the FP64 bit patterns as integers,
            // so that a warp whose columns all pass runs no FP64 instruction.
            bool zero_step = false;
            if constexpr (GM == 0) {
                if constexpr (sizeof(XT) == 4)
                    zero_step = a.problem == 0 && is_zero_bits(xi) && fabsf(float(acc)) <= lamf;
                else
                    zero_step = a.problem == 0 && is_zero_bits(xi) && abs_le_bits(double(acc), a.lambda);
            }
            if (!zero_step) {
                const double xn =
                    coord_step(a.problem, xi, double(acc), double(c0.invL), a.inv_beta, a.lambda, a.kappa);
                const double h64 = xn - xi;
                h0 = XT(h64);
                if (lane == 0 && h64 != 0.0) {
                    a.x[i0] = xn;
                    cnt.nonzero += 1;
                    cnt.scattered += (unsigned long long)c0.cnt;
                }
            }
            if (lane == 0) cnt.gathered += (unsigned long long)c0.cnt;
        }
        for (int64_t j = j0 + ngrp; j < a.tau; j += ngrp) gather_generic<W, VT, XT, GM>(a, S, j, lane, gmask, cnt);
        target += gridDim.x;
        if (!grid_sync(a.bar, target, a.status, a.timeout_ns)) return;

        // ---------------- phase 2: residual update, next sample
        // the chunk registers are free by now (reloaded from L2 for the few columns with h != 0)
        if (own && !is_zero_bits(h0)) column_scatter<W>(a, c0, lane, h0, 0);
        for (int64_t j = j0 + ngrp; j < a.tau; j += ngrp) scatter_generic<W>(a, S, j, lane);
        int32_t *Sn = sample_buf(a, k + 1);
        for (int64_t j = ngrp + gid; j < a.tau; j += nthreads) Sn[j] = sample_index(uint32_t(j), key);
        if (own) {
            i0 = i_next;
            c0 = c_next;
            if (lane == 0) Sn[j0] = i0;
        }
        target += gridDim.x;
        grid_arrive(a.bar);
        if (own) {
            if (lane * kE < c0.cnt) ld_chunk<kE>(ch, a.prow, a.pval, c0.pbeg + lane * kE);
            if (lane == 0 && c0.cnt > CH) {
                const int64_t tail = ((int64_t(c0.cnt) + G - 1) / G) * G - CH;
                prefetch_l2_bulk(a.prow + c0.pbeg + CH, uint32_t(tail * 4));
                prefetch_l2_bulk(a.pval + c0.pbeg + CH, uint32_t(tail * int64_t(sizeof(VT))));
            }
        }
        if (!grid_wait(a.bar, target, a.status, a.timeout_ns)) return;
    }
    flush_counters(cnt, a.counters);
}

// ---------------------------------------------------------------------------
// Pipelined persistent form: one lane per column, every sampled position owned
// by one thread (tau <= threads of the grid), one grid barrier per iteration.
// The residual lives in two buffers: at iteration k, buffer k&1 holds g_k and is
// only read (gathers), the other holds g_{k-1} and only receives atomic adds:
// the steps of iteration k-1 (it missed them) and of iteration k.  So the
// scatter of iteration k never touches what the gathers of iteration k read,
// the update stays Jacobi, and only the barrier that publishes g_{k+1} remains.
// Both buffers hold the same residual at every launch boundary.
// Thread j keeps i_k and i_{k+1} with their descriptors in registers; the first
// entries of column i_k sit in the thread's shared-memory slot, brought in by a
// TMA bulk copy issued during the previous iteration (completion on an
// mbarrier).  Per iteration k (k_fused_pipe_wide, after the helpers below):
//   gather   the gathers of g_k at the slot's rows are issued; the sample
//            i_{k+2} is drawn (integer work) while they are in flight and its
//            descriptor load is issued; then gradient, step, x;
//   scatter  the step of k-1 (from memory) and of k (from the slot) into the
//            other buffer;
//   barrier  release-arrive; then the bulk copy of column i_{k+1}'s first
//            entries into the slot; then wait
// On GB300 the scattered gathers saturate each SM's load/store pipe, so the
// bulk copies run on the TMA engine and the sampling is integer work only.
// Values of one 16-byte word of a shared chunk (16 / sizeof(VT) entries).
template <typename VT, typename XT>
__device__ __forceinline__ void decode_word(const uint4 u, XT (&v)[16 / sizeof(VT)])
{
    if constexpr (sizeof(VT) == 8) {
        v[0] = XT(__hiloint2double(int(u.y), int(u.x)));
        v[1] = XT(__hiloint2double(int(u.w), int(u.z)));
    } else if constexpr (sizeof(VT) == 4) {
        v[0] = XT(__uint_as_float(u.x));
        v[1] = XT(__uint_as_float(u.y));
        v[2] = XT(__uint_as_float(u.z));
        v[3] = XT(__uint_as_float(u.w));
    } else {
        const uint32_t q[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[2 * t + 0] = XT(__uint_as_float(q[t] << 16));
            v[2 * t + 1] = XT(__uint_as_float(q[t] & 0xFFFF0000u));
        }
    }
}

template <typename VT>
__host__ __device__ constexpr int pipe_value_words()
{
    return kLaneRun * int(sizeof(VT)) / 16;
}

// Shared-memory slot of one thread: kE row indices, kE values, 16 bytes of
// padding (with it, the 128-bit loads of 8 consecutive threads hit distinct banks).
template <typename VT>
__host__ __device__ constexpr int pipe_slot_bytes()
{
    return 16 * (4 + pipe_value_words<VT>()) + 16;
}

template <typename VT>
__host__ __device__ constexpr size_t pipe_smem_bytes(int threads)
{
    return size_t(2) * size_t(threads) * size_t(pipe_slot_bytes<VT>()) + 16;
}

// Scatter of one column's first chunk (from a shared slot) and of its tail
// (from memory) into g: g_r += a_ri * h.
template <typename VT, typename XT>
__device__ __forceinline__ void slot_scatter(const IterArgs<VT, XT> &a, const unsigned char *slot, const Col<XT> &d,
                                             XT h, XT *g, uint64_t pf, uint64_t pl)
{
    constexpr int VW = pipe_value_words<VT>();
    constexpr int EPW = 16 / int(sizeof(VT));
    int32_t row[kE];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 r4 = reinterpret_cast<const uint4 *>(slot)[q];
        row[4 * q + 0] = int32_t(r4.x);
        row[4 * q + 1] = int32_t(r4.y);
        row[4 * q + 2] = int32_t(r4.z);
        row[4 * q + 3] = int32_t(r4.w);
    }
#pragma unroll
    for (int w = 0; w < VW; ++w) {
        XT vw[EPW];
        decode_word<VT, XT>(reinterpret_cast<const uint4 *>(slot + 64)[w], vw);
#pragma unroll
        for (int q = 0; q < EPW; ++q)
            if (w * EPW + q < d.cnt) red_add(g + row[w * EPW + q], vw[q] * h, pl);
    }
    for (int cs = kE; cs < d.cnt; cs += kE) {
        Chunk<kE, XT> t;
        ld_chunk_hint<kE>(t, a.prow, a.pval, d.pbeg + cs, pf);
        chunk_scatter_hint<kE>(t, g, h, d.cnt - cs, pl);
    }
}

// Scatter of a whole column read from memory (A evict-first, g evict-last).
template <typename VT, typename XT>
__device__ __forceinline__ void mem_scatter(const IterArgs<VT, XT> &a, const Col<XT> &d, XT h, XT *g, uint64_t pf,
                                            uint64_t pl)
{
    for (int cs = 0; cs < d.cnt; cs += kE) {
        Chunk<kE, XT> t;
        ld_chunk_hint<kE>(t, a.prow, a.pval, d.pbeg + cs, pf);
        chunk_scatter_hint<kE>(t, g, h, d.cnt - cs, pl);
    }
}

// Shared-memory slot of one thread of the pipelined kernel: the column's first
// kE row indices and values (the head's layout), then its next wide_tail row indices
// and values, padded to an odd number of 16-byte words (with it, the 128-bit
// loads of 8 consecutive threads hit distinct banks).
template <typename VT>
__host__ __device__ constexpr int pipe_tail_off()
{
    return 64 + kLaneRun * int(sizeof(VT));   // the tail's row indices; its values 2 kLaneRun bytes on
}
template <typename VT>
__host__ __device__ constexpr int pipe_slot_raw()
{
    return pipe_tail_off<VT>() + wide_tail<VT>() * (4 + int(sizeof(VT)));
}
template <typename VT>
__host__ __device__ constexpr int pipe_slot_bytes1()
{
    return (pipe_slot_raw<VT>() / 16) % 2 == 0 ? pipe_slot_raw<VT>() + 16 : pipe_slot_raw<VT>();
}
template <typename VT>
__host__ __device__ constexpr size_t pipe_smem_bytes1(int threads)
{
    return size_t(threads) * size_t(pipe_slot_bytes1<VT>()) + 16;
}

// Row indices of a wide slot: the first kE entries, then the next wide_tail.
template <typename VT, typename XT>
__device__ __forceinline__ void slot_rows(const unsigned char *slot, int32_t (&row)[kE], int32_t (&tr)[wide_tail<VT>()])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 r4 = reinterpret_cast<const uint4 *>(slot)[q];
        row[4 * q + 0] = int32_t(r4.x);
        row[4 * q + 1] = int32_t(r4.y);
        row[4 * q + 2] = int32_t(r4.z);
        row[4 * q + 3] = int32_t(r4.w);
    }
#pragma unroll
    for (int q = 0; q < wide_tail<VT>() / 4; ++q) {
        const uint4 r4 = reinterpret_cast<const uint4 *>(slot + pipe_tail_off<VT>())[q];
        tr[4 * q + 0] = int32_t(r4.x);
        tr[4 * q + 1] = int32_t(r4.y);
        tr[4 * q + 2] = int32_t(r4.z);
        tr[4 * q + 3] = int32_t(r4.w);
    }
}

// Scatter of one column whose first kE + wide_tail entries sit in a slot (the rest
// from memory) into g: g_r += a_ri * h.
template <typename VT, typename XT>
__device__ __forceinline__ void slot_scatter1(const IterArgs<VT, XT> &a, const unsigned char *slot, const Col<XT> &d,
                                              XT h, XT *g, uint64_t pf, uint64_t pl)
{
    constexpr int VW = pipe_value_words<VT>();
    constexpr int kT = wide_tail<VT>();
    constexpr int VWT = kT * int(sizeof(VT)) / 16;
    constexpr int EPW = 16 / int(sizeof(VT));
    int32_t row[kE], tr[kT];
    slot_rows<VT, XT>(slot, row, tr);
#pragma unroll
    for (int w = 0; w < VW; ++w) {
        XT vw[EPW];
        decode_word<VT, XT>(reinterpret_cast<const uint4 *>(slot + 64)[w], vw);
#pragma unroll
        for (int o = 0; o < EPW; ++o)
            if (w * EPW + o < d.cnt) red_add(g + row[w * EPW + o], vw[o] * h, pl);
    }
    if (d.cnt > kE) {
#pragma unroll
        for (int w = 0; w < VWT; ++w) {
            XT vw[EPW];
            decode_word<VT, XT>(reinterpret_cast<const uint4 *>(slot + pipe_tail_off<VT>() + 4 * kT)[w], vw);
#pragma unroll
            for (int o = 0; o < EPW; ++o)
                if (kE + w * EPW + o < d.cnt) red_add(g + tr[w * EPW + o], vw[o] * h, pl);
        }
    }
    for (int cs = kE + kT; cs < d.cnt; cs += kE) {
        Chunk<kE, XT> t;
        ld_chunk_hint<kE>(t, a.prow, a.pval, d.pbeg + cs, pf);
        chunk_scatter_hint<kE>(t, g, h, d.cnt - cs, pl);
    }
}

// The pipelined kernel ("wide" slots): one slot per thread holds the column's
// first kE + wide_tail entries (one bulk copy of the column's head, or two to
// four from the CSC arrays without heads), so the gathers of entries
// kE .. kE + wide_tail - 1 need no dependent load; the slot is refilled after
// the grid barrier's arrive (its scatter done), and the previous iteration's
// step is scattered from memory.  Against the double-buffered form it replaced
// (two slots of kE entries per thread, the next kE / 2 entries loaded beside the
// first gathers), at the bench workload: FP64 18.6 -> 16.4 us per iteration (24
// entries), FP32 12.7 -> 11.8 us and BF16 12.2 -> 11.9 us (32 entries).
template <typename VT, typename XT, int GM = 0, bool ZC = false>
__global__ void __launch_bounds__(kPipeMaxBlock, 1) k_fused_pipe_wide(const IterArgs<VT, XT> a, int64_t k0, int64_t iters)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int VW = pipe_value_words<VT>();
    constexpr int SB = pipe_slot_bytes1<VT>();
    constexpr int TO = pipe_tail_off<VT>();
    constexpr int G = pad_granule<VT>();
    constexpr int kT = wide_tail<VT>();   // entries [kE, kE + kT) sit in the slot as well
    constexpr int VWT = kT * int(sizeof(VT)) / 16;
    static_assert(head_entries<VT>() == kE + kT, "the wide slot is filled from a wide head");
    const int nt = blockDim.x, t = threadIdx.x;
    // Sampled position j belongs to block j mod gridDim.x, thread j / gridDim.x:
    // with one block per SM the positions spread over every SM even when tau
    // does not fill the last block.
    const int64_t j0 = int64_t(t) * gridDim.x + blockIdx.x;
    const bool own = j0 < a.tau;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + size_t(nt) * SB);
    Counters cnt;
    const uint64_t pf = l2_evict_first();   // A, descriptors, x: touched once per iteration
    const uint64_t pl = l2_evict_last();    // the residual buffers: gathered at random rows
    const float lamf = __double2float_rd(a.lambda);   // the largest float <= lambda (ZeroCert)
    constexpr bool CERT = sizeof(XT) == 8 && GM == 0 && ZC;   // the FP64 form tries the FP32 certificate
    unsigned char *my = smem + size_t(t) * SB;
    // the residual buffer that holds g_k at iteration k
    auto gbuf = [&](int64_t kk) { return (kk & 1) ? a.g2 : a.g; };
    // This thread's share of filling the slots: arrive on the mbarrier and, for a
    // non-empty column, bulk-copy its first kE entries (one copy from the column's
    // head when the heads exist, else rows and values) and, for a longer column,
    // its next wide_tail entries (rows and values).
    auto fill = [&](const Col<XT> &d, int32_t ci, bool mine) {
        if (mine && d.cnt > 0) {
            const int64_t pc = (int64_t(d.cnt) + G - 1) / G * G;
            const uint32_t e = uint32_t(pc < kE ? pc : kE);
            const uint32_t br = e * 4u, bv = e * uint32_t(sizeof(VT));
            const uint32_t e2 = pc > kE ? uint32_t(pc - kE < kT ? pc - kE : kT) : 0u;
            const uint32_t br2 = e2 * 4u, bv2 = e2 * uint32_t(sizeof(VT));
            if (a.head) {
                // the head's layout is the slot's: one copy, up to the last tail value needed
                const uint32_t bytes = e2 > 0 ? uint32_t(TO + 4 * kT) + bv2 : 64u + bv;
                mbar_arrive_expect_tx(mbar, bytes);
                bulk_copy_g2s(my, a.head + int64_t(ci) * head_stride<VT>(), bytes, mbar, pf);
            } else {
                mbar_arrive_expect_tx(mbar, br + bv + br2 + bv2);
                bulk_copy_g2s(my, a.prow + d.pbeg, br, mbar, pf);
                bulk_copy_g2s(my + 64, a.pval + d.pbeg, bv, mbar, pf);
                if (e2 > 0) {
                    bulk_copy_g2s(my + TO, a.prow + d.pbeg + kE, br2, mbar, pf);
                    bulk_copy_g2s(my + TO + 4 * kT, a.pval + d.pbeg + kE, bv2, mbar, pf);
                }
            }
        } else {
            mbar_arrive(mbar);
        }
    };
    // The slots of iteration it are the mbarrier's it-th completion.
    auto wait_buf = [&](int64_t it) { return mbar_wait_bounded(mbar, uint32_t(it) & 1u, a.status, a.timeout_ns); };

    if (t == 0) {
        mbar_init(mbar, uint32_t(nt));
        fence_mbarrier_init();
    }
    __syncthreads();

    // Prologue: i_{k0} (drawn by the caller) and its entries; i_{k0+1} and its descriptor.
    int32_t i_cur = 0, i_nxt = 0;
    Col<XT> d_cur, d_nxt, d_prev;
    d_cur.pbeg = d_nxt.pbeg = d_prev.pbeg = 0;
    d_cur.cnt = d_nxt.cnt = d_prev.cnt = 0;
    d_cur.invL = d_nxt.invL = d_prev.invL = XT(0);
    XT h_prev = XT(0);   // the step of the previous iteration's column (still owed to one buffer)
    if (own) {
        i_cur = ldcg(sample_buf(a, k0) + j0);
        d_cur = load_col(a.desc, i_cur, pf);
        i_nxt = sample_index(uint32_t(j0), make_sample_key(a.seed, k0 + 1, a.n));
        d_nxt = load_col(a.desc, i_nxt, pf);
    }
    fill(d_cur, i_cur, own);

    constexpr int EPW = 16 / int(sizeof(VT));
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t k = k0 + it;
        // this iteration's entries (filled during the previous iteration)
        if (!wait_buf(it)) return;
        const XT *gk = gbuf(k);
        XT *gn = gbuf(k + 1);

        // ---------------- gather, step, x update (reads g_k)
        // The loads go first (x_i, the gathers of g at the slot's rows); the
        // sample of k+2 (integer work only) is drawn while they are in flight.
        XT h = XT(0);
        double xi = 0.0;
        int32_t i_nn = 0;
        Col<XT> d_nn = d_nxt;
        const int valid = own ? d_cur.cnt : 0;
        if (own) {
            xi = ldcg_hint(a.x + i_cur, pf);
            int32_t row[kE], tr[kT];
            slot_rows<VT, XT>(my, row, tr);
            // the step from the gradient (FP64), x_i and the counters
            auto take_step = [&](XT grad) {
                const double xn =
                    coord_step(a.problem, xi, double(grad), double(d_cur.invL), a.inv_beta, a.lambda, a.kappa);
                const double h64 = xn - xi;
                h = XT(h64);
                if (h64 != 0.0) {   // most steps are zero: x_i unchanged
                    st_hint(a.x + i_cur, xn, pf);
                    cnt.nonzero += 1;
                    cnt.scattered += (unsigned long long)valid;
                }
            };
            // the products of the slot's entries with gathered values gv (first chunk) and gt (next kT)
            auto slot_dot = [&](const XT (&gv)[kE], const XT (&gt)[kT]) {
                XT acc = XT(0);
#pragma unroll
                for (int w = 0; w < VW; ++w) {
                    XT vw[EPW];
                    decode_word<VT, XT>(reinterpret_cast<const uint4 *>(my + 64)[w], vw);
#pragma unroll
                    for (int q = 0; q < EPW; ++q)
                        if (w * EPW + q < valid) acc = fma(vw[q], grad_map<GM>(gv[w * EPW + q]), acc);
                }
                if (valid > kE) {
#pragma unroll
                    for (int w = 0; w < VWT; ++w) {
                        XT vw[EPW];
                        decode_word<VT, XT>(reinterpret_cast<const uint4 *>(my + TO + 4 * kT)[w], vw);
#pragma unroll
                        for (int q = 0; q < EPW; ++q)
                            if (kE + w * EPW + q < valid) acc = fma(vw[q], grad_map<GM>(gt[w * EPW + q]), acc);
                    }
                }
                return acc;
            };
            if constexpr (CERT) {
                // FP64 form with the FP32 certificate of a zero LASSO step (ZeroCert):
                // the slot's gathers stay in registers as FP64; entries past the slot
                // bring only the high words of g.  A lane the certificate does not
                // cover reads those entries again, from L2.
                XT gv[kE], gt[kT];
#pragma unroll
                for (int e = 0; e < kE; ++e) gv[e] = (e < valid) ? ldcg_hint(gk + row[e], pl) : XT(0);
#pragma unroll
                for (int e = 0; e < kT; ++e) gt[e] = (kE + e < valid) ? ldcg_hint(gk + tr[e], pl) : XT(0);
                i_nn = sample_index(uint32_t(j0), make_sample_key(a.seed, k + 2, a.n));
                d_nn = load_col(a.desc, i_nn, pf);
                bool zero_step = false;
                if (a.problem == 0 && is_zero_bits(xi)) {
                    ZeroCert zc;
#pragma unroll
                    for (int w = 0; w < VW; ++w) {
                        const uint4 u = reinterpret_cast<const uint4 *>(my + 64)[w];
                        if (2 * w < valid) zc.add(u.y, hi_word(gv[2 * w]));
                        if (2 * w + 1 < valid) zc.add(u.w, hi_word(gv[2 * w + 1]));
                    }
                    if (valid > kE) {
#pragma unroll
                        for (int w = 0; w < VWT; ++w) {
                            const uint4 u = reinterpret_cast<const uint4 *>(my + TO + 4 * kT)[w];
                            if (kE + 2 * w < valid) zc.add(u.y, hi_word(gt[2 * w]));
                            if (kE + 2 * w + 1 < valid) zc.add(u.w, hi_word(gt[2 * w + 1]));
                        }
                    }
                    for (int cs = kE + kT; cs < valid; cs += kT) {
                        Chunk<kT, XT> tc;
                        ld_chunk_hint<kT>(tc, a.prow, a.pval, d_cur.pbeg + cs, pf);
                        uint32_t gc[kT];
#pragma unroll
                        for (int e = 0; e < kT; ++e) gc[e] = (cs + e < valid) ? ldcg_hi_hint(gk + tc.row[e], pl) : 0u;
#pragma unroll
                        for (int e = 0; e < kT; ++e)
                            if (cs + e < valid) zc.add(hi_word(tc.val[e]), gc[e]);
                    }
                    zero_step = zc.below(valid, lamf);
                }
                if (!zero_step) {
                    // FP64 sum over the whole column: the slot's entries from registers,
                    // the rest from memory
                    XT acc = slot_dot(gv, gt);
                    for (int cs = kE + kT; cs < valid; cs += kE) {
                        Chunk<kE, XT> tc;
                        ld_chunk_hint<kE>(tc, a.prow, a.pval, d_cur.pbeg + cs, pf);
                        acc += chunk_dot_hint<kE, XT, XT, GM>(tc, gk, valid - cs, pl);
                    }
                    // the exact test on the FP64 sum (the bound may not have decided it)
                    if (!(a.problem == 0 && is_zero_bits(xi) && abs_le_bits(acc, a.lambda))) take_step(acc);
                }
            } else {
                XT gv[kE], gt[kT];
#pragma unroll
                for (int e = 0; e < kE; ++e) gv[e] = (e < valid) ? ldcg_hint(gk + row[e], pl) : XT(0);
#pragma unroll
                for (int e = 0; e < kT; ++e) gt[e] = (kE + e < valid) ? ldcg_hint(gk + tr[e], pl) : XT(0);
                i_nn = sample_index(uint32_t(j0), make_sample_key(a.seed, k + 2, a.n));
                d_nn = load_col(a.desc, i_nn, pf);
                XT acc = slot_dot(gv, gt);
                for (int cs = kE + kT; cs < valid; cs += kE) {
                    Chunk<kE, XT> tc;
                    ld_chunk_hint<kE>(tc, a.prow, a.pval, d_cur.pbeg + cs, pf);
                    acc += chunk_dot_hint<kE, XT, XT, GM>(tc, gk, valid - cs, pl);
                }
                // At x_i = 0 the LASSO step is 0 when |grad| <= lambda: tested in FP32
                // against lambda rounded down (FP32 and BF16 forms) or on the FP64
                // bit patterns as integers (FP64 form), with no FP64 instruction
                bool zero_step = false;
                if constexpr (GM == 0) {
                    if constexpr (sizeof(XT) == 4)
                        zero_step = a.problem == 0 && is_zero_bits(xi) && fabsf(float(acc)) <= lamf;
                    else
                        zero_step = a.problem == 0 && is_zero_bits(xi) && abs_le_bits(double(acc), a.lambda);
                }
                if (!zero_step) take_step(acc);
            }
            cnt.gathered += (unsigned long long)valid;
        }

        // ---------------- scatter into the other buffer (g_{k-1} -> g_{k+1})
        // No barrier is needed before it: every gather of iteration k reads g_k,
        // which nobody writes during iteration k.  The other buffer holds g_{k-1}
        // and receives the steps of iterations k-1 and k.  The previous column's
        // entries were replaced in the slot: it is scattered from memory.
        if (own && !is_zero_bits(h_prev)) mem_scatter<VT, XT>(a, d_prev, h_prev, gn, pf, pl);
        if (own && !is_zero_bits(h)) slot_scatter1<VT, XT>(a, my, d_cur, h, gn, pf, pl);
        h_prev = h;
        d_prev = d_cur;

        // ---------------- the only grid barrier of the iteration: g_{k+1} complete
        // Split: the release-arrive publishes x and the scatter; the bulk copies of
        // the next columns (reads of A only, nothing to publish) are issued after
        // it, into the slot this thread has finished reading, and overlap the wait.
        const unsigned long long target = (unsigned long long)(it + 1) * gridDim.x;
        grid_arrive(a.bar);
        fence_proxy_async_shared();
        fill(d_nxt, i_nxt, own);
        if (!grid_wait(a.bar, target, a.status, a.timeout_ns)) {
            wait_buf(it + 1);   // the copies just issued land before the block leaves
            return;
        }
        i_cur = i_nxt;
        d_cur = d_nxt;
        i_nxt = i_nn;
        d_nxt = d_nn;
    }
    // Both buffers equal again: the last iteration's steps go into the buffer
    // that holds g_{k0+iters-1}.
    if (iters > 0 && own && !is_zero_bits(h_prev))
        mem_scatter<VT, XT>(a, d_prev, h_prev, gbuf(k0 + iters - 1), pf, pl);
    // the last fill (the entries of i_{k0+iters}) lands before the block leaves
    wait_buf(iters);
    // S_{k0+iters} for the caller (the sample of the next launch).
    if (own) sample_buf(a, k0 + iters)[j0] = i_cur;
    flush_counters(cnt, a.counters);
}

// ---------------------------------------------------------------------------
// Pipelined kernel for tau larger than the grid: thread t of T owns positions
// t, t + T, ..., t + (R-1) T of every iteration ("rounds").  Its work items
// (k, r) form one stream: while item q is computed, the first chunk of item
// q+1 arrives in the other shared-memory slot (TMA bulk copies into
// two slots of kE entries per thread) and the sample of item q+2 is drawn.  The residual is double
// buffered (iteration k gathers from buffer k & 1, scatters into the other),
// so the only grid barrier is at the end of an iteration.  The step of
// position j in iteration k-1, still owed to the other buffer, is kept in
// H[j] with its column in S[(k-1) & 1][j] and re-scattered from memory when
// item (k, r) passes position j (most steps are zero).
template <typename VT, typename XT>
__global__ void __launch_bounds__(kPipeRoundsMaxBlock, 1) k_fused_pipe_rounds(const IterArgs<VT, XT> a, int64_t k0,
                                                                        int64_t iters, int64_t R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int VW = pipe_value_words<VT>();
    constexpr int SB = pipe_slot_bytes<VT>();
    constexpr int G = pad_granule<VT>();
    const int nt = blockDim.x, t = threadIdx.x;
    const int64_t T = int64_t(gridDim.x) * nt;
    const int64_t tg = int64_t(blockIdx.x) * nt + t;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + size_t(2) * nt * SB);
    unsigned long long target = 0;
    uint32_t phase = 0;
    Counters cnt;
    const uint64_t pf = l2_evict_first();
    const uint64_t pl = l2_evict_last();
    auto slot = [&](int b) { return smem + (size_t(b) * nt + t) * SB; };
    auto gbuf = [&](int64_t kk) { return (kk & 1) ? a.g2 : a.g; };
    auto fill = [&](int b, const Col<XT> &d, int32_t ci, bool mine) {
        if (mine && d.cnt > 0) {
            const int64_t pc = (int64_t(d.cnt) + G - 1) / G * G;
            const uint32_t e = uint32_t(pc < kE ? pc : kE);
            const uint32_t br = e * 4u, bv = e * uint32_t(sizeof(VT));
            if (a.head) {
                mbar_arrive_expect_tx(&mbar[b], 64u + bv);
                bulk_copy_g2s(slot(b), a.head + int64_t(ci) * head_stride<VT>(), 64u + bv, &mbar[b], pf);
            } else {
                mbar_arrive_expect_tx(&mbar[b], br + bv);
                bulk_copy_g2s(slot(b), a.prow + d.pbeg, br, &mbar[b], pf);
                bulk_copy_g2s(slot(b) + 64, a.pval + d.pbeg, bv, &mbar[b], pf);
            }
        } else {
            mbar_arrive(&mbar[b]);
        }
    };
    auto wait_buf = [&](int b) {
        const bool ok = mbar_wait_bounded(&mbar[b], (phase >> b) & 1u, a.status, a.timeout_ns);
        phase ^= 1u << b;
        return ok;
    };
    if (t == 0) {
        mbar_init(&mbar[0], uint32_t(nt));
        mbar_init(&mbar[1], uint32_t(nt));
        fence_mbarrier_init();
    }
    __syncthreads();

    const int64_t items = iters * R;
    // position and iteration of item q
    auto pos_of = [&](int64_t q) { return tg + (q % R) * T; };
    auto k_of = [&](int64_t q) { return k0 + q / R; };
    // sample of item q (key cached per iteration)
    SampleKey key = make_sample_key(a.seed, k0, a.n);
    int64_t key_k = k0;
    auto draw = [&](int64_t q, int32_t &i, Col<XT> &d) {
        const int64_t j = pos_of(q);
        const int64_t kq = k_of(q);
        if (q >= items || j >= a.tau) {
            i = 0;
            d.pbeg = 0;
            d.cnt = 0;
            d.invL = XT(0);
            return false;
        }
        if (kq != key_k) {
            key = make_sample_key(a.seed, kq, a.n);
            key_k = kq;
        }
        i = sample_index(uint32_t(j), key);
        d = load_col(a.desc, i, pf);
        return true;
    };

    int32_t i_cur = 0, i_nxt = 0;
    Col<XT> d_cur, d_nxt;
    bool own_cur = draw(0, i_cur, d_cur);
    bool own_nxt = draw(1, i_nxt, d_nxt);
    fill(0, d_cur, i_cur, own_cur);

    constexpr int kT = kE / 2;
    for (int64_t q = 0; q < items; ++q) {
        const int64_t k = k_of(q);
        const int64_t r = q % R;
        const int64_t j = pos_of(q);
        const int b = int(q & 1);
        if (!wait_buf(b)) return;
        const unsigned char *my = slot(b);
        const XT *gk = gbuf(k);
        XT *gn = gbuf(k + 1);
        int32_t i_nn = 0;
        Col<XT> d_nn;
        bool own_nn = false;
        if (own_cur) {
            const double xi = ldcg_hint(a.x + i_cur, pf);
            const int valid = d_cur.cnt;
            int32_t row[kE];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint4 r4 = reinterpret_cast<const uint4 *>(my)[w];
                row[4 * w + 0] = int32_t(r4.x);
                row[4 * w + 1] = int32_t(r4.y);
                row[4 * w + 2] = int32_t(r4.z);
                row[4 * w + 3] = int32_t(r4.w);
            }
            XT gv[kE];
#pragma unroll
            for (int e = 0; e < kE; ++e) gv[e] = (e < valid) ? ldcg_hint(gk + row[e], pl) : XT(0);
            Chunk<kT, XT> tl;
            if (valid > kE) ld_chunk_hint<kT>(tl, a.prow, a.pval, d_cur.pbeg + kE, pf);
            own_nn = draw(q + 2, i_nn, d_nn);
            XT gt[kT];
#pragma unroll
            for (int e = 0; e < kT; ++e) gt[e] = (kE + e < valid) ? ldcg_hint(gk + tl.row[e], pl) : XT(0);
            constexpr int EPW = 16 / int(sizeof(VT));
            XT acc = XT(0);
#pragma unroll
            for (int w = 0; w < VW; ++w) {
                XT vw[EPW];
                decode_word<VT, XT>(reinterpret_cast<const uint4 *>(my + 64)[w], vw);
#pragma unroll
                for (int e = 0; e < EPW; ++e)
                    if (w * EPW + e < valid) acc = fma(vw[e], gv[w * EPW + e], acc);
            }
#pragma unroll
            for (int e = 0; e < kT; ++e)
                if (kE + e < valid) acc = fma(tl.val[e], gt[e], acc);
            for (int cs = kE + kT; cs < valid; cs += kE) {
                Chunk<kE, XT> tc;
                ld_chunk_hint<kE>(tc, a.prow, a.pval, d_cur.pbeg + cs, pf);
                acc += chunk_dot_hint<kE, XT>(tc, gk, valid - cs, pl);
            }
            const double xn = prox_step(xi, double(acc), double(d_cur.invL), a.inv_beta, a.lambda);
            const double h64 = xn - xi;
            const XT h = XT(h64);
            if (h64 != 0.0) st_hint(a.x + i_cur, xn, pf);
            cnt.gathered += (unsigned long long)valid;
            if (h64 != 0.0) {
                cnt.nonzero += 1;
                cnt.scattered += (unsigned long long)valid;
            }
            // the step of iteration k-1 at this position, owed to the other buffer
            if (k > k0) {
                const XT hp = a.h[j];
                if (hp != XT(0)) mem_scatter<VT, XT>(a, load_col(a.desc, sample_buf(a, k - 1)[j], pf), hp, gn, pf, pl);
            }
            if (h != XT(0)) slot_scatter<VT, XT>(a, my, d_cur, h, gn, pf, pl);
            a.h[j] = h;
            sample_buf(a, k)[j] = i_cur;
        } else {
            own_nn = draw(q + 2, i_nn, d_nn);
        }
        if (r == R - 1) {
            // ---------------- end of iteration k: the only grid barrier
            target += gridDim.x;
            grid_arrive(a.bar);
            fence_proxy_async_shared();
            fill(b ^ 1, d_nxt, i_nxt, own_nxt);
            if (!grid_wait(a.bar, target, a.status, a.timeout_ns)) {
                wait_buf(b ^ 1);
                return;
            }
        } else {
            fence_proxy_async_shared();
            fill(b ^ 1, d_nxt, i_nxt, own_nxt);
        }
        i_cur = i_nxt;
        d_cur = d_nxt;
        own_cur = own_nxt;
        i_nxt = i_nn;
        d_nxt = d_nn;
        own_nxt = own_nn;
    }
    // Both buffers equal again: the last iteration's steps go into the buffer
    // that holds g_{k0+iters-1}.
    if (iters > 0) {
        const int64_t kl = k0 + iters - 1;
        for (int64_t r = 0; r < R; ++r) {
            const int64_t j = tg + r * T;
            if (j >= a.tau) break;
            const XT hp = a.h[j];
            if (hp != XT(0)) mem_scatter<VT, XT>(a, load_col(a.desc, sample_buf(a, kl)[j], pf), hp, gbuf(kl), pf, pl);
        }
    }
    wait_buf(int(items & 1));
    flush_counters(cnt, a.counters);
}

// ---------------------------------------------------------------------------
// Asynchronous PCDM (the shared-memory implementation mode of Sec. 8.1): every
// thread repeatedly takes the next update u of a global sequence, picks block
// i_u (the tau-independent pick with k = u, position 0, so that one thread
// reproduces the serial method with iid blocks), reads x_i and the residual as
// they are, computes the step of eq. (h(x)) with the given beta and applies it
// with atomic additions to x_i and to g.  No barrier: reads may see other
// threads' updates partially.  Updates u0 .. u0 + count - 1.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_async(const IterArgs<VT, XT> a, uint64_t u0, uint64_t count,
                                                  uint64_t nthreads)
{
    const uint64_t T = nthreads;   // threads taking part (the rest of the grid idles)
    Counters cnt;
    const uint64_t tid = uint64_t(blockIdx.x) * kBlock + threadIdx.x;
    for (uint64_t t = tid; tid < T && t < count; t += T) {
        const uint64_t u = u0 + t;
        const int32_t i = independent_pick(a.seed, int64_t(u), 0u, a.n);
        const Col<XT> c = load_col(a.desc, i);
        const double xi = ld_volatile_f64(a.x + i);
        XT acc = XT(0);
        for (int cs = 0; cs < c.cnt; cs += kE) {
            Chunk<kE, XT> ch;
            ld_chunk<kE>(ch, a.prow, a.pval, c.pbeg + cs);
            acc += chunk_dot<kE, XT, XT, XT>(ch, a.g, c.cnt - cs);
        }
        const double xn = prox_step(xi, double(acc), double(c.invL), a.inv_beta, a.lambda);
        const double h64 = xn - xi;
        cnt.gathered += (unsigned long long)c.cnt;
        if (h64 != 0.0) {
            atomicAdd(a.x + i, h64);
            const XT h = XT(h64);
            for (int cs = 0; cs < c.cnt; cs += kE) {
                Chunk<kE, XT> ch;
                ld_chunk<kE>(ch, a.prow, a.pval, c.pbeg + cs);
                chunk_scatter<kE>(ch, a.g, h, c.cnt - cs);
            }
            cnt.nonzero += 1;
            cnt.scattered += (unsigned long long)c.cnt;
        }
    }
    flush_counters(cnt, a.counters);
}

// ---------------------------------------------------------------------------
// Set-up on the caller's layout: one thread per column (runs once per matrix).
template <typename VT>
__device__ __forceinline__ double ld_orig(const VT *p);
template <>
__device__ __forceinline__ double ld_orig<double>(const double *p) { return *p; }
template <>
__device__ __forceinline__ double ld_orig<float>(const float *p) { return double(*p); }
template <>
__device__ __forceinline__ double ld_orig<bf16_t>(const bf16_t *p)
{
    return double(__uint_as_float(uint32_t(p->bits) << 16));
}

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
            const double v = ld_orig<VT>(val + p);
            if (!isfinite(v)) f |= FLAG_NONFINITE;
            s = __dadd_rn(s, __dmul_rn(v, v));   // no contraction: the same bits as a plain sum of squares
            atomicAdd(rowcnt + r, 1);
        }
        L[i] = s;
    }
    if (f) atomicOr(flags, f);
}

// Padded layout and descriptors (prow / pval zero-filled beforehand).
template <typename VT, typename XT>
__global__ void k_build_layout(const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
                               const VT *__restrict__ val, const int64_t *__restrict__ pbeg,
                               const double *__restrict__ L, int64_t n, ColDesc<XT> *__restrict__ desc,
                               int32_t *__restrict__ prow, VT *__restrict__ pval)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t s = col_ptr[i], c = col_ptr[i + 1] - s, pb = pbeg[i];
        for (int64_t p = 0; p < c; ++p) {
            prow[pb + p] = row_idx[s + p];
            pval[pb + p] = val[s + p];
        }
        ColDesc<XT> d;
        d.pb4 = uint32_t(pb / 4);
        d.cnt = int32_t(c);
        d.invL = L[i] > 0.0 ? XT(1.0 / L[i]) : XT(0);
        if constexpr (sizeof(XT) == 4) d.unused = 0.f;
        desc[i] = d;
    }
}

// Column heads: the first kE row indices (zero-padded) and values of every
// column.  Thread t fills entry t mod kE of column t / kE, so that a column's
// reads and writes are contiguous across kE neighbouring lanes.
template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_build_heads(const ColDesc<XT> *__restrict__ desc,
                                                        const int32_t *__restrict__ prow, const VT *__restrict__ pval,
                                                        int64_t n, unsigned char *__restrict__ head)
{
    constexpr int EH = head_entries<VT>();
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t t = int64_t(blockIdx.x) * kBlock + threadIdx.x; t < n * EH; t += stride) {
        const int64_t i = t / EH;
        const int e = int(t % EH);
        const Col<XT> c = load_col(desc, int32_t(i));
        // entries 0 .. kE-1: rows at 0, values at 4 kE; entries kE .. EH-1: rows, then values, after them
        unsigned char *h = head + i * head_stride<VT>() + (e < kE ? 0 : 4 * kE + kE * int(sizeof(VT)));
        const int q = e < kE ? e : e - kE;
        const int voff = e < kE ? 4 * kE : 4 * wide_tail<VT>();
        const bool in = e < c.cnt;
        reinterpret_cast<int32_t *>(h)[q] = in ? prow[c.pbeg + e] : 0;
        reinterpret_cast<VT *>(h + voff)[q] = in ? pval[c.pbeg + e] : VT{};
    }
}

// Refresh: g64 += a_i x_i over the columns with x_i != 0, in FP64.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_refresh_cols(const ColDesc<XT> *__restrict__ desc,
                                                         const int32_t *__restrict__ prow,
                                                         const VT *__restrict__ pval, const double *__restrict__ x,
                                                         int64_t n, double *__restrict__ g64)
{
    constexpr int CH = W * kE;
    const int lane = threadIdx.x & (W - 1);
    const int64_t ngrp = int64_t(gridDim.x) * kBlock / W;
    for (int64_t i = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W; i < n; i += ngrp) {
        const double xi = __ldg(x + i);
        if (xi == 0.0) continue;
        const Col<XT> c = load_col(desc, int32_t(i));
        for (int cs = 0; cs < c.cnt; cs += CH) {
            Chunk<kE, XT> t;
            const int st = cs + lane * kE;
            if (st >= c.cnt) continue;
            ld_chunk<kE>(t, prow, pval, c.pbeg + st);
            const int valid = c.cnt - st;
#pragma unroll
            for (int e = 0; e < kE; ++e)
                if (e < valid) red_add(g64 + t.row[e], double(t.val[e]) * xi);
        }
    }
}

// Gap, column part: c_i = a_i^T r in FP64; block partials of max|c_i|, sum|x_i|, sum x_i c_i.
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_gap_cols(const ColDesc<XT> *__restrict__ desc,
                                                     const int32_t *__restrict__ prow,
                                                     const VT *__restrict__ pval, const double *__restrict__ r,
                                                     const double *__restrict__ x, int64_t n, double *__restrict__ part)
{
    constexpr int CH = W * kE;
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t ngrp = int64_t(gridDim.x) * kBlock / W;
    double cmax = 0.0, l1 = 0.0, xc = 0.0;
    // A streams through once (evict-first); r is gathered at random rows (evict-last)
    const uint64_t pf = l2_evict_first(), pl = l2_evict_last();
    for (int64_t i = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W; i < n; i += ngrp) {
        const Col<XT> c = load_col(desc, int32_t(i), pf);
        double acc = 0.0;
        for (int cs = 0; cs < c.cnt; cs += CH) {
            Chunk<kE, XT> t;
            const int st = cs + lane * kE;
            if (st < c.cnt) ld_chunk_hint<kE>(t, prow, pval, c.pbeg + st, pf);
            acc += chunk_dot_hint<kE, XT, double>(t, r, c.cnt - st, pl);
        }
        acc = group_sum<W>(acc, gmask);
        if (lane == 0) {
            const double xi = __ldg(x + i);
            cmax = fmax(cmax, fabs(acc));
            l1 += fabs(xi);
            xc += xi * acc;
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

// Gap of the SVM dual and of logistic regression, column part (FP64, r = the
// refreshed g).  c_i = a_i^T phi(r) for the label-signed a_i; block partials:
//   problem 1 (SVM dual, s_i = c_i / kappa = y_i <w, A_i> with w = r/(lambda n)):
//     sum_i [(1 - s_i)_+ (1 - x_i) + (s_i - 1)_+ x_i],  sum_i (1 - s_i)_+,  sum_i x_i
//     (with ||r||^2 = x^T c the duality gap is the first sum over n, each term >= 0 on the box)
//   problem 2 (logistic, c = grad f):
//     sum_i (c_i + 2 lambda x_i)^2,  sum_i x_i^2,  sum_i c_i x_i
template <int W, typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_glm_gap_cols(int problem, const ColDesc<XT> *__restrict__ desc,
                                                         const int32_t *__restrict__ prow,
                                                         const VT *__restrict__ pval, const double *__restrict__ r,
                                                         const double *__restrict__ x, int64_t n, double lambda,
                                                         double kappa, double *__restrict__ part)
{
    constexpr int CH = W * kE;
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = group_mask<W>(threadIdx.x & 31);
    const int64_t ngrp = int64_t(gridDim.x) * kBlock / W;
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    const uint64_t pf = l2_evict_first(), pl = l2_evict_last();
    for (int64_t i = (int64_t(blockIdx.x) * kBlock + threadIdx.x) / W; i < n; i += ngrp) {
        const Col<XT> c = load_col(desc, int32_t(i), pf);
        double acc = 0.0;
        for (int cs = 0; cs < c.cnt; cs += CH) {
            Chunk<kE, XT> t;
            const int st = cs + lane * kE;
            if (st < c.cnt) ld_chunk_hint<kE>(t, prow, pval, c.pbeg + st, pf);
            acc += problem == 2 ? chunk_dot_hint<kE, XT, double, 1>(t, r, c.cnt - st, pl)
                                : chunk_dot_hint<kE, XT, double, 0>(t, r, c.cnt - st, pl);
        }
        acc = group_sum<W>(acc, gmask);
        if (lane == 0) {
            const double xi = __ldg(x + i);
            if (problem == 1) {
                const double s = acc / kappa;
                const double below = 1.0 - s > 0.0 ? 1.0 - s : 0.0, above = s - 1.0 > 0.0 ? s - 1.0 : 0.0;
                t1 += below * (1.0 - xi) + above * xi;
                t2 += below;
                t3 += xi;
            } else {
                const double q = fma(2.0 * lambda, xi, acc);
                t1 += q * q;
                t2 += xi * xi;
                t3 += acc * xi;
            }
        }
    }
    __shared__ double sm[3][kBlock / 32];
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    t3 = warp_sum(t3);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sm[0][w] = t1;
        sm[1][w] = t2;
        sm[2][w] = t3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) {
            a0 += sm[0][q];
            a1 += sm[1][q];
            a2 += sm[2][q];
        }
        part[3 * blockIdx.x + 0] = a0;
        part[3 * blockIdx.x + 1] = a1;
        part[3 * blockIdx.x + 2] = a2;
    }
}

// Labels folded into the stored values: the SVM dual signs column i by y_i
// (examples are columns), logistic regression signs entry (r, i) by y_r
// (examples are rows).  A sign flip is exact in every value type.
template <typename VT>
__device__ __forceinline__ VT negate_value(VT v)
{
    if constexpr (sizeof(VT) == 2) {
        VT o;
        o.bits = uint16_t(v.bits ^ 0x8000u);
        return o;
    } else {
        return -v;
    }
}

template <typename VT, typename XT>
__global__ void __launch_bounds__(kBlock) k_apply_labels(int problem, const ColDesc<XT> *__restrict__ desc,
                                                         const int32_t *__restrict__ prow, VT *__restrict__ pval,
                                                         int64_t n, const double *__restrict__ y)
{
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < n; i += stride) {
        const Col<XT> c = load_col(desc, int32_t(i));
        const bool col_neg = problem == 1 && y[i] < 0.0;
        for (int e = 0; e < c.cnt; ++e) {
            const int64_t p = c.pbeg + e;
            if (problem == 1 ? col_neg : (y[prow[p]] < 0.0)) pval[p] = negate_value(pval[p]);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers.
#define PCDM_DISPATCH_W(W, ...)                                    \
    switch (W) {                                                   \
    case 1: { constexpr int W_ = 1; __VA_ARGS__; } break;          \
    case 2: { constexpr int W_ = 2; __VA_ARGS__; } break;          \
    case 4: { constexpr int W_ = 4; __VA_ARGS__; } break;          \
    case 8: { constexpr int W_ = 8; __VA_ARGS__; } break;          \
    case 16: { constexpr int W_ = 16; __VA_ARGS__; } break;        \
    case 32: { constexpr int W_ = 32; __VA_ARGS__; } break;        \
    default: return cudaErrorInvalidValue;                         \
    }

static inline unsigned blocks_for_threads(int64_t threads, int64_t cap)
{
    int64_t b = (threads + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (cap > 0 && b > cap) b = cap;
    return unsigned(b);
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::gather(const IterArgs<VT, XT> &a, int W, int64_t k, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    if (a.problem == 2) {
        PCDM_DISPATCH_W(W, { k_gather<W_, VT, XT, 1><<<blocks_for_threads(a.tau * W_, 0), kBlock, 0, st>>>(a, k); });
    } else {
        PCDM_DISPATCH_W(W, { k_gather<W_, VT, XT, 0><<<blocks_for_threads(a.tau * W_, 0), kBlock, 0, st>>>(a, k); });
    }
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::scatter(const IterArgs<VT, XT> &a, int W, int64_t k, bool sample_next, cudaStream_t st)
{
    if (a.tau <= 0) return cudaSuccess;
    PCDM_DISPATCH_W(W, {
        k_scatter<W_, VT, XT><<<blocks_for_threads(a.tau * W_, 0), kBlock, 0, st>>>(a, k, sample_next ? 1 : 0);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
int Kernels<VT, XT>::fused_max_blocks(int W, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    // the same grid serves both gradient maps: the smaller co-resident grid of the two
    int per_sm_map = 0;
    cudaError_t e = cudaErrorInvalidValue, e2 = cudaErrorInvalidValue;
#define PCDM_FUSED_OCC(WW)                                                                            \
    case WW:                                                                                          \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<WW, VT, XT, 0>, threads, 0);   \
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_map, k_fused<WW, VT, XT, 1>, threads, 0); \
        break;
    switch (W) {
        PCDM_FUSED_OCC(1)
        PCDM_FUSED_OCC(2)
        PCDM_FUSED_OCC(4)
        PCDM_FUSED_OCC(8)
        PCDM_FUSED_OCC(16)
        PCDM_FUSED_OCC(32)
    default: return 0;
    }
#undef PCDM_FUSED_OCC
    if (e != cudaSuccess || e2 != cudaSuccess) return 0;
    return (per_sm < per_sm_map ? per_sm : per_sm_map) * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                   cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    const bool map = a.problem == 2;
    PCDM_DISPATCH_W(sh.W, {
        const void *fn = map ? (const void *)k_fused<W_, VT, XT, 1> : (const void *)k_fused<W_, VT, XT, 0>;
        return cudaLaunchCooperativeKernel(fn, dim3(unsigned(sh.blocks)), dim3(unsigned(sh.threads)), params, 0, st);
    });
    return cudaErrorInvalidValue;
}

template <typename VT, typename XT>
int Kernels<VT, XT>::pipe_max_blocks(int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    // the same grid serves every variant (gradient maps, zero-step certificate):
    // the smallest co-resident grid of them
    const size_t bytes = pipe_smem_bytes1<VT>(threads);
    const void *fns[3] = {(const void *)k_fused_pipe_wide<VT, XT, 0, false>,
                          (const void *)k_fused_pipe_wide<VT, XT, 1, false>,
                          (const void *)k_fused_pipe_wide<VT, XT, 0, true>};
    const int nf = sizeof(XT) == 8 ? 3 : 2;
    int best = -1;
    for (int f = 0; f < nf; ++f) {
        if (cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[f], threads, bytes) != cudaSuccess) return 0;
        if (best < 0 || per_sm < best) best = per_sm;
    }
    return best * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused_pipe(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0, int64_t iters,
                                        bool zero_cert, cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters};
    // the certificate applies to the FP64 form of LASSO (the FP32 forms test |grad| <= lambda exactly anyway)
    const void *fn = a.problem == 2 ? (const void *)k_fused_pipe_wide<VT, XT, 1, false>
                     : (sizeof(XT) == 8 && zero_cert && a.problem == 0) ? (const void *)k_fused_pipe_wide<VT, XT, 0, true>
                                                                       : (const void *)k_fused_pipe_wide<VT, XT, 0, false>;
    const size_t bytes = pipe_smem_bytes1<VT>(sh.threads);
    return cudaLaunchCooperativeKernel(fn, dim3(unsigned(sh.blocks)), dim3(unsigned(sh.threads)), params, bytes, st);
}

template <typename VT, typename XT>
int Kernels<VT, XT>::pipe_rounds_max_blocks(int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t bytes = pipe_smem_bytes<VT>(threads);
    if (cudaFuncSetAttribute(k_fused_pipe_rounds<VT, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_pipe_rounds<VT, XT>, threads, bytes) !=
        cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::fused_pipe_rounds(const IterArgs<VT, XT> &a, const FusedShape &sh, int64_t k0,
                                               int64_t iters, cudaStream_t st)
{
    if (iters <= 0 || a.tau <= 0) return cudaSuccess;
    IterArgs<VT, XT> args = a;
    const int64_t T = int64_t(sh.blocks) * sh.threads;
    int64_t R = (a.tau + T - 1) / T;
    void *params[] = {(void *)&args, (void *)&k0, (void *)&iters, (void *)&R};
    return cudaLaunchCooperativeKernel((const void *)k_fused_pipe_rounds<VT, XT>, dim3(unsigned(sh.blocks)),
                                       dim3(unsigned(sh.threads)), params, pipe_smem_bytes<VT>(sh.threads), st);
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::build_heads(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, int64_t n,
                                         unsigned char *head, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_build_heads<VT, XT><<<blocks_for_threads(n * head_entries<VT>(), 152 * 64), kBlock, 0, st>>>(desc, prow, pval,
                                                                                                   n, head);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::setup_cols(const int64_t *col_ptr, const int32_t *row_idx, const VT *val, int64_t m,
                                        int64_t n, double *L, int *rowcnt, int *flags, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_setup_cols<VT><<<blocks_for_threads(n, 152 * 64), kBlock, 0, st>>>(col_ptr, row_idx, val, m, n, L, rowcnt,
                                                                          flags);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::build_layout(const int64_t *col_ptr, const int32_t *row_idx, const VT *val,
                                          const int64_t *pbeg, const double *L, int64_t n, ColDesc<XT> *desc,
                                          int32_t *prow, VT *pval, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_build_layout<VT, XT><<<blocks_for_threads(n, 152 * 64), kBlock, 0, st>>>(col_ptr, row_idx, val, pbeg, L, n,
                                                                                desc, prow, pval);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::async(const IterArgs<VT, XT> &a, int blocks, uint64_t nthreads, uint64_t u0,
                                   uint64_t count, cudaStream_t st)
{
    k_async<VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(a, u0, count, nthreads);
    return cudaGetLastError();
}

template <typename VT, typename XT>
int Kernels<VT, XT>::async_max_blocks()
{
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_async<VT, XT>, kBlock, 0) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::refresh_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *x,
                                          int64_t n, double *g64, int W, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    PCDM_DISPATCH_W(W, {
        k_refresh_cols<W_, VT, XT><<<blocks_for_threads(n * W_, 152 * 16), kBlock, 0, st>>>(desc, prow, pval, x,
                                                                                              n, g64);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::glm_gap_cols(int problem, const ColDesc<XT> *desc, const int32_t *prow, const VT *pval,
                                          const double *r, const double *x, int64_t n, double lambda, double kappa,
                                          double *part, int blocks, int W, cudaStream_t st)
{
    PCDM_DISPATCH_W(W, {
        k_glm_gap_cols<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(problem, desc, prow, pval, r, x, n,
                                                                               lambda, kappa, part);
    });
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::apply_labels(int problem, const ColDesc<XT> *desc, const int32_t *prow, VT *pval,
                                          int64_t n, const double *y, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_apply_labels<VT, XT><<<blocks_for_threads(n, 152 * 64), kBlock, 0, st>>>(problem, desc, prow, pval, n, y);
    return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Kernels<VT, XT>::gap_cols(const ColDesc<XT> *desc, const int32_t *prow, const VT *pval, const double *r,
                                      const double *x, int64_t n, double *part, int blocks, int W, cudaStream_t st)
{
    PCDM_DISPATCH_W(W, {
        k_gap_cols<W_, VT, XT><<<dim3(unsigned(blocks)), kBlock, 0, st>>>(desc, prow, pval, r, x, n, part);
    });
    return cudaGetLastError();
}

}  // namespace pcdm

#include "stream_kernels.cuh"
#include "warp_kernels.cuh"

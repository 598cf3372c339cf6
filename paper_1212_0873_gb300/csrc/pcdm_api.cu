// Host implementation of the libpcdm C ABI (include/pcdm.h): argument checks,
// device memory ownership, kernel scheduling, and the solve loop.  Every step
// of the method runs in the kernels of kernels_*.cu; this file only moves
// pointers, sizes and scalars.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "pcdm_host.h"

using namespace pcdm;
using namespace pcdm_host;

thread_local std::string pcdm_host::g_free_error;

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};
uint64_t g_cache_limit = uint64_t(16) << 30;   // bytes of freed handle memory a pool keeps

// The persisting-L2 limit is a property of the device's context, shared by every
// handle on it.  It is raised when the first l2_persist handle of a device is
// created and put back (with the persisting lines reset) when the last one is
// destroyed, so that handles created and destroyed in any order neither drop
// another live handle's set-aside nor leave the raised limit behind.
std::mutex g_l2_mu;
struct L2Users {
    int count = 0;        // live l2_persist handles of the device
    size_t before = 0;    // the limit before the first of them raised it
};
L2Users g_l2_users[kMaxPoolDevices];

// Called with `device` current.
cudaError_t l2_persist_acquire(int device, size_t max_bytes)
{
    if (device < 0 || device >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_l2_mu);
    L2Users &u = g_l2_users[device];
    if (u.count == 0) {
        size_t before = 0;
        cudaError_t e = cudaDeviceGetLimit(&before, cudaLimitPersistingL2CacheSize);
        if (e == cudaSuccess) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, max_bytes);
        if (e != cudaSuccess) return e;
        u.before = before;
    }
    u.count += 1;
    return cudaSuccess;
}

void l2_persist_release(int device)
{
    if (device < 0 || device >= kMaxPoolDevices) return;
    std::lock_guard<std::mutex> lock(g_l2_mu);
    L2Users &u = g_l2_users[device];
    if (u.count <= 0 || --u.count > 0) return;
    int cur = -1;
    const bool switch_dev = cudaGetDevice(&cur) == cudaSuccess && cur != device;
    if (switch_dev) cudaSetDevice(device);
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, u.before);
    cudaCtxResetPersistingL2Cache();
    if (switch_dev) cudaSetDevice(cur);
}
}  // namespace

cudaError_t pcdm_host::handle_pool(int device, cudaMemPool_t *pool)
{
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (device < 0 || device >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    if (!g_pools[device]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t limit = g_cache_limit;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &limit);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[device] = p;
    }
    *pool = g_pools[device];
    return cudaSuccess;
}

namespace {

void free_all(pcdm_handle h)
{
    void *ptrs[] = {h->desc, h->prow, h->pval, h->b, h->L64, h->x, h->g, h->g2,
                    h->S[0], h->S[1], h->h, h->counters, h->bar, h->status, h->gap_part, h->gap_out,
                    h->as_sidx, h->as_c, h->as_sgn, h->as_u, h->as_dx, h->as_q, h->as_rowcnt, h->as_H,
                    h->as_S, h->as_part, h->win, h->head, h->det_rptr, h->det_rcol, h->det_rval, h->det_mark};
    for (void *p : ptrs) hfree(h, p);
    if (h->l2_set) {
        l2_persist_release(h->device);
        h->l2_set = false;
    }
    if (h->g64 && h->g64 != h->g) hfree(h, h->g64);
    if (h->host_buf) cudaFreeHost(h->host_buf);
    for (auto &pr : h->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
}

// Lanes per column: enough lanes of kLaneRun entries each to cover a column
// of average length in one chunk.
// beta of the handle's sampling (Theorem ESO-DU; ESO-nice for the tau-nice sampling).
double beta_for(pcdm_handle h, int64_t tau)
{
    if (h->opts.sampling == PCDM_SAMPLING_NICE) return beta_nice(h->omega, tau, h->n);
    double e1 = 0.0, e2 = 0.0;
    sampling_moments(h->opts.sampling, h->n, tau, h->opts.p_b, &e1, &e2);
    return beta_du(h->omega, e1, e2, h->n);
}

int auto_lanes(int64_t nnz, int64_t n)
{
    const double mean = n > 0 ? double(nnz) / double(n) : 0.0;
    int W = 1;
    while (W < 32 && double(W * kLaneRun) < mean) W *= 2;
    return W;
}

pcdm_status ensure_tau(pcdm_handle h, int64_t tau)
{
    if (tau <= h->tau_cap) return PCDM_OK;
    // Buffers are replaced only between calls; the stream must be idle first.
    CK(h, cudaStreamSynchronize(h->stream));
    for (int q = 0; q < 2; ++q) hfree(h, h->S[q]);
    hfree(h, h->h);
    h->S[0] = h->S[1] = nullptr;
    h->h = nullptr;
    h->tau_cap = 0;
    h->sample_valid = false;
    CK(h, halloc(h, &h->S[0], tau));
    CK(h, halloc(h, &h->S[1], tau));
    CK(h, halloc_bytes(h, &h->h, tau * dtype_bytes(h->xg_dtype)));
    h->tau_cap = tau;
    return PCDM_OK;
}

template <typename VT, typename XT>
IterArgs<VT, XT> iter_args(pcdm_handle h, int64_t tau, uint64_t seed)
{
    IterArgs<VT, XT> a;
    a.desc = static_cast<const ColDesc<XT> *>(h->desc);
    a.prow = h->prow;
    a.pval = static_cast<const VT *>(h->pval);
    a.x = static_cast<double *>(h->x);
    a.g = static_cast<XT *>(h->g);
    a.g2 = static_cast<XT *>(h->g2);
    a.h = static_cast<XT *>(h->h);
    a.S[0] = h->S[0];
    a.S[1] = h->S[1];
    a.inv_beta = 1.0 / beta_for(h, tau);
    a.sampling = h->opts.sampling;
    a.keep_T = binomial_threshold(h->opts.p_b);
    a.win = h->win;
    a.head = h->head;
    a.lambda = h->lambda;
    a.problem = h->problem;
    a.kappa = h->lambda * double(h->n);
    a.n = h->n;
    a.tau = tau;
    a.seed = seed;
    a.counters = h->counters;
    a.bar = h->bar;
    a.status = h->status;
    a.timeout_ns = h->opts.barrier_timeout_ns ? h->opts.barrier_timeout_ns : kDefaultTimeoutNs;
    return a;
}

// Launch shape of the fused kernel for tau: one group of W lanes per sampled
// column when the grid can hold them (spread over all SMs, one block each),
// otherwise full blocks at the co-residency limit.
template <typename VT, typename XT>
pcdm_status fused_shape(pcdm_handle h, int64_t tau, int W, FusedShape *sh)
{
    sh->W = W;
    const int64_t need = tau * W;
    int64_t blocks = (need + 63) / 64;
    if (blocks > h->sms) blocks = h->sms;
    if (blocks < 1) blocks = 1;
    int64_t threads = (need + blocks - 1) / blocks;
    threads = (threads + 31) / 32 * 32;
    if (threads > fused_max_block(W)) {
        threads = fused_max_block(W);
        blocks = (need + threads - 1) / threads;
    }
    const int cap = Kernels<VT, XT>::fused_max_blocks(W, int(threads));
    if (cap <= 0) return set_err(h, PCDM_ECUDA, "cooperative occupancy query failed");
    if (blocks > cap) blocks = cap;
    sh->blocks = int(blocks);
    sh->threads = int(threads);
    return PCDM_OK;
}

// Shape of the pipelined kernel for tau, if it applies: one lane per column,
// every position owned by one thread of a co-resident grid.
template <typename VT, typename XT>
bool pipe_shape(pcdm_handle h, int64_t tau, FusedShape *sh, int want_threads = 0)
{
    if (h->W != 1 && want_threads == 0) return false;
    int64_t threads = want_threads > 0 ? want_threads : (tau + h->sms - 1) / h->sms;
    threads = (threads + 31) / 32 * 32;
    if (threads < 32) threads = 32;
    if (threads > kPipeMaxBlock) return false;
    int64_t blocks = (tau + threads - 1) / threads;
    // the kernel deals positions round-robin over its blocks: one block per SM
    // when tau leaves SMs without a block
    if (blocks < h->sms) blocks = tau < h->sms ? tau : h->sms;
    const int cap = Kernels<VT, XT>::pipe_max_blocks(int(threads));
    if (cap <= 0 || blocks > cap) return false;
    sh->W = 1;
    sh->blocks = int(blocks);
    sh->threads = int(threads);
    return true;
}

// Shape of the streaming kernel for tau, if it applies: as the pipelined kernel,
// one lane per column, every position owned by one thread of a co-resident grid.
template <typename VT, typename XT>
bool stream_shape(pcdm_handle h, int64_t tau, FusedShape *sh, int want_threads)
{
    int64_t threads = want_threads > 0 ? want_threads : (tau + h->sms - 1) / h->sms;
    threads = (threads + 31) / 32 * 32;
    if (threads < 32) threads = 32;
    if (threads > kPipeMaxBlock) return false;
    int64_t blocks = (tau + threads - 1) / threads;
    if (blocks < h->sms) blocks = tau < h->sms ? tau : h->sms;
    const int cap = Kernels<VT, XT>::stream_max_blocks(int(threads));
    if (cap <= 0 || blocks > cap) return false;
    sh->W = 1;
    sh->blocks = int(blocks);
    sh->threads = int(threads);
    return true;
}

// Shape of the warp-cooperative kernel for tau, if it applies: blocks of
// `want_threads` (default kWarpMaxBlock) threads, as many co-resident blocks as
// give every warp a position, at most 32 positions per warp.
template <typename VT, typename XT>
bool warp_shape(pcdm_handle h, int64_t tau, FusedShape *sh, int want_threads)
{
    const int threads = want_threads > 0 ? want_threads : kWarpMaxBlock;
    if (threads % 32 != 0 || threads > kWarpMaxBlock) return false;
    const int wpb = threads / 32;
    const int cap = Kernels<VT, XT>::warp_max_blocks(threads);
    if (cap <= 0) return false;
    int64_t blocks = (tau + wpb - 1) / wpb;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (tau > 32 * int64_t(wpb) * blocks) return false;
    sh->W = 32;
    sh->blocks = int(blocks);
    sh->threads = threads;
    return true;
}

// The per-column heads of the pipelined kernels, built on their first use.
template <typename VT, typename XT>
pcdm_status ensure_heads(pcdm_handle h, IterArgs<VT, XT> &a)
{
    a.head = nullptr;
    if (!h->tune_heads || h->head_off) return PCDM_OK;
    if (!h->head) {
        const int64_t need = h->n * head_stride<VT>();
        size_t free_b = 0, total_b = 0;
        CK(h, cudaMemGetInfo(&free_b, &total_b));
        if (int64_t(free_b / 4) < need) {
            h->head_off = true;
            return PCDM_OK;
        }
        void *p = nullptr;
        CK(h, halloc_bytes(h, &p, need));
        h->head = static_cast<unsigned char *>(p);
        CK(h, Kernels<VT, XT>::build_heads(static_cast<const ColDesc<XT> *>(h->desc), h->prow,
                                           static_cast<const VT *>(h->pval), h->n, h->head, h->stream));
        h->st_kernels += 1;
    }
    a.head = h->head;
    return PCDM_OK;
}

// Run `iters` iterations starting at h->k with S_k already drawn.
template <typename VT, typename XT>
pcdm_status run_segment(pcdm_handle h, int64_t tau, uint64_t seed, int64_t iters)
{
    IterArgs<VT, XT> a = iter_args<VT, XT>(h, tau, seed);
    h->rounds_last = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->opts.profile) {
        CK(h, take_event(h, &e0));
        CK(h, take_event(h, &e1));
        CK(h, cudaEventRecord(e0, h->stream));
    }
    if (h->opts.deterministic_scatter) {
        // the deterministic two-kernel form: gather, scatter, then S_{k+1}
        CK(h, cudaMemsetAsync(h->det_mark, 0, size_t(h->n) * sizeof(unsigned long long), h->stream));
        const double beta = beta_for(h, tau);
        for (int64_t it = 0; it < iters; ++it) {
            const int64_t kk = h->k + it;
            CK(h, DetKernels<VT, XT>::gather(a, h->L64, beta, h->det_mark, kk, h->stream));
            CK(h, DetKernels<VT, XT>::scatter(a, h->det_rptr, h->det_rcol, static_cast<const VT *>(h->det_rval),
                                              h->det_mark, kk, h->stream));
            CK(h, launch_sample(seed, kk + 1, h->n, tau, a.S[(kk + 1) & 1], h->stream));
        }
        h->g2_valid = false;
        h->st_launches += iters;
        h->st_kernels += 3 * iters + 1;
    } else if (h->opts.sampling != PCDM_SAMPLING_NICE) {
        // the other samplings: draw, gather, scatter per iteration
        if (h->opts.sampling == PCDM_SAMPLING_INDEPENDENT) {
            if (!h->win) {
                CK(h, cudaStreamSynchronize(h->stream));
                CK(h, halloc(h, &h->win, h->n));
                a.win = h->win;
            }
            // keys of a later iteration than k would shadow this run's (after set_iteration)
            CK(h, cudaMemsetAsync(h->win, 0, sizeof(unsigned long long) * size_t(h->n), h->stream));
        }
        for (int64_t it = 0; it < iters; ++it) {
            const int64_t kk = h->k + it;
            CK(h, launch_sample_kind(h->opts.sampling, seed, kk, h->n, tau, a.keep_T, a.S[kk & 1],
                                     h->opts.sampling == PCDM_SAMPLING_INDEPENDENT ? h->win : nullptr, nullptr,
                                     h->stream));
            CK(h, Kernels<VT, XT>::gather(a, h->W, kk, h->stream));
            CK(h, Kernels<VT, XT>::scatter(a, h->W, kk, false, h->stream));
        }
        h->g2_valid = false;
        h->st_launches += iters;
        h->st_kernels += 3 * iters;
    } else if (h->opts.fused && h->tune_kernel != 2) {
        FusedShape sh;
        CK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
        // the streaming (4) and warp-cooperative (5) kernels: by the tuning only
        const bool warp = h->tune_kernel == 5 && warp_shape<VT, XT>(h, tau, &sh, h->tune_threads);
        const bool stream = h->tune_kernel == 4 && stream_shape<VT, XT>(h, tau, &sh, h->tune_threads);
        const bool pipe = (warp || stream || h->tune_kernel == 1 || h->tune_kernel == 3 || h->tune_kernel == 4 ||
                           h->tune_kernel == 5)
                              ? false
                              : pipe_shape<VT, XT>(h, tau, &sh, h->tune_kernel == 0 ? h->tune_threads : 0);
        // rounds: when chosen (pcdm_autotune / pcdm_set_tuning); on the workloads measured so far
        // it did not beat the fused kernel where the one-pass grid cannot hold tau
        bool rounds = false;
        if (!pipe && h->tune_kernel == 3 && h->problem == PCDM_PROBLEM_LASSO) {
            const int thr = h->tune_kernel == 3 && h->tune_threads > 0 ? h->tune_threads : kPipeRoundsMaxBlock;
            const int cap = Kernels<VT, XT>::pipe_rounds_max_blocks(thr);
            if (cap > 0) {
                sh.W = 1;
                sh.threads = thr;
                const int64_t need = (tau + thr - 1) / thr;
                sh.blocks = int(need < cap ? need : cap);
                rounds = true;
            }
        }
        h->rounds_last = rounds;
        if (rounds || pipe) {
            pcdm_status hs = ensure_heads<VT, XT>(h, a);
            if (hs != PCDM_OK) return hs;
        }
        if (warp) {
            const size_t gbytes = size_t(h->m) * size_t(dtype_bytes(h->xg_dtype));
            if (!h->g2) {
                CK(h, cudaStreamSynchronize(h->stream));
                CK(h, halloc_bytes(h, &h->g2, int64_t(gbytes)));
                a.g2 = static_cast<XT *>(h->g2);
                h->g2_valid = false;
            }
            if (!h->g2_valid) CK(h, cudaMemcpyAsync(h->g2, h->g, gbytes, cudaMemcpyDeviceToDevice, h->stream));
            // the FP32 zero-step certificate (FP64 form of LASSO): by the tuning, else while few
            // coordinates move (warp_cert)
            const bool wzc = h->tune_zc == 1 || (h->tune_zc < 0 && h->warp_cert);
            CK(h, Kernels<VT, XT>::fused_warp(a, sh, h->k, iters, wzc, h->stream));
            h->g2_valid = true;
        } else if (stream) {
            const size_t gbytes = size_t(h->m) * size_t(dtype_bytes(h->xg_dtype));
            if (!h->g2) {
                CK(h, cudaStreamSynchronize(h->stream));
                CK(h, halloc_bytes(h, &h->g2, int64_t(gbytes)));
                a.g2 = static_cast<XT *>(h->g2);
                h->g2_valid = false;
            }
            if (!h->g2_valid) CK(h, cudaMemcpyAsync(h->g2, h->g, gbytes, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, Kernels<VT, XT>::fused_stream(a, sh, h->k, iters, h->stream));
            h->g2_valid = true;
        } else if (rounds) {
            const size_t gbytes = size_t(h->m) * size_t(dtype_bytes(h->xg_dtype));
            if (!h->g2) {
                CK(h, cudaStreamSynchronize(h->stream));
                CK(h, halloc_bytes(h, &h->g2, int64_t(gbytes)));
                a.g2 = static_cast<XT *>(h->g2);
                h->g2_valid = false;
            }
            if (!h->g2_valid) CK(h, cudaMemcpyAsync(h->g2, h->g, gbytes, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, Kernels<VT, XT>::fused_pipe_rounds(a, sh, h->k, iters, h->stream));
            h->g2_valid = true;
        } else if (pipe) {
            const size_t gbytes = size_t(h->m) * size_t(dtype_bytes(h->xg_dtype));
            if (!h->g2) {
                CK(h, cudaStreamSynchronize(h->stream));
                CK(h, halloc_bytes(h, &h->g2, int64_t(gbytes)));
                a.g2 = static_cast<XT *>(h->g2);
                h->g2_valid = false;
            }
            if (!h->g2_valid) CK(h, cudaMemcpyAsync(h->g2, h->g, gbytes, cudaMemcpyDeviceToDevice, h->stream));
            // the FP64 zero-step certificate: by the tuning, else for short columns
            const bool zc = h->tune_zc < 0 ? (h->nnz <= 8 * h->n) : (h->tune_zc == 1);
            CK(h, Kernels<VT, XT>::fused_pipe(a, sh, h->k, iters, zc, h->stream));
            h->g2_valid = true;
        } else {
            pcdm_status s = fused_shape<VT, XT>(h, tau, h->tune_kernel == 1 ? h->tune_W : h->W, &sh);
            if (s != PCDM_OK) return s;
            CK(h, Kernels<VT, XT>::fused(a, sh, h->k, iters, h->stream));
            h->g2_valid = false;
        }
        h->st_launches += 1;
        h->st_kernels += 1;
    } else {
        const int W2 = h->tune_kernel == 2 && h->tune_W > 0 ? h->tune_W : h->W;
        for (int64_t it = 0; it < iters; ++it) {
            const int64_t kk = h->k + it;
            CK(h, Kernels<VT, XT>::gather(a, W2, kk, h->stream));
            CK(h, Kernels<VT, XT>::scatter(a, W2, kk, true, h->stream));
        }
        h->g2_valid = false;
        h->st_launches += iters;
        h->st_kernels += 2 * iters;
    }
    if (h->opts.profile) {
        CK(h, cudaEventRecord(e1, h->stream));
        h->ev_pending.emplace_back(e0, e1);
    }
    h->k += iters;
    h->sample_valid = !h->rounds_last;
    h->sample_seed = seed;
    h->sample_tau = tau;
    h->sample_k = h->k;
    h->st_iterations += iters;
    h->st_updates += iters * tau;
    return PCDM_OK;
}

template <typename VT, typename XT>
pcdm_status refresh_t(pcdm_handle h)
{
    double *target = h->g64;
    if (h->opts.deterministic_scatter) {
        CK(h, DetKernels<VT, XT>::refresh(h->det_rptr, h->det_rcol, static_cast<const VT *>(h->det_rval),
                                          static_cast<const double *>(h->x), h->b, h->m, target,
                                          static_cast<XT *>(h->g), h->stream));
        h->g2_valid = false;
        h->st_refreshes += 1;
        h->st_kernels += 1;
        return PCDM_OK;
    }
    CK(h, launch_neg_store<double>(target, h->b, h->m, h->stream));
    CK(h, Kernels<VT, XT>::refresh_cols(static_cast<const ColDesc<XT> *>(h->desc), h->prow,
                                        static_cast<const VT *>(h->pval), static_cast<const double *>(h->x), h->n,
                                        target, h->W, h->stream));
    if (sizeof(XT) == 4) CK(h, launch_store_from_f64<float>(static_cast<float *>(h->g), target, h->m, h->stream));
    h->g2_valid = false;
    h->st_refreshes += 1;
    h->st_kernels += sizeof(XT) == 4 ? 3 : 2;
    return PCDM_OK;
}

template <typename VT, typename XT>
pcdm_status gap_t(pcdm_handle h)
{
    pcdm_status s = refresh_t<VT, XT>(h);
    if (s != PCDM_OK) return s;
    double *part_c = h->gap_part;
    double *part_r = h->gap_part + 3 * h->gap_blocks;
    if (h->problem == PCDM_PROBLEM_LASSO) {
        CK(h, Kernels<VT, XT>::gap_cols(static_cast<const ColDesc<XT> *>(h->desc), h->prow,
                                        static_cast<const VT *>(h->pval), h->g64, static_cast<const double *>(h->x),
                                        h->n, part_c, h->gap_blocks, h->W, h->stream));
        CK(h, launch_gap_rows(h->g64, h->b, h->m, part_r, h->gap_row_blocks, h->stream));
        CK(h, launch_gap_finish(part_c, h->gap_blocks, part_r, h->gap_row_blocks, h->gap_out, h->lambda, h->stream));
    } else {
        CK(h, Kernels<VT, XT>::glm_gap_cols(h->problem, static_cast<const ColDesc<XT> *>(h->desc), h->prow,
                                            static_cast<const VT *>(h->pval), h->g64,
                                            static_cast<const double *>(h->x), h->n, h->lambda,
                                            h->lambda * double(h->n), part_c, h->gap_blocks, h->W, h->stream));
        CK(h, launch_glm_gap_rows(h->problem, h->g64, h->m, part_r, h->gap_row_blocks, h->stream));
        CK(h, launch_glm_gap_finish(h->problem, part_c, h->gap_blocks, part_r, h->gap_row_blocks, h->lambda, h->n,
                                    h->gap_out, h->stream));
    }
    CK(h, cudaMemcpyAsync(h->host_buf, h->gap_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    h->st_gaps += 1;
    h->st_kernels += 3;
    return sync_check(h);
}

pcdm_status do_refresh(pcdm_handle h)
{
    return dispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return refresh_t<VT, XT>(h);
    });
}

pcdm_status do_gap(pcdm_handle h, double *rec)
{
    pcdm_status s = dispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return gap_t<VT, XT>(h);
    });
    if (s != PCDM_OK) return s;
    for (int q = 0; q < 9; ++q) rec[q] = h->host_buf[q];
    return PCDM_OK;
}

pcdm_status reset_state(pcdm_handle h)
{
    CK(h, cudaMemsetAsync(h->x, 0, size_t(h->n) * sizeof(double), h->stream));
    if (h->xg_dtype == PCDM_F64)
        CK(h, launch_neg_store<double>(static_cast<double *>(h->g), h->b, h->m, h->stream));
    else
        CK(h, launch_neg_store<float>(static_cast<float *>(h->g), h->b, h->m, h->stream));
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    h->g2_valid = false;
    h->st_kernels += 1;   // the g = -b kernel
    h->k = 0;
    h->sample_valid = false;
    h->warp_cert = false;
    return PCDM_OK;
}

}  // namespace

// ============================================================================
extern "C" {

void pcdm_default_opts(pcdm_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->xg_dtype = PCDM_F64;
    o->fused = 1;
    o->refresh_every = 0;
    o->check_every = 0;
    o->lanes_per_col = 0;
    o->barrier_timeout_ns = kDefaultTimeoutNs;
    o->profile = 0;
    o->sampling = PCDM_SAMPLING_NICE;
    o->p_b = 1.0;
}

const char *pcdm_status_string(pcdm_status s)
{
    switch (s) {
    case PCDM_OK: return "PCDM_OK";
    case PCDM_EINVAL: return "PCDM_EINVAL";
    case PCDM_ENOMEM: return "PCDM_ENOMEM";
    case PCDM_ECUDA: return "PCDM_ECUDA";
    case PCDM_ETIMEOUT: return "PCDM_ETIMEOUT";
    case PCDM_ENOTCONV: return "PCDM_ENOTCONV";
    case PCDM_ESTATE: return "PCDM_ESTATE";
    default: return "PCDM_UNKNOWN";
    }
}

const char *pcdm_last_error(pcdm_handle h) { return h ? h->err.c_str() : g_free_error.c_str(); }

}  // extern "C"

namespace {

// pcdm_create (problem 0, b given) and pcdm_create_problem (problems 1 and 2:
// b = 0 and the labels y folded into the stored values).
pcdm_status create_impl(const pcdm_csc *A, const void *b, int32_t b_dtype, double lambda, const pcdm_opts *opts,
                        void *cuda_stream, pcdm_handle *out, int problem, const double *y)
{
    if (!out) return set_err(nullptr, PCDM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!A || (!b && problem == PCDM_PROBLEM_LASSO)) return set_err(nullptr, PCDM_EINVAL, "A or b is NULL");
    pcdm_opts o;
    pcdm_default_opts(&o);
    if (opts) o = *opts;
    if (A->m < 1 || A->n < 1 || A->m > 2147483647LL || A->n > 2147483647LL || A->nnz < 0)
        return set_err(nullptr, PCDM_EINVAL, "need 1 <= m, n < 2^31 and nnz >= 0");
    if (!A->col_ptr || (A->nnz > 0 && (!A->row_idx || !A->val)))
        return set_err(nullptr, PCDM_EINVAL, "NULL col_ptr, row_idx or val");
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return set_err(nullptr, PCDM_EINVAL, "lambda must be finite and >= 0");
    if (b_dtype != PCDM_F64 && b_dtype != PCDM_F32) return set_err(nullptr, PCDM_EINVAL, "b_dtype must be F64 or F32");
    const bool pair_ok = (A->val_dtype == PCDM_F64 && o.xg_dtype == PCDM_F64) ||
                         (A->val_dtype == PCDM_F32 && o.xg_dtype == PCDM_F32) ||
                         (A->val_dtype == PCDM_BF16 && o.xg_dtype == PCDM_F32);
    if (!pair_ok) return set_err(nullptr, PCDM_EINVAL, "dtype pair must be (F64,F64), (F32,F32) or (BF16,F32)");
    if (o.lanes_per_col != 0 && o.lanes_per_col != 4 && o.lanes_per_col != 8 && o.lanes_per_col != 16 &&
        o.lanes_per_col != 32)
        return set_err(nullptr, PCDM_EINVAL, "lanes_per_col must be 0, 4, 8, 16 or 32");
    if (o.refresh_every < 0 || o.check_every < 0) return set_err(nullptr, PCDM_EINVAL, "negative period");
    if (o.sampling < PCDM_SAMPLING_NICE || o.sampling > PCDM_SAMPLING_BINOMIAL)
        return set_err(nullptr, PCDM_EINVAL, "unknown sampling");
    if (o.sampling == PCDM_SAMPLING_BINOMIAL && !(o.p_b > 0.0 && o.p_b <= 1.0))
        return set_err(nullptr, PCDM_EINVAL, "p_b must be in (0, 1]");
    if (o.l2_persist != 0 && o.l2_persist != 1) return set_err(nullptr, PCDM_EINVAL, "l2_persist must be 0 or 1");
    if (o.deterministic_scatter != 0 && o.deterministic_scatter != 1)
        return set_err(nullptr, PCDM_EINVAL, "deterministic_scatter must be 0 or 1");
    if (o.deterministic_scatter && (problem != PCDM_PROBLEM_LASSO || o.sampling != PCDM_SAMPLING_NICE))
        return set_err(nullptr, PCDM_EINVAL, "deterministic_scatter needs LASSO with the tau-nice sampling");

    pcdm_ctx *h = new (std::nothrow) pcdm_ctx();
    if (!h) return set_err(nullptr, PCDM_ENOMEM, "host allocation failed");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->m = A->m;
    h->n = A->n;
    h->nnz = A->nnz;
    h->val_dtype = A->val_dtype;
    h->xg_dtype = o.xg_dtype;
    h->lambda = lambda;
    h->problem = problem;
    h->opts = o;
    h->W = o.lanes_per_col ? int(o.lanes_per_col) : auto_lanes(A->nnz, A->n);

    auto fail = [&](pcdm_status s) {
        g_free_error = h->err;
        free_all(h);
        delete h;
        return s;
    };
#define CKC(...)                                                            \
    do {                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                     \
        if (e_ != cudaSuccess) return fail(cuda_fail(h, e_, #__VA_ARGS__)); \
    } while (0)

    CKC(cudaGetDevice(&h->device));
    const int64_t vb = dtype_bytes(h->val_dtype), xb = dtype_bytes(h->xg_dtype);
    CKC(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
    if (o.l2_persist) {
        int maxp = 0;
        CKC(cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, h->device));
        if (maxp > 0) {
            CKC(l2_persist_acquire(h->device, size_t(maxp)));
            h->l2_set = true;
        }
    }
    {
        int64_t gb = (h->n * h->W + kBlock - 1) / kBlock;
        const int64_t cap = int64_t(h->sms) * 8;
        h->gap_blocks = int(gb < 1 ? 1 : (gb > cap ? cap : gb));
        int64_t rb = (h->m + kBlock - 1) / kBlock;
        h->gap_row_blocks = int(rb < 1 ? 1 : (rb > cap ? cap : rb));
    }
    CKC(halloc(h, &h->b, h->m));
    CKC(halloc(h, &h->L64, h->n));
    CKC(halloc(h, &h->x, h->n));
    CKC(halloc_bytes(h, &h->g, h->m * xb));
    if (h->xg_dtype == PCDM_F64)
        h->g64 = static_cast<double *>(h->g);
    else
        CKC(halloc(h, &h->g64, h->m));
    CKC(halloc(h, &h->counters, 3));
    CKC(halloc(h, &h->bar, 1));
    CKC(halloc(h, &h->status, 4));
    CKC(halloc(h, &h->gap_part, 3 * int64_t(h->gap_blocks) + 2 * int64_t(h->gap_row_blocks)));
    CKC(halloc(h, &h->gap_out, 9));
    CKC(cudaMallocHost(reinterpret_cast<void **>(&h->host_buf), 16 * sizeof(double)));

    // Stage the caller's CSC on the device (freed once the padded layout exists).
    struct Staging {
        int64_t *col_ptr = nullptr, *pbeg = nullptr, *tile = nullptr;
        int32_t *row_idx = nullptr;
        void *val = nullptr;
        int *rowcnt = nullptr;
        double *y = nullptr;
        cudaStream_t stream = nullptr;   // the handle's stream (the handle may be gone by destruction)
        ~Staging()
        {
            void *p[] = {col_ptr, pbeg, tile, row_idx, val, rowcnt, y};
            for (void *q : p)
                if (q) cudaFreeAsync(q, stream);
        }
    } stg;
    stg.stream = h->stream;
    cudaStream_t st = h->stream;
    const cudaMemcpyKind kin = copy_kind(A->on_device, 1);
    CKC(halloc(h, &stg.col_ptr, h->n + 1));
    CKC(halloc(h, &stg.row_idx, h->nnz));
    CKC(halloc_bytes(h, &stg.val, h->nnz * vb));
    CKC(cudaMemcpyAsync(stg.col_ptr, A->col_ptr, size_t(h->n + 1) * sizeof(int64_t), kin, st));
    if (h->nnz > 0) {
        CKC(cudaMemcpyAsync(stg.row_idx, A->row_idx, size_t(h->nnz) * sizeof(int32_t), kin, st));
        CKC(cudaMemcpyAsync(stg.val, A->val, size_t(h->nnz * vb), kin, st));
    }
    const int64_t ny = problem == PCDM_PROBLEM_SVM_DUAL ? h->n : h->m;   // labels: one per example
    if (problem != PCDM_PROBLEM_LASSO) {
        CKC(cudaMemsetAsync(h->b, 0, size_t(h->m) * sizeof(double), st));
        CKC(halloc(h, &stg.y, ny));
        CKC(cudaMemcpyAsync(stg.y, y, size_t(ny) * sizeof(double), kin, st));
    } else if (b_dtype == PCDM_F64) {
        CKC(cudaMemcpyAsync(h->b, b, size_t(h->m) * sizeof(double), kin, st));
    } else {
        // Stage the FP32 b in the g buffer (at least m floats) and widen it.
        CKC(cudaMemcpyAsync(h->g, b, size_t(h->m) * sizeof(float), kin, st));
        CKC(launch_convert_b(h->g, 1, h->m, h->b, st));
    }

    // Validation, first of col_ptr alone so that the column kernels index safely.
    int *flags = h->status + 1;
    int *omega_dev = h->status + 2;
    int *hflags = reinterpret_cast<int *>(h->host_buf + 10);
    CKC(cudaMemsetAsync(h->status, 0, 4 * sizeof(int), st));
    CKC(launch_check_colptr(stg.col_ptr, h->n, h->nnz, flags, st));
    CKC(cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (*hflags & FLAG_COLPTR) {
        h->err = "col_ptr must start at 0, be non-decreasing and end at nnz";
        return fail(PCDM_EINVAL);
    }
    CKC(halloc(h, &stg.rowcnt, h->m));
    CKC(cudaMemsetAsync(stg.rowcnt, 0, size_t(h->m) * sizeof(int), st));
    switch (h->val_dtype) {
    case PCDM_F64:
        CKC(Kernels<double, double>::setup_cols(stg.col_ptr, stg.row_idx, static_cast<const double *>(stg.val),
                                                h->m, h->n, h->L64, stg.rowcnt, flags, st));
        break;
    case PCDM_F32:
        CKC(Kernels<float, float>::setup_cols(stg.col_ptr, stg.row_idx, static_cast<const float *>(stg.val), h->m,
                                              h->n, h->L64, stg.rowcnt, flags, st));
        break;
    default:
        CKC(Kernels<bf16_t, float>::setup_cols(stg.col_ptr, stg.row_idx, static_cast<const bf16_t *>(stg.val),
                                               h->m, h->n, h->L64, stg.rowcnt, flags, st));
        break;
    }
    CKC(launch_check_finite(h->b, h->m, flags, st));
    if (problem != PCDM_PROBLEM_LASSO) CKC(launch_check_labels(stg.y, ny, flags, st));
    if (problem == PCDM_PROBLEM_LOGISTIC) CKC(launch_scale(h->L64, h->n, 0.25, st));   // L_i = ||a_i||^2 / 4
    CKC(launch_max_int(stg.rowcnt, h->m, omega_dev, st));
    CKC(cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    {
        const int f = hflags[0];
        if (f) {
            std::string msg = "invalid input:";
            if (f & FLAG_ROW_RANGE) msg += " row index outside [0, m);";
            if (f & FLAG_ROW_ORDER) msg += " rows of a column not strictly increasing;";
            if (f & FLAG_NONFINITE) msg += " non-finite value in A;";
            if (f & FLAG_B_NONFINITE) msg += " non-finite value in b;";
            if (f & FLAG_LABEL) msg += " a label other than -1 or +1;";
            h->err = msg;
            return fail(PCDM_EINVAL);
        }
    }
    h->omega = hflags[1];

    // Padded layout: exclusive scan of the padded lengths, then copy and descriptors.
    const int granule = h->val_dtype == PCDM_BF16 ? 8 : 4;
    CKC(halloc(h, &stg.pbeg, h->n + 1));
    CKC(halloc(h, &stg.tile, scan_tile_count(h->n) + 1));
    CKC(launch_padded_scan(stg.col_ptr, h->n, granule, stg.pbeg, stg.tile, st));
    int64_t *hP = reinterpret_cast<int64_t *>(h->host_buf + 11);
    CKC(cudaMemcpyAsync(hP, stg.pbeg + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    h->P = *hP;
    if (h->P / 4 > int64_t(0xFFFFFFFFu)) {
        h->err = "matrix too large for the padded layout (more than 2^34 padded entries)";
        return fail(PCDM_EINVAL);
    }
    CKC(halloc(h, &h->prow, h->P + kSlack));
    CKC(halloc_bytes(h, &h->pval, (h->P + kSlack) * vb));
    CKC(halloc_bytes(h, &h->desc, h->n * 16));
    CKC(cudaMemsetAsync(h->prow, 0, size_t(h->P + kSlack) * sizeof(int32_t), st));
    CKC(cudaMemsetAsync(h->pval, 0, size_t((h->P + kSlack) * vb), st));
    switch (h->val_dtype) {
    case PCDM_F64:
        CKC(Kernels<double, double>::build_layout(stg.col_ptr, stg.row_idx, static_cast<const double *>(stg.val),
                                                  stg.pbeg, h->L64, h->n, static_cast<ColDesc<double> *>(h->desc),
                                                  h->prow, static_cast<double *>(h->pval), st));
        break;
    case PCDM_F32:
        CKC(Kernels<float, float>::build_layout(stg.col_ptr, stg.row_idx, static_cast<const float *>(stg.val),
                                                stg.pbeg, h->L64, h->n, static_cast<ColDesc<float> *>(h->desc),
                                                h->prow, static_cast<float *>(h->pval), st));
        break;
    default:
        CKC(Kernels<bf16_t, float>::build_layout(stg.col_ptr, stg.row_idx, static_cast<const bf16_t *>(stg.val),
                                                 stg.pbeg, h->L64, h->n, static_cast<ColDesc<float> *>(h->desc),
                                                 h->prow, static_cast<bf16_t *>(h->pval), st));
        break;
    }
    if (problem != PCDM_PROBLEM_LASSO) {
        switch (h->val_dtype) {
        case PCDM_F64:
            CKC(Kernels<double, double>::apply_labels(problem, static_cast<const ColDesc<double> *>(h->desc), h->prow,
                                                      static_cast<double *>(h->pval), h->n, stg.y, st));
            break;
        case PCDM_F32:
            CKC(Kernels<float, float>::apply_labels(problem, static_cast<const ColDesc<float> *>(h->desc), h->prow,
                                                    static_cast<float *>(h->pval), h->n, stg.y, st));
            break;
        default:
            CKC(Kernels<bf16_t, float>::apply_labels(problem, static_cast<const ColDesc<float> *>(h->desc), h->prow,
                                                     static_cast<bf16_t *>(h->pval), h->n, stg.y, st));
            break;
        }
    }
    if (o.deterministic_scatter) {
        // row-major copy of A for the deterministic scatter and refresh
        CKC(halloc(h, &h->det_rptr, h->m + 1));
        CKC(halloc(h, &h->det_rcol, h->nnz > 0 ? h->nnz : 1));
        CKC(halloc_bytes(h, &h->det_rval, (h->nnz > 0 ? h->nnz : 1) * vb));
        CKC(halloc(h, &h->det_mark, h->n));
        int64_t *tile = nullptr;
        unsigned long long *cursor = nullptr;
        CKC(halloc(h, &tile, scan_tile_count(h->m) + 1));
        cudaError_t e = halloc(h, &cursor, h->m);
        if (e == cudaSuccess) e = launch_count_scan(stg.rowcnt, h->m, h->det_rptr, tile, st);
        if (e == cudaSuccess) {
            switch (h->val_dtype) {
            case PCDM_F64:
                e = DetKernels<double, double>::build_rows(stg.col_ptr, stg.row_idx,
                                                           static_cast<const double *>(stg.val), h->m, h->n,
                                                           h->det_rptr, cursor, h->det_rcol,
                                                           static_cast<double *>(h->det_rval), st);
                break;
            case PCDM_F32:
                e = DetKernels<float, float>::build_rows(stg.col_ptr, stg.row_idx, static_cast<const float *>(stg.val),
                                                         h->m, h->n, h->det_rptr, cursor, h->det_rcol,
                                                         static_cast<float *>(h->det_rval), st);
                break;
            default:
                e = DetKernels<bf16_t, float>::build_rows(stg.col_ptr, stg.row_idx,
                                                          static_cast<const bf16_t *>(stg.val), h->m, h->n,
                                                          h->det_rptr, cursor, h->det_rcol,
                                                          static_cast<bf16_t *>(h->det_rval), st);
                break;
            }
        }
        hfree(h, tile);
        hfree(h, cursor);
        CKC(e);
    }
    CKC(cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st));
    {
        pcdm_status s = reset_state(h);
        if (s != PCDM_OK) return fail(s);
    }
    CKC(cudaStreamSynchronize(st));
#undef CKC
    *out = h;
    return PCDM_OK;
}

}  // namespace

extern "C" {

pcdm_status pcdm_create(const pcdm_csc *A, const void *b, int32_t b_dtype, double lambda, const pcdm_opts *opts,
                        void *cuda_stream, pcdm_handle *out)
{
    return create_impl(A, b, b_dtype, lambda, opts, cuda_stream, out, PCDM_PROBLEM_LASSO, nullptr);
}

pcdm_status pcdm_create_problem(const pcdm_csc *A, int32_t problem, const double *y, double lambda,
                                const pcdm_opts *opts, void *cuda_stream, pcdm_handle *out)
{
    if (out) *out = nullptr;
    if (problem != PCDM_PROBLEM_SVM_DUAL && problem != PCDM_PROBLEM_LOGISTIC)
        return set_err(nullptr, PCDM_EINVAL, "problem must be PCDM_PROBLEM_SVM_DUAL or PCDM_PROBLEM_LOGISTIC");
    if (!y) return set_err(nullptr, PCDM_EINVAL, "y is NULL");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return set_err(nullptr, PCDM_EINVAL, "lambda must be finite and > 0");
    if (opts && opts->sampling != PCDM_SAMPLING_NICE)
        return set_err(nullptr, PCDM_EINVAL, "the SVM dual and logistic regression take the tau-nice sampling");
    return create_impl(A, nullptr, PCDM_F64, lambda, opts, cuda_stream, out, problem, y);
}

pcdm_status pcdm_problem_kind(pcdm_handle h, int32_t *problem)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!problem) return set_err(h, PCDM_EINVAL, "problem is NULL");
    *problem = h->problem;
    return PCDM_OK;
}

void pcdm_destroy(pcdm_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

pcdm_status pcdm_step(pcdm_handle h, int64_t tau, int64_t iters, uint64_t seed)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->n) return set_err(h, PCDM_EINVAL, "tau must be in [1, n]");
    if (iters < 0) return set_err(h, PCDM_EINVAL, "iters must be >= 0");
    if (iters == 0) return PCDM_OK;
    s = ensure_tau(h, tau);
    if (s != PCDM_OK) return s;
    int64_t left = iters;
    while (left > 0) {
        int64_t seg = left;
        if (h->opts.refresh_every > 0) {
            const int64_t to_refresh = h->opts.refresh_every - (h->k % h->opts.refresh_every);
            if (seg > to_refresh) seg = to_refresh;
        }
        if (h->opts.fused && seg > kMaxItersPerLaunch) seg = kMaxItersPerLaunch;
        if (!(h->sample_valid && h->sample_seed == seed && h->sample_tau == tau && h->sample_k == h->k)) {
            CK(h, launch_sample(seed, h->k, h->n, tau, (h->k & 1) ? h->S[1] : h->S[0], h->stream));
            h->st_kernels += 1;
        }
        s = dispatch(h, [&](auto *vt, auto *xt) {
            using VT = std::remove_pointer_t<decltype(vt)>;
            using XT = std::remove_pointer_t<decltype(xt)>;
            return run_segment<VT, XT>(h, tau, seed, seg);
        });
        if (s != PCDM_OK) return s;
        if (h->opts.refresh_every > 0 && h->k % h->opts.refresh_every == 0) {
            s = do_refresh(h);
            if (s != PCDM_OK) return s;
        }
        left -= seg;
    }
    return PCDM_OK;
}

pcdm_status pcdm_refresh(pcdm_handle h)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    return do_refresh(h);
}

pcdm_status pcdm_gap(pcdm_handle h, double *primal, double *dual, double *gap)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    double rec[9];
    s = do_gap(h, rec);
    if (s != PCDM_OK) return s;
    if (primal) *primal = rec[0];
    if (dual) *dual = rec[1];
    if (gap) *gap = rec[2];
    return PCDM_OK;
}

int64_t pcdm_next_check_interval(int64_t epoch, int64_t k_prev, double rel_prev, int64_t k_cur, double rel_cur,
                                 double rel_gap_tol)
{
    if (epoch < 1) epoch = 1;
    const int64_t lo = (epoch + 3) / 4, hi = 64 * epoch;
    const int64_t last = k_cur - k_prev;
    if (last < 1 || !(rel_prev > rel_cur) || !(rel_cur > 0.0) || !(rel_gap_tol > 0.0) || !(rel_cur > rel_gap_tol))
        return epoch;
    // linear rate of the last interval, extrapolated with a 5% margin
    const double rate = std::log(rel_prev / rel_cur) / double(last);
    const double pred = 1.05 * std::log(rel_cur / rel_gap_tol) / rate;
    int64_t next = pred < double(hi) ? int64_t(std::ceil(pred)) : hi;
    if (next > 2 * last) next = 2 * last;   // no long jumps from a short observation
    if (next < lo) next = lo;
    if (next > hi) next = hi;
    return next;
}

pcdm_status pcdm_solve(pcdm_handle h, int64_t tau, uint64_t seed, double rel_gap_tol, int64_t max_iters,
                       int64_t *iters_done, double *rel_gap)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->n) return set_err(h, PCDM_EINVAL, "tau must be in [1, n]");
    if (max_iters < 0 || !(rel_gap_tol >= 0.0)) return set_err(h, PCDM_EINVAL, "max_iters < 0 or bad tolerance");
    const int64_t epoch = (h->n + tau - 1) / tau;
    const bool fixed = h->opts.check_every > 0;
    int64_t every = fixed ? h->opts.check_every : first_check_interval(epoch, h->last_solve_iters);
    double rec[9];
    int64_t done = 0;
    s = do_gap(h, rec);
    if (s != PCDM_OK) return s;
    // the share of moving coordinates over each stretch between checks decides the
    // warp-cooperative kernel's certificate (counters read after the gap's synchronisation)
    unsigned long long *hc = reinterpret_cast<unsigned long long *>(h->host_buf + 12);
    auto moving = [&](unsigned long long *nonzero) -> pcdm_status {
        CK(h, cudaMemcpyAsync(hc, h->counters, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        *nonzero = hc[2];
        return PCDM_OK;
    };
    unsigned long long nz0 = 0, nz1 = 0;
    if ((s = moving(&nz0)) != PCDM_OK) return s;
    double rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300);
    while (rel > rel_gap_tol && done < max_iters) {
        const int64_t chunk = every < max_iters - done ? every : max_iters - done;
        s = pcdm_step(h, tau, chunk, seed);
        if (s != PCDM_OK) return s;
        const double rel_prev = rel;
        done += chunk;
        s = do_gap(h, rec);
        if (s != PCDM_OK) return s;
        if ((s = moving(&nz1)) != PCDM_OK) return s;
        h->warp_cert = 4 * (nz1 - nz0) <= (unsigned long long)(chunk * tau);
        nz0 = nz1;
        rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300);
        if (!fixed) every = pcdm_next_check_interval(epoch, done - chunk, rel_prev, done, rel, rel_gap_tol);
    }
    if (iters_done) *iters_done = done;
    if (rel_gap) *rel_gap = rel;
    h->last_solve_iters = done;
    if (rel > rel_gap_tol) return set_err(h, PCDM_ENOTCONV, "max_iters reached before the gap tolerance");
    return PCDM_OK;
}

pcdm_status pcdm_get_x(pcdm_handle h, void *x_out, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!x_out) return set_err(h, PCDM_EINVAL, "x_out is NULL");
    CK(h, cudaMemcpyAsync(x_out, h->x, size_t(h->n) * sizeof(double), copy_kind(1, on_device), h->stream));
    return sync_check(h);
}

pcdm_status pcdm_set_x(pcdm_handle h, const void *x_in, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!x_in) return set_err(h, PCDM_EINVAL, "x_in is NULL");
    CK(h, cudaMemcpyAsync(h->x, x_in, size_t(h->n) * sizeof(double), copy_kind(on_device, 1), h->stream));
    h->sample_valid = false;
    h->warp_cert = true;   // a warm start: most coordinates are expected to stay
    s = do_refresh(h);
    if (s != PCDM_OK) return s;
    return sync_check(h);
}

pcdm_status pcdm_get_residual(pcdm_handle h, void *g_out, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!g_out) return set_err(h, PCDM_EINVAL, "g_out is NULL");
    CK(h, cudaMemcpyAsync(g_out, h->g, size_t(h->m * dtype_bytes(h->xg_dtype)), copy_kind(1, on_device), h->stream));
    return sync_check(h);
}

pcdm_status pcdm_get_L(pcdm_handle h, double *L_out, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!L_out) return set_err(h, PCDM_EINVAL, "L_out is NULL");
    CK(h, cudaMemcpyAsync(L_out, h->L64, size_t(h->n) * sizeof(double), copy_kind(1, on_device), h->stream));
    return sync_check(h);
}

pcdm_status pcdm_set_lambda(pcdm_handle h, double lambda)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return set_err(h, PCDM_EINVAL, "lambda must be finite and >= 0");
    if (h->problem != PCDM_PROBLEM_LASSO && !(lambda > 0.0))
        return set_err(h, PCDM_EINVAL, "the SVM dual and logistic regression need lambda > 0");
    h->lambda = lambda;
    return PCDM_OK;
}

pcdm_status pcdm_omega(pcdm_handle h, int64_t *omega)
{
    if (!h || !omega) return set_err(h, PCDM_EINVAL, "NULL argument");
    *omega = h->omega;
    return PCDM_OK;
}

pcdm_status pcdm_beta(pcdm_handle h, int64_t tau, double *beta)
{
    if (!h || !beta) return set_err(h, PCDM_EINVAL, "NULL argument");
    if (tau < 1 || tau > h->n) return set_err(h, PCDM_EINVAL, "tau must be in [1, n]");
    *beta = beta_for(h, tau);
    return PCDM_OK;
}

pcdm_status pcdm_get_iteration(pcdm_handle h, int64_t *k)
{
    if (!h || !k) return set_err(h, PCDM_EINVAL, "NULL argument");
    *k = h->k;
    return PCDM_OK;
}

pcdm_status pcdm_set_iteration(pcdm_handle h, int64_t k)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (k < 0) return set_err(h, PCDM_EINVAL, "k must be >= 0");
    h->k = k;
    h->sample_valid = false;
    return PCDM_OK;
}

pcdm_status pcdm_reset(pcdm_handle h)
{
    if (!h) return set_err(nullptr, PCDM_EINVAL, "NULL handle");
    cudaGetLastError();
    h->failed = false;
    h->err.clear();
    for (auto &pr : h->ev_pending) {
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    h->last_solve_iters = 0;
    h->async_u = 0;
    pcdm_status s = reset_state(h);
    if (s != PCDM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    return PCDM_OK;
}

pcdm_status pcdm_get_stats(pcdm_handle h, pcdm_stats *out)
{
    if (!h || !out) return set_err(h, PCDM_EINVAL, "NULL argument");
    unsigned long long *hc = reinterpret_cast<unsigned long long *>(h->host_buf + 12);
    CK(h, cudaMemcpyAsync(hc, h->counters, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    pcdm_status s = sync_check(h);
    if (s != PCDM_OK && s != PCDM_ETIMEOUT) return s;
    std::memset(out, 0, sizeof(*out));
    out->iterations = h->st_iterations;
    out->updates = h->st_updates;
    out->gathered_nnz = int64_t(hc[0]);
    out->scattered_nnz = int64_t(hc[1]);
    out->nonzero_updates = int64_t(hc[2]);
    out->iter_launches = h->st_launches;
    out->iter_kernel_ms = h->st_kernel_ms;
    out->refreshes = h->st_refreshes;
    out->gaps = h->st_gaps;
    out->val_bytes = dtype_bytes(h->val_dtype);
    out->xg_bytes = dtype_bytes(h->xg_dtype);
    out->kernel_launches = h->st_kernels;
    return s;
}

pcdm_status pcdm_reset_stats(pcdm_handle h)
{
    if (!h) return set_err(nullptr, PCDM_EINVAL, "NULL handle");
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), h->stream));
    h->st_iterations = h->st_updates = h->st_launches = h->st_refreshes = h->st_gaps = 0;
    h->st_kernels = 0;
    h->st_kernel_ms = 0.0;
    for (auto &pr : h->ev_pending) {
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    return PCDM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Active-set solves: the polish of x on its support and the implicit backward.
namespace {

pcdm_status ensure_as(pcdm_handle h, int64_t tau)
{
    if (!h->as_sidx) {
        CK(h, halloc(h, &h->as_sidx, h->n));
        CK(h, halloc(h, &h->as_c, h->n));
        CK(h, halloc(h, &h->as_sgn, h->n));
        CK(h, halloc(h, &h->as_u, h->n));
        CK(h, halloc(h, &h->as_q, h->m));
        CK(h, halloc(h, &h->as_rowcnt, h->m + 4));
        const int64_t cap = int64_t(h->sms) * 4;
        int64_t blocks = (h->n + kBlock - 1) / kBlock;
        h->as_blocks = int(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
        CK(h, halloc(h, &h->as_part, 3 * int64_t(h->as_blocks)));
    }
    if (tau > h->as_tau_cap) {
        CK(h, cudaStreamSynchronize(h->stream));
        hfree(h, h->as_H);
        hfree(h, h->as_S);
        h->as_H = nullptr;
        h->as_S = nullptr;
        h->as_tau_cap = 0;
        CK(h, halloc(h, &h->as_H, tau));
        CK(h, halloc(h, &h->as_S, tau));
        h->as_tau_cap = tau;
    }
    return PCDM_OK;
}

// Relative residual ||A_S^T q - c|| / ||c|| over S (and sum_p w_p u_{i_p}).
template <typename VT, typename XT>
pcdm_status as_residual(pcdm_handle h, int64_t nS, const double *u, const double *w, double *rel, double *wu)
{
    CK(h, ActiveSetKernels<VT, XT>::resid(static_cast<const ColDesc<XT> *>(h->desc), h->prow,
                                          static_cast<const VT *>(h->pval), h->as_sidx, h->as_c, nS, h->as_q, w, u,
                                          h->as_part, h->as_blocks, h->stream));
    std::vector<double> part(size_t(3 * h->as_blocks));
    CK(h, cudaMemcpyAsync(part.data(), h->as_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->stream));
    pcdm_status s = sync_check(h);
    if (s != PCDM_OK) return s;
    double rr = 0.0, cc = 0.0, s_wu = 0.0;
    for (int b = 0; b < h->as_blocks; ++b) {
        rr += part[size_t(3 * b)];
        cc += part[size_t(3 * b + 1)];
        s_wu += part[size_t(3 * b + 2)];
    }
    *rel = cc > 0.0 ? std::sqrt(rr / cc) : std::sqrt(rr);
    if (wu) *wu = s_wu;
    h->st_kernels += 1;
    return PCDM_OK;
}

// Coordinate descent on Q(u) = 1/2 ||A_S u - y||^2 - c^T u over the support S
// of x: polish (u = x, y = b, c = -lambda sign(x_S)) or backward (u = as_u from
// 0, y = 0, c = dL/dx on S).  q = A_S u - y is kept in as_q and recomputed
// exactly before every convergence check.
template <typename VT, typename XT>
pcdm_status as_solve(pcdm_handle h, bool backward, const double *dx_dev, int64_t tau_req, uint64_t seed,
                     double tol, int64_t max_iters, int64_t *iters, double *rel_out, double *dlambda)
{
    const ColDesc<XT> *desc = static_cast<const ColDesc<XT> *>(h->desc);
    const VT *pval = static_cast<const VT *>(h->pval);
    cudaStream_t st = h->stream;
    pcdm_status s = ensure_as(h, 1);
    if (s != PCDM_OK) return s;
    // S, |S|
    int *cnt_dev = h->as_rowcnt + h->m;
    CK(h, launch_compact_support(h->x, h->n, h->as_sidx, cnt_dev, st));
    int hcnt[2] = {0, 0};
    CK(h, cudaMemcpyAsync(hcnt, cnt_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    s = sync_check(h);
    if (s != PCDM_OK) return s;
    const int64_t nS = hcnt[0];
    double *u = backward ? h->as_u : h->x;
    if (backward) CK(h, cudaMemsetAsync(h->as_u, 0, sizeof(double) * size_t(h->n), st));
    if (nS == 0) {
        if (backward) CK(h, cudaMemsetAsync(h->as_q, 0, sizeof(double) * size_t(h->m), st));
        if (iters) *iters = 0;
        if (rel_out) *rel_out = 0.0;
        if (dlambda) *dlambda = 0.0;
        return PCDM_OK;
    }
    const int64_t tau = tau_req > 0 ? (tau_req < nS ? tau_req : nS) : nS;
    s = ensure_as(h, tau);
    if (s != PCDM_OK) return s;
    CK(h, launch_as_linear(h->x, backward ? dx_dev : nullptr, h->as_sidx, nS, h->lambda, h->as_c, h->as_sgn, st));
    // omega_S: the largest row count of A_S
    CK(h, cudaMemsetAsync(h->as_rowcnt, 0, sizeof(int) * size_t(h->m + 4), st));
    CK(h, ActiveSetKernels<VT, XT>::rowcount(desc, h->prow, h->as_sidx, nS, h->as_rowcnt, st));
    CK(h, launch_max_int(h->as_rowcnt, h->m, cnt_dev + 1, st));
    CK(h, cudaMemcpyAsync(hcnt, cnt_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    s = sync_check(h);
    if (s != PCDM_OK) return s;
    const double inv_beta = 1.0 / beta_nice(hcnt[1], tau, nS);
    h->st_kernels += 4;

    auto exact_q = [&]() -> pcdm_status {
        if (backward)
            CK(h, cudaMemsetAsync(h->as_q, 0, sizeof(double) * size_t(h->m), st));
        else
            CK(h, launch_neg_store<double>(h->as_q, h->b, h->m, st));
        CK(h, ActiveSetKernels<VT, XT>::refresh(desc, h->prow, pval, h->as_sidx, nS, u, h->as_q, st));
        h->st_kernels += 2;
        return PCDM_OK;
    };
    s = exact_q();
    if (s != PCDM_OK) return s;
    double rel = 0.0, wu = 0.0;
    s = as_residual<VT, XT>(h, nS, u, h->as_sgn, &rel, &wu);
    if (s != PCDM_OK) return s;
    const int64_t check = 16;
    int64_t done = 0, k = 0;
    while (rel > tol && done < max_iters) {
        const int64_t chunk = check < max_iters - done ? check : max_iters - done;
        for (int64_t it = 0; it < chunk; ++it, ++k) {
            CK(h, ActiveSetKernels<VT, XT>::gather(desc, h->prow, pval, h->as_sidx, h->as_c, nS, tau, seed, k,
                                                   inv_beta, h->as_q, u, h->as_H, h->as_S, st));
            CK(h, ActiveSetKernels<VT, XT>::scatter(desc, h->prow, pval, tau, h->as_H, h->as_S, h->as_q, st));
        }
        h->st_kernels += 2 * chunk;
        done += chunk;
        s = exact_q();
        if (s != PCDM_OK) return s;
        s = as_residual<VT, XT>(h, nS, u, h->as_sgn, &rel, &wu);
        if (s != PCDM_OK) return s;
    }
    if (iters) *iters = done;
    if (rel_out) *rel_out = rel;
    if (dlambda) *dlambda = -wu;
    if (!backward) {
        s = do_refresh(h);   // g = A x - b for the polished x
        if (s != PCDM_OK) return s;
        h->sample_valid = false;
    }
    s = sync_check(h);
    if (s != PCDM_OK) return s;
    if (rel > tol) return set_err(h, PCDM_ENOTCONV, "max_iters reached before the active-set tolerance");
    return PCDM_OK;
}

}  // namespace

extern "C" {

pcdm_status pcdm_polish(pcdm_handle h, int64_t tau, uint64_t seed, double tol, int64_t max_iters, int64_t *iters,
                        double *rel_res)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (h->problem != PCDM_PROBLEM_LASSO) return set_err(h, PCDM_EINVAL, "pcdm_polish applies to LASSO handles only");
    if (tau < 0 || max_iters < 0 || !(tol >= 0.0)) return set_err(h, PCDM_EINVAL, "bad tau, max_iters or tol");
    return dispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return as_solve<VT, XT>(h, false, nullptr, tau, seed, tol, max_iters, iters, rel_res, nullptr);
    });
}

pcdm_status pcdm_backward(pcdm_handle h, const double *dx, int32_t dx_on_device, double *db, int32_t db_on_device,
                          double *dlambda, int64_t tau, uint64_t seed, double tol, int64_t max_iters, int64_t *iters,
                          double *rel_res)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (h->problem != PCDM_PROBLEM_LASSO) return set_err(h, PCDM_EINVAL, "pcdm_backward applies to LASSO handles only");
    if (!dx) return set_err(h, PCDM_EINVAL, "dx is NULL");
    if (tau < 0 || max_iters < 0 || !(tol >= 0.0)) return set_err(h, PCDM_EINVAL, "bad tau, max_iters or tol");
    s = ensure_as(h, 1);
    if (s != PCDM_OK) return s;
    const double *dx_dev = dx;
    if (!dx_on_device) {
        if (!h->as_dx) CK(h, halloc(h, &h->as_dx, h->n));
        CK(h, cudaMemcpyAsync(h->as_dx, dx, sizeof(double) * size_t(h->n), cudaMemcpyHostToDevice, h->stream));
        dx_dev = h->as_dx;
    }
    double dl = 0.0;
    s = dispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return as_solve<VT, XT>(h, true, dx_dev, tau, seed, tol, max_iters, iters, rel_res, &dl);
    });
    if (s != PCDM_OK && s != PCDM_ENOTCONV) return s;
    if (db) {
        CK(h, cudaMemcpyAsync(db, h->as_q, sizeof(double) * size_t(h->m), copy_kind(1, db_on_device), h->stream));
        pcdm_status s2 = sync_check(h);
        if (s2 != PCDM_OK) return s2;
    }
    if (dlambda) *dlambda = dl;
    return s;
}

pcdm_status pcdm_set_b(pcdm_handle h, const void *b, int32_t b_dtype, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (h->problem != PCDM_PROBLEM_LASSO) return set_err(h, PCDM_EINVAL, "pcdm_set_b applies to LASSO handles only");
    if (!b) return set_err(h, PCDM_EINVAL, "b is NULL");
    if (b_dtype != PCDM_F64 && b_dtype != PCDM_F32) return set_err(h, PCDM_EINVAL, "b_dtype must be F64 or F32");
    cudaStream_t st = h->stream;
    // stage in the refresh buffer (m doubles), then validate before replacing b
    double *stage = h->g64;
    if (b_dtype == PCDM_F64) {
        CK(h, cudaMemcpyAsync(stage, b, sizeof(double) * size_t(h->m), copy_kind(on_device, 1), st));
    } else {
        CK(h, cudaMemcpyAsync(h->b, b, sizeof(float) * size_t(h->m), copy_kind(on_device, 1), st));
        CK(h, launch_convert_b(h->b, 1, h->m, stage, st));
    }
    int *flags = h->status + 1;
    int *hflags = reinterpret_cast<int *>(h->host_buf + 10);
    CK(h, cudaMemsetAsync(flags, 0, sizeof(int), st));
    CK(h, launch_check_finite(stage, h->m, flags, st));
    CK(h, cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (*hflags) {
        // b was overwritten only in the FP32 case; recover it from nothing is not possible,
        // so the handle refuses further work until pcdm_set_b succeeds or pcdm_reset runs
        CK(h, cudaMemsetAsync(flags, 0, sizeof(int), st));
        if (b_dtype != PCDM_F64) h->failed = true;
        return set_err(h, PCDM_EINVAL, "a non-finite value in b");
    }
    CK(h, cudaMemcpyAsync(h->b, stage, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice, st));
    h->last_solve_iters = 0;
    s = do_refresh(h);
    if (s != PCDM_OK) return s;
    h->sample_valid = false;
    return sync_check(h);
}

pcdm_status pcdm_support_size(pcdm_handle h, int64_t *count)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!count) return set_err(h, PCDM_EINVAL, "count is NULL");
    s = ensure_as(h, 1);
    if (s != PCDM_OK) return s;
    int *cnt_dev = h->as_rowcnt + h->m;
    CK(h, launch_compact_support(h->x, h->n, h->as_sidx, cnt_dev, h->stream));
    int hc = 0;
    CK(h, cudaMemcpyAsync(&hc, cnt_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    s = sync_check(h);
    if (s != PCDM_OK) return s;
    *count = hc;
    return PCDM_OK;
}

pcdm_status pcdm_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S_device, void *cuda_stream)
{
    if (n < 1 || n > 2147483647LL || tau < 0 || tau > n || k < 0)
        return set_err(nullptr, PCDM_EINVAL, "need 1 <= n < 2^31, 0 <= tau <= n, k >= 0");
    if (tau > 0 && !S_device) return set_err(nullptr, PCDM_EINVAL, "S_device is NULL");
    cudaError_t e = launch_sample(seed, k, n, tau, S_device, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "launch_sample");
    return PCDM_OK;
}

pcdm_status pcdm_omega_noalloc(const pcdm_csc *A, int64_t *omega, void *cuda_stream)
{
    // Every check that needs no device comes first; nothing below allocates.
    if (!A || !omega) return set_err(nullptr, PCDM_EINVAL, "A or omega is NULL");
    if (A->on_device != 1) return set_err(nullptr, PCDM_EINVAL, "A must be in device memory (on_device = 1)");
    if (A->m < 1 || A->n < 1 || A->n > 2147483647LL || A->nnz < 0)
        return set_err(nullptr, PCDM_EINVAL, "need 1 <= m, n < 2^31 and nnz >= 0");
    if (A->m > PCDM_NOALLOC_MAX_ROWS)
        return set_err(nullptr, PCDM_EINVAL, "m exceeds PCDM_NOALLOC_MAX_ROWS (" +
                                                 std::to_string(PCDM_NOALLOC_MAX_ROWS) + ")");
    if (!A->col_ptr || (A->nnz > 0 && !A->row_idx)) return set_err(nullptr, PCDM_EINVAL, "col_ptr or row_idx is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    int *cnt = nullptr, *tail = nullptr;
    e = noalloc_rows_scratch(dev, &cnt, &tail);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the row-count scratch");
    // counters and the flags / result words start at zero
    e = cudaMemsetAsync(cnt, 0, size_t(A->m) * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tail, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = launch_rows_checked(A->col_ptr, A->row_idx, A->m, A->n, A->nnz, cnt, tail, st);
    if (e == cudaSuccess) e = launch_max_int(cnt, A->m, tail + 1, st);
    int host[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tail, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pcdm_omega_noalloc");
    if (host[0] & FLAG_COLPTR) return set_err(nullptr, PCDM_EINVAL, "col_ptr not monotone from 0 to nnz");
    if (host[0] & FLAG_ROW_RANGE) return set_err(nullptr, PCDM_EINVAL, "a row index outside [0, m)");
    if (host[0] & FLAG_ROW_ORDER) return set_err(nullptr, PCDM_EINVAL, "rows of a column not strictly increasing");
    *omega = host[1];
    return PCDM_OK;
}

// ---------------------------------------------------------------------------
// Asynchronous mode.
}  // extern "C"
namespace {

template <typename VT, typename XT>
pcdm_status async_t(pcdm_handle h, int64_t updates, uint64_t seed, int32_t threads, int64_t *used_threads)
{
    IterArgs<VT, XT> a = iter_args<VT, XT>(h, 1, seed);
    const int cap = Kernels<VT, XT>::async_max_blocks();
    if (cap <= 0) return set_err(h, PCDM_ECUDA, "occupancy query failed");
    int64_t T = threads > 0 ? threads : int64_t(cap) * kBlock;
    if (T > h->n) T = h->n;
    if (T < 1) T = 1;
    const int64_t blocks = (T + kBlock - 1) / kBlock;
    double e1 = 0.0, e2 = 0.0;
    sampling_moments(PCDM_SAMPLING_INDEPENDENT, h->n, T, 1.0, &e1, &e2);
    a.inv_beta = 1.0 / beta_du(h->omega, e1, e2, h->n);
    cudaEvent_t e0 = nullptr, ev1 = nullptr;
    if (h->opts.profile) {
        CK(h, take_event(h, &e0));
        CK(h, take_event(h, &ev1));
        CK(h, cudaEventRecord(e0, h->stream));
    }
    CK(h, Kernels<VT, XT>::async(a, int(blocks), uint64_t(T), h->async_u, uint64_t(updates), h->stream));
    if (h->opts.profile) {
        CK(h, cudaEventRecord(ev1, h->stream));
        h->ev_pending.emplace_back(e0, ev1);
    }
    h->async_u += uint64_t(updates);
    h->g2_valid = false;
    h->sample_valid = false;
    h->st_updates += updates;
    h->st_launches += 1;
    h->st_kernels += 1;
    if (used_threads) *used_threads = T;
    return PCDM_OK;
}

}  // namespace
extern "C" {

pcdm_status pcdm_step_async(pcdm_handle h, int64_t updates, uint64_t seed, int32_t threads)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (h->problem != PCDM_PROBLEM_LASSO) return set_err(h, PCDM_EINVAL, "pcdm_step_async applies to LASSO handles only");
    if (h->opts.deterministic_scatter)
        return set_err(h, PCDM_EINVAL, "the asynchronous mode has no fixed order (deterministic_scatter handle)");
    if (updates < 0 || threads < 0) return set_err(h, PCDM_EINVAL, "updates and threads must be >= 0");
    if (updates == 0) return PCDM_OK;
    s = dispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return async_t<VT, XT>(h, updates, seed, threads, nullptr);
    });
    if (s != PCDM_OK) return s;
    return sync_check(h);
}

pcdm_status pcdm_solve_async(pcdm_handle h, uint64_t seed, double rel_gap_tol, int64_t max_updates, int32_t threads,
                             int64_t *updates_done, double *rel_gap)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (h->problem != PCDM_PROBLEM_LASSO) return set_err(h, PCDM_EINVAL, "pcdm_solve_async applies to LASSO handles only");
    if (h->opts.deterministic_scatter)
        return set_err(h, PCDM_EINVAL, "the asynchronous mode has no fixed order (deterministic_scatter handle)");
    if (max_updates < 0 || threads < 0 || !(rel_gap_tol >= 0.0))
        return set_err(h, PCDM_EINVAL, "bad max_updates, threads or tolerance");
    const int64_t epoch = h->n;   // updates between the first checks
    int64_t every = epoch, done = 0, prev = 0;
    double rec[9];
    s = do_gap(h, rec);
    if (s != PCDM_OK) return s;
    double rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300), rel_prev = rel;
    while (rel > rel_gap_tol && done < max_updates) {
        const int64_t chunk = every < max_updates - done ? every : max_updates - done;
        s = dispatch(h, [&](auto *vt, auto *xt) {
            using VT = std::remove_pointer_t<decltype(vt)>;
            using XT = std::remove_pointer_t<decltype(xt)>;
            return async_t<VT, XT>(h, chunk, seed, threads, nullptr);
        });
        if (s != PCDM_OK) return s;
        prev = done;
        done += chunk;
        rel_prev = rel;
        s = do_gap(h, rec);   // refreshes g exactly
        if (s != PCDM_OK) return s;
        rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300);
        every = pcdm_next_check_interval(epoch, prev, rel_prev, done, rel, rel_gap_tol);
    }
    if (updates_done) *updates_done = done;
    if (rel_gap) *rel_gap = rel;
    if (rel > rel_gap_tol) return set_err(h, PCDM_ENOTCONV, "max_updates reached before the gap tolerance");
    return PCDM_OK;
}

pcdm_status pcdm_set_tuning(pcdm_handle h, const pcdm_tuning *t)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!t) {
        h->tune_kernel = -1;
        h->tune_W = 0;
        h->tune_threads = 0;
        h->tune_heads = 1;
        h->tune_zc = -1;
        return PCDM_OK;
    }
    if (t->heads != 0 && t->heads != 1) return set_err(h, PCDM_EINVAL, "heads must be 0 or 1");
    if (t->zero_cert < -1 || t->zero_cert > 1) return set_err(h, PCDM_EINVAL, "zero_cert must be -1, 0 or 1");
    if (h->problem != PCDM_PROBLEM_LASSO && t->kernel == 3)
        return set_err(h, PCDM_EINVAL, "the SVM dual and logistic regression run in kernels 0, 1 and 2");
    const bool lanes_ok = t->lanes_per_col == 1 || t->lanes_per_col == 2 || t->lanes_per_col == 4 ||
                          t->lanes_per_col == 8 || t->lanes_per_col == 16 || t->lanes_per_col == 32;
    if (t->kernel < 0 || t->kernel > 5 || !lanes_ok)
        return set_err(h, PCDM_EINVAL, "kernel must be 0..5 and lanes_per_col a power of two up to 32");
    if (((t->kernel == 0 || t->kernel == 4) && (t->threads_per_block < 32 || t->threads_per_block > kPipeMaxBlock)) ||
        (t->kernel == 5 && (t->threads_per_block < 32 || t->threads_per_block > kWarpMaxBlock)) ||
        (t->kernel == 3 && (t->threads_per_block < 32 || t->threads_per_block > kPipeRoundsMaxBlock)) ||
        t->threads_per_block % 32 != 0)
        return set_err(h, PCDM_EINVAL, "threads_per_block must be a multiple of 32 within the kernel's limit");
    h->tune_kernel = t->kernel;
    h->tune_W = t->lanes_per_col;
    h->tune_threads = t->threads_per_block;
    h->tune_heads = t->heads;
    h->tune_zc = t->zero_cert;
    return PCDM_OK;
}

pcdm_status pcdm_autotune(pcdm_handle h, int64_t tau, int64_t trial_iters, pcdm_tuning *best)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->n || trial_iters < 1) return set_err(h, PCDM_EINVAL, "bad tau or trial_iters");
    if (h->opts.sampling != PCDM_SAMPLING_NICE || !h->opts.fused || h->opts.deterministic_scatter)
        return set_err(h, PCDM_EINVAL, "autotuning applies to the fused tau-nice iteration kernels");
    s = ensure_tau(h, tau);
    if (s != PCDM_OK) return s;
    // the state the trials start from, restored after each one and at the end
    const size_t xbytes = sizeof(double) * size_t(h->n), gbytes = size_t(h->m) * size_t(dtype_bytes(h->xg_dtype));
    double *x0 = nullptr;
    void *g0 = nullptr;
    CK(h, halloc(h, &x0, h->n));
    cudaError_t e = halloc_bytes(h, &g0, int64_t(gbytes));
    if (e != cudaSuccess) {
        hfree(h, x0);
        return cuda_fail(h, e, "autotune state copy");
    }
    const int64_t k0 = h->k;
    const int64_t st_it = h->st_iterations, st_up = h->st_updates, st_la = h->st_launches, st_ke = h->st_kernels;
    const double st_ms = h->st_kernel_ms;
    const int keep[5] = {h->tune_kernel, h->tune_W, h->tune_threads, h->tune_heads, h->tune_zc};
    auto restore = [&]() -> pcdm_status {
        CK(h, cudaMemcpyAsync(h->x, x0, xbytes, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->g, g0, gbytes, cudaMemcpyDeviceToDevice, h->stream));
        h->k = k0;
        h->g2_valid = false;
        h->sample_valid = false;
        return PCDM_OK;
    };
    CK(h, cudaMemcpyAsync(x0, h->x, xbytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(g0, h->g, gbytes, cudaMemcpyDeviceToDevice, h->stream));
    struct Cand {
        int kernel, W, threads, heads, zc;
    };
    // the zero-step certificate is a choice of the FP64 form of LASSO only
    const bool zc_choice = h->xg_dtype == PCDM_F64 && h->problem == PCDM_PROBLEM_LASSO;
    std::vector<Cand> cands;
    for (int zc : {1, 0}) {
        if (zc == 0 && !zc_choice) continue;
        for (int hd : {1, 0})
            for (int t : {128, 192, 256, 320, 384, 448}) cands.push_back({0, 1, t, hd, zc_choice ? zc : -1});
    }
    for (int W : {1, 2, 4, 8, 16, 32}) cands.push_back({1, W, 0, 1, -1});
    for (int W : {1, 4, 16}) cands.push_back({2, W, 0, 1, -1});
    for (int t : {128, 256}) cands.push_back({3, 1, t, 1, -1});
    for (int t : {128, 256, 448}) cands.push_back({4, 1, t, 1, -1});
    for (int t : {128, 256, 512}) cands.push_back({5, 1, t, 1, -1});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    Cand bestc{-1, 0, 0, 1, -1};
    double best_us = 0.0;
    pcdm_status rs = PCDM_OK;
    for (const Cand &c : cands) {
        if (c.kernel == 0) {
            // the pipelined kernel must hold tau positions at this block size
            FusedShape sh;
            bool ok = false;
            dispatch(h, [&](auto *vt, auto *xt) {
                using VT = std::remove_pointer_t<decltype(vt)>;
                using XT = std::remove_pointer_t<decltype(xt)>;
                const int save_W = h->W;
                h->W = 1;
                ok = pipe_shape<VT, XT>(h, tau, &sh, c.threads);
                h->W = save_W;
                return PCDM_OK;
            });
            if (!ok) continue;
        }
        if (c.kernel == 4) {
            // the streaming kernel must hold tau positions at this block size
            FusedShape sh;
            bool ok = false;
            dispatch(h, [&](auto *vt, auto *xt) {
                using VT = std::remove_pointer_t<decltype(vt)>;
                using XT = std::remove_pointer_t<decltype(xt)>;
                ok = stream_shape<VT, XT>(h, tau, &sh, c.threads);
                return PCDM_OK;
            });
            if (!ok) continue;
        }
        if (c.kernel == 5) {
            // the warp-cooperative kernel must hold tau positions at this block size
            FusedShape sh;
            bool ok = false;
            dispatch(h, [&](auto *vt, auto *xt) {
                using VT = std::remove_pointer_t<decltype(vt)>;
                using XT = std::remove_pointer_t<decltype(xt)>;
                ok = warp_shape<VT, XT>(h, tau, &sh, c.threads);
                return PCDM_OK;
            });
            if (!ok) continue;
        }
        if (c.kernel == 0 && c.heads && h->head_off) continue;   // the heads do not fit
        if (h->problem != PCDM_PROBLEM_LASSO && c.kernel == 3) continue;
        h->tune_kernel = c.kernel;
        h->tune_W = c.W;
        h->tune_threads = c.threads;
        h->tune_heads = c.heads;
        h->tune_zc = c.zc;
        if ((rs = restore()) != PCDM_OK) break;
        if ((rs = pcdm_step(h, tau, 2, 0x5eedULL)) != PCDM_OK) break;   // warm-up (first launch of a shape)
        if ((rs = restore()) != PCDM_OK) break;
        if ((e = cudaEventRecord(e0, h->stream)) != cudaSuccess) break;
        if ((rs = pcdm_step(h, tau, trial_iters, 0x5eedULL)) != PCDM_OK) break;
        if ((e = cudaEventRecord(e1, h->stream)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        const double us = 1e3 * double(ms) / double(trial_iters);
        if (bestc.kernel < 0 || us < best_us) {
            bestc = c;
            best_us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs == PCDM_OK && e == cudaSuccess) rs = restore();
    if (rs == PCDM_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    hfree(h, x0);
    hfree(h, g0);
    h->st_iterations = st_it;
    h->st_updates = st_up;
    h->st_launches = st_la;
    h->st_kernels = st_ke;
    h->st_kernel_ms = st_ms;
    for (auto &pr : h->ev_pending) {   // timings of the trials are not kept
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    if (rs != PCDM_OK) {
        h->tune_kernel = keep[0];
        h->tune_W = keep[1];
        h->tune_threads = keep[2];
        h->tune_heads = keep[3];
        h->tune_zc = keep[4];
        return rs;
    }
    h->tune_kernel = bestc.kernel;
    h->tune_W = bestc.W;
    h->tune_threads = bestc.threads;
    h->tune_heads = bestc.heads;
    h->tune_zc = bestc.zc;
    if (best) {
        best->kernel = bestc.kernel;
        best->lanes_per_col = bestc.W;
        best->threads_per_block = bestc.threads;
        best->heads = bestc.heads && !h->head_off ? 1 : 0;
        // the warp-cooperative kernel's certificate follows the share of moving coordinates (tune_zc -1)
        best->zero_cert = !zc_choice ? 0 : bestc.kernel == 0 ? bestc.zc : bestc.kernel == 5 ? -1 : 0;
        best->us_per_iteration = best_us;
    }
    return PCDM_OK;
}

pcdm_status pcdm_sample_kind(int32_t kind, uint64_t seed, int64_t k, int64_t n, int64_t tau, double p_b,
                             int32_t *S_device, uint8_t *keep_device, void *cuda_stream)
{
    if (kind < PCDM_SAMPLING_NICE || kind > PCDM_SAMPLING_BINOMIAL)
        return set_err(nullptr, PCDM_EINVAL, "unknown sampling");
    if (n < 1 || n > 2147483647LL || tau < 0 || tau > n || k < 0)
        return set_err(nullptr, PCDM_EINVAL, "need 1 <= n < 2^31, 0 <= tau <= n, k >= 0");
    if (kind == PCDM_SAMPLING_BINOMIAL && !(p_b > 0.0 && p_b <= 1.0))
        return set_err(nullptr, PCDM_EINVAL, "p_b must be in (0, 1]");
    if (tau > 0 && !S_device) return set_err(nullptr, PCDM_EINVAL, "S_device is NULL");
    cudaError_t e = launch_sample_kind(kind, seed, k, n, tau, binomial_threshold(p_b), S_device, nullptr,
                                       kind == PCDM_SAMPLING_INDEPENDENT ? nullptr : keep_device,
                                       static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "launch_sample_kind");
    return PCDM_OK;
}

pcdm_status pcdm_set_memory_cache(uint64_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = handle_pool(dev, &pool);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        g_cache_limit = bytes;
        uint64_t limit = bytes;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &limit);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pcdm_set_memory_cache");
    return PCDM_OK;
}

pcdm_status pcdm_release_cached_memory(void)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = handle_pool(dev, &pool);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pcdm_release_cached_memory");
    return PCDM_OK;
}

pcdm_status pcdm_selftest_barrier_timeout(uint64_t timeout_ns, void *cuda_stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (timeout_ns == 0 || timeout_ns > 10000000000ull)
        return set_err(nullptr, PCDM_EINVAL, "timeout_ns must be in (0, 1e10]");
    unsigned long long *bar = nullptr;
    int *status = nullptr;
    int host_status = -1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&bar), sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&status), sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_barrier_selftest(bar, status, timeout_ns, 4, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bar) cudaFree(bar);
    if (status) cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "barrier self-test");
    if (host_status == DEV_TIMEOUT) return set_err(nullptr, PCDM_ETIMEOUT, "barrier wait timed out as designed");
    return PCDM_OK;
}

}  // extern "C"

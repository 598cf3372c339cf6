// Host implementation of the batched entry points of include/pcdm.h
// (pcdm_batch_*): several LASSO problems that share A, solved together by the
// kernels of batch_kernels.cuh.  A's device layout, L and omega come from an
// ordinary handle created for the first right-hand side; this file adds the
// interleaved right-hand sides, iterates and residuals and runs the solve loop.
#include <cmath>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "pcdm_host.h"

using namespace pcdm;
using namespace pcdm_host;

struct pcdm_batch_ctx {
    pcdm_handle base = nullptr;   // owns A's layout (desc, prow, pval), L, omega, the stream
    int64_t nrhs = 0;
    int bp = 4;                   // lanes per column: nrhs rounded up to 4, 8, 16 or 32
    double *X = nullptr;          // n x bp FP64 iterates, X[i * bp + l]
    void *G = nullptr;            // m x bp residuals in the iterate dtype
    double *G64 = nullptr;        // m x bp FP64 refresh target (aliases G in the FP64 form)
    double *Bm = nullptr;         // m x bp right-hand sides, FP64
    void *H = nullptr;            // tau_cap x bp steps of the listed columns
    int32_t *list = nullptr;      // tau_cap: columns with a nonzero step in the current iteration
    unsigned *list_cnt = nullptr; // [2]
    int64_t tau_cap = 0;
    double *lam_d = nullptr;      // bp lambdas (0 for padding lanes)
    int *active_d = nullptr;      // bp flags
    double *stage = nullptr;      // staging for get_x / set_x
    int64_t stage_len = 0;
    unsigned long long *counters = nullptr;   // [3]
    unsigned long long *bar = nullptr;
    int *status = nullptr;
    double *gap_part = nullptr;
    double *gap_out = nullptr;    // bp x 9
    int gap_blocks = 0, gap_row_blocks = 0, refresh_blocks = 0;
    double *host_buf = nullptr;   // pinned: bp x 9 gap doubles, then status
    std::vector<double> lam;
    std::vector<int> active;
    int64_t k = 0;
    int64_t last_solve_iters = 0;   // iterations of the last pcdm_batch_solve (0 after create / reset)
    int tune_blocks_per_sm = 0;     // grid of the iteration kernel chosen by pcdm_batch_autotune (0: built-in rule)
    bool failed = false;
    std::string err;
    int64_t st_iterations = 0, st_updates = 0, st_launches = 0, st_kernels = 0, st_refreshes = 0, st_gaps = 0;
    double st_kernel_ms = 0.0;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
};

namespace {

pcdm_status berr(pcdm_batch_handle h, pcdm_status s, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_free_error = msg;
    return s;
}

pcdm_status bfail(pcdm_batch_handle h, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return berr(h, PCDM_ENOMEM, msg);
    }
    if (h) h->failed = true;
    return berr(h, PCDM_ECUDA, msg);
}

#define BCK(h, ...)                                                 \
    do {                                                            \
        cudaError_t e_ = (__VA_ARGS__);                             \
        if (e_ != cudaSuccess) return bfail((h), e_, #__VA_ARGS__); \
    } while (0)

cudaStream_t bstream(pcdm_batch_handle h) { return h->base->stream; }

void bfree_all(pcdm_batch_handle h)
{
    void *ptrs[] = {h->X, h->G, h->Bm, h->H, h->list, h->list_cnt, h->lam_d, h->active_d, h->stage,
                    h->counters, h->bar, h->status, h->gap_part, h->gap_out};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->G64 && static_cast<void *>(h->G64) != h->G) cudaFree(h->G64);
    if (h->host_buf) cudaFreeHost(h->host_buf);
    for (auto &pr : h->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
    if (h->base) pcdm_destroy(h->base);
}

pcdm_status busable(pcdm_batch_handle h)
{
    if (!h) return berr(nullptr, PCDM_EINVAL, "NULL batch handle");
    if (h->failed) return berr(h, PCDM_ESTATE, "batch handle is in a failed state (" + h->err + ")");
    return PCDM_OK;
}

pcdm_status bsync(pcdm_batch_handle h)
{
    int *hs = reinterpret_cast<int *>(h->host_buf + 9 * h->bp);
    BCK(h, cudaMemcpyAsync(hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, bstream(h)));
    BCK(h, cudaStreamSynchronize(bstream(h)));
    for (auto &pr : h->ev_pending) {
        float ms = 0.f;
        BCK(h, cudaEventElapsedTime(&ms, pr.first, pr.second));
        h->st_kernel_ms += ms;
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    if (*hs != DEV_OK) {
        h->failed = true;
        return berr(h, PCDM_ETIMEOUT, "a grid-barrier wait of the batched kernel ran out of its time budget");
    }
    return PCDM_OK;
}

cudaError_t btake_event(pcdm_batch_handle h, cudaEvent_t *e)
{
    if (!h->ev_free.empty()) {
        *e = h->ev_free.back();
        h->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

template <typename F>
pcdm_status bdispatch(pcdm_batch_handle h, F &&f)
{
    const pcdm_handle b = h->base;
    if (b->val_dtype == PCDM_F64 && b->xg_dtype == PCDM_F64) return f((double *)nullptr, (double *)nullptr);
    if (b->val_dtype == PCDM_F32 && b->xg_dtype == PCDM_F32) return f((float *)nullptr, (float *)nullptr);
    if (b->val_dtype == PCDM_BF16 && b->xg_dtype == PCDM_F32) return f((bf16_t *)nullptr, (float *)nullptr);
    return berr(h, PCDM_EINVAL, "unsupported dtype pair");
}

pcdm_status upload_controls(pcdm_batch_handle h)
{
    BCK(h, cudaMemcpyAsync(h->lam_d, h->lam.data(), sizeof(double) * size_t(h->bp), cudaMemcpyHostToDevice,
                           bstream(h)));
    BCK(h, cudaMemcpyAsync(h->active_d, h->active.data(), sizeof(int) * size_t(h->bp), cudaMemcpyHostToDevice,
                           bstream(h)));
    // the host vectors must stay unchanged until the copies ran
    return bsync(h);
}

pcdm_status ensure_btau(pcdm_batch_handle h, int64_t tau)
{
    if (tau <= h->tau_cap) return PCDM_OK;
    BCK(h, cudaStreamSynchronize(bstream(h)));
    if (h->list) cudaFree(h->list);
    if (h->H) cudaFree(h->H);
    h->list = nullptr;
    h->H = nullptr;
    h->tau_cap = 0;
    BCK(h, dalloc(&h->list, tau));
    BCK(h, dalloc_bytes(&h->H, tau * h->bp * dtype_bytes(h->base->xg_dtype)));
    h->tau_cap = tau;
    return PCDM_OK;
}

pcdm_status ensure_stage(pcdm_batch_handle h, int64_t len)
{
    if (len <= h->stage_len) return PCDM_OK;
    BCK(h, cudaStreamSynchronize(bstream(h)));
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_len = 0;
    BCK(h, dalloc(&h->stage, len));
    h->stage_len = len;
    return PCDM_OK;
}

template <typename VT, typename XT>
pcdm_status brefresh_t(pcdm_batch_handle h)
{
    const pcdm_handle b = h->base;
    const int64_t total = b->m * h->bp;
    BCK(h, launch_neg_store<double>(h->G64, h->Bm, total, bstream(h)));
    BCK(h, BatchKernels<VT, XT>::refresh(static_cast<const ColDesc<XT> *>(b->desc), b->prow,
                                         static_cast<const VT *>(b->pval), h->X, b->n, h->bp, h->G64,
                                         h->refresh_blocks, bstream(h)));
    if (sizeof(XT) == 4) BCK(h, launch_store_from_f64<float>(static_cast<float *>(h->G), h->G64, total, bstream(h)));
    h->st_refreshes += 1;
    h->st_kernels += sizeof(XT) == 4 ? 3 : 2;
    return PCDM_OK;
}

template <typename VT, typename XT>
pcdm_status bgap_t(pcdm_batch_handle h)
{
    pcdm_status s = brefresh_t<VT, XT>(h);
    if (s != PCDM_OK) return s;
    const pcdm_handle b = h->base;
    double *pc = h->gap_part;
    double *pr = h->gap_part + int64_t(h->gap_blocks) * h->bp * 3;
    BCK(h, BatchKernels<VT, XT>::gap_cols(static_cast<const ColDesc<XT> *>(b->desc), b->prow,
                                          static_cast<const VT *>(b->pval), h->G64, h->X, b->n, h->bp, pc,
                                          h->gap_blocks, bstream(h)));
    BCK(h, launch_batch_gap_rows(h->G64, h->Bm, b->m, h->bp, pr, h->gap_row_blocks, bstream(h)));
    BCK(h, launch_batch_gap_finish(pc, h->gap_blocks, pr, h->gap_row_blocks, h->bp, h->lam_d, h->gap_out,
                                   bstream(h)));
    BCK(h, cudaMemcpyAsync(h->host_buf, h->gap_out, sizeof(double) * 9 * size_t(h->bp), cudaMemcpyDeviceToHost,
                           bstream(h)));
    h->st_gaps += 1;
    h->st_kernels += 3;
    return bsync(h);
}

pcdm_status bdo_refresh(pcdm_batch_handle h)
{
    return bdispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return brefresh_t<VT, XT>(h);
    });
}

pcdm_status bdo_gap(pcdm_batch_handle h)
{
    return bdispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return bgap_t<VT, XT>(h);
    });
}

template <typename VT, typename XT>
pcdm_status bsegment_t(pcdm_batch_handle h, int64_t tau, uint64_t seed, int64_t iters)
{
    const pcdm_handle b = h->base;
    BatchArgs<VT, XT> a;
    a.desc = static_cast<const ColDesc<XT> *>(b->desc);
    a.prow = b->prow;
    a.pval = static_cast<const VT *>(b->pval);
    a.X = h->X;
    a.G = static_cast<XT *>(h->G);
    a.H = static_cast<XT *>(h->H);
    a.list = h->list;
    a.list_cnt = h->list_cnt;
    a.lambda = h->lam_d;
    a.active = h->active_d;
    a.inv_beta = 1.0 / beta_nice(b->omega, tau, b->n);
    a.n = b->n;
    a.tau = tau;
    a.seed = seed;
    a.counters = h->counters;
    a.bar = h->bar;
    a.status = h->status;
    a.timeout_ns = b->opts.barrier_timeout_ns ? b->opts.barrier_timeout_ns : kDefaultTimeoutNs;
    const int cap = BatchKernels<VT, XT>::iter_max_blocks(h->bp);
    if (cap <= 0) return berr(h, PCDM_ECUDA, "cooperative occupancy query failed");
    int64_t blocks = (tau * h->bp + kBatchBlock - 1) / kBatchBlock;
    if (h->tune_blocks_per_sm > 0 && int64_t(h->tune_blocks_per_sm) * b->sms < blocks)
        blocks = int64_t(h->tune_blocks_per_sm) * b->sms;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->opts.profile) {
        BCK(h, btake_event(h, &e0));
        BCK(h, btake_event(h, &e1));
        BCK(h, cudaEventRecord(e0, bstream(h)));
    }
    BCK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), bstream(h)));
    BCK(h, cudaMemsetAsync(h->list_cnt, 0, 2 * sizeof(unsigned), bstream(h)));
    BCK(h, BatchKernels<VT, XT>::iter(a, h->bp, int(blocks), h->k, iters, bstream(h)));
    if (b->opts.profile) {
        BCK(h, cudaEventRecord(e1, bstream(h)));
        h->ev_pending.emplace_back(e0, e1);
    }
    int64_t act = 0;
    for (int l = 0; l < h->bp; ++l) act += h->active[l] ? 1 : 0;
    h->k += iters;
    h->st_iterations += iters;
    h->st_updates += iters * tau * act;
    h->st_launches += 1;
    h->st_kernels += 1;
    return PCDM_OK;
}

pcdm_status bstep(pcdm_batch_handle h, int64_t tau, int64_t iters, uint64_t seed)
{
    pcdm_status s = ensure_btau(h, tau);
    if (s != PCDM_OK) return s;
    const int64_t every = h->base->opts.refresh_every;
    int64_t left = iters;
    while (left > 0) {
        int64_t chunk = left < kMaxItersPerLaunch ? left : kMaxItersPerLaunch;
        if (every > 0) {
            const int64_t to_refresh = every - (h->k % every);   // refresh after iteration k when (k+1) % every == 0
            if (chunk > to_refresh) chunk = to_refresh;
        }
        s = bdispatch(h, [&](auto *vt, auto *xt) {
            using VT = std::remove_pointer_t<decltype(vt)>;
            using XT = std::remove_pointer_t<decltype(xt)>;
            return bsegment_t<VT, XT>(h, tau, seed, chunk);
        });
        if (s != PCDM_OK) return s;
        left -= chunk;
        if (every > 0 && h->k % every == 0) {
            s = bdo_refresh(h);
            if (s != PCDM_OK) return s;
        }
    }
    return PCDM_OK;
}

pcdm_status breset_state(pcdm_batch_handle h)
{
    const pcdm_handle b = h->base;
    BCK(h, cudaMemsetAsync(h->X, 0, sizeof(double) * size_t(b->n) * size_t(h->bp), bstream(h)));
    const int64_t total = b->m * h->bp;
    if (b->xg_dtype == PCDM_F64)
        BCK(h, launch_neg_store<double>(static_cast<double *>(h->G), h->Bm, total, bstream(h)));
    else
        BCK(h, launch_neg_store<float>(static_cast<float *>(h->G), h->Bm, total, bstream(h)));
    BCK(h, cudaMemsetAsync(h->status, 0, sizeof(int), bstream(h)));
    h->k = 0;
    h->last_solve_iters = 0;
    h->failed = false;
    return PCDM_OK;
}

}  // namespace

pcdm_status pcdm_batch_create(const pcdm_csc *A, int64_t nrhs, const void *B, int32_t b_dtype, const double *lambdas,
                              const pcdm_opts *opts, void *cuda_stream, pcdm_batch_handle *out)
{
    if (!out) return berr(nullptr, PCDM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!A || !B || !lambdas) return berr(nullptr, PCDM_EINVAL, "A, B or lambdas is NULL");
    if (nrhs < 1 || nrhs > 32) return berr(nullptr, PCDM_EINVAL, "nrhs must be in [1, 32]");
    for (int64_t l = 0; l < nrhs; ++l)
        if (!(lambdas[l] >= 0.0) || !std::isfinite(lambdas[l]))
            return berr(nullptr, PCDM_EINVAL, "every lambda must be finite and >= 0");
    if (b_dtype != PCDM_F64 && b_dtype != PCDM_F32) return berr(nullptr, PCDM_EINVAL, "b_dtype must be F64 or F32");
    if (opts && opts->sampling != PCDM_SAMPLING_NICE)
        return berr(nullptr, PCDM_EINVAL, "the batched solver runs the tau-nice sampling only");
    pcdm_handle base = nullptr;
    // A's validation and layout, with the first right-hand side
    pcdm_status s = pcdm_create(A, B, b_dtype, lambdas[0], opts, cuda_stream, &base);
    if (s != PCDM_OK) return s;

    pcdm_batch_ctx *h = new (std::nothrow) pcdm_batch_ctx();
    if (!h) {
        pcdm_destroy(base);
        return berr(nullptr, PCDM_ENOMEM, "host allocation failed");
    }
    h->base = base;
    h->nrhs = nrhs;
    h->bp = nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : 32;
    h->lam.assign(size_t(h->bp), 0.0);
    h->active.assign(size_t(h->bp), 0);
    for (int64_t l = 0; l < nrhs; ++l) {
        h->lam[size_t(l)] = lambdas[l];
        h->active[size_t(l)] = 1;
    }
    auto fail = [&](pcdm_status st) {
        g_free_error = h->err;
        bfree_all(h);
        delete h;
        return st;
    };
#define BCKC(...)                                                           \
    do {                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                     \
        if (e_ != cudaSuccess) return fail(bfail(h, e_, #__VA_ARGS__));     \
    } while (0)
    const int64_t m = base->m, n = base->n, bp = h->bp;
    const int64_t xb = dtype_bytes(base->xg_dtype);
    cudaStream_t st = base->stream;
    {
        const int64_t cap = int64_t(base->sms) * 8;
        int64_t gb = (n * bp + kBatchBlock - 1) / kBatchBlock;
        h->gap_blocks = int(gb < 1 ? 1 : (gb > cap ? cap : gb));
        h->refresh_blocks = h->gap_blocks;
        int64_t rb = (m * bp + kBlock - 1) / kBlock;
        h->gap_row_blocks = int(rb < 1 ? 1 : (rb > cap ? cap : rb));
    }
    BCKC(dalloc(&h->X, n * bp));
    BCKC(dalloc_bytes(&h->G, m * bp * xb));
    if (base->xg_dtype == PCDM_F64)
        h->G64 = static_cast<double *>(h->G);
    else
        BCKC(dalloc(&h->G64, m * bp));
    BCKC(dalloc(&h->Bm, m * bp));
    BCKC(dalloc(&h->lam_d, bp));
    BCKC(dalloc(&h->active_d, bp));
    BCKC(dalloc(&h->counters, 3));
    BCKC(dalloc(&h->list_cnt, 2));
    BCKC(dalloc(&h->bar, 1));
    BCKC(dalloc(&h->status, 4));
    BCKC(dalloc(&h->gap_part, int64_t(h->gap_blocks) * bp * 3 + int64_t(h->gap_row_blocks) * bp * 2));
    BCKC(dalloc(&h->gap_out, 9 * bp));
    BCKC(cudaMallocHost(reinterpret_cast<void **>(&h->host_buf), sizeof(double) * size_t(9 * bp + 8)));
    BCKC(cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), st));
    BCKC(cudaMemsetAsync(h->status, 0, 4 * sizeof(int), st));
    // right-hand sides: staged on the device when they are host memory, then interleaved
    const int64_t bbytes = dtype_bytes(b_dtype);
    const void *bsrc = B;
    double *tmp = nullptr;
    if (!A->on_device) {
        BCKC(dalloc(&tmp, (m * nrhs * bbytes + 7) / 8));
        BCKC(cudaMemcpyAsync(tmp, B, size_t(m * nrhs * bbytes), cudaMemcpyHostToDevice, st));
        bsrc = tmp;
    }
    cudaError_t e = launch_interleave(bsrc, b_dtype == PCDM_F32, m, int(nrhs), int(bp), h->Bm, st);
    int *flags = h->status + 1;
    if (e == cudaSuccess) e = launch_check_finite(h->Bm, m * bp, flags, st);
    int hflags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(bfail(h, e, "staging of the right-hand sides"));
    if (hflags) return fail(berr(h, PCDM_EINVAL, "a non-finite value in B"));
    BCKC(cudaMemsetAsync(flags, 0, sizeof(int), st));
    pcdm_status rs = breset_state(h);
    if (rs != PCDM_OK) return fail(rs);
    rs = upload_controls(h);
    if (rs != PCDM_OK) return fail(rs);
#undef BCKC
    *out = h;
    return PCDM_OK;
}

void pcdm_batch_destroy(pcdm_batch_handle h)
{
    if (!h) return;
    if (h->base) cudaStreamSynchronize(h->base->stream);
    bfree_all(h);
    delete h;
}

const char *pcdm_batch_last_error(pcdm_batch_handle h) { return h ? h->err.c_str() : g_free_error.c_str(); }

pcdm_status pcdm_batch_autotune(pcdm_batch_handle h, int64_t tau, int64_t trial_iters, int32_t *blocks_per_sm,
                                double *us_per_iteration)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    const pcdm_handle b = h->base;
    if (tau < 1 || tau > b->n || trial_iters < 1) return berr(h, PCDM_EINVAL, "bad tau or trial_iters");
    s = ensure_btau(h, tau);
    if (s != PCDM_OK) return s;
    s = bsync(h);
    if (s != PCDM_OK) return s;
    int cap = 0;
    bdispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        cap = BatchKernels<VT, XT>::iter_max_blocks(h->bp);
        return PCDM_OK;
    });
    if (cap <= 0) return berr(h, PCDM_ECUDA, "cooperative occupancy query failed");
    // the state the trials start from, restored after each one
    const size_t xbytes = sizeof(double) * size_t(b->n) * size_t(h->bp);
    const size_t gbytes = size_t(dtype_bytes(b->xg_dtype)) * size_t(b->m) * size_t(h->bp);
    double *x0 = nullptr;
    void *g0 = nullptr;
    BCK(h, dalloc(&x0, int64_t(b->n) * h->bp));
    cudaError_t e = dalloc_bytes(&g0, int64_t(gbytes));
    if (e != cudaSuccess) {
        cudaFree(x0);
        return berr(h, PCDM_ENOMEM, "autotune state copy");
    }
    unsigned long long c0[3] = {0, 0, 0};
    const int64_t k0 = h->k, st0[6] = {h->st_iterations, h->st_updates, h->st_launches, h->st_kernels,
                                       h->st_refreshes, h->st_gaps};
    const double ms0 = h->st_kernel_ms;
    const int keep = h->tune_blocks_per_sm;
    e = cudaMemcpy(c0, h->counters, sizeof(c0), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x0, h->X, xbytes, cudaMemcpyDeviceToDevice, bstream(h));
    if (e == cudaSuccess) e = cudaMemcpyAsync(g0, h->G, gbytes, cudaMemcpyDeviceToDevice, bstream(h));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    // candidates: 1, 2, ... blocks per SM up to the co-resident limit and the blocks tau needs
    const int64_t need = (tau * h->bp + kBatchBlock - 1) / kBatchBlock;
    int best = 0;
    double best_us = 0.0;
    for (int per_sm = 1; e == cudaSuccess && s == PCDM_OK && per_sm * b->sms <= cap; ++per_sm) {
        if (per_sm > 1 && int64_t(per_sm - 1) * b->sms >= need) break;
        h->tune_blocks_per_sm = per_sm;
        for (int rep = 0; rep < 2 && e == cudaSuccess && s == PCDM_OK; ++rep) {   // the first run warms up
            e = cudaEventRecord(t0, bstream(h));
            if (e != cudaSuccess) break;
            s = bdispatch(h, [&](auto *vt, auto *xt) {
                using VT = std::remove_pointer_t<decltype(vt)>;
                using XT = std::remove_pointer_t<decltype(xt)>;
                return bsegment_t<VT, XT>(h, tau, 0, trial_iters);
            });
            if (s != PCDM_OK) break;
            e = cudaEventRecord(t1, bstream(h));
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && rep == 1) {
                const double us = 1e3 * double(ms) / double(trial_iters);
                if (best == 0 || us < best_us) {
                    best = per_sm;
                    best_us = us;
                }
            }
            h->k = k0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->X, x0, xbytes, cudaMemcpyDeviceToDevice, bstream(h));
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->G, g0, gbytes, cudaMemcpyDeviceToDevice, bstream(h));
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->counters, c0, sizeof(c0), cudaMemcpyHostToDevice, bstream(h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(bstream(h));
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(x0);
    cudaFree(g0);
    h->k = k0;
    h->st_iterations = st0[0];
    h->st_updates = st0[1];
    h->st_launches = st0[2];
    h->st_kernels = st0[3];
    h->st_refreshes = st0[4];
    h->st_gaps = st0[5];
    h->st_kernel_ms = ms0;
    for (auto &pr : h->ev_pending) {   // the trials' profile events are not the handle's work
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    if (s != PCDM_OK) {
        h->tune_blocks_per_sm = keep;
        return s;
    }
    if (e != cudaSuccess) {
        h->tune_blocks_per_sm = keep;
        return berr(h, PCDM_ECUDA, std::string("pcdm_batch_autotune: ") + cudaGetErrorString(e));
    }
    h->tune_blocks_per_sm = best;
    if (blocks_per_sm) *blocks_per_sm = best;
    if (us_per_iteration) *us_per_iteration = best_us;
    return PCDM_OK;
}

pcdm_status pcdm_batch_step(pcdm_batch_handle h, int64_t tau, int64_t iters, uint64_t seed)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->base->n) return berr(h, PCDM_EINVAL, "tau must be in [1, n]");
    if (iters < 0) return berr(h, PCDM_EINVAL, "iters must be >= 0");
    s = bstep(h, tau, iters, seed);
    if (s != PCDM_OK) return s;
    return bsync(h);
}

pcdm_status pcdm_batch_refresh(pcdm_batch_handle h)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    s = bdo_refresh(h);
    if (s != PCDM_OK) return s;
    return bsync(h);
}

pcdm_status pcdm_batch_gap(pcdm_batch_handle h, double *primal, double *dual, double *gap)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    s = bdo_gap(h);
    if (s != PCDM_OK) return s;
    for (int64_t l = 0; l < h->nrhs; ++l) {
        const double *r = h->host_buf + 9 * l;
        if (primal) primal[l] = r[0];
        if (dual) dual[l] = r[1];
        if (gap) gap[l] = r[2];
    }
    return PCDM_OK;
}

pcdm_status pcdm_batch_solve(pcdm_batch_handle h, int64_t tau, uint64_t seed, double rel_gap_tol, int64_t max_iters,
                             int64_t *iters_done, double *rel_gaps)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->base->n) return berr(h, PCDM_EINVAL, "tau must be in [1, n]");
    if (max_iters < 0 || !(rel_gap_tol >= 0.0)) return berr(h, PCDM_EINVAL, "max_iters < 0 or bad tolerance");
    const int64_t epoch = (h->base->n + tau - 1) / tau;
    const bool fixed = h->base->opts.check_every > 0;
    int64_t every = fixed ? h->base->opts.check_every : first_check_interval(epoch, h->last_solve_iters);
    std::vector<double> rel(size_t(h->nrhs), 0.0);
    int64_t done = 0, prev_check = 0;
    double worst_prev = 0.0;
    for (;;) {
        s = bdo_gap(h);
        if (s != PCDM_OK) return s;
        double worst = 0.0;
        bool changed = false;
        for (int64_t l = 0; l < h->nrhs; ++l) {
            const double *r = h->host_buf + 9 * l;
            rel[size_t(l)] = r[2] / (r[0] > 1e-300 ? r[0] : 1e-300);
            const int want = rel[size_t(l)] > rel_gap_tol ? 1 : 0;
            // a problem that reached the tolerance is frozen for the rest of the solve
            if (h->active[size_t(l)] && !want) {
                h->active[size_t(l)] = 0;
                changed = true;
            }
            if (h->active[size_t(l)] && rel[size_t(l)] > worst) worst = rel[size_t(l)];
        }
        if (changed) {
            s = upload_controls(h);
            if (s != PCDM_OK) return s;
        }
        if (worst == 0.0 || done >= max_iters) break;
        if (done > 0 && !fixed)
            every = pcdm_next_check_interval(epoch, prev_check, worst_prev, done, worst, rel_gap_tol);
        worst_prev = worst;
        prev_check = done;
        const int64_t chunk = every < max_iters - done ? every : max_iters - done;
        s = bstep(h, tau, chunk, seed);
        if (s != PCDM_OK) return s;
        done += chunk;
    }
    bool all = true;
    for (int64_t l = 0; l < h->nrhs; ++l) {
        if (rel_gaps) rel_gaps[l] = rel[size_t(l)];
        if (rel[size_t(l)] > rel_gap_tol) all = false;
    }
    // the problems are active again for later calls
    for (int64_t l = 0; l < h->nrhs; ++l) h->active[size_t(l)] = 1;
    s = upload_controls(h);
    if (s != PCDM_OK) return s;
    if (iters_done) *iters_done = done;
    h->last_solve_iters = done;
    if (!all) return berr(h, PCDM_ENOTCONV, "max_iters reached before every problem met the gap tolerance");
    return PCDM_OK;
}

pcdm_status pcdm_batch_get_x(pcdm_batch_handle h, double *X_out, int32_t on_device)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    if (!X_out) return berr(h, PCDM_EINVAL, "X_out is NULL");
    const int64_t n = h->base->n;
    if (on_device) {
        BCK(h, launch_deinterleave(h->X, n, int(h->nrhs), h->bp, X_out, bstream(h)));
        return bsync(h);
    }
    s = ensure_stage(h, n * h->nrhs);
    if (s != PCDM_OK) return s;
    BCK(h, launch_deinterleave(h->X, n, int(h->nrhs), h->bp, h->stage, bstream(h)));
    BCK(h, cudaMemcpyAsync(X_out, h->stage, sizeof(double) * size_t(n * h->nrhs), cudaMemcpyDeviceToHost,
                           bstream(h)));
    return bsync(h);
}

pcdm_status pcdm_batch_set_x(pcdm_batch_handle h, const double *X_in, int32_t on_device)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    if (!X_in) return berr(h, PCDM_EINVAL, "X_in is NULL");
    const int64_t n = h->base->n;
    const void *src = X_in;
    if (!on_device) {
        s = ensure_stage(h, n * h->nrhs);
        if (s != PCDM_OK) return s;
        BCK(h, cudaMemcpyAsync(h->stage, X_in, sizeof(double) * size_t(n * h->nrhs), cudaMemcpyHostToDevice,
                               bstream(h)));
        src = h->stage;
    }
    BCK(h, launch_interleave(src, 0, n, int(h->nrhs), h->bp, h->X, bstream(h)));
    s = bdo_refresh(h);
    if (s != PCDM_OK) return s;
    return bsync(h);
}

pcdm_status pcdm_batch_set_lambda(pcdm_batch_handle h, const double *lambdas)
{
    pcdm_status s = busable(h);
    if (s != PCDM_OK) return s;
    if (!lambdas) return berr(h, PCDM_EINVAL, "lambdas is NULL");
    for (int64_t l = 0; l < h->nrhs; ++l)
        if (!(lambdas[l] >= 0.0) || !std::isfinite(lambdas[l]))
            return berr(h, PCDM_EINVAL, "every lambda must be finite and >= 0");
    for (int64_t l = 0; l < h->nrhs; ++l) h->lam[size_t(l)] = lambdas[l];
    return upload_controls(h);
}

pcdm_status pcdm_batch_reset(pcdm_batch_handle h)
{
    if (!h) return berr(nullptr, PCDM_EINVAL, "NULL batch handle");
    cudaGetLastError();
    pcdm_status s = breset_state(h);
    if (s != PCDM_OK) return s;
    return bsync(h);
}

pcdm_status pcdm_batch_get_stats(pcdm_batch_handle h, pcdm_stats *out)
{
    if (!h || !out) return berr(h, PCDM_EINVAL, "NULL argument");
    pcdm_status s = bsync(h);
    if (s != PCDM_OK) return s;
    unsigned long long c[3] = {0, 0, 0};
    BCK(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
    out->iterations = h->st_iterations;
    out->updates = h->st_updates;
    out->gathered_nnz = int64_t(c[0]);
    out->scattered_nnz = int64_t(c[1]);
    out->nonzero_updates = int64_t(c[2]);
    out->iter_launches = h->st_launches;
    out->iter_kernel_ms = h->st_kernel_ms;
    out->refreshes = h->st_refreshes;
    out->gaps = h->st_gaps;
    out->val_bytes = dtype_bytes(h->base->val_dtype);
    out->xg_bytes = dtype_bytes(h->base->xg_dtype);
    out->kernel_launches = h->st_kernels;
    return PCDM_OK;
}

pcdm_status pcdm_batch_reset_stats(pcdm_batch_handle h)
{
    if (!h) return berr(nullptr, PCDM_EINVAL, "NULL batch handle");
    pcdm_status s = bsync(h);
    if (s != PCDM_OK) return s;
    BCK(h, cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), bstream(h)));
    h->st_iterations = h->st_updates = h->st_launches = h->st_kernels = h->st_refreshes = h->st_gaps = 0;
    h->st_kernel_ms = 0.0;
    return bsync(h);
}

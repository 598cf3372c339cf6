// Host implementation of pcdm_multi_* (include/pcdm.h): many independent LASSO
// problems, each its own A, b and lambda, one thread block per problem
// (multi_kernels.cuh).  Each problem's layout, L and omega come from an
// ordinary handle; this file gathers their device pointers into one table and
// runs the solve loop as a captured CUDA graph: copy of the active flags,
// iterations, refresh + gap, copy of the gap records.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "pcdm_host.h"

using namespace pcdm;
using namespace pcdm_host;

struct pcdm_multi_ctx {
    std::vector<pcdm_handle> probs;
    int count = 0;
    int val_dtype = PCDM_F64, xg_dtype = PCDM_F64;
    cudaStream_t stream = nullptr;     // own stream: CUDA graphs cannot be captured on the legacy one
    void *inst = nullptr;              // device MultiInst<VT, XT>[count]
    int *active = nullptr;             // device flags
    int64_t *kcount = nullptr;         // device iteration counters
    double *rec = nullptr;             // device gap records, count x 9
    double *part = nullptr;            // device gap partials, count x kMultiSplit x 5
    unsigned long long *counters = nullptr;
    int *h_active = nullptr;           // pinned
    double *h_rec = nullptr;           // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_iters = -1, graph_tau = -1;
    uint64_t graph_seed = 0;
    int64_t st_iterations = 0, st_updates = 0, st_launches = 0, st_gaps = 0;
    bool failed = false;
    std::string err;
};

namespace {

pcdm_status merr(pcdm_multi_handle h, pcdm_status s, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_free_error = msg;
    return s;
}

pcdm_status mfail(pcdm_multi_handle h, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return merr(h, PCDM_ENOMEM, msg);
    }
    if (h) h->failed = true;
    return merr(h, PCDM_ECUDA, msg);
}

#define MCK(h, ...)                                                 \
    do {                                                            \
        cudaError_t e_ = (__VA_ARGS__);                             \
        if (e_ != cudaSuccess) return mfail((h), e_, #__VA_ARGS__); \
    } while (0)

void mfree_all(pcdm_multi_handle h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    void *ptrs[] = {h->inst, h->active, h->kcount, h->rec, h->part, h->counters};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->h_active) cudaFreeHost(h->h_active);
    if (h->h_rec) cudaFreeHost(h->h_rec);
    if (h->stream) cudaStreamDestroy(h->stream);
    for (pcdm_handle p : h->probs) pcdm_destroy(p);
}

template <typename F>
pcdm_status mdispatch(pcdm_multi_handle h, F &&f)
{
    if (h->val_dtype == PCDM_F64 && h->xg_dtype == PCDM_F64) return f((double *)nullptr, (double *)nullptr);
    if (h->val_dtype == PCDM_F32 && h->xg_dtype == PCDM_F32) return f((float *)nullptr, (float *)nullptr);
    if (h->val_dtype == PCDM_BF16 && h->xg_dtype == PCDM_F32) return f((bf16_t *)nullptr, (float *)nullptr);
    return merr(h, PCDM_EINVAL, "unsupported dtype pair");
}

// The device table for tau: tau_p = min(tau, n_p), beta of Theorem ESO-nice.
template <typename VT, typename XT>
pcdm_status upload_table(pcdm_multi_handle h, int64_t tau)
{
    std::vector<MultiInst<VT, XT>> tab(size_t(h->count));
    for (int p = 0; p < h->count; ++p) {
        const pcdm_handle q = h->probs[size_t(p)];
        MultiInst<VT, XT> &t = tab[size_t(p)];
        t.desc = static_cast<const ColDesc<XT> *>(q->desc);
        t.prow = q->prow;
        t.pval = static_cast<const VT *>(q->pval);
        t.x = q->x;
        t.g = static_cast<XT *>(q->g);
        t.g64 = q->g64;
        t.b = q->b;
        t.m = q->m;
        t.n = q->n;
        t.tau = tau < q->n ? tau : q->n;
        t.inv_beta = 1.0 / beta_nice(q->omega, t.tau, q->n);
        t.lambda = q->lambda;
    }
    MCK(h, cudaMemcpyAsync(h->inst, tab.data(), sizeof(MultiInst<VT, XT>) * tab.size(), cudaMemcpyHostToDevice,
                           h->stream));
    MCK(h, cudaStreamSynchronize(h->stream));
    return PCDM_OK;
}

// The graph of one check period: active flags in, iters iterations, gap, records out.
template <typename VT, typename XT>
pcdm_status build_graph(pcdm_multi_handle h, int64_t iters, uint64_t seed)
{
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    const auto *inst = static_cast<const MultiInst<VT, XT> *>(h->inst);
    MCK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(h->active, h->h_active, sizeof(int) * size_t(h->count), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess)
        e = MultiKernels<VT, XT>::iter(inst, h->active, h->kcount, h->count, iters, seed, h->counters, h->stream);
    if (e == cudaSuccess) e = MultiKernels<VT, XT>::gap(inst, h->active, h->count, h->part, h->rec, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_rec, h->rec, sizeof(double) * 9 * size_t(h->count), cudaMemcpyDeviceToHost,
                            h->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return mfail(h, e, "capture of the check period");
    }
    MCK(h, e2);
    h->graph = g;
    MCK(h, cudaGraphInstantiate(&h->exec, h->graph, 0));
    h->graph_iters = iters;
    h->graph_seed = seed;
    return PCDM_OK;
}

template <typename VT, typename XT>
pcdm_status multi_solve_t(pcdm_multi_handle h, int64_t tau, uint64_t seed, double tol, int64_t max_iters,
                          int64_t per_check, int64_t *iters_done, double *rel_gaps)
{
    pcdm_status s;
    if (tau != h->graph_tau) {
        s = upload_table<VT, XT>(h, tau);
        if (s != PCDM_OK) return s;
        h->graph_tau = tau;
    }
    if (!h->exec || h->graph_iters != per_check || h->graph_seed != seed) {
        s = build_graph<VT, XT>(h, per_check, seed);
        if (s != PCDM_OK) return s;
    }
    const auto *inst = static_cast<const MultiInst<VT, XT> *>(h->inst);
    std::vector<int64_t> done(size_t(h->count), 0);
    // first gap of every problem
    for (int p = 0; p < h->count; ++p) h->h_active[p] = 1;
    MCK(h, cudaMemcpyAsync(h->active, h->h_active, sizeof(int) * size_t(h->count), cudaMemcpyHostToDevice,
                           h->stream));
    MCK(h, MultiKernels<VT, XT>::gap(inst, h->active, h->count, h->part, h->rec, h->stream));
    MCK(h, cudaMemcpyAsync(h->h_rec, h->rec, sizeof(double) * 9 * size_t(h->count), cudaMemcpyDeviceToHost,
                           h->stream));
    MCK(h, cudaStreamSynchronize(h->stream));
    h->st_gaps += h->count;
    auto rel_of = [&](int p) {
        const double *r = h->h_rec + 9 * size_t(p);
        return r[2] / (r[0] > 1e-300 ? r[0] : 1e-300);
    };
    for (;;) {
        int nact = 0;
        for (int p = 0; p < h->count; ++p) {
            h->h_active[p] = (rel_of(p) > tol && done[size_t(p)] < max_iters) ? 1 : 0;
            nact += h->h_active[p];
        }
        if (nact == 0) break;
        MCK(h, cudaGraphLaunch(h->exec, h->stream));
        MCK(h, cudaStreamSynchronize(h->stream));
        for (int p = 0; p < h->count; ++p)
            if (h->h_active[p]) {
                done[size_t(p)] += per_check;
                const int64_t tp = tau < h->probs[size_t(p)]->n ? tau : h->probs[size_t(p)]->n;
                h->st_updates += per_check * tp;
            }
        h->st_iterations += per_check;
        h->st_launches += 1;
        h->st_gaps += nact;
    }
    bool all = true;
    for (int p = 0; p < h->count; ++p) {
        if (iters_done) iters_done[p] = done[size_t(p)];
        const double r = rel_of(p);
        if (rel_gaps) rel_gaps[p] = r;
        if (r > tol) all = false;
    }
    if (!all) return merr(h, PCDM_ENOTCONV, "max_iters reached before every problem met the gap tolerance");
    return PCDM_OK;
}

}  // namespace

pcdm_status pcdm_multi_create(int64_t count, const pcdm_csc *As, const void *const *bs, int32_t b_dtype,
                              const double *lambdas, const pcdm_opts *opts, void *cuda_stream,
                              pcdm_multi_handle *out)
{
    if (!out) return merr(nullptr, PCDM_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || count > 65535) return merr(nullptr, PCDM_EINVAL, "count must be in [1, 65535]");
    if (!As || !bs || !lambdas) return merr(nullptr, PCDM_EINVAL, "As, bs or lambdas is NULL");
    if (opts && opts->sampling != PCDM_SAMPLING_NICE)
        return merr(nullptr, PCDM_EINVAL, "the multi-problem solver runs the tau-nice sampling only");
    pcdm_multi_ctx *h = new (std::nothrow) pcdm_multi_ctx();
    if (!h) return merr(nullptr, PCDM_ENOMEM, "host allocation failed");
    h->count = int(count);
    auto fail = [&](pcdm_status st) {
        g_free_error = h->err;
        mfree_all(h);
        delete h;
        return st;
    };
    h->probs.reserve(size_t(count));
    for (int64_t p = 0; p < count; ++p) {
        pcdm_handle q = nullptr;
        pcdm_status s = pcdm_create(&As[p], bs[p], b_dtype, lambdas[p], opts, cuda_stream, &q);
        if (s != PCDM_OK) {
            h->err = "problem " + std::to_string(p) + ": " + g_free_error;
            return fail(s);
        }
        h->probs.push_back(q);
    }
    h->val_dtype = h->probs[0]->val_dtype;
    h->xg_dtype = h->probs[0]->xg_dtype;
    for (pcdm_handle q : h->probs)
        if (q->val_dtype != h->val_dtype || q->xg_dtype != h->xg_dtype) {
            h->err = "every problem must have the same dtype pair";
            return fail(PCDM_EINVAL);
        }
#define MCKC(...)                                                           \
    do {                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                     \
        if (e_ != cudaSuccess) return fail(mfail(h, e_, #__VA_ARGS__));     \
    } while (0)
    MCKC(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    MCKC(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    size_t isz = 0;
    mdispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        isz = sizeof(MultiInst<VT, XT>);
        return PCDM_OK;
    });
    MCKC(dalloc_bytes(&h->inst, int64_t(isz) * count));
    MCKC(dalloc(&h->active, count));
    MCKC(dalloc(&h->kcount, count));
    MCKC(dalloc(&h->rec, 9 * count));
    MCKC(dalloc(&h->part, int64_t(kMultiSplit) * 5 * count));
    MCKC(dalloc(&h->counters, 3));
    MCKC(cudaMallocHost(reinterpret_cast<void **>(&h->h_active), sizeof(int) * size_t(count)));
    MCKC(cudaMallocHost(reinterpret_cast<void **>(&h->h_rec), sizeof(double) * 9 * size_t(count)));
    MCKC(cudaMemsetAsync(h->kcount, 0, sizeof(int64_t) * size_t(count), h->stream));
    MCKC(cudaMemsetAsync(h->counters, 0, 3 * sizeof(unsigned long long), h->stream));
    MCKC(cudaStreamSynchronize(h->stream));
#undef MCKC
    *out = h;
    return PCDM_OK;
}

pcdm_status pcdm_multi_solve(pcdm_multi_handle h, int64_t tau, uint64_t seed, double rel_gap_tol, int64_t max_iters,
                             int64_t iters_per_check, int64_t *iters_done, double *rel_gaps)
{
    if (!h) return merr(nullptr, PCDM_EINVAL, "NULL multi handle");
    if (h->failed) return merr(h, PCDM_ESTATE, "multi handle is in a failed state (" + h->err + ")");
    if (tau < 1 || tau > kMultiBlock) return merr(h, PCDM_EINVAL, "tau must be in [1, 256]");
    if (iters_per_check < 1 || max_iters < 0 || !(rel_gap_tol >= 0.0))
        return merr(h, PCDM_EINVAL, "bad iters_per_check, max_iters or tolerance");
    return mdispatch(h, [&](auto *vt, auto *xt) {
        using VT = std::remove_pointer_t<decltype(vt)>;
        using XT = std::remove_pointer_t<decltype(xt)>;
        return multi_solve_t<VT, XT>(h, tau, seed, rel_gap_tol, max_iters, iters_per_check, iters_done, rel_gaps);
    });
}

pcdm_status pcdm_multi_get_x(pcdm_multi_handle h, int64_t p, double *x_out)
{
    if (!h || !x_out) return merr(h, PCDM_EINVAL, "NULL argument");
    if (p < 0 || p >= h->count) return merr(h, PCDM_EINVAL, "problem index out of range");
    MCK(h, cudaStreamSynchronize(h->stream));
    return pcdm_get_x(h->probs[size_t(p)], x_out, 0);
}

pcdm_status pcdm_multi_reset(pcdm_multi_handle h)
{
    if (!h) return merr(nullptr, PCDM_EINVAL, "NULL multi handle");
    MCK(h, cudaStreamSynchronize(h->stream));
    for (pcdm_handle q : h->probs) {
        pcdm_status s = pcdm_reset(q);
        if (s != PCDM_OK) return merr(h, s, std::string("reset of a problem: ") + pcdm_last_error(q));
    }
    MCK(h, cudaMemsetAsync(h->kcount, 0, sizeof(int64_t) * size_t(h->count), h->stream));
    MCK(h, cudaStreamSynchronize(h->stream));
    h->failed = false;
    return PCDM_OK;
}

pcdm_status pcdm_multi_get_stats(pcdm_multi_handle h, pcdm_stats *out)
{
    if (!h || !out) return merr(h, PCDM_EINVAL, "NULL argument");
    unsigned long long c[3] = {0, 0, 0};
    MCK(h, cudaStreamSynchronize(h->stream));
    MCK(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->iterations = h->st_iterations;
    out->updates = h->st_updates;
    out->gathered_nnz = int64_t(c[0]);
    out->scattered_nnz = int64_t(c[1]);
    out->nonzero_updates = int64_t(c[2]);
    out->iter_launches = h->st_launches;
    out->gaps = h->st_gaps;
    out->val_bytes = dtype_bytes(h->val_dtype);
    out->xg_bytes = dtype_bytes(h->xg_dtype);
    out->kernel_launches = 5 * h->st_launches;
    return PCDM_OK;
}

void pcdm_multi_destroy(pcdm_multi_handle h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    mfree_all(h);
    delete h;
}

const char *pcdm_multi_last_error(pcdm_multi_handle h) { return h ? h->err.c_str() : g_free_error.c_str(); }

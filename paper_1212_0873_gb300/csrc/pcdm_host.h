// Host-side state and helpers shared by the C-ABI implementation files
// (pcdm_api.cu: the single-right-hand-side solver; pcdm_batch_api.cu: the
// batched one).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "pcdm.h"
#include "pcdm_internal.h"

namespace pcdm_host {

using namespace pcdm;

extern thread_local std::string g_free_error;   // errors of calls without a handle (pcdm_api.cu)

constexpr int64_t kMaxItersPerLaunch = 1 << 16;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;

inline int64_t dtype_bytes(int dt)
{
    switch (dt) {
    case PCDM_F64: return 8;
    case PCDM_F32: return 4;
    case PCDM_BF16: return 2;
    default: return 0;
    }
}

}  // namespace pcdm_host

// The state behind a pcdm_handle.
struct pcdm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t m = 0, n = 0, nnz = 0;
    int val_dtype = PCDM_F64, xg_dtype = PCDM_F64;
    double lambda = 0.0;
    int problem = 0;              // PCDM_PROBLEM_*: LASSO, SVM dual, logistic regression
    bool l2_set = false;          // the handle counts among the device's l2_persist users
    pcdm_opts opts{};
    int W = 8;
    int sms = 0;

    void *desc = nullptr;         // ColDesc<XT>[n]: padded start, count, 1/L_i
    int32_t *prow = nullptr;      // padded row indices (P + kSlack)
    void *pval = nullptr;         // padded values (P + kSlack)
    int64_t P = 0;                // padded entries
    double *b = nullptr;          // FP64 copy of b
    double *L64 = nullptr;        // L_i in FP64
    double *x = nullptr;          // n FP64 entries
    void *g = nullptr;            // m entries of xg dtype
    void *g2 = nullptr;           // second residual buffer of the pipelined kernel
    unsigned char *head = nullptr;  // per-column heads of the pipelined kernels (built on first use)
    bool g2_valid = false;        // g2 holds the same residual as g
    double *g64 = nullptr;        // FP64 residual of the refresh (aliases g in the FP64 form)
    int32_t *S[2] = {nullptr, nullptr};
    void *h = nullptr;
    int64_t tau_cap = 0;
    unsigned long long *counters = nullptr;   // [3]
    unsigned long long *bar = nullptr;
    int *status = nullptr;
    double *gap_part = nullptr;
    double *gap_out = nullptr;    // 9 doubles
    int gap_blocks = 0, gap_row_blocks = 0;
    double *host_buf = nullptr;   // pinned: 9 gap doubles + status + counters

    // active-set solves (pcdm_polish / pcdm_backward), allocated on first use
    int32_t *as_sidx = nullptr;   // n: the support S of x
    double *as_c = nullptr;       // n: linear term c_p
    double *as_sgn = nullptr;     // n: sign(x_i) on S
    double *as_u = nullptr;       // n: the backward solution u (zero outside S)
    double *as_dx = nullptr;      // n: staging of a host dL/dx
    double *as_q = nullptr;       // m: A_S u - y in FP64
    int *as_rowcnt = nullptr;     // m + 4: row counts of A_S, then count / omega_S words
    double *as_H = nullptr;       // tau: steps of the iteration
    int32_t *as_S = nullptr;      // tau: columns of the iteration
    double *as_part = nullptr;    // residual partials
    int64_t as_tau_cap = 0;
    int as_blocks = 0;
    unsigned long long *win = nullptr;   // n: first-pick keys of the tau-independent sampling

    // deterministic two-kernel form (opts.deterministic_scatter)
    int64_t *det_rptr = nullptr;  // m + 1: row starts of the row-major copy of A
    int32_t *det_rcol = nullptr;  // nnz: its column indices, sorted within each row
    void *det_rval = nullptr;     // nnz: its values (the stored dtype)
    unsigned long long *det_mark = nullptr;   // n: stamps (lo32(k+1) << 32) | position of the nonzero steps

    int64_t omega = 0;
    int64_t k = 0;
    int64_t last_solve_iters = 0;   // iterations of the last pcdm_solve (0 after create / reset)
    uint64_t async_u = 0;           // next update number of the asynchronous mode
    // iteration kernel chosen by pcdm_autotune (-1: the built-in rule)
    int tune_kernel = -1;           // 0 pipelined, 1 fused with tune_W lanes, 2 two-kernel form, 3 pipelined rounds,
                                    // 4 streaming, 5 warp-cooperative
    int tune_W = 0;
    int tune_threads = 0;           // block size of the pipelined, streaming, warp kernels (0: built-in rule)
    int tune_heads = 1;             // pipelined kernels read the column heads (when they fit)
    int tune_zc = -1;               // FP32 certificate of zero steps in the FP64 pipelined kernel (-1: built-in rule)
    // The warp-cooperative kernel's FP32 certificate under tune_zc = -1: on when the last stretch of a
    // solve stepped at most a quarter of its sampled coordinates (pcdm_solve measures it between gap
    // checks); off after create and reset (from x = 0 most coordinates move), on after set_x
    bool warp_cert = false;
    bool head_off = false;          // the column heads did not fit in device memory
    bool rounds_last = false;       // the last segment ran the pipelined rounds kernel (S_{k} not left drawn)
    bool sample_valid = false;
    uint64_t sample_seed = 0;
    int64_t sample_tau = 0, sample_k = -1;
    bool failed = false;
    std::string err;

    int64_t st_iterations = 0, st_updates = 0, st_launches = 0, st_refreshes = 0, st_gaps = 0;
    int64_t st_kernels = 0;   // every kernel launched by this handle
    double st_kernel_ms = 0.0;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
};

namespace pcdm_host {

inline pcdm_status set_err(pcdm_handle h, pcdm_status s, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_free_error = msg;
    return s;
}

inline pcdm_status cuda_fail(pcdm_handle h, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(h, PCDM_ENOMEM, msg);
    }
    if (h) h->failed = true;
    return set_err(h, PCDM_ECUDA, msg);
}

#define CK(h, ...)                                                   \
    do {                                                             \
        cudaError_t e_ = (__VA_ARGS__);                              \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #__VA_ARGS__); \
    } while (0)

template <typename T>
inline cudaError_t dalloc(T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), size_t(count) * sizeof(T));
}

inline cudaError_t dalloc_bytes(void **p, int64_t bytes)
{
    *p = nullptr;
    if (bytes <= 0) bytes = 16;
    return cudaMalloc(p, size_t(bytes));
}

// Moments E|S|, E|S|^2 of the samplings (see pcdm.h) and beta of Theorem ESO-DU.
inline void sampling_moments(int kind, int64_t n, int64_t tau, double p_b, double *e1, double *e2)
{
    const double t = double(tau), nn = double(n);
    if (kind == PCDM_SAMPLING_INDEPENDENT) {
        const double a = std::exp(t * std::log1p(-1.0 / nn));
        const double a2 = n > 1 ? std::exp(t * std::log1p(-2.0 / nn)) : 0.0;
        *e1 = nn * (1.0 - a);
        *e2 = *e1 + nn * (nn - 1.0) * (1.0 - 2.0 * a + a2);
    } else if (kind == PCDM_SAMPLING_BINOMIAL) {
        *e1 = t * p_b;
        *e2 = t * p_b * (1.0 + t * p_b - p_b);
    } else {
        *e1 = t;
        *e2 = t * t;
    }
}

inline double beta_du(int64_t omega, double e1, double e2, int64_t n)
{
    const double om = double(omega < 1 ? 1 : omega);
    const double denom = double(n - 1 > 1 ? n - 1 : 1);
    return e1 > 0.0 ? 1.0 + (om - 1.0) * (e2 / e1 - 1.0) / denom : 1.0;
}

inline uint64_t binomial_threshold(double p_b)
{
    if (p_b >= 1.0) return uint64_t(1) << 32;
    if (p_b <= 0.0) return 0;
    return uint64_t(std::floor(p_b * 4294967296.0));
}

inline double beta_nice(int64_t omega, int64_t tau, int64_t n)
{
    const double om = double(omega < 1 ? 1 : omega);
    const double denom = double(n - 1 > 1 ? n - 1 : 1);
    return 1.0 + (om - 1.0) * (double(tau) - 1.0) / denom;
}

inline cudaMemcpyKind copy_kind(int on_device_src, int on_device_dst)
{
    if (on_device_src && on_device_dst) return cudaMemcpyDeviceToDevice;
    if (on_device_src) return cudaMemcpyDeviceToHost;
    if (on_device_dst) return cudaMemcpyHostToDevice;
    return cudaMemcpyHostToHost;
}

// Synchronise, fold finished event timings into the stats, and read the
// device status word.  Every call that returns host values goes through here.
// Device memory of single-problem handles comes from a per-device
// stream-ordered pool owned by the library (pcdm_api.cu).  The pool keeps
// freed blocks, up to the cache limit (pcdm_set_memory_cache), for the next
// handle: creating and destroying a handle then costs microseconds of
// allocation instead of milliseconds of cudaMalloc and cudaFree.
cudaError_t handle_pool(int device, cudaMemPool_t *pool);

inline cudaError_t halloc_bytes(pcdm_ctx *h, void **p, int64_t bytes)
{
    *p = nullptr;
    if (bytes <= 0) bytes = 16;
    cudaMemPool_t pool;
    cudaError_t e = handle_pool(h->device, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, size_t(bytes), pool, h->stream);
}

template <typename T>
inline cudaError_t halloc(pcdm_ctx *h, T **p, int64_t count)
{
    void *q = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = halloc_bytes(h, &q, count * int64_t(sizeof(T)));
    *p = static_cast<T *>(q);
    return e;
}

// Stream-ordered free of a halloc block (after the work already enqueued on the handle's stream).
inline void hfree(pcdm_ctx *h, void *p)
{
    if (p) cudaFreeAsync(p, h->stream);
}

inline pcdm_status sync_check(pcdm_handle h)
{
    int *hs = reinterpret_cast<int *>(h->host_buf + 9);
    CK(h, cudaMemcpyAsync(hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &pr : h->ev_pending) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, pr.first, pr.second));
        h->st_kernel_ms += ms;
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    if (*hs != DEV_OK) {
        h->failed = true;
        return set_err(h, PCDM_ETIMEOUT, "a grid-barrier wait of the fused kernel ran out of its time budget");
    }
    return PCDM_OK;
}

inline cudaError_t take_event(pcdm_handle h, cudaEvent_t *e)
{
    if (!h->ev_free.empty()) {
        *e = h->ev_free.back();
        h->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Dispatch on the (value, iterate) dtype pair.
template <typename F>
inline pcdm_status dispatch(pcdm_handle h, F &&f)
{
    if (h->val_dtype == PCDM_F64 && h->xg_dtype == PCDM_F64) return f((double *)nullptr, (double *)nullptr);
    if (h->val_dtype == PCDM_F32 && h->xg_dtype == PCDM_F32) return f((float *)nullptr, (float *)nullptr);
    if (h->val_dtype == PCDM_BF16 && h->xg_dtype == PCDM_F32) return f((bf16_t *)nullptr, (float *)nullptr);
    return set_err(h, PCDM_EINVAL, "unsupported dtype pair");
}

// First gap-check interval of a solve: one epoch, or, when the handle's last
// solve ran K iterations (a warm start, e.g. the next lambda of a path), half
// of K, so that a solve of similar length needs only a few checks.
inline int64_t first_check_interval(int64_t epoch, int64_t last_solve_iters)
{
    const int64_t guess = last_solve_iters / 2;
    return guess > epoch ? guess : epoch;
}

inline pcdm_status usable(pcdm_handle h)
{
    if (!h) return set_err(nullptr, PCDM_EINVAL, "NULL handle");
    if (h->failed) return set_err(h, PCDM_ESTATE, "handle is in a failed state (" + h->err + "); call pcdm_reset");
    return PCDM_OK;
}

}  // namespace pcdm_host

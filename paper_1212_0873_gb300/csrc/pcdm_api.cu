// Host implementation of the libpcdm C ABI (include/pcdm.h): argument checks,
// device memory ownership, kernel scheduling, and the solve loop.  Every step
// of the method runs in the kernels of kernels_*.cu; this file only moves
// pointers, sizes and scalars.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "pcdm.h"
#include "pcdm_internal.h"

using namespace pcdm;

namespace {

thread_local std::string g_free_error;   // errors of calls without a handle

constexpr int64_t kMaxItersPerLaunch = 1 << 16;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;

int64_t dtype_bytes(int dt)
{
    switch (dt) {
    case PCDM_F64: return 8;
    case PCDM_F32: return 4;
    case PCDM_BF16: return 2;
    default: return 0;
    }
}

}  // namespace

struct pcdm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t m = 0, n = 0, nnz = 0;
    int val_dtype = PCDM_F64, xg_dtype = PCDM_F64;
    double lambda = 0.0;
    pcdm_opts opts{};
    int W = 8;
    int fused_blocks_max = 0;

    int64_t *col_ptr = nullptr;
    int32_t *row_idx = nullptr;
    void *val = nullptr;
    double *b = nullptr;          // FP64 copy of b
    double *L64 = nullptr;        // L_i in FP64
    float *L32 = nullptr;         // L_i rounded to FP32 (FP32 iterate forms)
    void *x = nullptr;            // n entries of xg dtype
    void *g = nullptr;            // m entries of xg dtype
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

    int64_t omega = 0;
    int64_t k = 0;
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

namespace {

pcdm_status set_err(pcdm_handle h, pcdm_status s, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_free_error = msg;
    return s;
}

pcdm_status cuda_fail(pcdm_handle h, cudaError_t e, const char *what)
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
cudaError_t dalloc(T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), size_t(count) * sizeof(T));
}

cudaError_t dalloc_bytes(void **p, int64_t bytes)
{
    *p = nullptr;
    if (bytes <= 0) bytes = 16;
    return cudaMalloc(p, size_t(bytes));
}

void free_all(pcdm_handle h)
{
    void *ptrs[] = {h->col_ptr, h->row_idx, h->val, h->b, h->L64, h->L32, h->x, h->g,
                    h->S[0], h->S[1], h->h, h->counters, h->bar, h->status, h->gap_part, h->gap_out};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->g64 && h->g64 != h->g) cudaFree(h->g64);
    if (h->host_buf) cudaFreeHost(h->host_buf);
    for (auto &pr : h->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
}

int auto_lanes(int64_t nnz, int64_t n)
{
    const double mean = n > 0 ? double(nnz) / double(n) : 0.0;
    if (mean < 6.0) return 4;
    if (mean < 12.0) return 8;
    if (mean < 24.0) return 16;
    return 32;
}

double beta_nice(int64_t omega, int64_t tau, int64_t n)
{
    const double om = double(omega < 1 ? 1 : omega);
    const double denom = double(n - 1 > 1 ? n - 1 : 1);
    return 1.0 + (om - 1.0) * (double(tau) - 1.0) / denom;
}

cudaMemcpyKind copy_kind(int on_device_src, int on_device_dst)
{
    if (on_device_src && on_device_dst) return cudaMemcpyDeviceToDevice;
    if (on_device_src) return cudaMemcpyDeviceToHost;
    if (on_device_dst) return cudaMemcpyHostToDevice;
    return cudaMemcpyHostToHost;
}

// Synchronise, fold finished event timings into the stats, and read the
// device status word.  Every call that returns host values goes through here.
pcdm_status sync_check(pcdm_handle h)
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

cudaError_t take_event(pcdm_handle h, cudaEvent_t *e)
{
    if (!h->ev_free.empty()) {
        *e = h->ev_free.back();
        h->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

pcdm_status ensure_tau(pcdm_handle h, int64_t tau)
{
    if (tau <= h->tau_cap) return PCDM_OK;
    // Buffers are replaced only between calls; the stream must be idle first.
    CK(h, cudaStreamSynchronize(h->stream));
    for (int q = 0; q < 2; ++q)
        if (h->S[q]) cudaFree(h->S[q]);
    if (h->h) cudaFree(h->h);
    h->S[0] = h->S[1] = nullptr;
    h->h = nullptr;
    h->tau_cap = 0;
    h->sample_valid = false;
    CK(h, dalloc(&h->S[0], tau));
    CK(h, dalloc(&h->S[1], tau));
    CK(h, dalloc_bytes(&h->h, tau * dtype_bytes(h->xg_dtype)));
    h->tau_cap = tau;
    return PCDM_OK;
}

template <typename VT, typename XT>
IterArgs<VT, XT> iter_args(pcdm_handle h, int64_t tau, uint64_t seed)
{
    IterArgs<VT, XT> a;
    a.col_ptr = h->col_ptr;
    a.row_idx = h->row_idx;
    a.val = static_cast<const VT *>(h->val);
    if (sizeof(XT) == 8)
        a.L = reinterpret_cast<const XT *>(h->L64);
    else
        a.L = reinterpret_cast<const XT *>(h->L32);
    a.x = static_cast<XT *>(h->x);
    a.g = static_cast<XT *>(h->g);
    a.h = static_cast<XT *>(h->h);
    a.S[0] = h->S[0];
    a.S[1] = h->S[1];
    a.beta = XT(beta_nice(h->omega, tau, h->n));
    a.lambda = XT(h->lambda);
    a.n = h->n;
    a.tau = tau;
    a.seed = seed;
    a.counters = h->counters;
    a.bar = h->bar;
    a.status = h->status;
    a.timeout_ns = h->opts.barrier_timeout_ns ? h->opts.barrier_timeout_ns : kDefaultTimeoutNs;
    return a;
}

// Run `iters` iterations starting at h->k with S_k already drawn.
template <typename VT, typename XT>
pcdm_status run_segment(pcdm_handle h, int64_t tau, uint64_t seed, int64_t iters)
{
    IterArgs<VT, XT> a = iter_args<VT, XT>(h, tau, seed);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->opts.profile) {
        CK(h, take_event(h, &e0));
        CK(h, take_event(h, &e1));
        CK(h, cudaEventRecord(e0, h->stream));
    }
    if (h->opts.fused) {
        if (h->fused_blocks_max <= 0) {
            h->fused_blocks_max = Kernels<VT, XT>::fused_max_blocks(h->W);
            if (h->fused_blocks_max <= 0) return set_err(h, PCDM_ECUDA, "cooperative occupancy query failed");
        }
        const int64_t want = (tau * h->W + kBlock - 1) / kBlock;
        const int blocks = int(want < h->fused_blocks_max ? want : h->fused_blocks_max);
        CK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
        CK(h, Kernels<VT, XT>::fused(a, h->W, h->k, iters, blocks, h->stream));
        h->st_launches += 1;
        h->st_kernels += 1;
    } else {
        for (int64_t it = 0; it < iters; ++it) {
            const int64_t kk = h->k + it;
            CK(h, Kernels<VT, XT>::gather(a, h->W, kk, h->stream));
            CK(h, Kernels<VT, XT>::scatter(a, h->W, kk, true, h->stream));
        }
        h->st_launches += iters;
        h->st_kernels += 2 * iters;
    }
    if (h->opts.profile) {
        CK(h, cudaEventRecord(e1, h->stream));
        h->ev_pending.emplace_back(e0, e1);
    }
    h->k += iters;
    h->sample_valid = true;
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
    CK(h, launch_neg_store<double>(target, h->b, h->m, h->stream));
    CK(h, Kernels<VT, XT>::refresh_cols(h->col_ptr, h->row_idx, static_cast<const VT *>(h->val),
                                        static_cast<const XT *>(h->x), h->n, target, h->W, h->stream));
    if (sizeof(XT) == 4) CK(h, launch_store_from_f64<float>(static_cast<float *>(h->g), target, h->m, h->stream));
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
    CK(h, Kernels<VT, XT>::gap_cols(h->col_ptr, h->row_idx, static_cast<const VT *>(h->val), h->g64,
                                    static_cast<const XT *>(h->x), h->n, part_c, h->gap_blocks, h->W, h->stream));
    CK(h, launch_gap_rows(h->g64, h->b, h->m, part_r, h->gap_row_blocks, h->stream));
    CK(h, launch_gap_finish(part_c, h->gap_blocks, part_r, h->gap_row_blocks, h->gap_out, h->lambda, h->stream));
    CK(h, cudaMemcpyAsync(h->host_buf, h->gap_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    h->st_gaps += 1;
    h->st_kernels += 3;
    return sync_check(h);
}

// Dispatch on the (value, iterate) dtype pair.
template <typename F>
pcdm_status dispatch(pcdm_handle h, F &&f)
{
    if (h->val_dtype == PCDM_F64 && h->xg_dtype == PCDM_F64) return f((double *)nullptr, (double *)nullptr);
    if (h->val_dtype == PCDM_F32 && h->xg_dtype == PCDM_F32) return f((float *)nullptr, (float *)nullptr);
    if (h->val_dtype == PCDM_BF16 && h->xg_dtype == PCDM_F32) return f((bf16_t *)nullptr, (float *)nullptr);
    return set_err(h, PCDM_EINVAL, "unsupported dtype pair");
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

pcdm_status usable(pcdm_handle h)
{
    if (!h) return set_err(nullptr, PCDM_EINVAL, "NULL handle");
    if (h->failed) return set_err(h, PCDM_ESTATE, "handle is in a failed state (" + h->err + "); call pcdm_reset");
    return PCDM_OK;
}

pcdm_status reset_state(pcdm_handle h)
{
    CK(h, cudaMemsetAsync(h->x, 0, size_t(h->n) * size_t(dtype_bytes(h->xg_dtype)), h->stream));
    if (h->xg_dtype == PCDM_F64)
        CK(h, launch_neg_store<double>(static_cast<double *>(h->g), h->b, h->m, h->stream));
    else
        CK(h, launch_neg_store<float>(static_cast<float *>(h->g), h->b, h->m, h->stream));
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    h->st_kernels += 1;   // the g = -b kernel
    h->k = 0;
    h->sample_valid = false;
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

pcdm_status pcdm_create(const pcdm_csc *A, const void *b, int32_t b_dtype, double lambda, const pcdm_opts *opts,
                        void *cuda_stream, pcdm_handle *out)
{
    if (!out) return set_err(nullptr, PCDM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!A || !b) return set_err(nullptr, PCDM_EINVAL, "A or b is NULL");
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

    pcdm_ctx *h = new (std::nothrow) pcdm_ctx();
    if (!h) return set_err(nullptr, PCDM_ENOMEM, "host allocation failed");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->m = A->m;
    h->n = A->n;
    h->nnz = A->nnz;
    h->val_dtype = A->val_dtype;
    h->xg_dtype = o.xg_dtype;
    h->lambda = lambda;
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
    int sms = 0;
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    {
        int64_t gb = (h->n * h->W + kBlock - 1) / kBlock;
        const int64_t cap = int64_t(sms) * 8;
        h->gap_blocks = int(gb < 1 ? 1 : (gb > cap ? cap : gb));
        int64_t rb = (h->m + kBlock - 1) / kBlock;
        h->gap_row_blocks = int(rb < 1 ? 1 : (rb > cap ? cap : rb));
    }
    CKC(dalloc(&h->col_ptr, h->n + 1));
    CKC(dalloc(&h->row_idx, h->nnz));
    CKC(dalloc_bytes(&h->val, h->nnz * vb));
    CKC(dalloc(&h->b, h->m));
    CKC(dalloc(&h->L64, h->n));
    if (h->xg_dtype == PCDM_F32) CKC(dalloc(&h->L32, h->n));
    CKC(dalloc_bytes(&h->x, h->n * xb));
    CKC(dalloc_bytes(&h->g, h->m * xb));
    if (h->xg_dtype == PCDM_F64)
        h->g64 = static_cast<double *>(h->g);
    else
        CKC(dalloc(&h->g64, h->m));
    CKC(dalloc(&h->counters, 3));
    CKC(dalloc(&h->bar, 1));
    CKC(dalloc(&h->status, 4));
    CKC(dalloc(&h->gap_part, 3 * int64_t(h->gap_blocks) + 2 * int64_t(h->gap_row_blocks)));
    CKC(dalloc(&h->gap_out, 9));
    CKC(cudaMallocHost(reinterpret_cast<void **>(&h->host_buf), 16 * sizeof(double)));

    const cudaMemcpyKind kin = copy_kind(A->on_device, 1);
    cudaStream_t st = h->stream;
    CKC(cudaMemcpyAsync(h->col_ptr, A->col_ptr, size_t(h->n + 1) * sizeof(int64_t), kin, st));
    if (h->nnz > 0) {
        CKC(cudaMemcpyAsync(h->row_idx, A->row_idx, size_t(h->nnz) * sizeof(int32_t), kin, st));
        CKC(cudaMemcpyAsync(h->val, A->val, size_t(h->nnz * vb), kin, st));
    }
    if (b_dtype == PCDM_F64) {
        CKC(cudaMemcpyAsync(h->b, b, size_t(h->m) * sizeof(double), kin, st));
    } else {
        // Stage the FP32 b in the g buffer's space (g64 or g is at least m floats).
        void *stage = h->g;
        CKC(cudaMemcpyAsync(stage, b, size_t(h->m) * sizeof(float), kin, st));
        CKC(launch_convert_b(stage, 1, h->m, h->b, st));
    }

    // Validation, first of col_ptr alone so that the column kernels index safely.
    int *flags = h->status + 1;
    int *omega_dev = h->status + 2;
    int *hflags = reinterpret_cast<int *>(h->host_buf + 10);
    CKC(cudaMemsetAsync(h->status, 0, 4 * sizeof(int), st));
    CKC(launch_check_colptr(h->col_ptr, h->n, h->nnz, flags, st));
    CKC(cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (*hflags & FLAG_COLPTR) {
        h->err = "col_ptr must start at 0, be non-decreasing and end at nnz";
        return fail(PCDM_EINVAL);
    }
    int *rowcnt = nullptr;
    CKC(dalloc(&rowcnt, h->m));
    cudaError_t e = cudaMemsetAsync(rowcnt, 0, size_t(h->m) * sizeof(int), st);
    if (e == cudaSuccess) {
        switch (h->val_dtype) {
        case PCDM_F64:
            e = Kernels<double, double>::setup_cols(h->col_ptr, h->row_idx, static_cast<const double *>(h->val), h->m,
                                                    h->n, h->L64, rowcnt, flags, st);
            break;
        case PCDM_F32:
            e = Kernels<float, float>::setup_cols(h->col_ptr, h->row_idx, static_cast<const float *>(h->val), h->m,
                                                  h->n, h->L64, rowcnt, flags, st);
            break;
        default:
            e = Kernels<bf16_t, float>::setup_cols(h->col_ptr, h->row_idx, static_cast<const bf16_t *>(h->val), h->m,
                                                   h->n, h->L64, rowcnt, flags, st);
            break;
        }
    }
    if (e == cudaSuccess) e = launch_check_finite(h->b, h->m, flags, st);
    if (e == cudaSuccess) e = launch_max_int(rowcnt, h->m, omega_dev, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(rowcnt);
    if (e != cudaSuccess) return fail(cuda_fail(h, e, "set-up kernels"));
    const int f = hflags[0];
    if (f) {
        std::string msg = "invalid input:";
        if (f & FLAG_ROW_RANGE) msg += " row index outside [0, m);";
        if (f & FLAG_ROW_ORDER) msg += " rows of a column not strictly increasing;";
        if (f & FLAG_NONFINITE) msg += " non-finite value in A;";
        if (f & FLAG_B_NONFINITE) msg += " non-finite value in b;";
        h->err = msg;
        return fail(PCDM_EINVAL);
    }
    h->omega = hflags[1];
    if (h->xg_dtype == PCDM_F32) CKC(launch_f64_to_f32(h->L32, h->L64, h->n, st));
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

pcdm_status pcdm_solve(pcdm_handle h, int64_t tau, uint64_t seed, double rel_gap_tol, int64_t max_iters,
                       int64_t *iters_done, double *rel_gap)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (tau < 1 || tau > h->n) return set_err(h, PCDM_EINVAL, "tau must be in [1, n]");
    if (max_iters < 0 || !(rel_gap_tol >= 0.0)) return set_err(h, PCDM_EINVAL, "max_iters < 0 or bad tolerance");
    const int64_t every = h->opts.check_every > 0 ? h->opts.check_every : (h->n + tau - 1) / tau;
    double rec[9];
    int64_t done = 0;
    s = do_gap(h, rec);
    if (s != PCDM_OK) return s;
    double rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300);
    while (rel > rel_gap_tol && done < max_iters) {
        const int64_t chunk = every < max_iters - done ? every : max_iters - done;
        s = pcdm_step(h, tau, chunk, seed);
        if (s != PCDM_OK) return s;
        done += chunk;
        s = do_gap(h, rec);
        if (s != PCDM_OK) return s;
        rel = rec[2] / (rec[0] > 1e-300 ? rec[0] : 1e-300);
    }
    if (iters_done) *iters_done = done;
    if (rel_gap) *rel_gap = rel;
    if (rel > rel_gap_tol) return set_err(h, PCDM_ENOTCONV, "max_iters reached before the gap tolerance");
    return PCDM_OK;
}

pcdm_status pcdm_get_x(pcdm_handle h, void *x_out, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!x_out) return set_err(h, PCDM_EINVAL, "x_out is NULL");
    CK(h, cudaMemcpyAsync(x_out, h->x, size_t(h->n * dtype_bytes(h->xg_dtype)), copy_kind(1, on_device), h->stream));
    return sync_check(h);
}

pcdm_status pcdm_set_x(pcdm_handle h, const void *x_in, int32_t on_device)
{
    pcdm_status s = usable(h);
    if (s != PCDM_OK) return s;
    if (!x_in) return set_err(h, PCDM_EINVAL, "x_in is NULL");
    CK(h, cudaMemcpyAsync(h->x, x_in, size_t(h->n * dtype_bytes(h->xg_dtype)), copy_kind(on_device, 1), h->stream));
    h->sample_valid = false;
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
    *beta = beta_nice(h->omega, tau, h->n);
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

pcdm_status pcdm_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S_device, void *cuda_stream)
{
    if (n < 1 || n > 2147483647LL || tau < 0 || tau > n || k < 0)
        return set_err(nullptr, PCDM_EINVAL, "need 1 <= n < 2^31, 0 <= tau <= n, k >= 0");
    if (tau > 0 && !S_device) return set_err(nullptr, PCDM_EINVAL, "S_device is NULL");
    cudaError_t e = launch_sample(seed, k, n, tau, S_device, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "launch_sample");
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

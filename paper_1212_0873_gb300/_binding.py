"""ctypes binding of libpcdm (include/pcdm.h): the same entry-point names,
argument marshalling only.  Every call goes into the CUDA library; there is no
CPU fallback.  If the library has not been built, the first call raises.

Non-OK statuses raise PcdmError, except PCDM_ENOTCONV from pcdm_solve, which is
reported through its return value.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpcdm.so")

PCDM_OK, PCDM_EINVAL, PCDM_ENOMEM, PCDM_ECUDA, PCDM_ETIMEOUT, PCDM_ENOTCONV, PCDM_ESTATE = range(7)
PCDM_F64, PCDM_F32, PCDM_BF16 = 0, 1, 2
DTYPE_CODES = {"f64": PCDM_F64, "f32": PCDM_F32, "bf16": PCDM_BF16}

_i32, _i64, _u64, _dbl, _ptr = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class pcdm_csc(ctypes.Structure):
    _fields_ = [("m", _i64), ("n", _i64), ("nnz", _i64), ("col_ptr", _ptr), ("row_idx", _ptr), ("val", _ptr),
                ("val_dtype", _i32), ("on_device", _i32)]


class pcdm_tuning(ctypes.Structure):
    _fields_ = [("kernel", _i32), ("lanes_per_col", _i32), ("threads_per_block", _i32), ("heads", _i32),
                ("zero_cert", _i32), ("us_per_iteration", _dbl)]


class pcdm_opts(ctypes.Structure):
    _fields_ = [("xg_dtype", _i32), ("fused", _i32), ("refresh_every", _i64), ("check_every", _i64),
                ("lanes_per_col", _i64), ("barrier_timeout_ns", _u64), ("profile", _i32), ("sampling", _i32),
                ("p_b", _dbl), ("l2_persist", _i32), ("deterministic_scatter", _i32)]


class pcdm_stats(ctypes.Structure):
    _fields_ = [("iterations", _i64), ("updates", _i64), ("gathered_nnz", _i64), ("scattered_nnz", _i64),
                ("nonzero_updates", _i64), ("iter_launches", _i64), ("iter_kernel_ms", _dbl),
                ("refreshes", _i64), ("gaps", _i64), ("val_bytes", _i64), ("xg_bytes", _i64),
                ("kernel_launches", _i64)]


# Every function the header declares, with (restype, argtypes).
SIGNATURES = {
    "pcdm_default_opts": (None, [ctypes.POINTER(pcdm_opts)]),
    "pcdm_create": (_i32, [ctypes.POINTER(pcdm_csc), _ptr, _i32, _dbl, ctypes.POINTER(pcdm_opts), _ptr,
                           ctypes.POINTER(_ptr)]),
    "pcdm_create_problem": (_i32, [ctypes.POINTER(pcdm_csc), _i32, _ptr, _dbl, ctypes.POINTER(pcdm_opts), _ptr,
                                   ctypes.POINTER(_ptr)]),
    "pcdm_problem_kind": (_i32, [_ptr, ctypes.POINTER(_i32)]),
    "pcdm_set_memory_cache": (_i32, [_u64]),
    "pcdm_release_cached_memory": (_i32, []),
    "pcdm_step": (_i32, [_ptr, _i64, _i64, _u64]),
    "pcdm_refresh": (_i32, [_ptr]),
    "pcdm_gap": (_i32, [_ptr, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
    "pcdm_solve": (_i32, [_ptr, _i64, _u64, _dbl, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]),
    "pcdm_next_check_interval": (_i64, [_i64, _i64, ctypes.c_double, _i64, ctypes.c_double, ctypes.c_double]),
    "pcdm_omega_noalloc": (_i32, [ctypes.POINTER(pcdm_csc), ctypes.POINTER(_i64), _ptr]),
    "pcdm_gather_rate": (_i32, [_ptr, _i64, _i32, ctypes.POINTER(_dbl), _ptr]),
    "pcdm_batch_create": (_i32, [ctypes.POINTER(pcdm_csc), _i64, _ptr, _i32, _ptr, ctypes.POINTER(pcdm_opts), _ptr,
                                 _ptr]),
    "pcdm_batch_step": (_i32, [_ptr, _i64, _i64, _u64]),
    "pcdm_batch_refresh": (_i32, [_ptr]),
    "pcdm_batch_gap": (_i32, [_ptr, _ptr, _ptr, _ptr]),
    "pcdm_batch_solve": (_i32, [_ptr, _i64, _u64, _dbl, _i64, _ptr, _ptr]),
    "pcdm_batch_get_x": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_batch_set_x": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_batch_set_lambda": (_i32, [_ptr, _ptr]),
    "pcdm_batch_reset": (_i32, [_ptr]),
    "pcdm_batch_get_stats": (_i32, [_ptr, ctypes.POINTER(pcdm_stats)]),
    "pcdm_batch_reset_stats": (_i32, [_ptr]),
    "pcdm_batch_destroy": (None, [_ptr]),
    "pcdm_batch_last_error": (ctypes.c_char_p, [_ptr]),
    "pcdm_batch_autotune": (_i32, [_ptr, _i64, _i64, ctypes.POINTER(_i32), ctypes.POINTER(_dbl)]),
    "pcdm_set_b": (_i32, [_ptr, _ptr, _i32, _i32]),
    "pcdm_support_size": (_i32, [_ptr, _ptr]),
    "pcdm_polish": (_i32, [_ptr, _i64, _u64, _dbl, _i64, _ptr, _ptr]),
    "pcdm_backward": (_i32, [_ptr, _ptr, _i32, _ptr, _i32, _ptr, _i64, _u64, _dbl, _i64, _ptr, _ptr]),
    "pcdm_sample_kind": (_i32, [_i32, _u64, _i64, _i64, _i64, _dbl, _ptr, _ptr, _ptr]),
    "pcdm_step_async": (_i32, [_ptr, _i64, _u64, _i32]),
    "pcdm_solve_async": (_i32, [_ptr, _u64, _dbl, _i64, _i32, _ptr, _ptr]),
    "pcdm_multi_create": (_i32, [_i64, _ptr, _ptr, _i32, _ptr, ctypes.POINTER(pcdm_opts), _ptr, _ptr]),
    "pcdm_multi_solve": (_i32, [_ptr, _i64, _u64, _dbl, _i64, _i64, _ptr, _ptr]),
    "pcdm_multi_get_x": (_i32, [_ptr, _i64, _ptr]),
    "pcdm_multi_reset": (_i32, [_ptr]),
    "pcdm_multi_get_stats": (_i32, [_ptr, ctypes.POINTER(pcdm_stats)]),
    "pcdm_multi_destroy": (None, [_ptr]),
    "pcdm_multi_last_error": (ctypes.c_char_p, [_ptr]),
    "pcdm_autotune": (_i32, [_ptr, _i64, _i64, ctypes.POINTER(pcdm_tuning)]),
    "pcdm_set_tuning": (_i32, [_ptr, ctypes.POINTER(pcdm_tuning)]),
    "pcdm_get_x": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_set_x": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_get_residual": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_get_L": (_i32, [_ptr, _ptr, _i32]),
    "pcdm_set_lambda": (_i32, [_ptr, _dbl]),
    "pcdm_omega": (_i32, [_ptr, ctypes.POINTER(_i64)]),
    "pcdm_beta": (_i32, [_ptr, _i64, ctypes.POINTER(_dbl)]),
    "pcdm_get_iteration": (_i32, [_ptr, ctypes.POINTER(_i64)]),
    "pcdm_set_iteration": (_i32, [_ptr, _i64]),
    "pcdm_reset": (_i32, [_ptr]),
    "pcdm_get_stats": (_i32, [_ptr, ctypes.POINTER(pcdm_stats)]),
    "pcdm_reset_stats": (_i32, [_ptr]),
    "pcdm_sample": (_i32, [_u64, _i64, _i64, _i64, _ptr, _ptr]),
    "pcdm_selftest_barrier_timeout": (_i32, [_u64, _ptr]),
    "pcdm_destroy": (None, [_ptr]),
    "pcdm_last_error": (ctypes.c_char_p, [_ptr]),
    "pcdm_status_string": (ctypes.c_char_p, [_i32]),
}

_lib = None


class PcdmError(RuntimeError):
    def __init__(self, status, message):
        self.status = int(status)
        super().__init__("%s: %s" % (_STATUS_NAMES.get(int(status), str(status)), message))


_STATUS_NAMES = {0: "PCDM_OK", 1: "PCDM_EINVAL", 2: "PCDM_ENOMEM", 3: "PCDM_ECUDA", 4: "PCDM_ETIMEOUT",
                 5: "PCDM_ENOTCONV", 6: "PCDM_ESTATE"}


def lib():
    """The loaded libpcdm; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpcdm.so is not built (%s). Build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`; there is no CPU fallback."
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != PCDM_OK:
        msg = lib().pcdm_last_error(handle)
        raise PcdmError(status, (msg or b"").decode(errors="replace"))


def _stream(stream):
    return ctypes.c_void_p(int(stream) if stream else 0)


# ---------------------------------------------------------------------------- entry points
def pcdm_default_opts():
    o = pcdm_opts()
    lib().pcdm_default_opts(ctypes.byref(o))
    return o


def pcdm_create(A, b_ptr, b_dtype, lam, opts=None, stream=0):
    h = _ptr()
    st = lib().pcdm_create(ctypes.byref(A), _ptr(b_ptr), int(b_dtype), float(lam),
                           ctypes.byref(opts) if opts is not None else None, _stream(stream), ctypes.byref(h))
    _check(st, None)
    return h


PROBLEM_CODES = {"lasso": 0, "svm_dual": 1, "logistic": 2}


def pcdm_create_problem(A, problem, y_ptr, lam, opts=None, stream=0):
    h = _ptr()
    st = lib().pcdm_create_problem(ctypes.byref(A), int(PROBLEM_CODES[problem]), _ptr(y_ptr), float(lam),
                                   ctypes.byref(opts) if opts is not None else None, _stream(stream),
                                   ctypes.byref(h))
    _check(st, None)
    return h


def pcdm_problem_kind(h):
    v = _i32()
    _check(lib().pcdm_problem_kind(h, ctypes.byref(v)), h)
    return {c: k for k, c in PROBLEM_CODES.items()}[v.value]


def pcdm_step(h, tau, iters, seed):
    _check(lib().pcdm_step(h, int(tau), int(iters), int(seed) & (2**64 - 1)), h)


def pcdm_refresh(h):
    _check(lib().pcdm_refresh(h), h)


def pcdm_gap(h):
    p, d, g = _dbl(), _dbl(), _dbl()
    _check(lib().pcdm_gap(h, ctypes.byref(p), ctypes.byref(d), ctypes.byref(g)), h)
    return p.value, d.value, g.value


def pcdm_solve(h, tau, seed, rel_gap_tol, max_iters):
    """Returns (converged, iters_done, rel_gap)."""
    it, rel = _i64(), _dbl()
    st = lib().pcdm_solve(h, int(tau), int(seed) & (2**64 - 1), float(rel_gap_tol), int(max_iters),
                          ctypes.byref(it), ctypes.byref(rel))
    if st == PCDM_ENOTCONV:
        return False, it.value, rel.value
    _check(st, h)
    return True, it.value, rel.value


def pcdm_get_x(h, ptr, on_device):
    _check(lib().pcdm_get_x(h, _ptr(ptr), int(on_device)), h)


def pcdm_set_x(h, ptr, on_device):
    _check(lib().pcdm_set_x(h, _ptr(ptr), int(on_device)), h)


def pcdm_get_residual(h, ptr, on_device):
    _check(lib().pcdm_get_residual(h, _ptr(ptr), int(on_device)), h)


def pcdm_get_L(h, ptr, on_device):
    _check(lib().pcdm_get_L(h, _ptr(ptr), int(on_device)), h)


def pcdm_set_lambda(h, lam):
    _check(lib().pcdm_set_lambda(h, float(lam)), h)


def pcdm_omega(h):
    v = _i64()
    _check(lib().pcdm_omega(h, ctypes.byref(v)), h)
    return v.value


def pcdm_beta(h, tau):
    v = _dbl()
    _check(lib().pcdm_beta(h, int(tau), ctypes.byref(v)), h)
    return v.value


def pcdm_get_iteration(h):
    v = _i64()
    _check(lib().pcdm_get_iteration(h, ctypes.byref(v)), h)
    return v.value


def pcdm_set_iteration(h, k):
    _check(lib().pcdm_set_iteration(h, int(k)), h)


def pcdm_reset(h):
    _check(lib().pcdm_reset(h), h)


def pcdm_get_stats(h):
    s = pcdm_stats()
    _check(lib().pcdm_get_stats(h, ctypes.byref(s)), h)
    return {name: getattr(s, name) for name, _ in pcdm_stats._fields_}


def pcdm_reset_stats(h):
    _check(lib().pcdm_reset_stats(h), h)


def pcdm_sample(seed, k, n, tau, S_device_ptr, stream=0):
    _check(lib().pcdm_sample(int(seed) & (2**64 - 1), int(k), int(n), int(tau), _ptr(S_device_ptr),
                             _stream(stream)), None)


def pcdm_selftest_barrier_timeout(timeout_ns, stream=0):
    """Returns the raw status (PCDM_ETIMEOUT is the expected outcome)."""
    return int(lib().pcdm_selftest_barrier_timeout(int(timeout_ns), _stream(stream)))


def pcdm_gather_rate(src_device_ptr, n, elem_bytes, stream=0):
    """Random gathers per second from a device vector of n elem_bytes-wide values."""
    out = _dbl(0.0)
    _check(lib().pcdm_gather_rate(_ptr(src_device_ptr), int(n), int(elem_bytes), ctypes.byref(out),
                                  _stream(stream)), None)
    return float(out.value)


def pcdm_destroy(h):
    lib().pcdm_destroy(h)


def pcdm_last_error(h=None):
    msg = lib().pcdm_last_error(h)
    return (msg or b"").decode(errors="replace")


def pcdm_status_string(status):
    return lib().pcdm_status_string(int(status)).decode()


def pcdm_next_check_interval(epoch, k_prev, rel_prev, k_cur, rel_cur, rel_gap_tol):
    return int(lib().pcdm_next_check_interval(int(epoch), int(k_prev), float(rel_prev), int(k_cur), float(rel_cur),
                                              float(rel_gap_tol)))


PCDM_NOALLOC_MAX_ROWS = 1048576


def pcdm_omega_noalloc(csc, stream):
    """omega of a device CSC (a pcdm_csc with on_device = 1) without any allocation."""
    out = _i64(0)
    _check(lib().pcdm_omega_noalloc(ctypes.byref(csc), ctypes.byref(out), _stream(stream)), None)
    return int(out.value)


# ---------------------------------------------------------------------------- batched solver
def _bcheck(status, handle=None):
    if status != PCDM_OK:
        msg = lib().pcdm_batch_last_error(handle)
        raise PcdmError(status, (msg or b"").decode(errors="replace"))


def pcdm_batch_create(A, nrhs, B_ptr, b_dtype, lambdas, opts=None, stream=0):
    lam = (ctypes.c_double * int(nrhs))(*[float(v) for v in lambdas])
    h = _ptr()
    st = lib().pcdm_batch_create(ctypes.byref(A), int(nrhs), _ptr(B_ptr), int(b_dtype), ctypes.cast(lam, _ptr),
                                 ctypes.byref(opts) if opts is not None else None, _stream(stream), ctypes.byref(h))
    _bcheck(st, None)
    return h


def pcdm_batch_step(h, tau, iters, seed):
    _bcheck(lib().pcdm_batch_step(h, int(tau), int(iters), int(seed) & (2**64 - 1)), h)


def pcdm_batch_refresh(h):
    _bcheck(lib().pcdm_batch_refresh(h), h)


def pcdm_batch_gap(h, nrhs):
    p, d, g = (ctypes.c_double * nrhs)(), (ctypes.c_double * nrhs)(), (ctypes.c_double * nrhs)()
    _bcheck(lib().pcdm_batch_gap(h, ctypes.cast(p, _ptr), ctypes.cast(d, _ptr), ctypes.cast(g, _ptr)), h)
    return list(p), list(d), list(g)


def pcdm_batch_solve(h, nrhs, tau, seed, rel_gap_tol, max_iters):
    """Returns (converged, iters_done, [rel_gap per problem])."""
    it = _i64()
    rel = (ctypes.c_double * nrhs)()
    st = lib().pcdm_batch_solve(h, int(tau), int(seed) & (2**64 - 1), float(rel_gap_tol), int(max_iters),
                                ctypes.byref(it), ctypes.cast(rel, _ptr))
    if st == PCDM_ENOTCONV:
        return False, it.value, list(rel)
    _bcheck(st, h)
    return True, it.value, list(rel)


def pcdm_batch_get_x(h, ptr, on_device):
    _bcheck(lib().pcdm_batch_get_x(h, _ptr(ptr), int(on_device)), h)


def pcdm_batch_set_x(h, ptr, on_device):
    _bcheck(lib().pcdm_batch_set_x(h, _ptr(ptr), int(on_device)), h)


def pcdm_batch_set_lambda(h, lambdas):
    lam = (ctypes.c_double * len(lambdas))(*[float(v) for v in lambdas])
    _bcheck(lib().pcdm_batch_set_lambda(h, ctypes.cast(lam, _ptr)), h)


def pcdm_batch_reset(h):
    _bcheck(lib().pcdm_batch_reset(h), h)


def pcdm_batch_get_stats(h):
    s = pcdm_stats()
    _bcheck(lib().pcdm_batch_get_stats(h, ctypes.byref(s)), h)
    return {name: getattr(s, name) for name, _ in pcdm_stats._fields_}


def pcdm_batch_reset_stats(h):
    _bcheck(lib().pcdm_batch_reset_stats(h), h)


def pcdm_batch_autotune(h, tau, trial_iters):
    bps, us = _i32(0), _dbl(0.0)
    _bcheck(lib().pcdm_batch_autotune(h, int(tau), int(trial_iters), ctypes.byref(bps), ctypes.byref(us)), h)
    return {"blocks_per_sm": int(bps.value), "us_per_iteration": float(us.value)}


def pcdm_batch_destroy(h):
    lib().pcdm_batch_destroy(h)


def pcdm_batch_last_error(h=None):
    msg = lib().pcdm_batch_last_error(h)
    return (msg or b"").decode(errors="replace")


# ---------------------------------------------------------------------------- derivatives
def pcdm_set_b(h, ptr, b_dtype, on_device):
    _check(lib().pcdm_set_b(h, _ptr(ptr), int(b_dtype), int(on_device)), h)


def pcdm_support_size(h):
    v = _i64()
    _check(lib().pcdm_support_size(h, ctypes.byref(v)), h)
    return v.value


def pcdm_polish(h, tau, seed, tol, max_iters):
    """Returns (converged, iterations, relative residual)."""
    it, rel = _i64(), _dbl()
    st = lib().pcdm_polish(h, int(tau), int(seed) & (2**64 - 1), float(tol), int(max_iters), ctypes.byref(it),
                           ctypes.byref(rel))
    if st == PCDM_ENOTCONV:
        return False, it.value, rel.value
    _check(st, h)
    return True, it.value, rel.value


def pcdm_backward(h, dx_ptr, dx_on_device, db_ptr, db_on_device, tau, seed, tol, max_iters):
    """Returns (converged, dlambda, iterations, relative residual); db written in place."""
    dl, it, rel = _dbl(), _i64(), _dbl()
    st = lib().pcdm_backward(h, _ptr(dx_ptr), int(dx_on_device), _ptr(db_ptr), int(db_on_device), ctypes.byref(dl),
                             int(tau), int(seed) & (2**64 - 1), float(tol), int(max_iters), ctypes.byref(it),
                             ctypes.byref(rel))
    if st == PCDM_ENOTCONV:
        return False, dl.value, it.value, rel.value
    _check(st, h)
    return True, dl.value, it.value, rel.value


PCDM_SAMPLING_NICE, PCDM_SAMPLING_INDEPENDENT, PCDM_SAMPLING_BINOMIAL = 0, 1, 2
SAMPLING_CODES = {"nice": 0, "independent": 1, "binomial": 2}


def pcdm_sample_kind(kind, seed, k, n, tau, p_b, S_device_ptr, keep_device_ptr=None, stream=0):
    _check(lib().pcdm_sample_kind(int(kind), int(seed) & (2**64 - 1), int(k), int(n), int(tau), float(p_b),
                                  _ptr(S_device_ptr), _ptr(keep_device_ptr), _stream(stream)), None)


def pcdm_step_async(h, updates, seed, threads=0):
    _check(lib().pcdm_step_async(h, int(updates), int(seed) & (2**64 - 1), int(threads)), h)


def pcdm_solve_async(h, seed, rel_gap_tol, max_updates, threads=0):
    """Returns (converged, updates_done, rel_gap)."""
    u, rel = _i64(), _dbl()
    st = lib().pcdm_solve_async(h, int(seed) & (2**64 - 1), float(rel_gap_tol), int(max_updates), int(threads),
                                ctypes.byref(u), ctypes.byref(rel))
    if st == PCDM_ENOTCONV:
        return False, u.value, rel.value
    _check(st, h)
    return True, u.value, rel.value


# ---------------------------------------------------------------------------- many problems
def _mcheck(status, handle=None):
    if status != PCDM_OK:
        msg = lib().pcdm_multi_last_error(handle)
        raise PcdmError(status, (msg or b"").decode(errors="replace"))


def pcdm_multi_create(cscs, b_ptrs, b_dtype, lambdas, opts=None, stream=0):
    count = len(cscs)
    arr = (pcdm_csc * count)(*cscs)
    bp = (ctypes.c_void_p * count)(*[int(p) for p in b_ptrs])
    lam = (ctypes.c_double * count)(*[float(v) for v in lambdas])
    h = _ptr()
    st = lib().pcdm_multi_create(count, ctypes.cast(arr, _ptr), ctypes.cast(bp, _ptr), int(b_dtype),
                                 ctypes.cast(lam, _ptr), ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream), ctypes.byref(h))
    _mcheck(st, None)
    return h


def pcdm_multi_solve(h, count, tau, seed, tol, max_iters, iters_per_check):
    """Returns (all converged, [iterations], [relative gap])."""
    it = (ctypes.c_int64 * count)()
    rel = (ctypes.c_double * count)()
    st = lib().pcdm_multi_solve(h, int(tau), int(seed) & (2**64 - 1), float(tol), int(max_iters),
                                int(iters_per_check), ctypes.cast(it, _ptr), ctypes.cast(rel, _ptr))
    if st == PCDM_ENOTCONV:
        return False, list(it), list(rel)
    _mcheck(st, h)
    return True, list(it), list(rel)


def pcdm_multi_get_x(h, p, ptr):
    _mcheck(lib().pcdm_multi_get_x(h, int(p), _ptr(ptr)), h)


def pcdm_multi_reset(h):
    _mcheck(lib().pcdm_multi_reset(h), h)


def pcdm_multi_get_stats(h):
    s = pcdm_stats()
    _mcheck(lib().pcdm_multi_get_stats(h, ctypes.byref(s)), h)
    return {name: getattr(s, name) for name, _ in pcdm_stats._fields_}


def pcdm_multi_destroy(h):
    lib().pcdm_multi_destroy(h)


def pcdm_autotune(h, tau, trial_iters):
    t = pcdm_tuning()
    _check(lib().pcdm_autotune(h, int(tau), int(trial_iters), ctypes.byref(t)), h)
    return {name: getattr(t, name) for name, _ in pcdm_tuning._fields_}


def pcdm_set_tuning(h, kernel=None, lanes_per_col=1, threads_per_block=0, heads=1, zero_cert=-1):
    """kernel None: back to the built-in rule."""
    if kernel is None:
        _check(lib().pcdm_set_tuning(h, None), h)
        return
    t = pcdm_tuning(int(kernel), int(lanes_per_col), int(threads_per_block), int(heads), int(zero_cert), 0.0)
    _check(lib().pcdm_set_tuning(h, ctypes.byref(t)), h)


def pcdm_set_memory_cache(nbytes):
    _check(lib().pcdm_set_memory_cache(int(nbytes)), None)


def pcdm_release_cached_memory():
    _check(lib().pcdm_release_cached_memory(), None)

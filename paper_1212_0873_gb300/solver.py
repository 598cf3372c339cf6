"""A LASSO instance resident on the GPU and solved by PCDM1 through libpcdm.

Marshalling only: arrays are numpy (host memory, copied by the library) or
torch CUDA tensors (device memory, copied device to device); every step of the
method runs in the library's kernels.
"""
import numpy as np

from . import _binding as B

_NP_VAL = {np.dtype(np.float64): "f64", np.dtype(np.float32): "f32", np.dtype(np.uint16): "bf16"}


def _torch():
    import torch
    return torch


def _is_tensor(a):
    return type(a).__module__.startswith("torch")


def _ptr_and_device(a):
    if _is_tensor(a):
        if not a.is_cuda:
            raise ValueError("torch tensors must be CUDA tensors (host data goes in as numpy arrays)")
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous numpy arrays or CUDA tensors")
    return a.ctypes.data, 0


def _val_code(val):
    if _is_tensor(val):
        torch = _torch()
        table = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}
        return table[val.dtype]
    return _NP_VAL[val.dtype]


def current_stream():
    """The torch current CUDA stream handle (0 if torch has no CUDA)."""
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Lasso:
    """min 1/2 ||A x - b||^2 + lam ||x||_1 with A in CSC form, on one GPU."""

    def __init__(self, m, n, col_ptr, row_idx, val, b, lam, *, xg_dtype=None, fused=True, refresh_every=0,
                 check_every=0, lanes_per_col=0, profile=False, barrier_timeout_ns=None, stream=None,
                 sampling="nice", p_b=1.0, l2_persist=False, deterministic_scatter=False):
        val_dtype = _val_code(val)
        if xg_dtype is None:
            xg_dtype = "f64" if val_dtype == "f64" else "f32"
        self.m, self.n = int(m), int(n)
        self.val_dtype, self.xg_dtype = val_dtype, xg_dtype
        p_cp, d_cp = _ptr_and_device(col_ptr)
        p_ri, d_ri = _ptr_and_device(row_idx)
        p_v, d_v = _ptr_and_device(val)
        p_b_ptr, d_b = _ptr_and_device(b)
        if len({d_cp, d_ri, d_v, d_b}) != 1:
            raise ValueError("A and b must all be host arrays or all be device tensors")
        nnz = int(col_ptr[-1]) if not _is_tensor(col_ptr) else int(col_ptr[-1].item())
        A = B.pcdm_csc(self.m, self.n, nnz, p_cp, p_ri, p_v, B.DTYPE_CODES[val_dtype], d_cp)
        opts = B.pcdm_default_opts()
        opts.xg_dtype = B.DTYPE_CODES[xg_dtype]
        opts.fused = 1 if fused else 0
        opts.refresh_every = int(refresh_every)
        opts.check_every = int(check_every)
        opts.lanes_per_col = int(lanes_per_col)
        opts.profile = 1 if profile else 0
        opts.sampling = B.SAMPLING_CODES[sampling]
        opts.p_b = float(p_b)
        opts.l2_persist = 1 if l2_persist else 0
        opts.deterministic_scatter = 1 if deterministic_scatter else 0
        if barrier_timeout_ns is not None:
            opts.barrier_timeout_ns = int(barrier_timeout_ns)
        b_dt = B.PCDM_F32 if (str(getattr(b, "dtype", "")) in ("float32", "torch.float32")) else B.PCDM_F64
        self.stream = current_stream() if stream is None else stream
        self._h = B.pcdm_create(A, p_b_ptr, b_dt, lam, opts, self.stream)
        self.lam = float(lam)

    @classmethod
    def from_instance(cls, inst, **kw):
        return cls(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, inst.b, inst.lam, **kw)

    # -------------------------------------------------------------- the method
    def step(self, tau, iters, seed=0):
        B.pcdm_step(self._h, tau, iters, seed)

    def refresh(self):
        B.pcdm_refresh(self._h)

    def gap(self):
        p, d, g = B.pcdm_gap(self._h)
        return dict(primal=p, dual=d, gap=g, rel_gap=g / max(p, 1e-300))

    def solve(self, tau, seed=0, tol=1e-6, max_iters=10**9):
        """Returns (converged, iterations, relative gap)."""
        return B.pcdm_solve(self._h, tau, seed, tol, max_iters)

    # -------------------------------------------------------------- state
    def _np_g(self, count):
        return np.empty(count, dtype=np.float64 if self.xg_dtype == "f64" else np.float32)

    def x(self):
        out = np.empty(self.n, dtype=np.float64)
        B.pcdm_get_x(self._h, out.ctypes.data, 0)
        return out

    def x_into(self, tensor):
        """Copy x into a CUDA float64 tensor of n entries."""
        B.pcdm_get_x(self._h, tensor.data_ptr(), 1)
        return tensor

    def set_x(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64) if not _is_tensor(x) else x
        p, d = _ptr_and_device(x)
        B.pcdm_set_x(self._h, p, d)

    def autotune(self, tau, trial_iters=50):
        """Pick the fastest iteration kernel for tau on this matrix (pcdm_autotune)."""
        return B.pcdm_autotune(self._h, tau, trial_iters)

    def set_tuning(self, kernel=None, lanes_per_col=1, threads_per_block=0, heads=1, zero_cert=-1):
        """Choose the iteration kernel (0 pipelined, 1 fused, 2 two-kernel, 3 pipelined
        rounds, 4 streaming, 5 warp-cooperative) by hand, whether the pipelined kernels read the column heads, and
        whether the FP64 pipelined kernel certifies zero steps in FP32 first (-1: the
        built-in rule); None returns to the built-in rule."""
        B.pcdm_set_tuning(self._h, kernel, lanes_per_col, threads_per_block, heads, zero_cert)

    def step_async(self, updates, seed=0, threads=0):
        """Asynchronous updates (pcdm_step_async); threads = 1 is the serial method."""
        B.pcdm_step_async(self._h, updates, seed, threads)

    def solve_async(self, seed=0, tol=1e-6, max_updates=10**12, threads=0):
        """Returns (converged, updates, relative gap)."""
        return B.pcdm_solve_async(self._h, seed, tol, max_updates, threads)

    def set_b(self, b):
        """New right-hand side (m entries, numpy or CUDA tensor); x is kept."""
        if not _is_tensor(b):
            b = np.ascontiguousarray(b, dtype=np.float64)
        b_dt = B.PCDM_F32 if (str(getattr(b, "dtype", "")) in ("float32", "torch.float32")) else B.PCDM_F64
        p, d = _ptr_and_device(b)
        B.pcdm_set_b(self._h, p, b_dt, d)

    def support_size(self):
        return B.pcdm_support_size(self._h)

    def polish(self, tol=1e-13, max_iters=100_000, tau=0, seed=0):
        """Solve the optimality system on the current support and signs
        (pcdm_polish); returns (converged, iterations, relative residual)."""
        return B.pcdm_polish(self._h, tau, seed, tol, max_iters)

    def backward(self, dx, tol=1e-12, max_iters=100_000, tau=0, seed=0, db_out=None):
        """dL/db (m) and dL/dlambda at the current x for dx = dL/dx (pcdm_backward).
        dx: numpy or CUDA float64; db_out: optional CUDA float64 tensor of m.
        Returns (db, dlambda, converged, iterations, relative residual)."""
        if not _is_tensor(dx):
            dx = np.ascontiguousarray(dx, dtype=np.float64)
        p_dx, d_dx = _ptr_and_device(dx)
        if db_out is None:
            db_out = np.empty(self.m, dtype=np.float64)
        p_db, d_db = _ptr_and_device(db_out)
        ok, dl, it, rel = B.pcdm_backward(self._h, p_dx, d_dx, p_db, d_db, tau, seed, tol, max_iters)
        return db_out, dl, ok, it, rel

    def residual(self):
        out = self._np_g(self.m)
        B.pcdm_get_residual(self._h, out.ctypes.data, 0)
        return out

    def L(self):
        out = np.empty(self.n, dtype=np.float64)
        B.pcdm_get_L(self._h, out.ctypes.data, 0)
        return out

    @property
    def omega(self):
        return B.pcdm_omega(self._h)

    def beta(self, tau):
        return B.pcdm_beta(self._h, tau)

    @property
    def iteration(self):
        return B.pcdm_get_iteration(self._h)

    @iteration.setter
    def iteration(self, k):
        B.pcdm_set_iteration(self._h, k)

    def set_lambda(self, lam):
        B.pcdm_set_lambda(self._h, lam)
        self.lam = float(lam)

    def reset(self):
        B.pcdm_reset(self._h)

    def stats(self):
        return B.pcdm_get_stats(self._h)

    def reset_stats(self):
        B.pcdm_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None):
            B.pcdm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchLasso:
    """nrhs <= 32 problems min 1/2 ||A x - b_l||^2 + lam_l ||x||_1 sharing A, solved together
    (pcdm_batch_*).  B is (nrhs, m): row l is b_l."""

    def __init__(self, m, n, col_ptr, row_idx, val, B_rhs, lams, *, xg_dtype=None, refresh_every=0, check_every=0,
                 profile=False, barrier_timeout_ns=None, stream=None):
        val_dtype = _val_code(val)
        if xg_dtype is None:
            xg_dtype = "f64" if val_dtype == "f64" else "f32"
        self.m, self.n = int(m), int(n)
        self.nrhs = int(B_rhs.shape[0])
        if tuple(B_rhs.shape) != (self.nrhs, self.m):
            raise ValueError("B must have shape (nrhs, m)")
        self.val_dtype, self.xg_dtype = val_dtype, xg_dtype
        p_cp, d_cp = _ptr_and_device(col_ptr)
        p_ri, d_ri = _ptr_and_device(row_idx)
        p_v, d_v = _ptr_and_device(val)
        p_b, d_b = _ptr_and_device(B_rhs)
        if len({d_cp, d_ri, d_v, d_b}) != 1:
            raise ValueError("A and B must all be host arrays or all be device tensors")
        nnz = int(col_ptr[-1]) if not _is_tensor(col_ptr) else int(col_ptr[-1].item())
        A = B.pcdm_csc(self.m, self.n, nnz, p_cp, p_ri, p_v, B.DTYPE_CODES[val_dtype], d_cp)
        opts = B.pcdm_default_opts()
        opts.xg_dtype = B.DTYPE_CODES[xg_dtype]
        opts.refresh_every = int(refresh_every)
        opts.check_every = int(check_every)
        opts.profile = 1 if profile else 0
        if barrier_timeout_ns is not None:
            opts.barrier_timeout_ns = int(barrier_timeout_ns)
        b_dt = B.PCDM_F32 if (str(getattr(B_rhs, "dtype", "")) in ("float32", "torch.float32")) else B.PCDM_F64
        self.stream = current_stream() if stream is None else stream
        self.lams = [float(v) for v in lams]
        if len(self.lams) != self.nrhs:
            raise ValueError("one lambda per right-hand side")
        self._h = B.pcdm_batch_create(A, self.nrhs, p_b, b_dt, self.lams, opts, self.stream)

    def step(self, tau, iters, seed=0):
        B.pcdm_batch_step(self._h, tau, iters, seed)

    def refresh(self):
        B.pcdm_batch_refresh(self._h)

    def gap(self):
        p, d, g = B.pcdm_batch_gap(self._h, self.nrhs)
        p, d, g = np.array(p), np.array(d), np.array(g)
        return dict(primal=p, dual=d, gap=g, rel_gap=g / np.maximum(p, 1e-300))

    def solve(self, tau, seed=0, tol=1e-6, max_iters=10**9):
        """Returns (all converged, iterations, relative gap per problem)."""
        ok, it, rel = B.pcdm_batch_solve(self._h, self.nrhs, tau, seed, tol, max_iters)
        return ok, it, np.array(rel)

    def x(self):
        out = np.empty((self.nrhs, self.n), dtype=np.float64)
        B.pcdm_batch_get_x(self._h, out.ctypes.data, 0)
        return out

    def set_x(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64) if not _is_tensor(X) else X
        if tuple(X.shape) != (self.nrhs, self.n):
            raise ValueError("X must have shape (nrhs, n)")
        p, d = _ptr_and_device(X)
        B.pcdm_batch_set_x(self._h, p, d)

    def set_lambda(self, lams):
        lams = [float(v) for v in lams]
        if len(lams) != self.nrhs:
            raise ValueError("one lambda per right-hand side")
        B.pcdm_batch_set_lambda(self._h, lams)
        self.lams = lams

    def autotune(self, tau, trial_iters=20):
        """Pick the grid of the batched iteration kernel for tau (pcdm_batch_autotune)."""
        return B.pcdm_batch_autotune(self._h, tau, trial_iters)

    def reset(self):
        B.pcdm_batch_reset(self._h)

    def stats(self):
        return B.pcdm_batch_get_stats(self._h)

    def reset_stats(self):
        B.pcdm_batch_reset_stats(self._h)

    def close(self):
        if getattr(self, "_h", None):
            B.pcdm_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiLasso:
    """Many independent LASSO problems (each its own A, b, lambda; numpy host
    arrays), one GPU thread block per problem (pcdm_multi_*)."""

    def __init__(self, problems, *, xg_dtype=None, stream=None):
        """problems: sequence of (m, n, col_ptr, row_idx, val, b, lam)."""
        vals = {_val_code(pr[4]) for pr in problems}
        if len(vals) != 1:
            raise ValueError("every problem must store its values in the same dtype")
        val_dtype = vals.pop()
        if xg_dtype is None:
            xg_dtype = "f64" if val_dtype == "f64" else "f32"
        self._keep = []
        cscs, bps, lams, self.ns = [], [], [], []
        for m, n, col_ptr, row_idx, val, b, lam in problems:
            col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int64)
            row_idx = np.ascontiguousarray(row_idx, dtype=np.int32)
            val = np.ascontiguousarray(val)
            b = np.ascontiguousarray(b, dtype=np.float64)
            self._keep += [col_ptr, row_idx, val, b]
            cscs.append(B.pcdm_csc(int(m), int(n), int(col_ptr[-1]), col_ptr.ctypes.data, row_idx.ctypes.data,
                                   val.ctypes.data, B.DTYPE_CODES[val_dtype], 0))
            bps.append(b.ctypes.data)
            lams.append(float(lam))
            self.ns.append(int(n))
        opts = B.pcdm_default_opts()
        opts.xg_dtype = B.DTYPE_CODES[xg_dtype]
        self.count = len(cscs)
        self.stream = current_stream() if stream is None else stream
        self._h = B.pcdm_multi_create(cscs, bps, B.PCDM_F64, lams, opts, self.stream)
        self._keep = None

    def solve(self, tau=256, seed=0, tol=1e-6, max_iters=10**7, iters_per_check=64):
        ok, it, rel = B.pcdm_multi_solve(self._h, self.count, tau, seed, tol, max_iters, iters_per_check)
        return ok, np.array(it), np.array(rel)

    def x(self, p):
        out = np.empty(self.ns[p], dtype=np.float64)
        B.pcdm_multi_get_x(self._h, p, out.ctypes.data)
        return out

    def reset(self):
        B.pcdm_multi_reset(self._h)

    def stats(self):
        return B.pcdm_multi_get_stats(self._h)

    def close(self):
        if getattr(self, "_h", None):
            B.pcdm_multi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LabeledProblem(Lasso):
    """PCDM1 on the SVM dual (Sec. 8.3, problem "svm_dual": A is d x n with one
    example per column and y one label per column) or on L2-regularised logistic
    regression (Sec. 8.4, problem "logistic": one example per row, y one label
    per row), through pcdm_create_problem.  Same methods as Lasso; residual()
    returns sum_i y_i x_i A_i (SVM dual) or the margins y_j A_j^T x (logistic),
    and gap() the primal, dual and duality gap of that problem."""

    def __init__(self, problem, m, n, col_ptr, row_idx, val, y, lam, *, xg_dtype=None, fused=True, refresh_every=0,
                 check_every=0, lanes_per_col=0, profile=False, barrier_timeout_ns=None, stream=None,
                 sampling="nice", p_b=1.0):
        val_dtype = _val_code(val)
        if xg_dtype is None:
            xg_dtype = "f64" if val_dtype == "f64" else "f32"
        self.m, self.n = int(m), int(n)
        self.val_dtype, self.xg_dtype = val_dtype, xg_dtype
        self.problem = problem
        p_cp, d_cp = _ptr_and_device(col_ptr)
        p_ri, d_ri = _ptr_and_device(row_idx)
        p_v, d_v = _ptr_and_device(val)
        if not _is_tensor(y):
            y = np.ascontiguousarray(y, dtype=np.float64)
        p_y, d_y = _ptr_and_device(y)
        if len({d_cp, d_ri, d_v, d_y}) != 1:
            raise ValueError("A and y must all be host arrays or all be device tensors")
        nnz = int(col_ptr[-1]) if not _is_tensor(col_ptr) else int(col_ptr[-1].item())
        A = B.pcdm_csc(self.m, self.n, nnz, p_cp, p_ri, p_v, B.DTYPE_CODES[val_dtype], d_cp)
        opts = B.pcdm_default_opts()
        opts.xg_dtype = B.DTYPE_CODES[xg_dtype]
        opts.fused = 1 if fused else 0
        opts.refresh_every = int(refresh_every)
        opts.check_every = int(check_every)
        opts.lanes_per_col = int(lanes_per_col)
        opts.profile = 1 if profile else 0
        opts.sampling = B.SAMPLING_CODES[sampling]
        opts.p_b = float(p_b)
        if barrier_timeout_ns is not None:
            opts.barrier_timeout_ns = int(barrier_timeout_ns)
        self.stream = current_stream() if stream is None else stream
        self._h = B.pcdm_create_problem(A, problem, p_y, lam, opts, self.stream)
        self.lam = float(lam)

    @classmethod
    def from_instance(cls, inst, **kw):
        return cls(inst.problem, inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, inst.y, inst.lam, **kw)

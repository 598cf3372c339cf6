"""Plain FP64 CPU oracle for PCDM1 (arXiv:1212.0873) on LASSO, the SVM dual and
L2-regularised logistic regression.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py, never by the product package.  The arithmetic
lives in pcdm_oracle.c (single-threaded IEEE double, steps in the paper's order);
this module only marshals numpy arrays into it.

Citations (sections, equations and tables of the paper):
  sample         tau-nice sampling, Sec. 4.1 item 3, via the keyed permutation spec
                 in pcdm_oracle.c
  col_sqnorms    L_i = ||a_i||^2 (Sec. 3, "Partial separability" item)
  omega          max_j ||A_j||_0 (Sec. 1, examples of partially separable functions)
  beta_nice      Theorem ESO-nice, Table ESO
  iteration      Algorithm 1 step 4 with h(x) of eq. (h(x)) for Omega = lambda ||.||_1
  residual       g = A x - b
  objective      F(x) of eq. (P) for LASSO (Sec. 8.1)
  gap            LASSO duality gap at theta = min(1, lambda/||A^T g||_inf) g
  run            iterations of Algorithm 1 with periodic residual refresh
  sample_independent, binomial_keep, q_independent, moments, beta_du, run_sampling
                 the tau-independent and (tau, p_b)-binomial samplings (Sec. 4.1
                 items 4 and 5) and beta of Theorem ESO-DU
  glm_*, GlmState
                 PCDM1 on the SVM dual (Sec. 8.3) and on L2-regularised logistic
                 regression (Sec. 8.4): L_i, the kept vector (u or A x), the
                 gradient, objective, duality gap, iteration and run
                 (pcdm_oracle_glm.c)
  active_set_solution, implicit_grad
                 the LASSO optimality condition on a fixed support and sign
                 pattern, and the implicit-function derivatives of the solution
                 (dense numpy solves; tiny inputs only).  The paper has no
                 derivatives; these are the definitions the GPU backward is
                 checked against.

Every function here is pinned by a -m "not gpu" test in tests/test_oracle_*.py.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def use_library(path):
    """Point the wrapper at another build of pcdm_oracle.c (the mutation test
    loads copies with planted mistakes); None returns to the normal build."""
    global _lib
    _lib = None
    if path is not None:
        _lib = _declare(ctypes.CDLL(path))


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


def _declare(L):
    if True:
        L.pcdm_oracle_philox4x32_10.argtypes = [_ptr, _ptr, _ptr]
        L.pcdm_oracle_philox4x32_10.restype = None
        L.pcdm_oracle_sample.argtypes = [_u64, _i64, _i64, _i64, _ptr]
        L.pcdm_oracle_sample.restype = ctypes.c_int
        L.pcdm_oracle_sample_many.argtypes = [_u64, _i64, _i64, _i64, _i64, _ptr]
        L.pcdm_oracle_sample_many.restype = ctypes.c_int
        L.pcdm_oracle_feistel_rounds.argtypes = []
        L.pcdm_oracle_feistel_rounds.restype = ctypes.c_int
        L.pcdm_oracle_col_sqnorms.argtypes = [_i64, _ptr, _ptr, _ptr]
        L.pcdm_oracle_col_sqnorms.restype = None
        L.pcdm_oracle_omega.argtypes = [_i64, _i64, _ptr, _ptr]
        L.pcdm_oracle_omega.restype = _i64
        L.pcdm_oracle_beta_nice.argtypes = [_i64, _i64, _i64]
        L.pcdm_oracle_beta_nice.restype = _dbl
        L.pcdm_oracle_iteration.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, _i64,
                                            _ptr, _ptr, _ptr, _ptr, _ptr]
        L.pcdm_oracle_iteration.restype = None
        L.pcdm_oracle_residual.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr]
        L.pcdm_oracle_residual.restype = None
        L.pcdm_oracle_objective.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl]
        L.pcdm_oracle_objective.restype = _dbl
        L.pcdm_oracle_sample_independent.argtypes = [_u64, _i64, _i64, _i64, _ptr, _ptr]
        L.pcdm_oracle_sample_independent.restype = ctypes.c_int
        L.pcdm_oracle_binomial_keep.argtypes = [_u64, _i64, _i64, _dbl, _ptr]
        L.pcdm_oracle_binomial_keep.restype = None
        L.pcdm_oracle_q_independent.argtypes = [_i64, _i64, _ptr]
        L.pcdm_oracle_q_independent.restype = None
        L.pcdm_oracle_moments.argtypes = [ctypes.c_int, _i64, _i64, _dbl, _ptr, _ptr]
        L.pcdm_oracle_moments.restype = None
        L.pcdm_oracle_beta_du.argtypes = [_i64, _dbl, _dbl, _i64]
        L.pcdm_oracle_beta_du.restype = _dbl
        L.pcdm_oracle_run_sampling.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, ctypes.c_int,
                                               _dbl, _i64, _u64, _i64, _i64, _i64, _ptr, _ptr]
        L.pcdm_oracle_run_sampling.restype = ctypes.c_int
        L.pcdm_oracle_gap.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _ptr]
        L.pcdm_oracle_gap.restype = None
        L.pcdm_oracle_run.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, _i64,
                                      _u64, _i64, _i64, _i64, _ptr, _ptr]
        L.pcdm_oracle_run.restype = ctypes.c_int
        L.pcdm_oracle_run_threads.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, _i64,
                                              _u64, _i64, _i64, _i64, _ptr, _ptr, ctypes.c_int]
        L.pcdm_oracle_run_threads.restype = ctypes.c_int
        L.pcdm_oracle_sample_range.argtypes = [_u64, _i64, _i64, _i64, _i64, _ptr]
        L.pcdm_oracle_sample_range.restype = ctypes.c_int
        _ci = ctypes.c_int
        L.pcdm_oracle_glm_lipschitz.argtypes = [_ci, _i64, _ptr, _ptr, _dbl, _ptr]
        L.pcdm_oracle_glm_lipschitz.restype = None
        L.pcdm_oracle_glm_residual.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr]
        L.pcdm_oracle_glm_residual.restype = None
        L.pcdm_oracle_glm_gradient.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _ptr]
        L.pcdm_oracle_glm_gradient.restype = None
        L.pcdm_oracle_glm_objective.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl]
        L.pcdm_oracle_glm_objective.restype = _dbl
        L.pcdm_oracle_glm_gap.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _ptr]
        L.pcdm_oracle_glm_gap.restype = None
        L.pcdm_oracle_glm_iteration.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, _i64,
                                                _ptr, _ptr, _ptr, _ptr, _ptr]
        L.pcdm_oracle_glm_iteration.restype = None
        L.pcdm_oracle_glm_run.argtypes = [_ci, _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _dbl, _dbl, _i64, _u64,
                                          _i64, _i64, _i64, _ptr, _ptr]
        L.pcdm_oracle_glm_run.restype = ctypes.c_int
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Csc:
    """A in compressed sparse column form with FP64 values (the stored values of
    an FP32 or BF16 instance promoted exactly to FP64)."""

    def __init__(self, m, n, col_ptr, row_idx, val):
        self.m = int(m)
        self.n = int(n)
        self.col_ptr = _c(col_ptr, np.int64)
        self.row_idx = _c(row_idx, np.int32)
        self.val = _c(val, np.float64)
        assert self.col_ptr.shape == (self.n + 1,)
        assert self.row_idx.shape == self.val.shape == (int(self.col_ptr[-1]),)

    def args(self):
        return (self.m, self.n, _p(self.col_ptr), _p(self.row_idx), _p(self.val))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().pcdm_oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sample_many(seed, k0, K, n, tau):
    """Samples of iterations k0..k0+K-1 as a (K, tau) int32 array."""
    out = np.zeros((int(K), int(tau)), dtype=np.int32)
    rc = lib().pcdm_oracle_sample_many(int(seed) & (2**64 - 1), int(k0), int(K), int(n), int(tau), _p(out))
    if rc != 0:
        raise ValueError("bad sampler sizes")
    return out


def feistel_rounds():
    return int(lib().pcdm_oracle_feistel_rounds())


def sample(seed, k, n, tau):
    S = np.zeros(max(int(tau), 1), dtype=np.int32)
    rc = lib().pcdm_oracle_sample(int(seed) & (2**64 - 1), int(k), int(n), int(tau), _p(S))
    if rc != 0:
        raise ValueError("bad sampler sizes")
    return S[: int(tau)]


def col_sqnorms(A: Csc):
    L = np.zeros(max(A.n, 1), dtype=np.float64)
    lib().pcdm_oracle_col_sqnorms(A.n, _p(A.col_ptr), _p(A.val), _p(L))
    return L[: A.n]


def omega(A: Csc):
    return int(lib().pcdm_oracle_omega(A.m, A.n, _p(A.col_ptr), _p(A.row_idx)))


def beta_nice(omega_, tau, n):
    return float(lib().pcdm_oracle_beta_nice(int(omega_), int(tau), int(n)))


def residual(A: Csc, b, x):
    b = _c(b, np.float64)
    x = _c(x, np.float64)
    g = np.zeros(max(A.m, 1), dtype=np.float64)
    lib().pcdm_oracle_residual(*A.args(), _p(b), _p(x), _p(g))
    return g[: A.m]


def objective(A: Csc, b, x, lam):
    b = _c(b, np.float64)
    x = _c(x, np.float64)
    return float(lib().pcdm_oracle_objective(*A.args(), _p(b), _p(x), float(lam)))


GAP_FIELDS = ("primal", "dual", "gap", "cinf", "s", "rr", "br", "l1", "xc")


def gap(A: Csc, b, x, r, lam):
    """Duality-gap record at x with residual r (dict keyed by GAP_FIELDS)."""
    b = _c(b, np.float64)
    x = _c(x, np.float64)
    r = _c(r, np.float64)
    out = np.zeros(9, dtype=np.float64)
    lib().pcdm_oracle_gap(*A.args(), _p(b), _p(x), _p(r), float(lam), _p(out))
    return dict(zip(GAP_FIELDS, (float(v) for v in out)))


def iteration(A: Csc, L, lam, beta, S, x, g):
    """One Jacobi PCDM1 iteration on the explicit coordinate set S (in place on x, g)."""
    S = _c(S, np.int32)
    L = _c(L, np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    assert g.dtype == np.float64 and g.flags.c_contiguous
    tau = S.shape[0]
    hbuf = np.zeros(max(tau, 1))
    xbuf = np.zeros(max(tau, 1))
    lib().pcdm_oracle_iteration(*A.args(), _p(L), float(lam), float(beta), tau, _p(S), _p(x), _p(g),
                                _p(hbuf), _p(xbuf))


class State:
    """Oracle state (x, g, k) of one PCDM1 run on one instance."""

    def __init__(self, A: Csc, b, lam, x0=None):
        self.A = A
        self.b = _c(b, np.float64)
        self.lam = float(lam)
        self.L = col_sqnorms(A)
        self.omega = omega(A)
        self.x = np.zeros(A.n) if x0 is None else _c(x0, np.float64).copy()
        self.g = residual(A, self.b, self.x)
        self.k = 0

    def beta(self, tau):
        return beta_nice(self.omega, tau, self.A.n)

    def run(self, tau, iters, seed, refresh_every=0, beta=None):
        b_ = self.beta(tau) if beta is None else float(beta)
        rc = lib().pcdm_oracle_run(*self.A.args(), _p(self.b), _p(self.L), self.lam, b_, int(tau),
                                   int(seed) & (2**64 - 1), int(self.k), int(iters), int(refresh_every),
                                   _p(self.x), _p(self.g))
        if rc != 0:
            raise ValueError("oracle run failed")
        self.k += int(iters)

    def run_threads(self, tau, iters, seed, threads, refresh_every=0, beta=None):
        """run() on `threads` host threads (the timing mode of the CPU baseline):
        the same iterations, equal to run() bit for bit."""
        b_ = self.beta(tau) if beta is None else float(beta)
        rc = lib().pcdm_oracle_run_threads(*self.A.args(), _p(self.b), _p(self.L), self.lam, b_, int(tau),
                                           int(seed) & (2**64 - 1), int(self.k), int(iters), int(refresh_every),
                                           _p(self.x), _p(self.g), int(threads))
        if rc != 0:
            raise ValueError("oracle threaded run failed")
        self.k += int(iters)

    def run_sampling(self, kind, tau, iters, seed, p_b=1.0, refresh_every=0, beta=None):
        """run() with the sampling `kind` ("nice", "independent", "binomial") and
        beta of Theorem ESO-DU unless given."""
        b_ = beta_sampling(self.omega, kind, tau, self.A.n, p_b) if beta is None else float(beta)
        rc = lib().pcdm_oracle_run_sampling(*self.A.args(), _p(self.b), _p(self.L), self.lam, b_, SAMPLINGS[kind],
                                            float(p_b), int(tau), int(seed) & (2**64 - 1), int(self.k), int(iters),
                                            int(refresh_every), _p(self.x), _p(self.g))
        if rc != 0:
            raise ValueError("oracle run failed")
        self.k += int(iters)

    def refresh(self):
        self.g = residual(self.A, self.b, self.x)

    def gap(self):
        """Refresh the residual (as the library's gap call does) and return the gap record."""
        self.refresh()
        return gap(self.A, self.b, self.x, self.g, self.lam)

    def objective(self):
        return objective(self.A, self.b, self.x, self.lam)

    def solve(self, tau, seed, rel_gap_tol, max_iters, check_every, refresh_every=0):
        """Iterate in chunks of check_every until gap/P <= rel_gap_tol; returns (iters, rel_gap)."""
        done = 0
        rec = self.gap()
        rel = rec["gap"] / max(rec["primal"], 1e-300)
        while rel > rel_gap_tol and done < max_iters:
            chunk = min(check_every, max_iters - done)
            self.run(tau, chunk, seed, refresh_every)
            done += chunk
            rec = self.gap()
            rel = rec["gap"] / max(rec["primal"], 1e-300)
        return done, rel


# ----------------------------------------------------------------------------- other samplings
SAMPLINGS = {"nice": 0, "independent": 1, "binomial": 2}


def sample_independent(seed, k, n, tau):
    """(picks, active): tau iid picks and the first-occurrence flags (Sec. 4.1 item 4)."""
    S = np.empty(tau, dtype=np.int32)
    act = np.empty(tau, dtype=np.uint8)
    if lib().pcdm_oracle_sample_independent(int(seed) & (2**64 - 1), int(k), int(n), int(tau), _p(S), _p(act)):
        raise ValueError("bad sizes")
    return S, act.astype(bool)


def binomial_keep(seed, k, tau, p_b):
    act = np.empty(tau, dtype=np.uint8)
    lib().pcdm_oracle_binomial_keep(int(seed) & (2**64 - 1), int(k), int(tau), float(p_b), _p(act))
    return act.astype(bool)


def q_independent(n, tau):
    q = np.zeros(int(tau) + 1)
    lib().pcdm_oracle_q_independent(int(n), int(tau), _p(q))
    return q


def moments(kind, n, tau, p_b=1.0):
    e1, e2 = _dbl(), _dbl()
    lib().pcdm_oracle_moments(SAMPLINGS[kind], int(n), int(tau), float(p_b), ctypes.byref(e1), ctypes.byref(e2))
    return e1.value, e2.value


def beta_du(omega_, e1, e2, n):
    return float(lib().pcdm_oracle_beta_du(int(omega_), float(e1), float(e2), int(n)))


def beta_sampling(omega_, kind, tau, n, p_b=1.0):
    e1, e2 = moments(kind, n, tau, p_b)
    return beta_du(omega_, e1, e2, n)


# ----------------------------------------------------------------------------- derivatives (dense)
def _dense_columns(A: Csc, S):
    cp, ri, v = A.col_ptr, A.row_idx, A.val
    D = np.zeros((A.m, len(S)))
    for q, i in enumerate(S):
        D[ri[cp[i]:cp[i + 1]], q] = v[cp[i]:cp[i + 1]]
    return D


def active_set_solution(A: Csc, b, lam, S, s):
    """x with x_S solving A_S^T (A_S x_S - b) + lam s = 0 and x = 0 off S."""
    S = np.asarray(S, dtype=np.int64)
    x = np.zeros(A.n)
    if S.size:
        AS = _dense_columns(A, S)
        x[S] = np.linalg.solve(AS.T @ AS, AS.T @ np.asarray(b, dtype=np.float64) - lam * np.asarray(s, float))
    return x


def implicit_grad(A: Csc, x, lam, dx):
    """(dL/db, dL/dlam) at a LASSO solution x for dL/dx = dx: with S = supp(x),
    s = sign(x_S) and (A_S^T A_S) u = dx_S, dL/db = A_S u, dL/dlam = -s^T u."""
    x = np.asarray(x, dtype=np.float64)
    S = np.nonzero(x)[0]
    if S.size == 0:
        return np.zeros(A.m), 0.0
    AS = _dense_columns(A, S)
    u = np.linalg.solve(AS.T @ AS, np.asarray(dx, dtype=np.float64)[S])
    return AS @ u, float(-np.sign(x[S]) @ u)


# ----------------------------------------------------------------------------- SVM dual and logistic
# problem codes: 1 = dual of the L2-regularised hinge-loss SVM (Sec. 8.3),
# 2 = L2-regularised logistic regression (Sec. 8.4); see pcdm_oracle_glm.c.
SVM_DUAL = 1
LOGISTIC = 2


def glm_lipschitz(problem, A: Csc, lam):
    L = np.zeros(max(A.n, 1))
    lib().pcdm_oracle_glm_lipschitz(int(problem), A.n, _p(A.col_ptr), _p(A.val), float(lam), _p(L))
    return L[: A.n]


def glm_residual(problem, A: Csc, y, x):
    """SVM: u = sum_i y_i x_i A_i.  Logistic: z = A x."""
    y = _c(y, np.float64)
    x = _c(x, np.float64)
    v = np.zeros(max(A.m, 1))
    lib().pcdm_oracle_glm_residual(int(problem), *A.args(), _p(y), _p(x), _p(v))
    return v[: A.m]


def glm_gradient(problem, A: Csc, y, v, lam):
    y = _c(y, np.float64)
    v = _c(v, np.float64)
    gr = np.zeros(max(A.n, 1))
    lib().pcdm_oracle_glm_gradient(int(problem), *A.args(), _p(y), _p(v), float(lam), _p(gr))
    return gr[: A.n]


def glm_objective(problem, A: Csc, y, x, lam):
    y = _c(y, np.float64)
    x = _c(x, np.float64)
    return float(lib().pcdm_oracle_glm_objective(int(problem), *A.args(), _p(y), _p(x), float(lam)))


def glm_gap(problem, A: Csc, y, x, lam):
    """{primal, dual, gap} at x, from scratch."""
    y = _c(y, np.float64)
    x = _c(x, np.float64)
    out = np.zeros(3)
    lib().pcdm_oracle_glm_gap(int(problem), *A.args(), _p(y), _p(x), float(lam), _p(out))
    return {"primal": float(out[0]), "dual": float(out[1]), "gap": float(out[2])}


def glm_iteration(problem, A: Csc, y, L, lam, beta, S, x, v):
    """One Jacobi iteration on the explicit set S (in place on x, v)."""
    y = _c(y, np.float64)
    L = _c(L, np.float64)
    S = _c(S, np.int32)
    assert x.dtype == np.float64 and x.flags.c_contiguous and v.dtype == np.float64 and v.flags.c_contiguous
    tau = S.shape[0]
    hb = np.zeros(max(tau, 1))
    xb = np.zeros(max(tau, 1))
    lib().pcdm_oracle_glm_iteration(int(problem), *A.args(), _p(y), _p(L), float(lam), float(beta), tau, _p(S),
                                    _p(x), _p(v), _p(hb), _p(xb))


class GlmState:
    """Oracle state (x, v, k) of one PCDM1 run on the SVM dual or logistic regression."""

    def __init__(self, problem, A: Csc, y, lam, x0=None):
        self.problem = int(problem)
        self.A = A
        self.y = _c(y, np.float64)
        self.lam = float(lam)
        self.L = glm_lipschitz(problem, A, lam)
        self.omega = omega(A)
        self.x = np.zeros(A.n) if x0 is None else _c(x0, np.float64).copy()
        self.v = glm_residual(problem, A, self.y, self.x)
        self.k = 0

    def beta(self, tau):
        return beta_nice(self.omega, tau, self.A.n)

    def run(self, tau, iters, seed, refresh_every=0, beta=None):
        b_ = self.beta(tau) if beta is None else float(beta)
        rc = lib().pcdm_oracle_glm_run(self.problem, *self.A.args(), _p(self.y), _p(self.L), self.lam, b_, int(tau),
                                       int(seed) & (2**64 - 1), int(self.k), int(iters), int(refresh_every),
                                       _p(self.x), _p(self.v))
        if rc != 0:
            raise ValueError("oracle run failed")
        self.k += int(iters)

    def refresh(self):
        self.v = glm_residual(self.problem, self.A, self.y, self.x)

    def gradient(self):
        return glm_gradient(self.problem, self.A, self.y, self.v, self.lam)

    def objective(self):
        return glm_objective(self.problem, self.A, self.y, self.x, self.lam)

    def gap(self):
        return glm_gap(self.problem, self.A, self.y, self.x, self.lam)

"""Parity at the benchmark's full size, in the launch configuration bench.py times:
m = n = 4e6, omega = 16 per row (nnz = 6.4e7), tau = 65536, the iteration kernel
and tuning pcdm_autotune picks (the persisting-L2 window in FP64, as the bench).

- The first iterations: the oracle runs them too (tau columns per iteration is
  cheap), so x and g are compared in full: FP64 to 1e-10 after 1 and 3
  iterations; FP32 and BF16 values (FP32 residual, FP64 refresh every 64) to
  1e-5 after 1, 3 and 64 iterations.
- The zero decisions of the soft threshold, coordinate by coordinate: from one
  common state (x and g of the GPU), one iteration on both sides; wherever
  exactly one of the two new x_i is 0, the oracle's u_i = beta L_i x_i - grad_i
  must lie within the GPU's summation error of the threshold, | |u_i| - lambda |
  <= 2 (c_i + 2) eps sum_r |a_ri g_r| + 8 eps (|beta L_i x_i| + |grad_i| + lambda)
  (eps = 2^-24 in the FP32 forms, 2^-53 in FP64): the two sums' error bounds
  and the step's own roundings, so a decision may differ only where rounding
  can flip it.  The max-norm
  tolerance alone would hide a wrong zero (it moves x_i by about
  (|grad_i| - lambda) / (beta L_i)).
- A complete solve to relative gap 1e-6: the oracle recomputes the residual and
  the duality gap of the GPU's final x from scratch and checks the KKT
  conditions of LASSO on sampled coordinates.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, instances

pytestmark = pytest.mark.gpu

N, OMEGA, TAU = 4_000_000, 16, 65536


@pytest.fixture(scope="module")
def inst():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return instances.row_omega_instance(N, N, OMEGA, density=0.01, noise=0.01, lam_frac=0.05, seed=1002)


@pytest.fixture(scope="module")
def ref_state(inst):
    return oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def test_first_iterations_match_in_full(inst, ref_state):
    with Lasso.from_instance(inst) as s:
        assert s.omega == ref_state.omega == OMEGA
        assert np.array_equal(s.L(), ref_state.L)
        for upto in (1, 3):
            s.step(TAU, upto - s.iteration, 0)
            ref_state.run(TAU, upto - ref_state.k, 0)
            assert _rel(s.x(), ref_state.x) <= 1e-10
            assert _rel(s.residual(), ref_state.g) <= 1e-10
        got, want = s.gap(), ref_state.gap()
        assert abs(got["gap"] - want["gap"]) <= 1e-10 * want["primal"]
        assert abs(got["primal"] - want["primal"]) <= 1e-10 * want["primal"]


def test_solve_certified_by_the_oracle(inst):
    tol = 1e-6
    with Lasso.from_instance(inst) as s:
        ok, it, rel = s.solve(TAU, 0, tol, 200_000)
        assert ok and rel <= tol
        x = s.x()
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    r = oracle.residual(A, inst.b, x)
    rec = oracle.gap(A, inst.b, x, r, inst.lam)
    assert rec["gap"] <= tol * rec["primal"] * (1 + 1e-6)
    # KKT on sampled coordinates, c_i = a_i^T (A x - b) computed by the oracle's residual
    rng = np.random.default_rng(0)
    support = np.nonzero(x)[0]
    picks = np.concatenate([rng.choice(inst.n, 2000, replace=False), rng.choice(support, min(2000, support.size),
                                                                               replace=False)])
    for i in picks:
        s_, e_ = inst.col_ptr[i], inst.col_ptr[i + 1]
        c = float(np.dot(inst.val64[s_:e_], r[inst.row_idx[s_:e_]]))
        if x[i] == 0:
            assert abs(c) <= inst.lam * (1 + 1e-2)
        else:
            assert abs(c + inst.lam * np.sign(x[i])) <= 1e-2 * inst.lam


REFRESH = 64
TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-5}
EPS = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}


def _bench_handle(inst, dtype):
    """The handle the bench times: FP32 residual with an FP64 refresh every 64
    iterations in the FP32/BF16 forms, the persisting-L2 window in FP64, and the
    autotuner's kernel choice."""
    s = Lasso.from_instance(inst, refresh_every=0 if dtype == "f64" else REFRESH, l2_persist=(dtype == "f64"))
    s.autotune(TAU, 20)
    s.reset()
    return s


def _zero_decisions_agree(inst, ref, s, dtype, seed):
    """One iteration from the GPU's current state on both sides; the mismatched
    zero decisions must sit within the rounding bound of the threshold."""
    k = s.iteration
    ref.x[:] = s.x()
    ref.g[:] = s.residual().astype(np.float64)
    ref.k = k
    x0, g0 = ref.x.copy(), ref.g.copy()
    S = oracle.sample(seed, k, inst.n, TAU)
    s.step(TAU, 1, seed)
    ref.run(TAU, 1, seed, refresh_every=0 if dtype == "f64" else REFRESH)
    xg, xr = s.x()[S], ref.x[S]
    cp, ri, v = inst.col_ptr, inst.row_idx, inst.val64
    lens = cp[S + 1] - cp[S]
    pos = np.repeat(cp[S] - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())
    owner = np.repeat(np.arange(S.size), lens)
    prod = v[pos] * g0[ri[pos]]
    grad = np.bincount(owner, weights=prod, minlength=S.size)
    sabs = np.bincount(owner, weights=np.abs(prod), minlength=S.size)
    beta = ref.beta(TAU)
    u = beta * ref.L[S] * x0[S] - grad
    # the two sums, then the step's own roundings (1/L and 1/beta stored rounded, the products)
    bound = (2.0 * (lens + 2) * EPS[dtype] * sabs
             + 8.0 * EPS[dtype] * (np.abs(beta * ref.L[S] * x0[S]) + np.abs(grad) + inst.lam))
    mism = (xg == 0) != (xr == 0)
    slack = np.abs(np.abs(u) - inst.lam)
    assert np.all(slack[mism] <= bound[mism]), (dtype, int(mism.sum()), float((slack[mism] / inst.lam).max()))
    return int(mism.sum()), float((slack[mism] / inst.lam).max()) if mism.any() else 0.0


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_bench_configuration_follows_the_oracle(dtype):
    inst = instances.row_omega_instance(N, N, OMEGA, density=0.01, noise=0.01, lam_frac=0.05, val_dtype=dtype,
                                        seed=1002)
    ref = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)
    refresh = 0 if dtype == "f64" else REFRESH
    s = _bench_handle(inst, dtype)
    try:
        for upto in ((1, 3) if dtype == "f64" else (1, 3, 64)):
            s.step(TAU, upto - s.iteration, 0)
            ref.run(TAU, upto - ref.k, 0, refresh_every=refresh)
            assert _rel(s.x(), ref.x) <= TOL[dtype], (dtype, upto)
            assert _rel(s.residual().astype(np.float64), ref.g) <= TOL[dtype], (dtype, upto)
        # zero decisions from a common state, early (many crossings) and after a few epochs
        _zero_decisions_agree(inst, ref, s, dtype, 0)
        s.step(TAU, 300, 0)
        _zero_decisions_agree(inst, ref, s, dtype, 0)
    finally:
        s.close()

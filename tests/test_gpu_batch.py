"""The batched solver (pcdm_batch_*): every right-hand side must follow the
oracle's single-problem PCDM1 run with the same seed (the batch only shares the
reads of A), the solve must certify every problem by the oracle's duality gap,
and a regularisation path with warm starts must too."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import BatchLasso, Lasso, PcdmError, PCDM_EINVAL, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _rhs(inst, nrhs, seed, lam_fracs=None):
    """nrhs right-hand sides b_l = A x*_l + noise on the stored (promoted) values."""
    rng = np.random.default_rng(seed)
    cols = np.repeat(np.arange(inst.n), np.diff(inst.col_ptr))
    Bm = np.empty((nrhs, inst.m))
    lams = []
    for l in range(nrhs):
        xs = np.zeros(inst.n)
        sup = rng.choice(inst.n, max(1, inst.n // 20), replace=False)
        xs[sup] = rng.choice([-1.0, 1.0], sup.size) * rng.uniform(1, 2, sup.size)
        Bm[l] = np.bincount(inst.row_idx, weights=inst.val64 * xs[cols], minlength=inst.m) \
            + 0.01 * rng.standard_normal(inst.m)
        atb = np.bincount(cols, weights=inst.val64 * Bm[l][inst.row_idx], minlength=inst.n)
        frac = 0.1 if lam_fracs is None else lam_fracs[l]
        lams.append(frac * float(np.max(np.abs(atb))))
    return Bm, lams


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _inst(val_dtype):
    return instances.per_col_instance(2000, 1000, 10, nnz_star=50, val_dtype=val_dtype, seed=1001) \
        if val_dtype != "f64" else instances.tiny_instance()


TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-5}


@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 5, 16, 32])
def test_each_problem_follows_the_oracle(val_dtype, nrhs):
    inst = _inst(val_dtype)
    Bm, lams = _rhs(inst, nrhs, 7, lam_fracs=np.linspace(0.05, 0.5, nrhs))
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    iters, tau, seed = 60, 32, 3
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, lams) as bt:
        bt.step(tau, iters, seed)
        X = bt.x()
        st = bt.stats()
    assert st["iterations"] == iters and st["updates"] == iters * tau * nrhs
    for l in range(nrhs):
        ref = oracle.State(A, Bm[l], lams[l])
        ref.run(tau, iters, seed)
        assert _rel(X[l], ref.x) <= TOL[val_dtype], l


def test_batch_equals_single_problem_handles():
    inst = instances.tiny_instance()
    Bm, lams = _rhs(inst, 4, 11)
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, lams) as bt:
        bt.step(48, 80, 5)
        X = bt.x()
        gp = bt.gap()
    for l in range(4):
        with Lasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm[l].copy(), lams[l]) as s:
            s.step(48, 80, 5)
            assert _rel(X[l], s.x()) <= 1e-12
            g = s.gap()
            assert abs(g["gap"] - gp["gap"][l]) <= 1e-10 * g["primal"]
            assert abs(g["primal"] - gp["primal"][l]) <= 1e-12 * g["primal"]


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-8), ("f32", 1e-6), ("bf16", 1e-6)])
def test_solve_is_certified_by_the_oracle(val_dtype, tol):
    inst = _inst(val_dtype)
    Bm, lams = _rhs(inst, 8, 13, lam_fracs=np.geomspace(0.5, 0.02, 8))
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, lams,
                    refresh_every=0 if val_dtype == "f64" else 64) as bt:
        ok, it, rel = bt.solve(32, 0, tol, 200_000)
        X = bt.x()
    assert ok and np.all(rel <= tol)
    for l in range(8):
        r = oracle.residual(A, Bm[l], X[l])
        rec = oracle.gap(A, Bm[l], X[l], r, lams[l])
        assert rec["gap"] <= tol * rec["primal"] * (1 + 1e-6), l


def test_regularisation_path_with_warm_starts():
    inst = _inst("bf16")
    Bm, lmax = _rhs(inst, 16, 17, lam_fracs=np.ones(16))
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    path = np.geomspace(1.0, 1e-2, 6)
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, [lmax[l] * path[0] for l in range(16)],
                    refresh_every=64) as bt:
        for f in path:
            lams = [lmax[l] * f for l in range(16)]
            bt.set_lambda(lams)
            ok, it, rel = bt.solve(64, 1, 1e-6, 200_000)
            assert ok
            X = bt.x()
            for l in (0, 7, 15):
                r = oracle.residual(A, Bm[l], X[l])
                rec = oracle.gap(A, Bm[l], X[l], r, lams[l])
                assert rec["gap"] <= 1e-6 * rec["primal"] * (1 + 1e-6)
        # at lambda >= lambda_max the solution is 0; at the end of the path it is not
        assert np.count_nonzero(X) > 0


def test_warm_start_and_reset():
    inst = instances.tiny_instance()
    Bm, lams = _rhs(inst, 3, 19)
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, lams) as bt:
        bt.step(32, 40, 2)
        X = bt.x()
        bt.reset()
        assert np.count_nonzero(bt.x()) == 0
        bt.set_x(X)
        g1 = bt.gap()
        for l in range(3):
            A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
            rec = oracle.gap(A, Bm[l], X[l], oracle.residual(A, Bm[l], X[l]), lams[l])
            assert abs(g1["gap"][l] - rec["gap"]) <= 1e-10 * rec["primal"]


@pytest.mark.parametrize("case", ["nrhs0", "nrhs33", "neg_lambda", "nan_b", "shape"])
def test_invalid_batches_are_rejected(case):
    inst = instances.tiny_instance()
    Bm, lams = _rhs(inst, 2, 23)
    if case == "nrhs0":
        Bm, lams = Bm[:0], []
    elif case == "nrhs33":
        Bm = np.tile(Bm[:1], (33, 1))
        lams = lams[:1] * 33
    elif case == "neg_lambda":
        lams = [lams[0], -1.0]
    elif case == "nan_b":
        Bm = Bm.copy()
        Bm[1, 5] = np.nan
    elif case == "shape":
        with pytest.raises(ValueError):
            BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm[:, :-1].copy(), lams)
        return
    with pytest.raises(PcdmError) as e:
        BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, np.ascontiguousarray(Bm), lams)
    assert e.value.status == PCDM_EINVAL


@pytest.mark.parametrize("val_dtype", ["f64", "bf16"])
def test_batch_autotune_restores_the_state_and_keeps_parity(val_dtype):
    # a larger instance, so that several grids are tried; the FP32 residuals use the
    # four-problem vector reductions of the scatter (16 right-hand sides)
    inst = instances.per_col_instance(400_000, 200_000, 15, nnz_star=1000, val_dtype=val_dtype, seed=1013)
    Bm, lams = _rhs(inst, 16, 17, lam_fracs=np.geomspace(0.5, 0.05, 16))
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    tau, seed = 8192, 9
    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, Bm, lams) as bt:
        bt.step(tau, 3, seed)
        X3 = bt.x().copy()
        st3 = bt.stats()
        choice = bt.autotune(tau, 5)
        assert choice["blocks_per_sm"] >= 1 and choice["us_per_iteration"] > 0
        assert np.array_equal(bt.x(), X3)
        st = bt.stats()
        assert st["iterations"] == st3["iterations"] and st["gathered_nnz"] == st3["gathered_nnz"]
        bt.step(tau, 9, seed)
        X = bt.x()
    for l in (0, 7, 15):
        ref = oracle.State(A, Bm[l], lams[l])
        ref.run(tau, 12, seed)
        assert _rel(X[l], ref.x) <= TOL[val_dtype], l

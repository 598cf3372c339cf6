"""Derivatives of the LASSO solution on the GPU (pcdm_polish, pcdm_backward and
the torch.autograd layer) against the oracle's dense implicit-function
definitions and against FP64 central finite differences."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    t.cuda.set_device(0)
    return t


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _solved(inst, tol):
    s = Lasso.from_instance(inst, refresh_every=0 if inst.val_dtype == "f64" else 64)
    ok, it, rel = s.solve(64, 0, tol, 200_000)
    assert ok
    return s


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-7), ("bf16", 1e-7)])
def test_polish_reaches_the_active_set_solution(torch, val_dtype, tol):
    inst = instances.per_col_instance(2000, 1000, 10, nnz_star=50, val_dtype=val_dtype, seed=1001)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    with _solved(inst, tol) as s:
        ok, it, res = s.polish(1e-14)
        assert ok and res <= 1e-14
        x = s.x()
        S = np.nonzero(x)[0]
        want = oracle.active_set_solution(A, inst.b, inst.lam, S, np.sign(x[S]))
        assert _rel(x, want) <= 1e-12
        g = s.gap()
        assert g["rel_gap"] <= 1e-12
        assert s.support_size() == S.size


@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
def test_backward_matches_the_dense_implicit_gradient(torch, val_dtype):
    inst = instances.per_col_instance(2000, 1000, 10, nnz_star=50, val_dtype=val_dtype, seed=1001)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    rng = np.random.default_rng(5)
    with _solved(inst, 1e-10 if val_dtype == "f64" else 1e-7) as s:
        s.polish(1e-14)
        x = s.x()
        dx = rng.standard_normal(inst.n)
        db, dlam, ok, it, res = s.backward(dx, tol=1e-13)
        assert ok
        want_db, want_dlam = oracle.implicit_grad(A, x, inst.lam, dx)
        assert _rel(db, want_db) <= 1e-10
        assert abs(dlam - want_dlam) <= 1e-10 * max(1.0, abs(want_dlam))
        # device in, device out
        t_dx = torch.from_numpy(dx).cuda()
        t_db = torch.empty(inst.m, dtype=torch.float64, device="cuda")
        s.backward(t_dx, tol=1e-13, db_out=t_db)
        assert _rel(t_db.cpu().numpy(), want_db) <= 1e-10


def test_backward_at_zero_solution_is_zero(torch):
    inst = instances.tiny_instance()
    with Lasso.from_instance(inst) as s:
        s.set_lambda(2.0 * inst.lam / 0.1)            # above lambda_max
        ok, it, rel = s.solve(32, 0, 1e-10, 10_000)
        assert ok and s.support_size() == 0
        db, dlam, ok, it, res = s.backward(np.ones(inst.n))
        assert ok and not np.any(db) and dlam == 0.0


def test_set_b_recomputes_the_residual(torch):
    inst = instances.tiny_instance()
    rng = np.random.default_rng(3)
    with Lasso.from_instance(inst) as s:
        s.step(32, 50, 1)
        x = s.x()
        b2 = inst.b + 0.1 * rng.standard_normal(inst.m)
        s.set_b(b2)
        A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
        assert _rel(s.residual(), oracle.residual(A, b2, x)) <= 1e-13
        assert np.array_equal(s.x(), x)
        bad = b2.copy()
        bad[3] = np.inf
        with pytest.raises(Exception):
            s.set_b(bad)


def _fd_check(torch, inst, x_target, directions, eps=1e-6, tol_rel=1e-6, seed=0):
    from paper_1212_0873_gb300.autograd import LassoLayer
    layer = LassoLayer(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val,
                       refresh_every=0 if inst.val_dtype == "f64" else 64,
                       tol=1e-9 if inst.val_dtype == "f64" else 1e-6)
    try:
        b = torch.from_numpy(inst.b).cuda().requires_grad_(True)
        lam = torch.tensor(inst.lam, dtype=torch.float64, device="cuda", requires_grad=True)
        t = torch.from_numpy(x_target).cuda()
        x = layer(b, lam)
        L = 0.5 * torch.sum((x - t) ** 2)
        L.backward()
        gb, gl = b.grad.detach().cpu().numpy(), float(lam.grad)

        def Lval(bv, lv):
            with torch.no_grad():
                xv = layer.solve(torch.from_numpy(bv).cuda(), lv)
                return 0.5 * float(torch.sum((xv - t) ** 2))

        rng = np.random.default_rng(seed)
        worst = 0.0
        for _ in range(directions):
            d = rng.standard_normal(inst.m)
            fd = (Lval(inst.b + eps * d, inst.lam) - Lval(inst.b - eps * d, inst.lam)) / (2 * eps)
            an = float(gb @ d)
            worst = max(worst, abs(fd - an) / max(abs(fd), 1e-12))
        fd = (Lval(inst.b, inst.lam + eps) - Lval(inst.b, inst.lam - eps)) / (2 * eps)
        worst_l = abs(fd - gl) / max(abs(fd), 1e-12)
        assert worst <= tol_rel, worst
        assert worst_l <= tol_rel, worst_l
    finally:
        layer.close()


def test_autograd_matches_finite_differences_small(torch):
    inst = instances.per_col_instance(600, 300, 8, nnz_star=30, seed=77)
    _fd_check(torch, inst, inst.x_star, directions=8)


def test_autograd_matches_finite_differences_at_scale(torch):
    """m = 1e6, n = 5e5, 12 FP32 nonzeros per column, x* 1% dense, noise variance
    1e-4, lambda = 0.1 ||A^T b||_inf, L = 1/2 ||x(b, lambda) - x*||^2, 32 random
    directions in b and one in lambda, central differences with step 1e-6."""
    inst = instances.per_col_instance(1_000_000, 500_000, 12, density=0.01, noise=0.01, lam_frac=0.1,
                                      val_dtype="f32", seed=1005)
    _fd_check(torch, inst, inst.x_star, directions=32)

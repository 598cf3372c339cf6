"""Many independent problems, one thread block each (pcdm_multi_*): every
problem's trajectory against the oracle's single-problem run (same seed, its
tau_p = min(tau, n_p), FP64 refresh at each check), and every solve certified
by the oracle's duality gap."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import MultiLasso, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _problems(val_dtype, sizes, seed=40):
    out = []
    for q, n in enumerate(sizes):
        inst = instances.per_col_instance(2 * n, n, 8, density=0.01, lam_frac=0.1, val_dtype=val_dtype,
                                          seed=seed + q)
        out.append(inst)
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
def test_each_problem_follows_the_oracle(val_dtype, tol):
    insts = _problems(val_dtype, [100, 700, 1500, 4000])
    K, tau, seed = 16, 256, 5
    with MultiLasso([(i.m, i.n, i.col_ptr, i.row_idx, i.val, i.b, i.lam) for i in insts]) as ml:
        ok, iters, rel = ml.solve(tau=tau, seed=seed, tol=1e-300, max_iters=3 * K, iters_per_check=K)
        assert not ok and np.all(iters == 3 * K)
        for p, inst in enumerate(insts):
            A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
            ref = oracle.State(A, inst.b, inst.lam)
            ref.run(min(tau, inst.n), int(iters[p]), seed, refresh_every=K)
            assert _rel(ml.x(p), ref.x) <= tol, p


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-8), ("bf16", 1e-6)])
def test_every_solve_is_certified(val_dtype, tol):
    insts = _problems(val_dtype, [64, 1000, 3000, 12000, 30000], seed=60)
    with MultiLasso([(i.m, i.n, i.col_ptr, i.row_idx, i.val, i.b, i.lam) for i in insts]) as ml:
        ok, iters, rel = ml.solve(tau=256, seed=1, tol=tol, max_iters=10**6, iters_per_check=64)
        assert ok and np.all(rel <= tol)
        st = ml.stats()
        assert st["updates"] == sum(int(it) * min(256, i.n) for it, i in zip(iters, insts))
        for p, inst in enumerate(insts):
            A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
            x = ml.x(p)
            rec = oracle.gap(A, inst.b, x, oracle.residual(A, inst.b, x), inst.lam)
            assert rec["gap"] <= tol * rec["primal"] * (1 + 1e-6), p
        # a second solve after reset follows the same path
        ml.reset()
        ok2, iters2, rel2 = ml.solve(tau=256, seed=1, tol=tol, max_iters=10**6, iters_per_check=64)
        assert ok2 and np.array_equal(iters2, iters)

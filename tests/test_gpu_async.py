"""Asynchronous mode (pcdm_step_async / pcdm_solve_async): one thread is the
serial method with iid blocks, which the oracle runs exactly; many threads
converge to a LASSO solution certified by the oracle's duality gap."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-12), ("f32", 1e-5), ("bf16", 1e-5)])
def test_one_thread_is_the_serial_iid_method(val_dtype, tol):
    inst = instances.per_col_instance(2000, 1000, 10, nnz_star=50, val_dtype=val_dtype, seed=1001)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    with Lasso.from_instance(inst) as s:
        for upto in (1, 50, 3000):
            s.step_async(upto - ref.k, seed=21, threads=1)
            ref.run_sampling("independent", 1, upto - ref.k, 21)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto


@pytest.mark.parametrize("val_dtype", ["f64", "bf16"])
def test_many_threads_converge(val_dtype):
    inst = instances.per_col_instance(20_000, 10_000, 10, nnz_star=200, val_dtype=val_dtype, seed=31)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    tol = 1e-8 if val_dtype == "f64" else 1e-6
    with Lasso.from_instance(inst) as s:
        ok, updates, rel = s.solve_async(seed=3, tol=tol, max_updates=10**9)
        assert ok and rel <= tol
        x = s.x()
    rec = oracle.gap(A, inst.b, x, oracle.residual(A, inst.b, x), inst.lam)
    assert rec["gap"] <= tol * rec["primal"] * (1 + 1e-6)

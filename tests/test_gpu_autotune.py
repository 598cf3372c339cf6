"""pcdm_autotune: it returns one of its candidates with a measured time, leaves
x, g, the iteration counter and the counters as they were, and the solver
keeps matching the oracle with the kernel it picked."""
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


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("bf16", 1e-5)])
def test_autotune_keeps_state_and_parity(val_dtype, tol):
    inst = instances.per_col_instance(20_000, 10_000, 12, nnz_star=100, val_dtype=val_dtype, seed=77)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    with Lasso.from_instance(inst) as s:
        s.step(512, 7, 3)
        ref.run(512, 7, 3)
        x_before, g_before, st_before = s.x(), s.residual(), s.stats()
        best = s.autotune(512, trial_iters=10)
        assert best["kernel"] in (0, 1, 2, 3, 4, 5) and best["us_per_iteration"] > 0
        assert best["heads"] in (0, 1)
        # kernel 5 reports -1: its certificate follows the share of moving coordinates
        assert best["zero_cert"] in ((-1,) if best["kernel"] == 5 and val_dtype == "f64" else (0, 1))
        assert val_dtype == "f64" or best["zero_cert"] == 0
        assert best["lanes_per_col"] in (1, 2, 4, 8, 16, 32)
        assert np.array_equal(s.x(), x_before) and np.array_equal(s.residual(), g_before)
        assert s.iteration == 7
        st_after = s.stats()
        for key in ("iterations", "updates", "iter_launches"):
            assert st_after[key] == st_before[key]
        s.step(512, 30, 3)
        ref.run(512, 30, 3)
        assert _rel(s.x(), ref.x) <= tol
        assert _rel(s.residual(), ref.g) <= tol

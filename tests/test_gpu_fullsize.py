"""Parity at the benchmark's full size, in the launch configuration bench.py times:
m = n = 4e6, omega = 16 per row (nnz = 6.4e7), tau = 65536, fused persistent kernel.

- The first iterations: the oracle runs them too (tau columns per iteration is
  cheap), so x and g are compared in full, FP64 to 1e-10.
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

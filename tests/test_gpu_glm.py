"""PCDM1 on the SVM dual (Sec. 8.3) and on L2-regularised logistic regression
(Sec. 8.4) on the GPU against the oracle: the same tau-nice samples, iterate by
iterate, in every kernel that runs these problems (pipelined, fused with 1, 8
and 32 lanes per column, two-kernel form with 1 and 4) and every precision pair; the duality-gap record;
solves to a tight gap; edge cases (an all-zero example, columns longer than one
chunk, ragged tau, bad labels)."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import LabeledProblem, PcdmError, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


PROBLEMS = {"svm_dual": oracle.SVM_DUAL, "logistic": oracle.LOGISTIC}


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _instance(problem, val_dtype, seed, big=False):
    if problem == "svm_dual":
        # about 20 features per example (so columns pass one 16-entry chunk), popular features
        if big:   # uniform feature popularity: omega near 100, so tau = 1024 gives beta near 20;
            # lambda n = 0.5 leaves about a third of the x_i at each bound and a third inside
            return instances.svm_instance(3000, 5000, 40, lam=1e-4, zipf=0.0, val_dtype=val_dtype, seed=seed)
        return instances.svm_instance(400, 900, 24, lam=1e-3, zipf=0.6, val_dtype=val_dtype, seed=seed)
    return instances.logistic_instance(6000 if big else 1200, 2500 if big else 300, 12, lam=0.01 if big else 0.5,
                                       val_dtype=val_dtype, seed=seed)


def _oracle_state(inst):
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    return oracle.GlmState(PROBLEMS[inst.problem], A, inst.y, inst.lam)


def _gpu_residual_as_oracle(inst, g):
    # the library keeps y_j A_j^T x for logistic regression (labels folded into the rows)
    return g * inst.y if inst.problem == "logistic" else g


# (kernel, lanes per column, threads per block, heads)
CHOICES = [(0, 1, 64, 1), (0, 1, 160, 0), (1, 1, 0, 1), (1, 8, 0, 1), (1, 32, 0, 1), (2, 1, 0, 1), (2, 4, 0, 1), (4, 1, 64, 1), (5, 1, 64, 1)]


@pytest.mark.parametrize("problem", sorted(PROBLEMS))
@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
@pytest.mark.parametrize("choice", CHOICES)
def test_iterates_follow_the_oracle(problem, val_dtype, tol, choice):
    inst = _instance(problem, val_dtype, seed=2001)
    ref = _oracle_state(inst)
    tau = 203                                           # ragged: not a multiple of any block size
    with LabeledProblem.from_instance(inst) as s:
        s.set_tuning(*choice)
        for upto in (1, 7, 30):
            s.step(tau, upto - s.iteration, 5)
            ref.run(tau, upto - ref.k, 5)
            assert _rel(s.x(), ref.x) <= tol, (choice, upto)
            assert _rel(_gpu_residual_as_oracle(inst, s.residual()), ref.v) <= tol, (choice, upto)


@pytest.mark.parametrize("problem", sorted(PROBLEMS))
def test_gap_record_matches_the_oracle(problem):
    inst = _instance(problem, "f64", seed=2002)
    ref = _oracle_state(inst)
    with LabeledProblem.from_instance(inst) as s:
        for upto in (0, 5, 40):
            if upto:
                s.step(128, upto - s.iteration, 1)
                ref.run(128, upto - ref.k, 1)
            rec = s.gap()
            P, D, gap = rec["primal"], rec["dual"], rec["gap"]
            r = ref.gap()
            assert P == pytest.approx(r["primal"], rel=1e-10)
            assert D == pytest.approx(r["dual"], rel=1e-10, abs=1e-12 * abs(r["primal"]))
            assert gap == pytest.approx(r["gap"], rel=1e-8, abs=1e-11 * abs(r["primal"]))
            assert gap >= 0.0


@pytest.mark.parametrize("problem", sorted(PROBLEMS))
@pytest.mark.parametrize("val_dtype", ["f64", "bf16"])
def test_solve_reaches_the_gap_the_oracle_certifies(problem, val_dtype):
    inst = _instance(problem, val_dtype, seed=2003, big=True)
    tol = 1e-7 if val_dtype == "f64" else 1e-6
    with LabeledProblem.from_instance(inst, refresh_every=0 if val_dtype == "f64" else 32) as s:
        ok, it, rel = s.solve(1024, 3, tol, 200_000)
        assert ok and rel <= tol
        x = s.x()
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    r = oracle.glm_gap(PROBLEMS[problem], A, inst.y, x, inst.lam)
    assert r["gap"] <= 1.01 * tol * r["primal"] + 1e-12
    if problem == "svm_dual":
        assert np.all((x >= 0.0) & (x <= 1.0))


def test_svm_all_zero_example_goes_to_one_and_full_tau():
    Ad = np.zeros((6, 5))
    Ad[:2, 0] = [1.0, 0.5]
    Ad[2:4, 2] = [0.3, -1.0]
    Ad[4:, 3] = [2.0, 1.0]
    Ad[0, 4] = 0.7
    y = np.array([1.0, -1.0, 1.0, -1.0, 1.0])
    inst = instances.labeled_from_dense(Ad, y, 0.05, "svm_dual")
    ref = _oracle_state(inst)
    with LabeledProblem.from_instance(inst) as s:
        s.step(5, 3, 0)
        ref.run(5, 3, 0)
        x = s.x()
    assert x[1] == 1.0
    assert _rel(x, ref.x) <= 1e-12


def test_bad_labels_and_lasso_only_calls_are_rejected():
    inst = _instance("logistic", "f64", seed=2004)
    y = inst.y.copy()
    y[3] = 0.5
    with pytest.raises(PcdmError):
        LabeledProblem(inst.problem, inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, y, inst.lam)
    with LabeledProblem.from_instance(inst) as s:
        with pytest.raises(PcdmError):
            s.polish()
        with pytest.raises(PcdmError):
            s.step_async(100)
        with pytest.raises(PcdmError):
            s.set_tuning(3, 1, 128)
        s.step(64, 2, 0)                                # the handle stays usable

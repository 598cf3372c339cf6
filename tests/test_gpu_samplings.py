"""The tau-independent and (tau, p_b)-binomial samplings (Sec. 4.1 items 4, 5)
on the GPU: the drawn lists bit-exact against the oracle, iterates against the
oracle's runs with the same sampling, beta of Theorem ESO-DU, and solves."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, PcdmError, PCDM_EINVAL, instances
from paper_1212_0873_gb300 import _binding as B

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


@pytest.mark.parametrize("n,tau", [(1, 1), (10, 8), (1000, 32), (4097, 4097), (1_000_003, 65536)])
def test_sampled_lists_are_bit_exact(torch, n, tau):
    S = torch.empty(tau, dtype=torch.int32, device="cuda")
    keep = torch.empty(tau, dtype=torch.uint8, device="cuda")
    for seed, k in [(0, 0), (7, 3), (2**63 + 5, 12345)]:
        B.pcdm_sample_kind(B.PCDM_SAMPLING_INDEPENDENT, seed, k, n, tau, 1.0, S.data_ptr())
        want, _ = oracle.sample_independent(seed, k, n, tau)
        assert np.array_equal(S.cpu().numpy(), want)
        B.pcdm_sample_kind(B.PCDM_SAMPLING_BINOMIAL, seed, k, n, tau, 0.37, S.data_ptr(), keep.data_ptr())
        assert np.array_equal(S.cpu().numpy(), oracle.sample(seed, k, n, tau))
        assert np.array_equal(keep.cpu().numpy().astype(bool), oracle.binomial_keep(seed, k, tau, 0.37))


@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("kind,p_b", [("independent", 1.0), ("binomial", 0.6)])
def test_iterates_match_the_oracle(torch, val_dtype, kind, p_b):
    inst = instances.per_col_instance(2000, 1000, 10, nnz_star=50, val_dtype=val_dtype, seed=1001)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    tol = 1e-10 if val_dtype == "f64" else 1e-5
    ref = oracle.State(A, inst.b, inst.lam)
    with Lasso.from_instance(inst, sampling=kind, p_b=p_b) as s:
        assert s.beta(64) == pytest.approx(oracle.beta_sampling(ref.omega, kind, 64, inst.n, p_b), rel=1e-14)
        for upto in (1, 10, 60):
            s.step(64, upto - s.iteration, 9)
            ref.run_sampling(kind, 64, upto - ref.k, 9, p_b=p_b)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto


@pytest.mark.parametrize("kind,p_b", [("independent", 1.0), ("binomial", 0.5)])
def test_solve_is_certified(torch, kind, p_b):
    inst = instances.tiny_instance()
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    with Lasso.from_instance(inst, sampling=kind, p_b=p_b) as s:
        ok, it, rel = s.solve(32, 0, 1e-8, 200_000)
        assert ok and rel <= 1e-8
        x = s.x()
    rec = oracle.gap(A, inst.b, x, oracle.residual(A, inst.b, x), inst.lam)
    assert rec["gap"] <= 1e-8 * rec["primal"] * (1 + 1e-6)


def test_binomial_with_p_one_is_the_nice_sampling(torch):
    inst = instances.tiny_instance()
    with Lasso.from_instance(inst, sampling="binomial", p_b=1.0) as a, \
            Lasso.from_instance(inst, fused=False) as b:
        a.step(48, 30, 4)
        b.step(48, 30, 4)
        assert np.array_equal(a.x(), b.x())


@pytest.mark.parametrize("kw", [dict(sampling="binomial", p_b=0.0), dict(sampling="binomial", p_b=1.5)])
def test_bad_sampling_options(torch, kw):
    inst = instances.tiny_instance()
    with pytest.raises(PcdmError) as e:
        Lasso.from_instance(inst, **kw)
    assert e.value.status == PCDM_EINVAL

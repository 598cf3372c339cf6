"""The theory-versus-reality experiment (Sec. 8.2): the iteration speedup of
PCDM1 with the tau-nice sampling on least squares with equal-valued rows of
omega nonzeros follows tau / beta (Theorem ESO-nice).  The paper gives the
comparison only as a figure, so this is a shape check: the empirical speedup
increases with tau and stays within 20% of the theoretical one."""
import pytest

pytestmark = pytest.mark.gpu


def test_speedup_follows_tau_over_beta():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build, experiments
    build.build()
    rows = experiments.theory_vs_reality(omegas=(5, 50), taus=(1, 8, 64, 1000))
    for omega in (5, 50):
        sel = [r for r in rows if r["omega"] == omega]
        emp = [r["empirical"] for r in sel]
        assert all(b > a for a, b in zip(emp, emp[1:])), sel
        for r in sel:
            assert 0.8 <= r["empirical"] / r["theory"] <= 1.2, r

"""The deterministic two-kernel form (pcdm_opts.deterministic_scatter).

Algorithm 1, step 4 (Jacobi), with every gradient summed in column order and
every residual entry updated in increasing sampled position, products and sums
rounded on their own.  In FP64 these are the operations of the oracle's
sequential run, so x and g must equal the oracle's BIT FOR BIT (compared as
64-bit patterns), through refreshes and gap evaluations.  FP32 and BF16 runs
must repeat bit for bit and stay within the usual 1e-5 of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, PcdmError, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ref(inst):
    return oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)


def _bits(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64)).view(np.uint64)


def _assert_bit_equal(s, ref, what):
    x, g = s.x(), s.residual()
    bx, bg = _bits(x) != _bits(ref.x), _bits(g) != _bits(ref.g)
    assert not bx.any(), (what, "x differs at", np.flatnonzero(bx)[:8], x[bx][:4], ref.x[bx][:4])
    assert not bg.any(), (what, "g differs at", np.flatnonzero(bg)[:8], g[bg][:4], ref.g[bg][:4])


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b))) / max(float(np.max(np.abs(b))), 1e-300)


def test_fp64_equals_the_oracle_bit_for_bit_on_the_tiny_config():
    # 2000 x 1000, 10 nonzeros per column, tau = 32: 400 iterations
    inst = instances.tiny_instance("f64")
    ref = _ref(inst)
    with Lasso.from_instance(inst, deterministic_scatter=True) as s:
        for upto in (1, 2, 10, 100, 400):
            s.step(32, upto - s.iteration, 0)
            ref.run(32, upto - ref.k, 0)
            _assert_bit_equal(s, ref, upto)
        assert np.count_nonzero(ref.x) > 0


@pytest.mark.parametrize("refresh_every", [1, 16])
def test_fp64_bit_for_bit_through_refreshes_and_gaps(refresh_every):
    inst = instances.tiny_instance("f64")
    ref = _ref(inst)
    with Lasso.from_instance(inst, deterministic_scatter=True, refresh_every=refresh_every) as s:
        s.step(32, 50, 3)
        ref.run(32, 50, 3, refresh_every=refresh_every)
        _assert_bit_equal(s, ref, "after 50")
        d = s.gap()                               # refreshes g first, as the oracle's gap does
        P, gap = d["primal"], d["gap"]
        ref.refresh()
        _assert_bit_equal(s, ref, "after the gap")
        rec = ref.gap()
        assert abs(P - rec["primal"]) <= 1e-12 * abs(rec["primal"])
        assert abs(gap - rec["gap"]) <= 1e-10 * abs(rec["primal"])
        s.step(32, 70, 3)
        ref.run(32, 70, 3, refresh_every=refresh_every)
        _assert_bit_equal(s, ref, "after 120")


@pytest.mark.parametrize("kind", ["per_col", "row_omega"])
def test_fp64_bit_for_bit_at_larger_sizes(kind):
    # several hundred blocks of positions, rows shared by many sampled columns
    if kind == "per_col":
        inst = instances.per_col_instance(400_000, 200_000, 10, nnz_star=2000, val_dtype="f64", seed=91)
    else:
        inst = instances.row_omega_instance(200_000, 200_000, 16, density=0.01, val_dtype="f64", seed=92)
    ref = _ref(inst)
    tau = 4096 + 37                                # ragged: not a multiple of the block
    with Lasso.from_instance(inst, deterministic_scatter=True, refresh_every=8) as s:
        for upto in (1, 9, 25):
            s.step(tau, upto - s.iteration, 5)
            ref.run(tau, upto - ref.k, 5, refresh_every=8)
            _assert_bit_equal(s, ref, (kind, upto))


def test_fp64_bit_for_bit_with_every_column_and_empty_columns():
    # tau = n (beta = omega, every column each iteration) and two empty columns (x_i stays 0)
    rng = np.random.default_rng(7)
    Ad = rng.standard_normal((60, 40)) * (rng.random((60, 40)) < 0.2)
    Ad[:, 5] = 0.0
    Ad[:, 31] = 0.0
    b = rng.standard_normal(60)
    inst = instances.from_dense(Ad, b, 0.1 * float(np.max(np.abs(Ad.T @ b))))
    ref = _ref(inst)
    with Lasso.from_instance(inst, deterministic_scatter=True) as s:
        for upto in (1, 30, 200):
            s.step(40, upto - s.iteration, 1)
            ref.run(40, upto - ref.k, 1)
            _assert_bit_equal(s, ref, upto)
        assert s.x()[5] == 0.0 and s.x()[31] == 0.0


@pytest.mark.parametrize("val_dtype", ["f32", "bf16"])
def test_fp32_forms_repeat_bit_for_bit_and_follow_the_oracle(val_dtype):
    inst = instances.per_col_instance(400_000, 200_000, 10, nnz_star=2000, val_dtype=val_dtype, seed=93)
    ref = _ref(inst)
    runs = []
    for _ in range(2):
        with Lasso.from_instance(inst, deterministic_scatter=True, refresh_every=8) as s:
            s.step(4096, 20, 11)
            runs.append((s.x().copy(), s.residual().copy()))
    ref.run(4096, 20, 11, refresh_every=8)
    assert np.array_equal(runs[0][0].view(np.uint64), runs[1][0].view(np.uint64))
    assert np.array_equal(np.ascontiguousarray(runs[0][1]).view(np.uint32), np.ascontiguousarray(runs[1][1]).view(np.uint32))
    assert _rel(runs[0][0], ref.x) <= 1e-5 and _rel(runs[0][1], ref.g) <= 1e-5


def test_deterministic_solve_is_certified_and_repeats():
    inst = instances.tiny_instance("f64")
    out = []
    for _ in range(2):
        with Lasso.from_instance(inst, deterministic_scatter=True) as s:
            ok, it, rel = s.solve(32, 0, 1e-8, 200_000)
            assert ok and rel <= 1e-8
            out.append((it, s.x()))
    assert out[0][0] == out[1][0] and np.array_equal(_bits(out[0][1]), _bits(out[1][1]))
    ref = _ref(inst)
    ref.x[:] = out[0][1]
    rec = ref.gap()
    assert rec["gap"] <= 1.01e-8 * rec["primal"]


def test_deterministic_handle_refuses_the_unordered_calls():
    inst = instances.tiny_instance("f64")
    with Lasso.from_instance(inst, deterministic_scatter=True) as s:
        with pytest.raises(PcdmError):
            s.autotune(32, 5)
        with pytest.raises(PcdmError):
            s.step_async(100)
        s.step(32, 3, 0)                           # still usable

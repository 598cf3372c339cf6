"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by element.

Tolerances (max-abs difference over max-abs of the oracle's vector):
  FP64 values, FP64 x/g ............ 1e-10 on x, g and F
  FP32 values or BF16 values, FP32 x/g .. 1e-5
The sampled coordinate sets and omega are integers: bit-exact.  L_i is summed in
the same order with no contraction on both sides: bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, PcdmError, instances
from paper_1212_0873_gb300 import _binding as B

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


def _torch():
    import torch
    return torch


def _ref(inst):
    return oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)


def _rel(a, b):
    scale = max(float(np.max(np.abs(b))) if b.size else 0.0, 1e-300)
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b))) / scale if b.size else 0.0


def _assert_close(solver, ref, tol, what=""):
    x = solver.x().astype(np.float64)
    g = solver.residual().astype(np.float64)
    ex, eg = _rel(x, ref.x), _rel(g, ref.g)
    F_gpu = oracle.objective(ref.A, ref.b, x, ref.lam)
    F_ref = ref.objective()
    eF = abs(F_gpu - F_ref) / max(abs(F_ref), 1e-300)
    assert ex <= tol and eg <= tol and eF <= tol, (what, ex, eg, eF)


# --------------------------------------------------------------------------- sampler
@pytest.mark.parametrize("n,tau", [(1, 1), (2, 2), (3, 1), (10, 10), (17, 5), (1000, 32), (4096, 4096),
                                   (4097, 1000), (65536, 65536), (4_000_000, 65536), (500_000_000, 4096),
                                   (2_147_483_647, 1000)])
def test_sampler_bit_exact(n, tau):
    torch = _torch()
    S = torch.empty(tau, dtype=torch.int32, device="cuda")
    for seed, k in [(0, 0), (0, 1), (12345, 77), (2**40 + 3, 2**33 + 5)]:
        B.pcdm_sample(seed, k, n, tau, S.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(S.cpu().numpy(), oracle.sample(seed, k, n, tau)), (n, tau, seed, k)


# --------------------------------------------------------------------------- set-up
@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
def test_setup_L_and_omega_exact(val_dtype):
    inst = instances.tiny_instance(val_dtype=val_dtype)
    ref = _ref(inst)
    with Lasso.from_instance(inst) as s:
        assert s.omega == ref.omega
        assert np.array_equal(s.L(), ref.L)
        for tau in (1, 32, 1000):
            assert s.beta(tau) == ref.beta(tau)
        assert np.array_equal(s.x(), np.zeros(inst.n))
        assert _rel(s.residual().astype(np.float64), -inst.b) <= (0 if val_dtype == "f64" else 1e-7)


# --------------------------------------------------------------------------- iterates
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
def test_iterates_match_oracle_tiny(val_dtype, fused):
    """The 2000 x 1000 parity workload, tau = 32, at several checkpoints."""
    inst = instances.tiny_instance(val_dtype=val_dtype)
    refresh = 0 if val_dtype == "f64" else 64
    ref = _ref(inst)
    tau, seed = 32, 0
    with Lasso.from_instance(inst, fused=fused, refresh_every=refresh) as s:
        done = 0
        for upto in (1, 10, 100, 400):
            s.step(tau, upto - done, seed)
            ref.run(tau, upto - done, seed, refresh_every=refresh)
            done = upto
            _assert_close(s, ref, TOL[val_dtype], "k=%d" % upto)
        assert s.iteration == 400


@pytest.mark.parametrize("W", [4, 8, 16, 32])
def test_lane_widths_agree(W):
    inst = instances.per_col_instance(700, 500, 37, nnz_star=20, seed=31)   # 37 > 32: several rounds per lane
    ref = _ref(inst)
    ref.run(64, 60, 3)
    for fused in (True, False):
        with Lasso.from_instance(inst, lanes_per_col=W, fused=fused) as s:
            s.step(64, 60, 3)
            _assert_close(s, ref, TOL["f64"], "W=%d fused=%s" % (W, fused))


def test_gap_matches_oracle():
    inst = instances.tiny_instance()
    ref = _ref(inst)
    with Lasso.from_instance(inst) as s:
        for k in (0, 50, 300):
            if k:
                s.step(32, k - s.iteration, 0)
                ref.run(32, k - ref.k, 0)
            got = s.gap()
            want = ref.gap()
            P = want["primal"]
            assert abs(got["primal"] - P) <= 1e-10 * P
            assert abs(got["dual"] - want["dual"]) <= 1e-10 * P
            assert abs(got["gap"] - want["gap"]) <= 1e-10 * P
            _assert_close(s, ref, TOL["f64"], "after gap at k=%d" % k)


@pytest.mark.parametrize("val_dtype", ["f64", "f32", "bf16"])
def test_solve_matches_oracle_and_kkt(val_dtype):
    inst = instances.tiny_instance(val_dtype=val_dtype)
    tol = 1e-8 if val_dtype == "f64" else 1e-6
    refresh = 0 if val_dtype == "f64" else 64
    ref = _ref(inst)
    with Lasso.from_instance(inst, refresh_every=refresh, check_every=32) as s:
        ok, it, rel = s.solve(32, 0, tol, 4000)
        assert ok and rel <= tol
        if val_dtype == "f64":
            it_ref, _ = ref.solve(32, 0, tol, 4000, check_every=32, refresh_every=refresh)
            assert it == it_ref
        else:
            # the same schedule (gap, hence a refresh, every 32 iterations) for exactly `it` iterations
            ref.solve(32, 0, 0.0, it, check_every=32, refresh_every=refresh)
        _assert_close(s, ref, TOL[val_dtype], "solved")
        A = instances.dense(inst)
        x = s.x().astype(np.float64)
        c = A.T @ (A @ x - inst.b)
        on = x != 0
        kkt = 1e-3 if val_dtype == "f64" else 3e-2
        assert np.max(np.abs(c[~on])) <= inst.lam * (1 + kkt)
        assert np.max(np.abs(c[on] + inst.lam * np.sign(x[on]))) <= kkt * inst.lam


def test_step_is_additive_and_resumable():
    inst = instances.tiny_instance()
    with Lasso.from_instance(inst) as a, Lasso.from_instance(inst) as b:
        a.step(32, 10, 5)
        a.step(32, 15, 5)
        b.step(32, 25, 5)
        assert _rel(a.x(), b.x()) <= 1e-12
        # checkpoint (x, k), restore into a fresh handle, continue
        x_ck, k_ck = a.x(), a.iteration
        a.step(32, 20, 5)
        with Lasso.from_instance(inst) as c:
            c.set_x(x_ck)
            c.iteration = k_ck
            c.step(32, 20, 5)
            assert _rel(c.x(), a.x()) <= 1e-10


def test_stats_count_the_work():
    inst = instances.tiny_instance()
    counts = np.diff(inst.col_ptr)
    with Lasso.from_instance(inst) as s:
        s.reset_stats()
        s.step(32, 30, 9)
        st = s.stats()
    want = sum(int(counts[oracle.sample(9, k, inst.n, 32)].sum()) for k in range(30))
    assert st["iterations"] == 30 and st["updates"] == 960
    assert st["gathered_nnz"] == want
    assert 0 < st["nonzero_updates"] <= 960
    assert st["scattered_nnz"] <= want


# --------------------------------------------------------------------------- edge cases
def _dense_instance(A, b, lam, val_dtype="f64"):
    return instances.from_dense(np.asarray(A, dtype=float), np.asarray(b, dtype=float), lam, val_dtype)


@pytest.mark.parametrize("case", ["n1", "m1", "tau_n", "tau_1", "empty_cols", "all_empty", "lam0", "lam_max",
                                  "long_col"])
def test_edge_cases(case):
    rng = np.random.default_rng(5)
    tau, iters = 3, 40
    if case == "n1":
        inst = _dense_instance(rng.standard_normal((5, 1)), rng.standard_normal(5), 0.1)
        tau = 1
    elif case == "m1":
        inst = _dense_instance(rng.standard_normal((1, 6)), [2.0], 0.05)
    elif case == "tau_n":
        inst = instances.per_col_instance(60, 40, 4, nnz_star=4, seed=1)
        tau = 40
    elif case == "tau_1":
        inst = instances.per_col_instance(60, 40, 4, nnz_star=4, seed=2)
        tau, iters = 1, 300
    elif case == "empty_cols":
        A = rng.standard_normal((30, 20)) * (rng.random((30, 20)) < 0.2)
        A[:, [0, 7, 19]] = 0.0
        inst = _dense_instance(A, rng.standard_normal(30), 0.1)
    elif case == "all_empty":
        inst = _dense_instance(np.zeros((4, 6)), rng.standard_normal(4), 0.1)
    elif case == "lam0":
        inst = instances.per_col_instance(60, 40, 4, nnz_star=4, lam_frac=0.0, seed=3)
    elif case == "lam_max":
        inst = instances.per_col_instance(60, 40, 4, nnz_star=4, lam_frac=1.0 + 1e-9, seed=4)
    else:   # a 1500-entry column among short ones
        A = rng.standard_normal((3000, 8)) * (rng.random((3000, 8)) < 0.01)
        A[:1500, 3] = rng.standard_normal(1500)
        inst = _dense_instance(A, rng.standard_normal(3000), 0.2)
    ref = _ref(inst)
    ref.run(tau, iters, 11)
    for fused in (True, False):
        with Lasso.from_instance(inst, fused=fused) as s:
            s.step(tau, iters, 11)
            _assert_close(s, ref, TOL["f64"], case)
            if case in ("all_empty", "lam_max"):
                assert np.all(s.x() == 0)
            g = s.gap()
            assert g["gap"] >= -1e-12 * g["primal"]


# --------------------------------------------------------------------------- invalid input
def _small_valid():
    A = np.array([[1.0, 0.0, 2.0], [0.0, 3.0, 0.0], [4.0, 0.0, 5.0]])
    inst = _dense_instance(A, [1.0, 2.0, 3.0], 0.1)
    return inst


@pytest.mark.parametrize("case", ["colptr_decreasing", "colptr_start", "row_out_of_range", "row_negative",
                                  "rows_unsorted", "rows_duplicate", "nan_value", "inf_b"])
def test_invalid_matrix_is_rejected(case):
    inst = _small_valid()
    col_ptr, row_idx, val, b = inst.col_ptr.copy(), inst.row_idx.copy(), inst.val.copy(), inst.b.copy()
    if case == "colptr_decreasing":
        col_ptr[1], col_ptr[2] = col_ptr[2], col_ptr[1]
    elif case == "colptr_start":
        col_ptr[0] = 1
    elif case == "row_out_of_range":
        row_idx[1] = 3
    elif case == "row_negative":
        row_idx[0] = -1
    elif case == "rows_unsorted":
        row_idx[0], row_idx[1] = row_idx[1], row_idx[0]
    elif case == "rows_duplicate":
        row_idx[1] = row_idx[0]
    elif case == "nan_value":
        val[2] = np.nan
    else:
        b[1] = np.inf
    with pytest.raises(PcdmError) as e:
        Lasso(inst.m, inst.n, col_ptr, row_idx, val, b, inst.lam)
    assert e.value.status == B.PCDM_EINVAL
    with Lasso.from_instance(inst) as s:       # the device is still fine
        s.step(2, 3, 0)


def test_step_rejects_bad_tau():
    inst = _small_valid()
    with Lasso.from_instance(inst) as s:
        for tau in (0, -1, 4):
            with pytest.raises(PcdmError) as e:
                s.step(tau, 1, 0)
            assert e.value.status == B.PCDM_EINVAL
        s.step(3, 1, 0)


# --------------------------------------------------------------------------- device inputs, bounded waits
def test_device_inputs_match_host_inputs():
    torch = _torch()
    inst = instances.tiny_instance()
    d = dict(col_ptr=torch.from_numpy(inst.col_ptr).cuda(), row_idx=torch.from_numpy(inst.row_idx).cuda(),
             val=torch.from_numpy(inst.val).cuda(), b=torch.from_numpy(inst.b).cuda())
    with Lasso(inst.m, inst.n, d["col_ptr"], d["row_idx"], d["val"], d["b"], inst.lam) as s1, \
            Lasso.from_instance(inst) as s2:
        s1.step(32, 50, 1)
        s2.step(32, 50, 1)
        assert _rel(s1.x(), s2.x()) <= 1e-12
        xt = torch.empty(inst.n, dtype=torch.float64, device="cuda")
        s1.x_into(xt)
        assert np.array_equal(xt.cpu().numpy(), s1.x())


def test_barrier_wait_is_bounded():
    """The fused kernel's grid-barrier waits give up after their time budget and
    report PCDM_ETIMEOUT; the device keeps working afterwards."""
    torch = _torch()
    st = B.pcdm_selftest_barrier_timeout(2_000_000, torch.cuda.current_stream().cuda_stream)
    assert st == B.PCDM_ETIMEOUT
    inst = instances.tiny_instance()
    with Lasso.from_instance(inst) as s:
        s.step(32, 5, 0)
        assert s.gap()["primal"] > 0

"""Every iteration kernel (pipelined, fused with several lane widths, two-kernel,
pipelined rounds, streaming, warp-cooperative; the pipelined ones with and without the
column heads, the pipelined one also with and without the FP32 certificate of zero
steps) selected by hand through pcdm_set_tuning follows the oracle; the pipelined kernel
also on columns shorter and longer than its shared-memory slot; the rounds kernel
also with several positions per thread (tau beyond the grid), the warp-cooperative one
also with many positions per warp, empty columns and columns of several items."""
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


# (kernel, lanes per column, threads per block, column heads[, zero-step certificate])
CHOICES = [(0, 1, 64, 1), (0, 1, 448, 1), (0, 1, 128, 0), (0, 1, 64, 1, 1), (0, 1, 128, 0, 1), (0, 1, 448, 1, 0),
           (1, 1, 0, 1), (1, 4, 0, 1), (1, 32, 0, 1), (2, 1, 0, 1), (2, 16, 0, 1), (3, 1, 128, 1), (3, 1, 256, 0),
           (4, 1, 64, 1), (4, 1, 448, 1), (5, 1, 32, 1), (5, 1, 512, 1, 1), (5, 1, 128, 1, 0)]


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
@pytest.mark.parametrize("choice", CHOICES)
def test_each_kernel_follows_the_oracle(val_dtype, tol, choice):
    inst = instances.per_col_instance(2000, 1000, 20, nnz_star=50, val_dtype=val_dtype, seed=1001)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    with Lasso.from_instance(inst) as s:
        s.set_tuning(*choice)
        for upto in (1, 9, 40):
            s.step(96, upto - s.iteration, 2)
            ref.run(96, upto - ref.k, 2)
            assert _rel(s.x(), ref.x) <= tol, (choice, upto)
            assert _rel(s.residual(), ref.g) <= tol, (choice, upto)


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("bf16", 1e-5)])
def test_rounds_kernel_with_several_positions_per_thread(val_dtype, tol):
    # tau = 2^17 is beyond one pass of the grid: two or more positions per thread
    inst = instances.per_col_instance(400_000, 200_000, 10, nnz_star=2000, val_dtype=val_dtype, seed=91)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    tau = 1 << 17
    with Lasso.from_instance(inst) as s:
        s.set_tuning(3, 1, 256)
        for upto in (1, 4, 12):
            s.step(tau, upto - s.iteration, 8)
            ref.run(tau, upto - ref.k, 8)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto
        s.set_tuning(3, 1, 128, 0)                    # more rounds per iteration, no heads
        s.step(tau, 5, 8)
        ref.run(tau, 5, 8)
        assert _rel(s.x(), ref.x) <= tol
        ok, it, rel = s.solve(tau, 8, 1e-8 if val_dtype == "f64" else 1e-6, 100_000)
        assert ok


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
@pytest.mark.parametrize("per_col,threads", [(150, 448), (37, 128), (1, 64)])
def test_streaming_kernel_on_long_and_short_columns(val_dtype, tol, per_col, threads):
    # the streaming kernel copies every chunk of a column: 150 entries are ten chunks
    # (the last one ragged); 37 three; 1 a single ragged chunk; ragged tau
    inst = instances.per_col_instance(20_000, 4_000, per_col, nnz_star=200, val_dtype=val_dtype, seed=1021)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    tau = min(2048 + 5, inst.n)
    refresh = 0 if val_dtype == "f64" else 16
    with Lasso.from_instance(inst, refresh_every=refresh) as s:
        s.set_tuning(4, 1, threads, 1)
        for upto in (1, 3, 30):
            s.step(tau, upto - s.iteration, 6)
            ref.run(tau, upto - ref.k, 6, refresh_every=refresh)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto
        ok, it, rel = s.solve(tau, 6, 1e-8 if val_dtype == "f64" else 1e-6, 100_000)
        assert ok


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
@pytest.mark.parametrize("per_col,choice", [(1, (0, 1, 64, 1)), (17, (0, 1, 128, 0)), (25, (0, 1, 448, 1)),
                                            (33, (0, 1, 448, 0)), (33, (0, 1, 128, 1, 1)), (150, (0, 1, 448, 1)),
                                            (150, (0, 1, 64, 0, 1))])
def test_pipelined_kernel_on_long_and_short_columns(val_dtype, tol, per_col, choice):
    # the pipelined kernel's slot holds a column's first 24 (FP64) or 32 (FP32, BF16) entries;
    # the rest is read from memory in chunks of 16, in the gradient and in both scatters (this
    # iteration's from the slot, the previous one's from memory).  1 entry: a single padded
    # entry; 17: one entry past the first chunk; 25: one past the FP64 slot; 33: one past the
    # FP32 / BF16 slot; 150: several chunks past it, the last one ragged.  With and without
    # the column heads (one bulk copy, or two to four from the CSC arrays), FP64 also with the
    # FP32 certificate of zero steps; ragged tau over blocks of 64 to 448 threads
    inst = instances.per_col_instance(20_000, 4_000, per_col, nnz_star=200, val_dtype=val_dtype, seed=1027)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    tau = min(2048 + 5, inst.n)
    refresh = 0 if val_dtype == "f64" else 16
    with Lasso.from_instance(inst, refresh_every=refresh) as s:
        s.set_tuning(*choice)
        for upto in (1, 3, 30):
            s.step(tau, upto - s.iteration, 6)
            ref.run(tau, upto - ref.k, 6, refresh_every=refresh)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto
        ok, it, rel = s.solve(tau, 6, 1e-8 if val_dtype == "f64" else 1e-6, 100_000)
        assert ok


@pytest.mark.parametrize("val_dtype,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16", 1e-5)])
@pytest.mark.parametrize("per_col,threads", [(600, 512), (150, 128), (37, 32), (1, 64)])
def test_warp_kernel_on_long_and_short_columns(val_dtype, tol, per_col, threads):
    # the warp-cooperative kernel copies runs of up to 256 entries: 600 entries are three
    # items (the last one ragged), 150 and 37 one, 1 a single padded entry; ragged tau
    # (m grows with the column length: the generator draws each column's distinct rows)
    m = 400_000 if per_col > 200 else 20_000
    inst = instances.per_col_instance(m, 4_000, per_col, nnz_star=200, val_dtype=val_dtype, seed=1021)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    tau = min(2048 + 5, inst.n)
    refresh = 0 if val_dtype == "f64" else 16
    with Lasso.from_instance(inst, refresh_every=refresh) as s:
        s.set_tuning(5, 1, threads, 1)
        for upto in (1, 3, 30):
            s.step(tau, upto - s.iteration, 6)
            ref.run(tau, upto - ref.k, 6, refresh_every=refresh)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto
        ok, it, rel = s.solve(tau, 6, 1e-8 if val_dtype == "f64" else 1e-6, 100_000)
        assert ok


def _warps_of_grid(threads):
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count * (threads // 32)


@pytest.mark.parametrize("val_dtype,tol,zc", [("f64", 1e-10, 1), ("f64", 1e-10, 0), ("bf16", 1e-5, -1)])
def test_warp_kernel_with_many_positions_per_warp(val_dtype, tol, zc):
    # about 28 positions per warp (blocks of 512 threads, one per SM): several groups of
    # four (FP64) or eight columns per warp reduction, the last one ragged; about a
    # quarter of the columns empty (Poisson column counts of mean 1.5); FP64 with and
    # without the FP32 certificate
    warps = _warps_of_grid(512)
    n = 30 * warps
    inst = instances.row_omega_instance(n // 2, n, 3, density=0.01, val_dtype=val_dtype, seed=1051)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    assert np.sum(np.diff(inst.col_ptr) == 0) > n // 8
    tau = 28 * warps + 7
    with Lasso.from_instance(inst) as s:
        s.set_tuning(5, 1, 512, 1, zc)
        for upto in (1, 2, 7):
            s.step(tau, upto - s.iteration, 9)
            ref.run_threads(tau, upto - ref.k, 9, 8)
            assert _rel(s.x(), ref.x) <= tol, upto
            assert _rel(s.residual(), ref.g) <= tol, upto


def _cu_limit_persisting_l2():
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    v = ctypes.c_size_t(0)
    assert cu.cuCtxGetLimit(ctypes.byref(v), 0x06) == 0        # CU_LIMIT_PERSISTING_L2_CACHE_SIZE (read only)
    return v.value


def test_l2_persist_option_is_scoped_to_the_handle():
    import torch
    torch.zeros(1, device="cuda")
    before = _cu_limit_persisting_l2()
    inst = instances.per_col_instance(2000, 1000, 20, nnz_star=50, val_dtype="f64", seed=1003)
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    with Lasso.from_instance(inst, l2_persist=True) as s:
        assert _cu_limit_persisting_l2() >= before
        s.step(96, 12, 2)
        ref.run(96, 12, 2)
        assert _rel(s.x(), ref.x) <= 1e-10
    assert _cu_limit_persisting_l2() == before


@pytest.mark.parametrize("first_destroyed", ["first_created", "last_created"])
def test_l2_persist_limit_is_shared_by_the_handles_of_a_device(first_destroyed):
    # the limit is the context's: it stays raised while any l2_persist handle lives,
    # and goes back to the value from before the first one when the last one goes
    import torch
    torch.zeros(1, device="cuda")
    before = _cu_limit_persisting_l2()
    inst = instances.per_col_instance(2000, 1000, 20, nnz_star=50, val_dtype="f64", seed=1003)
    a = Lasso.from_instance(inst, l2_persist=True)
    raised = _cu_limit_persisting_l2()
    assert raised >= before
    b = Lasso.from_instance(inst, l2_persist=True)
    plain = Lasso.from_instance(inst)
    assert _cu_limit_persisting_l2() == raised
    order = (a, b) if first_destroyed == "first_created" else (b, a)
    order[0].close()
    assert _cu_limit_persisting_l2() == raised       # the other handle still holds its set-aside
    order[1].step(96, 3, 2)
    plain.close()
    assert _cu_limit_persisting_l2() == raised
    order[1].close()
    assert _cu_limit_persisting_l2() == before


def test_handle_memory_comes_back_from_the_pool():
    # destroyed handles leave their memory in the library's pool; the next handle
    # reuses it, and pcdm_release_cached_memory returns it to the device
    import torch
    from paper_1212_0873_gb300 import _binding as B
    torch.cuda.synchronize()
    B.pcdm_release_cached_memory()
    free0, _ = torch.cuda.mem_get_info()
    inst = instances.per_col_instance(400_000, 200_000, 20, nnz_star=100, val_dtype="f64", seed=1041)
    xs = []
    for _ in range(3):
        with Lasso.from_instance(inst) as s:
            s.step(4096, 5, 1)
            xs.append(s.x())
        torch.cuda.synchronize()
    assert all(np.array_equal(xs[0], x) for x in xs[1:])
    B.pcdm_set_memory_cache(0)                 # keep nothing: freed memory goes back at synchronisation
    torch.cuda.synchronize()
    B.pcdm_release_cached_memory()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    B.pcdm_set_memory_cache(16 << 30)


@pytest.fixture(scope="module")
def omega128_inst():
    # 128 nonzeros in every row (the long-column end of the scale workload), smaller m = n
    return instances.row_omega_instance(200_000, 200_000, 128, density=0.01, val_dtype="f64", seed=1031)


@pytest.mark.parametrize("choice", [(1, 2, 0, 1), (2, 4, 0, 1), (4, 1, 448, 1), (0, 1, 448, 1), (5, 1, 512, 1, 1),
                                    (5, 1, 256, 1, 0)])
def test_omega128_rows_follow_the_oracle(omega128_inst, choice):
    inst = omega128_inst
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    assert ref.omega == 128
    tau = 8192
    with Lasso.from_instance(inst, l2_persist=True) as s:
        assert s.omega == 128
        s.set_tuning(*choice)
        for upto in (1, 4, 12):
            s.step(tau, upto - s.iteration, 4)
            ref.run_threads(tau, upto - ref.k, 4, 8)
            assert _rel(s.x(), ref.x) <= 1e-10, (choice, upto)
            assert _rel(s.residual(), ref.g) <= 1e-10, (choice, upto)

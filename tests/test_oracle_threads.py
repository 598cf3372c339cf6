"""The oracle's threaded timing mode (the multicore CPU baseline of the bench)
equals its single-threaded run, which stays the parity reference, bit for bit:
the same Algorithm 1 iterations with the per-position steps spread over threads
and the updates of g applied in the same order."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import instances


def _state(inst):
    return oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
@pytest.mark.parametrize("case", ["tiny", "per_col"])
def test_threaded_run_equals_the_serial_run(threads, case):
    if case == "tiny":
        inst, tau, iters, refresh = instances.tiny_instance("f64"), 32, 300, 16
    else:
        inst = instances.per_col_instance(40_000, 20_000, 10, nnz_star=400, val_dtype="f64", seed=95)
        tau, iters, refresh = 1000 + 7, 30, 8
    a, b = _state(inst), _state(inst)
    a.run(tau, iters, 4, refresh_every=refresh)
    b.run_threads(tau, iters // 3, 4, threads, refresh_every=refresh)
    b.run_threads(tau, iters - iters // 3, 4, threads, refresh_every=refresh)
    assert a.k == b.k
    assert np.array_equal(a.x.view(np.uint64), b.x.view(np.uint64))
    assert np.array_equal(a.g.view(np.uint64), b.g.view(np.uint64))
    assert np.count_nonzero(a.x) > 0


def test_threaded_run_with_more_threads_than_positions_and_bad_sizes():
    inst = instances.tiny_instance("f64")
    a, b = _state(inst), _state(inst)
    a.run(3, 50, 9)
    b.run_threads(3, 50, 9, threads=16)               # capped at tau threads
    assert np.array_equal(a.x, b.x) and np.array_equal(a.g, b.g)
    with pytest.raises(ValueError):
        b.run_threads(inst.n + 1, 1, 0, threads=2)
    with pytest.raises(ValueError):
        b.run_threads(4, 1, 0, threads=0)


def test_sample_range_pieces_make_the_sample():
    import ctypes
    n, tau, seed, k = 100_003, 5000, 77, 12
    full = oracle.sample(seed, k, n, tau)
    S = np.zeros(tau, dtype=np.int32)
    for j0, j1 in ((0, 1), (1, 999), (999, 4321), (4321, 5000)):
        assert oracle.lib().pcdm_oracle_sample_range(seed, k, n, j0, j1, ctypes.c_void_p(S.ctypes.data)) == 0
    assert np.array_equal(S, full)

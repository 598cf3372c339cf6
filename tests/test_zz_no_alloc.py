"""pcdm_omega_noalloc: the row-count / omega computation of the set-up with its
scratch in a fixed device array of the library (no allocation), against the
omega that pcdm_create computes (pcdm_omega) and the oracle's."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, _binding as B, instances

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


def _device_csc(torch, inst):
    d = dict(col_ptr=torch.from_numpy(inst.col_ptr).cuda(), row_idx=torch.from_numpy(inst.row_idx).cuda())
    csc = B.pcdm_csc(m=inst.m, n=inst.n, nnz=int(inst.col_ptr[-1]), col_ptr=d["col_ptr"].data_ptr(),
                     row_idx=d["row_idx"].data_ptr(), val=0, val_dtype=B.PCDM_F64, on_device=1)
    return csc, d


def _omega_both_ways(torch, inst):
    csc, keep = _device_csc(torch, inst)
    stream = torch.cuda.current_stream().cuda_stream
    first = B.pcdm_omega_noalloc(csc, stream)
    second = B.pcdm_omega_noalloc(csc, stream)
    with Lasso.from_instance(inst) as s:
        existing = s.omega
    return first, second, existing


@pytest.mark.parametrize("make", [
    lambda: instances.tiny_instance(),
    lambda: instances.per_col_instance(50_000, 20_000, 12, nnz_star=100, seed=7),
    lambda: instances.row_omega_instance(1_000_000, 1_000_000, 16, density=0.01, noise=0.01, lam_frac=0.05,
                                         seed=1002),
])
def test_matches_pcdm_omega_twice_in_a_row(torch, make):
    inst = make()
    first, second, existing = _omega_both_ways(torch, inst)
    assert first == second == existing
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    assert first == oracle.omega(A)


def test_largest_allowed_m(torch):
    m = B.PCDM_NOALLOC_MAX_ROWS
    rng = np.random.default_rng(3)
    n, per = 2000, 6
    rows = np.sort(np.stack([rng.choice(m, per, replace=False) for _ in range(n)]), axis=1)
    rows[0, -1] = m - 1            # the last row is touched
    rows[1, -1] = m - 1            # twice
    rows.sort(axis=1)
    col_ptr = np.arange(0, n * per + 1, per, dtype=np.int64)
    row_idx = rows.reshape(-1).astype(np.int32)
    val = rng.standard_normal(n * per)
    b = rng.standard_normal(m)
    t_cp, t_ri = torch.from_numpy(col_ptr).cuda(), torch.from_numpy(row_idx).cuda()
    csc = B.pcdm_csc(m=m, n=n, nnz=n * per, col_ptr=t_cp.data_ptr(), row_idx=t_ri.data_ptr(), val=0,
                     val_dtype=B.PCDM_F64, on_device=1)
    got = B.pcdm_omega_noalloc(csc, torch.cuda.current_stream().cuda_stream)
    want = int(np.bincount(row_idx, minlength=m).max())
    assert got == want >= 2
    with Lasso(m, n, col_ptr, row_idx, val, b, 0.1) as s:
        assert s.omega == got


def test_no_device_memory_is_taken(torch):
    inst = instances.tiny_instance()
    csc, keep = _device_csc(torch, inst)
    stream = torch.cuda.current_stream().cuda_stream
    B.pcdm_omega_noalloc(csc, stream)          # set-up (first call on this device) already done or done here
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.pcdm_omega_noalloc(csc, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_invalid_matrix_then_valid_again(torch):
    inst = instances.tiny_instance()
    bad_rows = inst.row_idx.copy()
    bad_rows[5] = inst.m            # out of range: skipped by the kernel and reported
    t_cp, t_ri = torch.from_numpy(inst.col_ptr).cuda(), torch.from_numpy(bad_rows).cuda()
    csc = B.pcdm_csc(m=inst.m, n=inst.n, nnz=int(inst.col_ptr[-1]), col_ptr=t_cp.data_ptr(),
                     row_idx=t_ri.data_ptr(), val=0, val_dtype=B.PCDM_F64, on_device=1)
    with pytest.raises(B.PcdmError) as ei:
        B.pcdm_omega_noalloc(csc, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == B.PCDM_EINVAL
    first, second, existing = _omega_both_ways(torch, inst)
    assert first == second == existing

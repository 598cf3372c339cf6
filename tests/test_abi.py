"""The C ABI on the CPU: the library loads, exports every function that
include/pcdm.h declares, its structs have the layout the binding uses, and the
argument checks that run before any CUDA call reject bad input.  No GPU needed:
no call here reaches a kernel."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcdm.h")


@pytest.fixture(scope="module")
def B():
    from paper_1212_0873_gb300 import build
    build.build()
    from paper_1212_0873_gb300 import _binding
    _binding.lib()
    return _binding


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcdm_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pcdm_create", "pcdm_step", "pcdm_gap", "pcdm_solve", "pcdm_get_x", "pcdm_set_x",
                     "pcdm_set_lambda", "pcdm_omega", "pcdm_destroy", "pcdm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(B):
    lib = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared_functions()) == set(B.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_header(B):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "pcdm.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(pcdm_csc), sizeof(pcdm_opts), sizeof(pcdm_stats), sizeof(pcdm_tuning));
  printf("%zu %zu %zu %zu\n", offsetof(pcdm_csc, val_dtype), offsetof(pcdm_opts, barrier_timeout_ns),
         offsetof(pcdm_stats, iter_kernel_ms), offsetof(pcdm_tuning, us_per_iteration));
  printf("%zu\n", offsetof(pcdm_opts, deterministic_scatter));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[0] == ctypes.sizeof(B.pcdm_csc)
    assert sizes[1] == ctypes.sizeof(B.pcdm_opts)
    assert sizes[2] == ctypes.sizeof(B.pcdm_stats)
    assert sizes[3] == ctypes.sizeof(B.pcdm_tuning)
    assert sizes[4] == B.pcdm_csc.val_dtype.offset
    assert sizes[5] == B.pcdm_opts.barrier_timeout_ns.offset
    assert sizes[6] == B.pcdm_stats.iter_kernel_ms.offset
    assert sizes[7] == B.pcdm_tuning.us_per_iteration.offset
    assert sizes[8] == B.pcdm_opts.deterministic_scatter.offset


def test_default_opts_and_status_strings(B):
    o = B.pcdm_default_opts()
    assert (o.xg_dtype, o.fused, o.refresh_every, o.check_every, o.lanes_per_col, o.profile) == (0, 1, 0, 0, 0, 0)
    assert o.barrier_timeout_ns == 2_000_000_000
    for code, name in enumerate(["PCDM_OK", "PCDM_EINVAL", "PCDM_ENOMEM", "PCDM_ECUDA", "PCDM_ETIMEOUT",
                                 "PCDM_ENOTCONV", "PCDM_ESTATE"]):
        assert B.pcdm_status_string(code) == name


def _csc(B, m=4, n=3, nnz=0, val_dtype=0):
    import numpy as np
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    keep = [col_ptr]
    A = B.pcdm_csc(m, n, nnz, col_ptr.ctypes.data, None, None, val_dtype, 0)
    return A, keep


@pytest.mark.parametrize("case", ["null_A", "null_b", "m0", "n0", "neg_nnz", "huge_m", "lam_neg", "lam_nan",
                                  "lam_inf", "pair_f64_f32", "pair_bf16_f64", "bad_bdtype", "bad_lanes",
                                  "neg_refresh", "null_rows", "det_flag_2", "det_independent"])
def test_create_rejects_bad_arguments_before_any_cuda_call(B, case):
    import numpy as np
    b = np.zeros(4)
    A, keep = _csc(B)
    opts = B.pcdm_default_opts()
    lam = 0.1
    bdt = B.PCDM_F64
    a_arg, b_arg = A, b.ctypes.data
    if case == "null_A":
        a_arg = None
    elif case == "null_b":
        b_arg = None
    elif case == "m0":
        A.m = 0
    elif case == "n0":
        A.n = 0
    elif case == "neg_nnz":
        A.nnz = -1
    elif case == "huge_m":
        A.m = 2**31
    elif case == "lam_neg":
        lam = -1.0
    elif case == "lam_nan":
        lam = float("nan")
    elif case == "lam_inf":
        lam = float("inf")
    elif case == "pair_f64_f32":
        opts.xg_dtype = B.PCDM_F32
    elif case == "pair_bf16_f64":
        A.val_dtype = B.PCDM_BF16
    elif case == "bad_bdtype":
        bdt = B.PCDM_BF16
    elif case == "bad_lanes":
        opts.lanes_per_col = 12
    elif case == "neg_refresh":
        opts.refresh_every = -1
    elif case == "null_rows":
        A.nnz = 5
    elif case == "det_flag_2":
        opts.deterministic_scatter = 2
    elif case == "det_independent":
        opts.deterministic_scatter = 1
        opts.sampling = B.SAMPLING_CODES["independent"]
    h = ctypes.c_void_p()
    st = B.lib().pcdm_create(ctypes.byref(a_arg) if a_arg is not None else None, b_arg, bdt, lam,
                             ctypes.byref(opts), None, ctypes.byref(h))
    assert st == B.PCDM_EINVAL, (case, st, B.pcdm_last_error(None))
    assert not h.value
    assert B.pcdm_last_error(None)
    del keep


def test_calls_on_a_null_handle_are_rejected(B):
    L = B.lib()
    assert L.pcdm_step(None, 1, 1, 0) == B.PCDM_EINVAL
    assert L.pcdm_gap(None, None, None, None) == B.PCDM_EINVAL
    assert L.pcdm_solve(None, 1, 0, 1e-6, 10, None, None) == B.PCDM_EINVAL
    assert L.pcdm_refresh(None) == B.PCDM_EINVAL
    assert L.pcdm_reset(None) == B.PCDM_EINVAL
    k = ctypes.c_int64()
    assert L.pcdm_omega(None, ctypes.byref(k)) == B.PCDM_EINVAL
    L.pcdm_destroy(None)


@pytest.mark.parametrize("args", [(0, 0, 0, 1), (0, 0, 5, 6), (0, -1, 5, 1), (0, 0, 2**31, 1), (0, 0, 5, -1)])
def test_sample_rejects_bad_sizes(B, args):
    seed, k, n, tau = args
    assert B.lib().pcdm_sample(seed, k, n, tau, None, None) == B.PCDM_EINVAL


def test_selftest_rejects_bad_timeout(B):
    assert B.lib().pcdm_selftest_barrier_timeout(0, None) == B.PCDM_EINVAL


def test_check_schedule_extrapolates_the_linear_rate(B):
    """pcdm_solve's adaptive gap-check schedule: host arithmetic, no device."""
    f = B.pcdm_next_check_interval
    E = 62
    # gap fell 1e-1 -> 1e-2 over one epoch: 4 more decades to 1e-6 is 4 epochs,
    # + 5%, but at most twice the last interval
    assert f(E, 0, 1e-1, E, 1e-2, 1e-6) == 2 * E
    # the same rate over a 4-epoch window: ceil(1.05 * 4 E)
    assert f(E, 0, 1e-1 ** 4, 4 * E, 1e-1 ** 8, 1e-12) == int(__import__("math").ceil(1.05 * 4 * E))
    # almost there: never below a quarter epoch
    assert f(E, 0, 2e-6, 10 * E, 1.0000001e-6, 1e-6) == (E + 3) // 4
    # slow progress: never beyond 64 epochs
    assert f(E, 0, 1.0, 100 * E, 0.5, 1e-9) == 64 * E
    # no decrease, non-positive gaps, zero interval: one epoch
    assert f(E, 0, 1e-3, E, 2e-3, 1e-6) == E
    assert f(E, 0, 1e-3, E, 0.0, 1e-6) == E
    assert f(E, E, 1e-2, E, 1e-3, 1e-6) == E
    assert f(0, 0, 1e-1, 1, 1e-2, 1e-6) == 2      # epoch < 1 is taken as 1


def test_omega_noalloc_host_checks(B):
    """pcdm_omega_noalloc rejects, before any device work, what it cannot serve."""
    L = B.lib()
    out = ctypes.c_int64(-1)
    ok = dict(m=10, n=4, nnz=0, col_ptr=1, row_idx=0, val=0, val_dtype=B.PCDM_F64, on_device=1)
    for case, change in [("host arrays", dict(on_device=0)), ("too many rows", dict(m=B.PCDM_NOALLOC_MAX_ROWS + 1)),
                         ("negative n", dict(n=-1)), ("no rows", dict(m=0)), ("no columns", dict(n=0)),
                         ("n of 2^31", dict(n=2**31)), ("negative nnz", dict(nnz=-1)), ("no col_ptr", dict(col_ptr=0)),
                         ("no row_idx", dict(nnz=5))]:
        csc = B.pcdm_csc(**dict(ok, **change))
        assert L.pcdm_omega_noalloc(ctypes.byref(csc), ctypes.byref(out), None) == B.PCDM_EINVAL, case
    assert L.pcdm_omega_noalloc(None, ctypes.byref(out), None) == B.PCDM_EINVAL
    assert out.value == -1
    assert B.PCDM_NOALLOC_MAX_ROWS == int(re.search(r"#define PCDM_NOALLOC_MAX_ROWS (\d+)",
                                                    open(HEADER).read()).group(1))


def test_batch_create_host_checks(B):
    """pcdm_batch_create rejects its own arguments before any device work."""
    L = B.lib()
    h = ctypes.c_void_p()
    csc = B.pcdm_csc(m=10, n=4, nnz=0, col_ptr=1, row_idx=0, val=0, val_dtype=B.PCDM_F64, on_device=1)
    lam = (ctypes.c_double * 40)(*([0.5] * 40))
    bad = (ctypes.c_double * 2)(0.5, -1.0)
    for nrhs, lams in [(0, lam), (33, lam), (2, bad)]:
        st = L.pcdm_batch_create(ctypes.byref(csc), nrhs, ctypes.c_void_p(1), B.PCDM_F64,
                                 ctypes.cast(lams, ctypes.c_void_p), None, None, ctypes.byref(h))
        assert st == B.PCDM_EINVAL and not h.value
    assert L.pcdm_batch_step(None, 1, 1, 0) == B.PCDM_EINVAL
    assert L.pcdm_batch_gap(None, None, None, None) == B.PCDM_EINVAL
    L.pcdm_batch_destroy(None)


def test_generator_library_exports_its_header():
    from paper_1212_0873_gb300 import build
    build.build_gen()
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "pcdm_gen.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(pcdm_[A-Za-z_0-9]+)\s*\(", text)))
    assert names == ["pcdm_gen_per_col"]
    lib = ctypes.CDLL(build.GEN_LIB)
    assert all(hasattr(lib, n) for n in names)


def test_create_problem_rejects_bad_arguments_before_device_work(B):
    L = B.lib()
    A = B.pcdm_csc(4, 3, 0, None, None, None, B.PCDM_F64, 0)
    y = (ctypes.c_double * 4)(1.0, -1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    opts = B.pcdm_default_opts()
    assert L.pcdm_create_problem(ctypes.byref(A), 0, y, 1.0, None, None, ctypes.byref(h)) == B.PCDM_EINVAL
    assert L.pcdm_create_problem(ctypes.byref(A), 3, y, 1.0, None, None, ctypes.byref(h)) == B.PCDM_EINVAL
    assert L.pcdm_create_problem(ctypes.byref(A), 1, None, 1.0, None, None, ctypes.byref(h)) == B.PCDM_EINVAL
    for lam in (0.0, -1.0, float("inf"), float("nan")):
        assert L.pcdm_create_problem(ctypes.byref(A), 2, y, lam, None, None, ctypes.byref(h)) == B.PCDM_EINVAL
    opts.sampling = 1
    assert L.pcdm_create_problem(ctypes.byref(A), 1, y, 1.0, ctypes.byref(opts), None,
                                 ctypes.byref(h)) == B.PCDM_EINVAL
    # the deterministic form is LASSO-only (a valid empty matrix, so that only the option is wrong)
    col_ptr = (ctypes.c_int64 * 4)(0, 0, 0, 0)
    A2 = B.pcdm_csc(4, 3, 0, ctypes.addressof(col_ptr), None, None, B.PCDM_F64, 0)
    opts = B.pcdm_default_opts()
    opts.deterministic_scatter = 1
    assert L.pcdm_create_problem(ctypes.byref(A2), 1, y, 1.0, ctypes.byref(opts), None,
                                 ctypes.byref(h)) == B.PCDM_EINVAL
    msg = B.pcdm_last_error(None)
    assert "deterministic" in (msg.decode() if isinstance(msg, bytes) else msg)
    assert not h.value
    assert L.pcdm_problem_kind(None, None) != 0


def test_gather_rate_rejects_bad_arguments(B):
    L = B.lib()
    out = ctypes.c_double(-1.0)
    buf = ctypes.c_void_p(1 << 20)                  # never dereferenced: every case fails before device work
    assert L.pcdm_gather_rate(None, 10, 8, ctypes.byref(out), None) == B.PCDM_EINVAL
    assert L.pcdm_gather_rate(buf, 10, 8, None, None) == B.PCDM_EINVAL
    for n, eb in ((0, 8), (-1, 4), (2**32, 4), (10, 2), (10, 16)):
        assert L.pcdm_gather_rate(buf, n, eb, ctypes.byref(out), None) == B.PCDM_EINVAL, (n, eb)
    assert out.value == -1.0

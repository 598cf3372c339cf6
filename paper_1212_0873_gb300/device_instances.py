"""Seeded synthetic instances generated on the GPU (libpcdm_gen, include/pcdm_gen.h).

Input generation only: these arrays feed the solver and the tests alike.  Used
for sizes that host generation cannot reach (the huge mixed-precision instance:
m = 1e9, n = 5e8, 8 nonzeros per column, 4e9 nonzeros)."""
import ctypes
import os

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.GEN_LIB
        if not os.path.exists(path):
            raise RuntimeError("libpcdm_gen.so is not built (run paper_1212_0873_gb300.build.build())")
        L = ctypes.CDLL(path)
        L.pcdm_gen_per_col.restype = ctypes.c_int
        L.pcdm_gen_per_col.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int32] + [ctypes.c_void_p] * 8
        _lib = L
    return _lib


def per_col_on_device(m, n, per_col, *, seed=1008, val_dtype="bf16", x_density=1e-4, noise_sd=1e-2,
                      b_dtype="f32", stream=None):
    """Returns dict(col_ptr, row_idx, val, b, x_star: CUDA tensors; lambda_max: float);
    val is int16-typed storage for bf16 values (their bit patterns)."""
    import torch
    dev = "cuda"
    vt = {"f64": (0, torch.float64), "f32": (1, torch.float32), "bf16": (2, torch.bfloat16)}[val_dtype]
    bt = {"f64": (0, torch.float64), "f32": (1, torch.float32)}[b_dtype]
    col_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    row_idx = torch.empty(n * per_col, dtype=torch.int32, device=dev)
    val = torch.empty(n * per_col, dtype=vt[1], device=dev)
    b = torch.empty(m, dtype=bt[1], device=dev)
    x_star = torch.empty(n, dtype=torch.float64, device=dev)
    scratch = torch.empty(m, dtype=torch.float64, device=dev)
    lam_max = ctypes.c_double()
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = lib().pcdm_gen_per_col(int(m), int(n), int(per_col), int(seed) & (2**64 - 1), vt[0], float(x_density),
                                float(noise_sd), bt[0], col_ptr.data_ptr(), row_idx.data_ptr(), val.data_ptr(),
                                b.data_ptr(), x_star.data_ptr(), scratch.data_ptr(), ctypes.byref(lam_max),
                                ctypes.c_void_p(st))
    del scratch
    if rc != 0:
        raise RuntimeError("pcdm_gen_per_col failed (cudaError %d)" % rc)
    return dict(col_ptr=col_ptr, row_idx=row_idx, val=val, b=b, x_star=x_star, lambda_max=lam_max.value)

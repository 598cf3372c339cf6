"""Device-generated instances at scale (libpcdm_gen): the first PCDM1 iterations
against the oracle on the subproblem they touch.  The oracle draws S_k itself
(the full n), takes the touched columns and rows from the generated instance,
computes omega from all row indices and L from its columns, and runs the same
iterations; the GPU's x on those columns and g on those rows must agree.
The huge configuration (m = 1e9, n = 5e8, 8 BF16 nonzeros per column, 4e9
nonzeros, tau = 2^20) is marked slow: about 140 GB of device memory."""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso, device_instances

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _bf16_to_f64(t):
    return t.float().double()


def _first_iterations_match(m, n, per_col, tau, K, lam_frac=0.1, seed=1008, refresh_every=32):
    torch = _torch()
    gen = device_instances.per_col_on_device(m, n, per_col, seed=seed, val_dtype="bf16", x_density=1e-4,
                                             noise_sd=1e-2, b_dtype="f32")
    lam = lam_frac * gen["lambda_max"]
    with Lasso(m, n, gen["col_ptr"], gen["row_idx"], gen["val"], gen["b"], lam,
               refresh_every=refresh_every) as s:
        # omega from every row index, on the host (int32 -> bincount)
        rows_all = gen["row_idx"].cpu().numpy()
        omega = int(np.bincount(rows_all, minlength=m).max())
        del rows_all
        assert s.omega == omega
        beta = oracle.beta_nice(omega, tau, n)
        assert s.beta(tau) == pytest.approx(beta, rel=1e-15)
        s.step(tau, K, seed)
        S = [oracle.sample(seed, k, n, tau) for k in range(K)]
        cols = np.unique(np.concatenate(S))
        t_cols = torch.from_numpy(cols.astype(np.int64)).cuda()
        # the touched columns (per_col entries each) and the rows they touch
        idx = (t_cols[:, None] * per_col + torch.arange(per_col, device="cuda")[None, :]).reshape(-1)
        rows = gen["row_idx"][idx].cpu().numpy().astype(np.int64)
        vals = _bf16_to_f64(gen["val"][idx]).cpu().numpy()
        urows, rmap = np.unique(rows, return_inverse=True)
        b_sub = gen["b"][torch.from_numpy(urows).cuda()].double().cpu().numpy()
        ncol = cols.size
        A_sub = oracle.Csc(urows.size, ncol, np.arange(ncol + 1, dtype=np.int64) * per_col,
                           rmap.astype(np.int32), vals)
        L = oracle.col_sqnorms(A_sub)
        x = np.zeros(ncol)
        g = -b_sub.copy()
        pos = {int(c): q for q, c in enumerate(cols)}
        for k in range(K):
            Sk = np.array([pos[int(c)] for c in S[k]], dtype=np.int32)
            oracle.iteration(A_sub, L, lam, beta, Sk, x, g)
        x_gpu = torch.empty(n, dtype=torch.float64, device="cuda")
        s.x_into(x_gpu)
        x_gpu = x_gpu[t_cols].cpu().numpy()
        g_gpu = torch.empty(m, dtype=torch.float32, device="cuda")
        from paper_1212_0873_gb300 import _binding as B
        B.pcdm_get_residual(s._h, g_gpu.data_ptr(), 1)
        g_gpu = g_gpu[torch.from_numpy(urows).cuda()].double().cpu().numpy()
        scale_x = max(float(np.max(np.abs(x))), 1e-300)
        assert float(np.max(np.abs(x_gpu - x))) <= 1e-5 * scale_x
        assert float(np.max(np.abs(g_gpu - g))) <= 1e-5 * max(float(np.max(np.abs(g))), 1e-300)
        assert np.count_nonzero(x) > 0
        return s.stats()


def test_first_iterations_at_1e7_columns():
    _first_iterations_match(m=20_000_000, n=10_000_000, per_col=8, tau=1 << 20, K=3)


@pytest.mark.slow
def test_first_iterations_huge():
    _first_iterations_match(m=1_000_000_000, n=500_000_000, per_col=8, tau=1 << 20, K=2)

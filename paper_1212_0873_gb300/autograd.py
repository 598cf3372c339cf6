"""torch.autograd for the LASSO solution map (b, lambda) -> x(b, lambda).

Forward: pcdm_solve (PCDM1) to a relative duality gap, then pcdm_polish on the
identified support and signs, so x is accurate to machine precision.
Backward: the implicit function theorem on the active set S = supp(x) with
s = sign(x_S): u solves (A_S^T A_S) u = dL/dx_S (pcdm_backward, the coordinate
kernel without the prox), dL/db = A_S u and dL/dlambda = -s^T u.  Nothing is
unrolled: a forward keeps only x (n doubles) for its backward.
"""
import torch

from .solver import Lasso


class LassoLayer:
    """A fixed sparse A (CSC) on the GPU; calling the layer with (b, lam) returns
    x(b, lam) as a differentiable CUDA float64 tensor.

    The forward solve only has to settle the support and signs (tol: relative
    duality gap; the FP32 forms bottom out near 1e-7); the FP64 polish then
    solves the optimality system on that support to polish_tol."""

    def __init__(self, m, n, col_ptr, row_idx, val, *, tau=None, tol=1e-9, polish_tol=1e-14, seed=0,
                 refresh_every=0, max_iters=10**6, backward_tol=1e-13):
        self.m, self.n = int(m), int(n)
        zeros = torch.zeros(self.m, dtype=torch.float64, device="cuda")
        if isinstance(col_ptr, torch.Tensor):
            self.solver = Lasso(m, n, col_ptr, row_idx, val, zeros, 0.0, refresh_every=refresh_every)
        else:
            import numpy as np
            self.solver = Lasso(m, n, col_ptr, row_idx, val, np.zeros(self.m), 0.0, refresh_every=refresh_every)
        self.tau = tau if tau is not None else min(self.n, 4096)
        self.tol, self.polish_tol, self.seed = tol, polish_tol, seed
        self.max_iters, self.backward_tol = max_iters, backward_tol

    def solve(self, b, lam):
        """x(b, lam) without autograd (warm-started from the previous x)."""
        s = self.solver
        s.set_b(b.detach().contiguous())
        s.set_lambda(float(lam))
        ok, it, rel = s.solve(self.tau, self.seed, self.tol, self.max_iters)
        if not ok:
            raise RuntimeError("forward solve did not reach the gap tolerance (%d iterations, %g)" % (it, rel))
        ok, it, rel = s.polish(self.polish_tol, self.max_iters)
        if not ok:
            raise RuntimeError("polish did not converge (%d iterations, residual %g)" % (it, rel))
        x = torch.empty(self.n, dtype=torch.float64, device="cuda")
        s.x_into(x)
        return x

    def __call__(self, b, lam):
        if not isinstance(lam, torch.Tensor):
            lam = torch.tensor(float(lam), dtype=torch.float64, device="cuda")
        return _LassoFn.apply(b, lam, self)

    def close(self):
        self.solver.close()


class _LassoFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, lam, layer):
        x = layer.solve(b, float(lam))
        ctx.layer = layer
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        layer = ctx.layer
        s = layer.solver
        s.set_x(x)                       # the support and signs of this forward
        db = torch.empty(layer.m, dtype=torch.float64, device="cuda")
        db, dlam, ok, it, rel = s.backward(gx.detach().to(torch.float64).contiguous(), tol=layer.backward_tol,
                                           max_iters=layer.max_iters, db_out=db)
        if not ok:
            raise RuntimeError("backward solve did not converge (%d iterations, residual %g)" % (it, rel))
        return db, torch.tensor(dlam, dtype=torch.float64, device="cuda"), None

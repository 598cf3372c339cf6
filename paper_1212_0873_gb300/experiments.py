"""The paper's "theory versus reality" experiment (Sec. 8.2) on the GPU solver.

min 1/2 ||A x - b||^2 (lambda = 0) with A 3000 x 1000 whose every row holds
exactly omega nonzeros, all equal (instances.equal_rows_instance).  For each tau
PCDM1 with the tau-nice sampling runs from x = 0 until F(x_k) - F* <= eps; the
empirical speedup is iterations(tau = 1) / iterations(tau), the theoretical one
tau / beta with beta of Theorem ESO-nice (the tau-nice row of the paper's table
of speedup factors).  F* comes from a dense FP64 least-squares solve (numpy) of
the same A and b, not from the GPU.  The paper shows the comparison only as a
figure, so there are no printed numbers to match: the result is a table.
"""
import numpy as np

from . import instances
from .solver import Lasso


def iterations_to_eps(solver, tau, f_star, eps, seed=0, resolution=8, max_iters=10**8):
    """Iterations of PCDM1 from the solver's current x until F - F* <= eps,
    checked every max(1, epoch / resolution) iterations (epoch = n / tau)."""
    every = max(1, (solver.n + tau - 1) // tau // resolution)
    k = 0
    while k < max_iters:
        if solver.gap()["primal"] - f_star <= eps:
            return k
        solver.step(tau, every, seed)
        k += every
    raise RuntimeError("no eps-solution within max_iters")


def theory_vs_reality(omegas=(5, 10, 50, 100), taus=(1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1000), eps=1e-6,
                      m=3000, n=1000, seed=0, resolution=8):
    rows = []
    for omega in omegas:
        inst = instances.equal_rows_instance(m, n, omega)
        A = instances.dense(inst)
        x_ls = np.linalg.lstsq(A, inst.b, rcond=None)[0]
        f_star = 0.5 * float(np.sum((A @ x_ls - inst.b) ** 2))
        serial = None
        for tau in taus:
            with Lasso.from_instance(inst) as s:
                it = iterations_to_eps(s, tau, f_star, eps, seed, resolution)
            if tau == 1:
                serial = it
            beta = 1.0 + (omega - 1) * (tau - 1) / max(1, n - 1)
            rows.append(dict(omega=omega, tau=tau, iterations=it, beta=beta, theory=tau / beta,
                             empirical=(serial / it) if serial else None))
    return rows

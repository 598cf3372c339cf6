"""PCDM1 with tau-nice sampling for LASSO on one GB300 (sm_103a).

Richtarik & Takac, "Parallel Coordinate Descent Methods for Big Data
Optimization" (arXiv:1212.0873), Algorithm 1 with the step of eq. (h(x)) and
beta of Theorem ESO-nice, on a column-stored sparse A.

  _binding   ctypes binding of libpcdm (include/pcdm.h), same entry-point names
  solver     Lasso: one instance resident on the GPU (numpy or torch CUDA inputs);
             BatchLasso: up to 32 right-hand sides / lambdas sharing A;
             MultiLasso: many independent small problems, one block each
             LabeledProblem: the SVM dual (Sec. 8.3) and logistic regression (Sec. 8.4)
  instances  seeded synthetic instances (numpy only)
  build      nvcc build of libpcdm.so for sm_103a

The CUDA library is loaded on first use; without it every call raises.
"""
from . import instances  # noqa: F401
from ._binding import (PCDM_BF16, PCDM_EINVAL, PCDM_F32, PCDM_F64, PcdmError, pcdm_beta, pcdm_create,  # noqa: F401
                       pcdm_csc, pcdm_default_opts, pcdm_destroy, pcdm_gap, pcdm_get_iteration, pcdm_get_L,
                       pcdm_get_residual, pcdm_get_stats, pcdm_get_x, pcdm_last_error, pcdm_omega, pcdm_opts,
                       pcdm_refresh, pcdm_reset, pcdm_reset_stats, pcdm_sample, pcdm_selftest_barrier_timeout,
                       pcdm_set_iteration, pcdm_set_lambda, pcdm_set_x, pcdm_solve, pcdm_stats,
                       pcdm_status_string, pcdm_step)
from .solver import BatchLasso, LabeledProblem, Lasso, MultiLasso, current_stream  # noqa: F401

"""The zero-step shortcuts of the iteration kernels change no result.

At x_i = 0 the LASSO step is zero exactly when |grad_i| <= lambda.  The
pipelined and warp-cooperative kernels can decide that in FP32 before any FP64
work (FP64 form: a sum over FP32 images of the operands with an error bound);
they and the lanes-per-column kernel test the finished gradient exactly (FP32 and BF16 forms:
the FP32 gradient against lambda rounded down; FP64 form: the bit patterns
compared as integers) and run no FP64 instruction for a lane that passes.  A
wrong certificate zeroes a step that should be nonzero, so these instances put
|grad_i| just above lambda for whole families of columns (nonzero but tiny
steps, which the oracle computes in FP64) next to columns just below it, with
operands chosen so that truncated FP32 images land below lambda, and with
magnitudes at the edges of the FP32 range (images clamped to 2^-126 or to inf).
Every kernel choice must then follow the oracle, and a zeroed step shows up as
a 100 % error on the tiny iterates.

Tolerance: the nonzero steps here are differences of two nearly equal FP64
numbers (u - t in the soft threshold), so the oracle and the kernel may differ
in their last 2^-53 / eps bits (eps the relative distance of |grad| to lambda);
the bound used is 1e-6 relative to the largest step (FP64) and 1e-4 (FP32).
"""
import numpy as np
import pytest

import oracle
from paper_1212_0873_gb300 import Lasso

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


# Column lengths: inside the first chunk, in the tail run, beyond both.
LENGTHS = [1, 2, 3, 4, 7, 8, 15, 16, 17, 23, 24, 25, 31, 32, 33, 40, 48, 57]


def _instance(n, m, scale_v, scale_b, seed):
    """Dyadic values with column sums of +-1 ("hot" columns) or +-1/2 ("cold"),
    so a_i^T b is exact in FP64 in any order; b = scale_b * beta0 * (+-1)
    with beta0 = 1 + 2^-25 + 2^-30 (bits below the 20 an FP32 image keeps)."""
    rng = np.random.default_rng(seed)
    beta0 = 1.0 + 2.0 ** -25 + 2.0 ** -30
    sgn_b = np.where(rng.random(m) < 0.5, -1.0, 1.0)
    b = scale_b * beta0 * sgn_b
    col_ptr = [0]
    rows, vals = [], []
    hot = np.zeros(n, dtype=bool)
    for i in range(n):
        c = LENGTHS[i % len(LENGTHS)]
        r = np.sort(rng.choice(m, size=c, replace=False))
        target = 1.0 if i % 3 != 2 else 0.5           # two columns in three are hot
        hot[i] = target == 1.0
        # split `target` into c dyadic parts of mixed signs: parts 2^-k, the first absorbs the rest
        parts = np.where(rng.random(c) < 0.5, -1.0, 1.0) * 2.0 ** -rng.integers(1, 6, size=c)
        parts[0] = 0.0
        parts[0] = target - parts.sum()
        v = parts * sgn_b[r]                           # so that v . b / (scale_b beta0) = target
        rows.append(r)
        vals.append(v * scale_v)
        col_ptr.append(col_ptr[-1] + c)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    row_idx = np.concatenate(rows).astype(np.int32)
    val = np.concatenate(vals)
    G = scale_v * scale_b * beta0                      # |a_i^T b| of a hot column, exactly
    return m, n, col_ptr, row_idx, val, b, G, hot


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


# (scale of the values, scale of b): ordinary; large b with small values; images
# of the values clamped to 2^-126; images of b infinite; products underflowing FP32.
SCALES = [(1.0, 1.0), (2.0 ** -100, 2.0 ** 100), (2.0 ** -130, 2.0 ** 20), (1.0, 2.0 ** 130), (2.0 ** -70, 2.0 ** -70)]
# (kernel, lanes per column, threads per block, column heads, zero-step certificate):
# the pipelined kernel with the FP32 certificate, without it (the exact test on the
# FP64 sum alone), the lanes-per-column kernel with 1 and 4 lanes, and the
# warp-cooperative kernel with its certificate and without it
CHOICES = [(0, 1, 448, 1, 1), (0, 1, 64, 0, 1), (0, 1, 448, 1, 0), (1, 1, 0, 1, -1), (1, 4, 0, 1, -1),
           (5, 1, 128, 1, 1), (5, 1, 32, 1, 0)]


@pytest.mark.parametrize("choice", CHOICES)
@pytest.mark.parametrize("scales", SCALES)
@pytest.mark.parametrize("eps", [2.0 ** -26, 2.0 ** -18])
def test_fp64_certificate_never_zeroes_a_nonzero_step(choice, scales, eps):
    m, n, col_ptr, row_idx, val, b, G, hot = _instance(611, 5000, *scales, seed=7)
    lam = G * (1.0 - eps)            # hot columns: |grad| just above lambda; cold ones: far below
    ref = oracle.State(oracle.Csc(m, n, col_ptr, row_idx, val), b, lam)
    ref.run(n, 1, 3)
    assert np.count_nonzero(ref.x[hot]) == np.count_nonzero(hot) and not np.any(ref.x[~hot])
    with Lasso(m, n, col_ptr, row_idx, val, b, lam) as s:
        s.set_tuning(*choice)
        s.step(n, 1, 3)
        x = s.x()
        assert np.count_nonzero(x[hot]) == np.count_nonzero(hot) and not np.any(x[~hot])
        assert _rel(x, ref.x) <= 1e-6
        # a second iteration: the hot columns now sit at x_i != 0 (no certificate)
        s.step(n, 1, 3)
        ref.run(n, 1, 3)
        assert _rel(s.x(), ref.x) <= 1e-6


@pytest.mark.parametrize("choice", CHOICES)
def test_fp64_ties_and_steps_just_below_lambda_are_zero(choice):
    m, n, col_ptr, row_idx, val, b, G, hot = _instance(611, 5000, 1.0, 1.0, seed=8)
    for lam in (G, G * (1.0 + 2.0 ** -40)):
        with Lasso(m, n, col_ptr, row_idx, val, b, lam) as s:
            s.set_tuning(*choice)
            s.step(n, 1, 5)
            assert not np.any(s.x())


@pytest.mark.parametrize("choice", CHOICES)
def test_fp32_gradient_against_lambda_rounded_down(choice):
    # FP32 values and residual: powers of two make the FP32 gradient exact, so
    # lambda a hair below |grad| must give nonzero steps (lambda rounded to
    # nearest in FP32 would equal |grad| and zero them)
    m, n, col_ptr, row_idx, val, b, G, hot = _instance(611, 5000, 1.0, 1.0, seed=9)
    b = np.sign(b)                                   # |b_r| = 1: exact in FP32
    G = 1.0
    lam = G * (1.0 - 2.0 ** -30)
    val32 = val.astype(np.float32)
    assert np.array_equal(val32.astype(np.float64), val)
    ref = oracle.State(oracle.Csc(m, n, col_ptr, row_idx, val), b, lam)
    ref.run(n, 1, 11)
    with Lasso(m, n, col_ptr, row_idx, val32, b, lam) as s:
        s.set_tuning(*choice)
        s.step(n, 1, 11)
        x = s.x()
        assert np.count_nonzero(x[hot]) == np.count_nonzero(hot) and not np.any(x[~hot])
        assert _rel(x, ref.x) <= 1e-4

"""Seeded synthetic instances (numpy only): LASSO, and labelled data for the
SVM dual and logistic regression.

This module only synthesises inputs: sparse matrices, planted solutions,
right-hand sides and the regularisation weight.  It holds none of the method's
arithmetic, imports nothing from the CUDA binding or the oracle, and is the one
piece of code that both sides read, so that both solve the same instance.

The paper's LASSO workload (Sec. 8.1) is a column-stored A with a fixed number
of nonzeros per column and a planted sparse optimum.  Its own generator is not
given, so the recipes here follow the workload shapes named in the design notes:

  tiny_instance        m x n, exactly `per_col` nonzeros per column at distinct
                       uniform rows, N(0,1) values, x* with `nnz_star` entries
                       +-U[1,2], b = A x* + N(0, noise^2), lambda = frac ||A^T b||_inf
  row_omega_instance   every row has exactly `omega` nonzeros at distinct uniform
                       columns (so the degree of partial separability is omega
                       exactly), N(0,1) values, x* `density`-dense +-U[1,2]
  per_col_instance     like tiny_instance at scale, with a density for x*

Values are stored in one of three dtypes: float64, float32 (round to nearest
even) or bfloat16 (round to nearest even directly from float64, kept as uint16
bit patterns).  `val64` always holds the stored values promoted exactly to
float64, and b is built from the stored values, so the instance is the stored A.
"""
from dataclasses import dataclass, field

import numpy as np

VAL_DTYPES = ("f64", "f32", "bf16")


@dataclass
class Instance:
    m: int
    n: int
    col_ptr: np.ndarray          # int64[n+1]
    row_idx: np.ndarray          # int32[nnz], ascending within each column
    val: np.ndarray              # stored values: float64, float32 or uint16 (bf16 bits)
    val_dtype: str               # "f64" | "f32" | "bf16"
    val64: np.ndarray            # stored values promoted exactly to float64
    b: np.ndarray                # float64[m]
    lam: float
    x_star: np.ndarray           # float64[n], the planted vector
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.col_ptr[-1])


def bf16_round(x):
    """Round float64 values to bfloat16 with round-to-nearest-even in one step
    (no detour through float32).  Returns (uint16 bit patterns, float64 values).
    Inputs must be finite and either zero or of magnitude >= 2**-126."""
    x = np.asarray(x, dtype=np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("non-finite value")
    ax = np.abs(x)
    if np.any((ax > 0) & (ax < 2.0 ** -126)):
        raise ValueError("value below the bfloat16 normal range")
    mant, expo = np.frexp(x)                 # x = mant * 2**expo, 0.5 <= |mant| < 1
    q = np.rint(mant * 256.0)                # 8 significant bits, ties to even (exact scaling)
    y = np.ldexp(q, expo - 8)                # exact in float64, 8 significant bits
    if np.any(np.abs(y) > 3.3895313892515355e38):
        raise ValueError("value above the bfloat16 range")
    f32 = y.astype(np.float32)               # exact: 8 significant bits fit in float32
    bits = (f32.view(np.uint32) >> 16).astype(np.uint16)
    return bits, y


def bf16_bits_to_f64(bits):
    bits = np.asarray(bits, dtype=np.uint16)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _store(val, val_dtype):
    if val_dtype == "f64":
        v = np.ascontiguousarray(val, dtype=np.float64)
        return v, v
    if val_dtype == "f32":
        v = np.ascontiguousarray(val, dtype=np.float32)
        return v, v.astype(np.float64)
    if val_dtype == "bf16":
        bits, v64 = bf16_round(val)
        return bits, v64
    raise ValueError(val_dtype)


def _distinct_rows(rng, count, width, high):
    """`count` sorted rows of `width` distinct integers drawn uniformly from [0, high)."""
    if width > high:
        raise ValueError("cannot draw %d distinct values from [0, %d)" % (width, high))
    idx = np.sort(rng.integers(0, high, size=(count, width), dtype=np.int64), axis=1)
    while True:
        if width < 2:
            break
        bad = np.nonzero(np.any(idx[:, 1:] == idx[:, :-1], axis=1))[0]
        if bad.size == 0:
            break
        idx[bad] = np.sort(rng.integers(0, high, size=(bad.size, width), dtype=np.int64), axis=1)
    return idx


def _planted(rng, n, count):
    x = np.zeros(n)
    count = int(min(max(count, 0), n))
    if count:
        where = rng.choice(n, size=count, replace=False)
        x[where] = rng.uniform(1.0, 2.0, size=count) * rng.choice([-1.0, 1.0], size=count)
    return x


def _finish(rng, m, n, col_ptr, row_idx, cols_of_entries, val, val_dtype, x_star, noise, lam_frac, meta):
    stored, val64 = _store(val, val_dtype)
    rows = row_idx.astype(np.int64)
    b = np.bincount(rows, weights=val64 * x_star[cols_of_entries], minlength=m)
    if noise > 0:
        b = b + rng.normal(0.0, noise, size=m)
    atb = np.bincount(cols_of_entries, weights=val64 * b[rows], minlength=n)
    lam = float(lam_frac * np.max(np.abs(atb))) if atb.size else 0.0
    return Instance(m=m, n=n, col_ptr=col_ptr, row_idx=row_idx.astype(np.int32), val=stored,
                    val_dtype=val_dtype, val64=val64, b=np.ascontiguousarray(b, dtype=np.float64),
                    lam=lam, x_star=x_star, meta=meta)


def per_col_instance(m, n, per_col, nnz_star=None, density=None, noise=0.01, lam_frac=0.1,
                     val_dtype="f64", seed=1001):
    """Exactly `per_col` nonzeros per column at distinct uniform rows, N(0,1) values."""
    rng = np.random.default_rng(seed)
    rows = _distinct_rows(rng, n, per_col, m)                       # (n, per_col), sorted per column
    col_ptr = np.arange(n + 1, dtype=np.int64) * per_col
    row_idx = rows.reshape(-1)
    cols = np.repeat(np.arange(n, dtype=np.int64), per_col)
    val = rng.standard_normal(n * per_col)
    if nnz_star is None:
        nnz_star = int(round((density or 0.0) * n))
    x_star = _planted(rng, n, nnz_star)
    meta = dict(kind="per_col", per_col=per_col, seed=seed, noise=noise, lam_frac=lam_frac)
    return _finish(rng, m, n, col_ptr, row_idx, cols, val, val_dtype, x_star, noise, lam_frac, meta)


def tiny_instance(val_dtype="f64", seed=1001):
    """A is 2000 x 1000 with exactly 10 nonzeros per column; x* has 50 nonzeros;
    b = A x* + N(0, 0.01^2); lambda = 0.1 ||A^T b||_inf."""
    return per_col_instance(2000, 1000, 10, nnz_star=50, noise=0.01, lam_frac=0.1,
                            val_dtype=val_dtype, seed=seed)


def row_omega_instance(m, n, omega, density=0.01, noise=0.01, lam_frac=0.05, val_dtype="f64",
                       seed=1002):
    """Every row has exactly `omega` nonzeros at distinct uniform columns (so the
    degree of partial separability is exactly omega); column counts are then
    about Poisson(m*omega/n).  Defaults follow the square scale workload:
    x* 1%-dense +-U[1,2], noise standard deviation 1e-2, lambda = 0.05 ||A^T b||_inf."""
    rng = np.random.default_rng(seed)
    cols = _distinct_rows(rng, m, omega, n)                        # (m, omega) distinct columns per row
    # CSC order = sort by (column, row): pack both into one int64 key and sort in place
    key = cols.reshape(-1)
    key <<= 32
    key |= np.repeat(np.arange(m, dtype=np.int64), omega)
    del cols
    key.sort()
    cols_sorted = key >> 32
    row_idx = (key & 0xFFFFFFFF).astype(np.int32)
    del key
    counts = np.bincount(cols_sorted, minlength=n)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    # values are i.i.d. and independent of the pattern: draw them in storage order
    val = rng.standard_normal(m * omega)
    x_star = _planted(rng, n, int(round(density * n)))
    meta = dict(kind="row_omega", omega=omega, seed=seed, noise=noise, lam_frac=lam_frac)
    return _finish(rng, m, n, col_ptr, row_idx, cols_sorted, val, val_dtype, x_star, noise, lam_frac, meta)


def from_dense(Adense, b, lam, val_dtype="f64"):
    """CSC instance from a small dense matrix (tests and examples)."""
    Adense = np.asarray(Adense, dtype=np.float64)
    m, n = Adense.shape
    col_ptr = [0]
    rows, vals, cols = [], [], []
    for i in range(n):
        nz = np.nonzero(Adense[:, i])[0]
        rows.extend(nz.tolist())
        vals.extend(Adense[nz, i].tolist())
        cols.extend([i] * len(nz))
        col_ptr.append(len(rows))
    stored, val64 = _store(np.array(vals, dtype=np.float64), val_dtype)
    return Instance(m=m, n=n, col_ptr=np.array(col_ptr, dtype=np.int64),
                    row_idx=np.array(rows, dtype=np.int32), val=stored, val_dtype=val_dtype,
                    val64=val64, b=np.ascontiguousarray(b, dtype=np.float64), lam=float(lam),
                    x_star=np.zeros(n), meta=dict(kind="dense"))


def dense(inst: Instance):
    """Dense float64 copy of the stored A (small instances only)."""
    A = np.zeros((inst.m, inst.n))
    for i in range(inst.n):
        s, e = inst.col_ptr[i], inst.col_ptr[i + 1]
        A[inst.row_idx[s:e], i] = inst.val64[s:e]
    return A


def multi_rhs(inst, nrhs, density=0.005, noise=0.01, seed=1004):
    """nrhs right-hand sides on inst's matrix (its stored values): b_l = A x*_l +
    N(0, noise^2), x*_l `density`-dense with +-U[1,2] entries.  Returns
    (B of shape (nrhs, m), the nrhs values lambda_max,l = ||A^T b_l||_inf)."""
    rng = np.random.default_rng(seed)
    cols = np.repeat(np.arange(inst.n, dtype=np.int64), np.diff(inst.col_ptr))
    rows = inst.row_idx.astype(np.int64)
    B = np.empty((nrhs, inst.m))
    lam_max = []
    for l in range(nrhs):
        xs = _planted(rng, inst.n, int(round(density * inst.n)))
        b = np.bincount(rows, weights=inst.val64 * xs[cols], minlength=inst.m)
        if noise > 0:
            b = b + rng.normal(0.0, noise, size=inst.m)
        B[l] = b
        atb = np.bincount(cols, weights=inst.val64 * b[rows], minlength=inst.n)
        lam_max.append(float(np.max(np.abs(atb))))
    return B, lam_max


def batched_path_instance(m=4_000_000, n=2_000_000, per_col=15, nrhs=16, val_dtype="bf16", seed=1003):
    """The batched regularisation-path workload: A is m x n with `per_col` N(0,1)
    nonzeros per column at distinct uniform rows (stored as val_dtype), and nrhs
    right-hand sides b_l = A x*_l + N(0, 1e-4), x*_l 0.5%-dense +-U[1,2].
    Returns (inst, B, lambda_max)."""
    inst = per_col_instance(m, n, per_col, density=0.005, noise=0.01, lam_frac=0.1, val_dtype=val_dtype, seed=seed)
    B, lam_max = multi_rhs(inst, nrhs, density=0.005, noise=0.01, seed=seed + 1)
    return inst, B, lam_max


def equal_rows_instance(m=3000, n=1000, omega=5, seed=1006):
    """The theory-versus-reality matrix (Sec. 8.2): every row has exactly omega
    nonzeros, all equal to 1, at distinct uniform columns (the 0-1 construction
    for which the DSO bound is tight, Sec. 5.1); b ~ N(0, 1); lambda = 0
    (least squares).  Returns an Instance with lam = 0 and x_star = 0."""
    rng = np.random.default_rng(seed)
    cols = _distinct_rows(rng, m, omega, n)
    key = cols.reshape(-1)
    key <<= 32
    key |= np.repeat(np.arange(m, dtype=np.int64), omega)
    key.sort()
    cols_sorted = key >> 32
    row_idx = (key & 0xFFFFFFFF).astype(np.int32)
    counts = np.bincount(cols_sorted, minlength=n)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    val = np.ones(row_idx.size)
    b = rng.standard_normal(m)
    meta = dict(kind="equal_rows", omega=omega, seed=seed)
    return Instance(m=m, n=n, col_ptr=col_ptr, row_idx=row_idx, val=val, val_dtype="f64", val64=val.copy(),
                    b=b, lam=0.0, x_star=np.zeros(n), meta=meta)


def small_instances(count=256, lo=1_000, hi=100_000, per_col=8, val_dtype="bf16", seed=1007):
    """The batch of independent small problems: n log-uniform in [lo, hi], m = 2n,
    `per_col` N(0,1) nonzeros per column, x* 1% dense, noise variance 1e-4,
    lambda = 0.1 ||A^T b||_inf (one per_col_instance per problem)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    return [per_col_instance(2 * int(n), int(n), per_col, density=0.01, noise=0.01, lam_frac=0.1,
                             val_dtype=val_dtype, seed=seed + 1 + q) for q, n in enumerate(ns)]


# ----------------------------------------------------------------------------- labelled data
@dataclass
class LabeledInstance:
    """A sparse data matrix with +-1 labels, for the SVM dual (labels on the
    columns: one per example) and for logistic regression (labels on the rows)."""
    m: int
    n: int
    col_ptr: np.ndarray          # int64[n+1]
    row_idx: np.ndarray          # int32[nnz], ascending within each column
    val: np.ndarray              # stored values: float64, float32 or uint16 (bf16 bits)
    val_dtype: str
    val64: np.ndarray            # stored values promoted exactly to float64
    y: np.ndarray                # float64 labels in {-1, +1}: n of them (SVM) or m (logistic)
    lam: float
    problem: str                 # "svm_dual" | "logistic"
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.col_ptr[-1])


def svm_instance(d, n, per_example, lam, zipf=0.0, label_noise=0.05, val_dtype="f64", seed=1008):
    """Data for the dual of the L2-regularised hinge-loss SVM (Sec. 8.3).

    A is d x n: column i is example i.  Each example draws `per_example`
    features with replacement, with feature r drawn with probability proportional
    to (r + 1)^-zipf (zipf = 0: uniform); repeats are dropped, so an example has
    at most `per_example` distinct features.  A large zipf makes a few features
    common to many examples, which is what gives rcv1 its large omega.  Values
    are |N(0,1)| scaled to unit norm per example (tf-idf-like, nonnegative).
    Labels: y_i = sign(<w*, A_i>) with w* ~ N(0, I_d), each flipped with
    probability label_noise."""
    rng = np.random.default_rng(seed)
    if zipf > 0:
        cdf = np.cumsum((np.arange(d) + 1.0) ** -float(zipf))
        cdf /= cdf[-1]
        draws = np.minimum(np.searchsorted(cdf, rng.random((n, per_example)), side="right"), d - 1)
    else:
        draws = rng.integers(0, d, size=(n, per_example))
    draws.sort(axis=1)
    keep = np.ones(draws.shape, dtype=bool)
    keep[:, 1:] = draws[:, 1:] != draws[:, :-1]
    counts = keep.sum(axis=1)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    row_idx = draws[keep].astype(np.int32)
    del draws, keep
    cols = np.repeat(np.arange(n, dtype=np.int64), counts)
    val = np.abs(rng.standard_normal(row_idx.size))
    norms = np.sqrt(np.bincount(cols, weights=val * val, minlength=n))
    val /= norms[cols]
    stored, val64 = _store(val, val_dtype)
    w = rng.standard_normal(d)
    score = np.bincount(cols, weights=val64 * w[row_idx], minlength=n)
    y = np.where(score >= 0.0, 1.0, -1.0)
    flip = rng.random(n) < label_noise
    y[flip] = -y[flip]
    meta = dict(kind="svm", per_example=per_example, zipf=zipf, label_noise=label_noise, seed=seed)
    return LabeledInstance(m=d, n=n, col_ptr=col_ptr, row_idx=row_idx, val=stored, val_dtype=val_dtype,
                           val64=val64, y=y, lam=float(lam), problem="svm_dual", meta=meta)


def logistic_instance(m, n, per_row, lam=1.0, val_dtype="f64", seed=1009):
    """Data for L2-regularised logistic regression (Sec. 8.4).

    A is m x n: row j is example j, with exactly `per_row` distinct features at
    uniform columns (so omega = per_row exactly, as the paper stresses for
    KDDB), N(0,1)/sqrt(per_row) values.  Labels: y_j = +1 with probability
    1/(1 + exp(-A_j^T x*)), x* ~ N(0, I_n), else -1."""
    rng = np.random.default_rng(seed)
    cols = _distinct_rows(rng, m, per_row, n)
    key = cols.reshape(-1)
    key <<= 32
    key |= np.repeat(np.arange(m, dtype=np.int64), per_row)
    del cols
    key.sort()
    cols_sorted = key >> 32
    row_idx = (key & 0xFFFFFFFF).astype(np.int32)
    del key
    counts = np.bincount(cols_sorted, minlength=n)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    val = rng.standard_normal(row_idx.size) / np.sqrt(per_row)
    stored, val64 = _store(val, val_dtype)
    x_star = rng.standard_normal(n)
    margin = np.bincount(row_idx.astype(np.int64), weights=val64 * x_star[cols_sorted], minlength=m)
    y = np.where(rng.random(m) < 1.0 / (1.0 + np.exp(-margin)), 1.0, -1.0)
    meta = dict(kind="logistic", per_row=per_row, seed=seed)
    return LabeledInstance(m=m, n=n, col_ptr=col_ptr, row_idx=row_idx, val=stored, val_dtype=val_dtype,
                           val64=val64, y=y, lam=float(lam), problem="logistic", meta=meta)


def labeled_from_dense(Adense, y, lam, problem, val_dtype="f64"):
    """LabeledInstance from a small dense matrix (tests)."""
    inst = from_dense(Adense, np.zeros(np.asarray(Adense).shape[0]), lam, val_dtype)
    return LabeledInstance(m=inst.m, n=inst.n, col_ptr=inst.col_ptr, row_idx=inst.row_idx, val=inst.val,
                           val_dtype=val_dtype, val64=inst.val64, y=np.asarray(y, dtype=np.float64),
                           lam=float(lam), problem=problem, meta=dict(kind="dense"))

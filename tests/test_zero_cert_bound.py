"""The error bound of the FP32 zero-step certificate, restated exactly on the CPU.

The FP64 forms of the pipelined and warp-cooperative kernels may decide a
LASSO step at x_i = 0 without FP64 work: they sum FP32 images of the operands
(made from their high words with integer operations) and certify
|a_i^T g| <= lambda when

    |acc32| + (c + 40) 2^-24 sabs32 + c 2^-123 mx + 2^-120  <=  lambda rounded down to FP32,

the left side rounded upwards (acc32, sabs32: FP32 FMA sums of v g and |v||g|;
mx: the largest image magnitude; c <= 1024 products).  This test restates that
arithmetic with exact rationals and correctly rounded FP32 operations, and
checks on random and adversarial columns that a certificate is only ever
issued when the FP64 sum the kernel would otherwise compute (in any order, with
or without FMA) is at most lambda in magnitude: the only property the kernels
rely on.  The warp-cooperative kernel sums in another order (per lane, then a
five-level tree) and takes the bound with c + 5 for c: certify_warp restates
it.  The GPU side of the same claim is tests/test_gpu_zero_cert.py.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

U32 = 0xFFFFFFFF


def hi_word(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0] >> 32


def f32_image(hi):
    """The kernel's image: sign, exponent and 20 mantissa bits of the double whose
    high word is hi, magnitude clamped to [2^-126, inf]."""
    m = min(max(hi & 0x7FFFFFFF, 0x38100000), 0x47F00000)
    bits = (((m - 0x38000000) << 3) & U32) | (hi & 0x80000000)
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def round_f32(q, up=False):
    """Fraction -> the nearest FP32 value (ties to even), or the smallest FP32
    value >= q when up; inf beyond the largest finite value."""
    if q == 0:
        return 0.0
    neg = q < 0
    a = -q if neg else q
    # exponent e with 2^e <= a < 2^(e+1)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                                  # subnormals share the exponent -126
    scale = Fraction(2) ** (23 - e)                   # 24 significant bits (fewer below 2^-126)
    t = a * scale
    n, r = divmod(t.numerator, t.denominator)
    rem = Fraction(r, t.denominator)
    if up:
        if (rem > 0) and not neg:
            n += 1
    else:
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
            n += 1
    val = Fraction(n) / scale
    if val > Fraction((2 ** 24 - 1) * 2 ** 104):
        return -math.inf if neg else math.inf
    f = float(val)
    return -f if neg else f


def fma32(a, b, c, up=False):
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        return a * b + c                              # inf or NaN, as the hardware gives
    return round_f32(Fraction(a) * Fraction(b) + Fraction(c), up)


def certify(v, g, lam):
    """The kernel's ZeroCert: True when the bound shows |FP64 sum| <= lambda."""
    c = len(v)
    if c > 1024:
        return False
    acc = sabs = mx = 0.0
    for vv, gg in zip(v, g):
        vi, gi = f32_image(hi_word(vv)), f32_image(hi_word(gg))
        acc = fma32(vi, gi, acc)
        sabs = fma32(abs(vi), abs(gi), sabs)
        mx = max(mx, abs(vi), abs(gi))
    if any(math.isnan(t) or math.isinf(t) for t in (acc, sabs, mx)):
        return False
    lamf = round_f32(Fraction(lam))                   # then rounded down
    if math.isinf(lamf) or Fraction(lamf) > Fraction(lam):
        lamf = float(np.nextafter(np.float32(lamf), np.float32(0)))
    lhs = round_f32(Fraction(abs(acc)) + Fraction(2) ** -120, up=True)
    lhs = fma32(mx, c * 2.0 ** -123, lhs, up=True)
    lhs = fma32(sabs, (c + 40) * 2.0 ** -24, lhs, up=True)
    return lhs <= lamf


def fp64_sums(v, g):
    """FP64 sums the kernel may form: sequential without FMA (two roundings per
    term), sequential in reverse, and in chunks of 16 added together."""
    s1 = 0.0
    for a, b in zip(v, g):
        s1 = s1 + a * b
    s2 = 0.0
    for a, b in zip(reversed(v), reversed(g)):
        s2 = s2 + a * b
    s3 = 0.0
    for k in range(0, len(v), 16):
        part = 0.0
        for a, b in zip(v[k:k + 16], g[k:k + 16]):
            part = part + a * b
        s3 = s3 + part
    return s1, s2, s3


def _column(rng, c, kind):
    sgn = lambda n: np.where(rng.random(n) < 0.5, -1.0, 1.0)
    if kind == "normal":
        v, g = rng.standard_normal(c), rng.standard_normal(c)
    elif kind == "spread":                            # exponents over a wide range
        v = sgn(c) * 2.0 ** rng.uniform(-60, 60, c)
        g = sgn(c) * 2.0 ** rng.uniform(-60, 60, c)
    elif kind == "cancel":                            # large terms that cancel to a small sum
        base = rng.standard_normal(c // 2 + 1) * 1e3
        v = np.concatenate([base, -base])[:c] * (1 + 1e-9 * rng.standard_normal(c))
        g = np.ones(c) + 2.0 ** -30 * rng.standard_normal(c)
    elif kind == "tiny":                              # below the FP32 normal range
        v = sgn(c) * 2.0 ** rng.uniform(-160, -120, c)
        g = sgn(c) * 2.0 ** rng.uniform(-10, 10, c)
    elif kind == "huge":                              # beyond the FP32 range (images inf)
        v = sgn(c) * 2.0 ** rng.uniform(129, 140, c)
        g = sgn(c) * 2.0 ** rng.uniform(-10, 10, c)
    elif kind == "lowbits":                           # low mantissa bits the images drop
        v = sgn(c) * (1.0 + 2.0 ** -21 + 2.0 ** -40)
        g = sgn(c) * (1.0 + 2.0 ** -22 + 2.0 ** -45)
    else:
        raise ValueError(kind)
    return [float(x) for x in v], [float(x) for x in g]


@pytest.mark.parametrize("kind", ["normal", "spread", "cancel", "tiny", "huge", "lowbits"])
def test_certificate_only_when_the_fp64_sum_is_within_lambda(kind):
    rng = np.random.default_rng(hash(kind) % (2 ** 32))
    issued = 0
    for trial in range(120):
        c = int(rng.choice([1, 2, 3, 7, 16, 17, 24, 31, 48, 64]))
        v, g = _column(rng, c, kind)
        D = math.fsum(float(Fraction(a) * Fraction(b)) for a, b in zip(v, g))
        base = abs(D) if D != 0 else 2.0 ** -100
        # lambda just above, at, and just below |D|, and far above it
        for rel in (-2.0 ** -10, -2.0 ** -20, -2.0 ** -40, 0.0, 2.0 ** -40, 2.0 ** -20, 2.0 ** -10, 1.0):
            lam = base * (1.0 + rel)
            if not (lam > 0 and math.isfinite(lam)):
                continue
            if certify(v, g, lam):
                issued += 1
                for s in fp64_sums(v, g):
                    assert abs(s) <= lam, (kind, c, rel, s, lam)
    if kind in ("normal", "lowbits", "spread"):
        assert issued > 0          # the certificate is not vacuous on ordinary columns
    if kind == "huge":
        assert issued == 0         # images beyond the FP32 range never certify


def test_images_and_rounding_helpers():
    # the image keeps sign, exponent and 20 mantissa bits, clamps below 2^-126
    assert f32_image(hi_word(1.0)) == 1.0
    assert f32_image(hi_word(-3.5)) == -3.5
    assert f32_image(hi_word(1.0 + 2.0 ** -21)) == 1.0          # bit 21 is dropped
    assert f32_image(hi_word(1.0 + 2.0 ** -20)) == 1.0 + 2.0 ** -20
    assert f32_image(hi_word(0.0)) == 2.0 ** -126
    assert f32_image(hi_word(2.0 ** -140)) == 2.0 ** -126
    assert math.isinf(f32_image(hi_word(2.0 ** 130)))
    assert math.isinf(f32_image(hi_word(float("nan"))))
    # correctly rounded FP32 against numpy on random values (nearest-even)
    rng = np.random.default_rng(5)
    for x in rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200):
        assert round_f32(Fraction(float(x))) == float(np.float32(x))
    assert round_f32(Fraction(1) + Fraction(1, 2 ** 30), up=True) == float(np.nextafter(np.float32(1), np.float32(2)))


def certify_warp(v, g, lam):
    """The warp-cooperative kernel's certificate: lane l sums the products of
    entries 64r + 2l and 64r + 2l + 1 (r = 0, 1, ...) with FP32 FMAs in that
    order, the 32 lane sums are added by the five levels of the warp reduction
    (partners at distance 16, 8, 4, 2, 1), the maxima likewise, and the bound
    is taken with c + 5 in place of c."""
    c = len(v)
    if c + 5 > 1024:
        return False
    acc, sabs, mx = [0.0] * 32, [0.0] * 32, [0.0] * 32
    for e in range(c):
        l = (e % 64) // 2
        vi, gi = f32_image(hi_word(v[e])), f32_image(hi_word(g[e]))
        acc[l] = fma32(vi, gi, acc[l])
        sabs[l] = fma32(abs(vi), abs(gi), sabs[l])
        mx[l] = max(mx[l], abs(vi), abs(gi))
    for d in (16, 8, 4, 2, 1):
        acc = [fma32(1.0, acc[l], acc[l ^ d]) for l in range(32)]
        sabs = [fma32(1.0, sabs[l], sabs[l ^ d]) for l in range(32)]
        mx = [max(mx[l], mx[l ^ d]) for l in range(32)]
    acc, sabs, mx = acc[0], sabs[0], mx[0]
    if any(math.isnan(t) or math.isinf(t) for t in (acc, sabs, mx)):
        return False
    lamf = round_f32(Fraction(lam))
    if math.isinf(lamf) or Fraction(lamf) > Fraction(lam):
        lamf = float(np.nextafter(np.float32(lamf), np.float32(0)))
    cc = c + 5
    lhs = round_f32(Fraction(abs(acc)) + Fraction(2) ** -120, up=True)
    lhs = fma32(mx, cc * 2.0 ** -123, lhs, up=True)
    lhs = fma32(sabs, (cc + 40) * 2.0 ** -24, lhs, up=True)
    return lhs <= lamf


def fp64_warp_sum(v, g):
    """The FP64 sum the warp-cooperative kernel falls back to: lane l takes the
    entries l, l + 32, ... with FMAs, then the five-level reduction."""
    acc = [0.0] * 32
    for e, (a, b) in enumerate(zip(v, g)):
        acc[e % 32] = float(Fraction(a) * Fraction(b) + Fraction(acc[e % 32]))
    for d in (16, 8, 4, 2, 1):
        acc = [acc[l] + acc[l ^ d] for l in range(32)]
    return acc[0]


@pytest.mark.parametrize("kind", ["normal", "spread", "cancel", "tiny", "huge", "lowbits"])
def test_warp_order_certificate_only_when_the_fp64_sum_is_within_lambda(kind):
    # columns up to a few hundred entries: several products per lane, then the tree
    rng = np.random.default_rng((hash(kind) + 7) % (2 ** 32))
    issued = 0
    for trial in range(40):
        c = int(rng.choice([1, 3, 31, 32, 33, 64, 100, 128, 150, 300]))
        v, g = _column(rng, c, kind)
        D = math.fsum(float(Fraction(a) * Fraction(b)) for a, b in zip(v, g))
        base = abs(D) if D != 0 else 2.0 ** -100
        for rel in (-2.0 ** -10, -2.0 ** -20, 0.0, 2.0 ** -20, 2.0 ** -10, 1.0):
            lam = base * (1.0 + rel)
            if not (lam > 0 and math.isfinite(lam)):
                continue
            if certify_warp(v, g, lam):
                issued += 1
                for s in list(fp64_sums(v, g)) + [fp64_warp_sum(v, g)]:
                    assert abs(s) <= lam, (kind, c, rel, s, lam)
    if kind in ("normal", "lowbits", "spread"):
        assert issued > 0
    if kind == "huge":
        assert issued == 0

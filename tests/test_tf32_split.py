"""The operand split of the tensor-core tiles, checked on the CPU.

The tiles hand the tensor core u = hi + lo with hi = u rounded to TF32 (10
explicit mantissa bits, nearest, ties away from zero) by integer arithmetic
on the bits, (bits + 0x1000) & 0xFFFFE000, and lo = u - hi in FP32, unrounded.
The MMA uses the leading 19 bits of each operand.  Here, in numpy FP32:

* the integer form equals exact rounding to nearest, ties away, for every
  finite input tried (random bit patterns, ties, mantissa carries into the
  exponent, subnormals);
* lo = u - hi is exact (hi + lo == u, and the FP32 subtraction loses nothing);
* keeping only the leading 19 bits of hi and lo (truncation) represents u to
  2^-21 relative, the bound the design relies on.
"""
from fractions import Fraction

import numpy as np


def tf32_int(x):
    b = x.view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def trunc19(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def rna_exact(v):
    """v (a finite float32, as Python float) rounded to 10 explicit mantissa
    bits, nearest, ties away from zero, with float32's exponent range."""
    if v == 0.0:
        return 0.0
    f = Fraction(v)
    sign = -1 if f < 0 else 1
    f = abs(f)
    e = f.numerator.bit_length() - f.denominator.bit_length()
    if Fraction(2) ** e > f:
        e -= 1
    e = max(e, -126)                        # subnormals share the smallest exponent
    q = Fraction(2) ** (e - 10)             # spacing of 10-bit mantissas at this exponent
    n = f / q
    r = int(n) + (1 if n - int(n) >= Fraction(1, 2) else 0)
    return sign * float(r * q)


def _samples():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < np.float32(3e38))]
    ties = ((rng.integers(0, 2 ** 19, 2000, dtype=np.uint64).astype(np.uint32) << np.uint32(13))
            | np.uint32(0x1000)).view(np.float32)                       # exactly half-way cases
    carries = (np.uint32(0x3F800000) | np.uint32(0x7FF000)).reshape(1).view(np.float32)   # rounds up into 2.0
    sub = (rng.integers(1, 2 ** 23, 2000, dtype=np.uint64).astype(np.uint32)).view(np.float32)
    return np.concatenate([x, ties[np.isfinite(ties)], -ties[np.isfinite(ties)], carries, sub, -sub])


def test_integer_rounding_is_nearest_ties_away():
    x = _samples()
    hi = tf32_int(x)
    pick = np.random.default_rng(3).choice(len(x), 20_000, replace=False)
    for v, h in zip(x[pick], hi[pick]):
        assert float(h) == rna_exact(float(v)), (float(v), float(h))
    c = np.float32(np.uint32(0x3FFFF000).view(np.float32))     # 1.999..., mantissa all ones above the tie
    assert float(tf32_int(np.array([c]))[0]) == 2.0


def test_low_part_is_exact_and_pair_is_within_2_to_minus_21():
    x = _samples()
    x = x[(x != 0) & (np.abs(x) > np.float32(1e-30))]          # away from subnormal results
    hi = tf32_int(x)
    lo = (x - hi).astype(np.float32)
    # exact: the FP32 difference equals the real difference
    assert np.all(hi.astype(np.float64) + lo.astype(np.float64) == x.astype(np.float64))
    # what the MMA sees when it keeps 19 leading bits of each part
    seen = trunc19(hi).astype(np.float64) + trunc19(lo).astype(np.float64)
    rel = np.abs(seen - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -21, rel.max()

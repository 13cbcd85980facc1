"""The FP32 field-rotation arithmetic of the kernels, emulated on the CPU.

The rotation exp(-i mu E dt / hbar) turns each coherence pair (j, k) of the
dipole eigenbasis by theta_jk = (lambda_j - lambda_k) E dt / hbar (Sec. 2.2).
The kernels form sin theta and cos theta - 1 (never 1 - 1) by Taylor
polynomials to x^7 and x^8 while |theta| <= 1/2; larger angles go to the
library routine (per angle, or for a whole warp after a vote in the
two-level tiles), and the tensor-core tiles derive the pairs (j, k), j > 0,
from theta_0k and theta_0j by the angle-difference identities written in
sin and cos - 1.  In FP32 with fused multiply-adds (emulated: each fma
rounded once from exact float64 products):

* the polynomials hold sin x to 2 ulp and cos x - 1 to 3 ulp of the result
  on |x| <= 1/2 (the omitted terms are below half an ulp there), and fail
  beyond |x| ~ 1, which is what the guards are for;
* the identities reproduce sin and cos - 1 of the difference to 3 x 2^-24
  absolute, the order of rounding the difference angle itself in FP32
  (the rotation's entries are of order 1), and a wrong sign in either
  would fail by far.
"""
import numpy as np

f32 = np.float32


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def taylor_half(x):
    x = f32(x)
    t = f32(x * x)
    ps = fma(t, f32(-1.0 / 5040.0), f32(1.0 / 120.0))
    ps = fma(t, ps, f32(-1.0 / 6.0))
    ps = fma(t, ps, f32(1.0))
    s = f32(x * ps)
    pc = fma(t, f32(1.0 / 40320.0), f32(-1.0 / 720.0))
    pc = fma(t, pc, f32(1.0 / 24.0))
    pc = fma(t, pc, f32(-0.5))
    return s, f32(t * pc)


def ulp(v):
    return np.spacing(np.abs(f32(v))).astype(np.float64)


def cosm1(x):
    return -2.0 * np.sin(x / 2.0) ** 2


def test_angle_difference_identities():
    rng = np.random.default_rng(9)
    worst_s, worst_c = 0.0, 0.0
    for _ in range(5_000):
        a, b = rng.uniform(-0.5, 0.5, 2).astype(np.float32)   # theta_0k, theta_0j
        sk, ck = taylor_half(a)   # the tensor-core tiles' polynomials
        sj, cj = taylor_half(b)
        sv = f32(f32(sk - sj) + fma(sk, cj, -f32(ck * sj)))
        mv = fma(ck, cj, fma(sk, sj, f32(ck + cj)))
        d = np.float64(a) - np.float64(b)
        worst_s = max(worst_s, abs(np.float64(sv) - np.sin(d)))
        worst_c = max(worst_c, abs(np.float64(mv) - cosm1(d)))
    assert worst_s <= 3 * 2.0 ** -24, worst_s
    assert worst_c <= 3 * 2.0 ** -24, worst_c


def test_short_polynomials_on_half_the_range():
    rng = np.random.default_rng(6)
    xs = np.concatenate([rng.uniform(-0.5, 0.5, 20_000), np.geomspace(1e-12, 0.5, 2_000),
                         -np.geomspace(1e-12, 0.5, 2_000), [0.5, -0.5]]).astype(np.float32)
    es, ec = 0.0, 0.0
    for x in xs:
        s, c = taylor_half(x)
        xd = np.float64(x)
        es = max(es, abs(np.float64(s) - np.sin(xd)) / ulp(np.sin(xd)))
        if xd != 0.0:
            ec = max(ec, abs(np.float64(c) - cosm1(xd)) / ulp(cosm1(xd)))
    assert es <= 2.0, es
    assert ec <= 3.0, ec
    s1, c1 = taylor_half(1.0)   # beyond the vote's range the shorter series fails
    assert abs(np.float64(s1) - np.sin(1.0)) / ulp(np.sin(1.0)) > 10

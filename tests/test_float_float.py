"""The float-float field and Kahan state arithmetic of the FP32 kernels,
emulated on the CPU.

FP32 fields are unevaluated pairs hi + lo of floats.  The update
f += c (xr - xl) + extra takes the neighbour difference with TwoSum, the
product with TwoProd (one fused multiply-add), and adds into the pair either
renormalised or lazily (hi takes the rounded sum of the high words, lo
collects the exact rounding error and the low terms; the tiles renormalise
once per launch).  In numpy FP32 (fused multiply-adds emulated by one
rounding of the exact float64 result):

* TwoSum and TwoProd are error-free: s + e == a + b and p + e == a * b exactly;
* a long run of updates, lazily accumulated and renormalised every 24
  steps, stays within 1e-9 of the same recurrence in FP64 (measured 3.5e-11
  over 6,000 steps: the low word itself collects the small terms between
  renormalisations and rounds at their scale), where a single FP32 word
  drifts by more than 1e-7;
* the tiles' per-step form (one subtraction for the neighbour difference,
  Fast2Sum for the accumulation, both exact away from zero crossings) carries
  a 1D Yee pulse 6,000 steps within 2e-7 of FP64, where one FP32 word per
  field drifts past 1e-5;
* the blocked accumulation of the two-level tiles (a tile's increments
  summed in one FP32 word, folded into the deviation by TwoSum at the tile's
  end) keeps increments below half an ulp of the deviation as Kahan does,
  and rounds larger ones against the block's partial sum: within 1 % of the
  worst-case bound (T + 1) 2^-24 sum |x|, 100 times below plain FP32.
"""
import numpy as np

f32 = np.float32


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def two_prod(a, b):
    p = f32(a * b)
    return p, fma(a, b, -p)


def axpy_diff(fh, fl, c, xrh, xrl, xlh, xll, extra, lazy):
    dh, de = two_sum(xrh, f32(-xlh))
    dl = f32(de + f32(xrl - xll))
    ph, pe = two_prod(c, dh)
    b = f32(fma(c, dl, pe) + extra)
    s, e = two_sum(fh, ph)
    if lazy:
        return s, f32(e + f32(fl + b))
    e = f32(e + f32(fl + b))
    h = f32(s + e)
    return h, f32(e - f32(h - s))


def renorm(h, l):
    s = f32(h + l)
    return s, f32(l - f32(s - h))


def test_two_sum_and_two_prod_are_exact():
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(20_000) * 10.0 ** rng.integers(-6, 7, 20_000)).astype(np.float32)
    b = (rng.standard_normal(20_000) * 10.0 ** rng.integers(-6, 7, 20_000)).astype(np.float32)
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        assert np.float64(s) + np.float64(e) == np.float64(x) + np.float64(y)
        p, q = two_prod(x, y)
        assert np.float64(p) + np.float64(q) == np.float64(x) * np.float64(y)


def test_lazy_float_float_tracks_fp64():
    rng = np.random.default_rng(2)
    n = 6_000
    c = f32(0.37)
    xr = rng.uniform(-1e9, 1e9, n)
    xl = rng.uniform(-1e9, 1e9, n)
    extra = rng.uniform(-1e3, 1e3, n)
    fh, fl = f32(1.3e9), f32(0.0)
    ref = np.float64(fh)
    single = f32(fh)
    worst, worst_single = 0.0, 0.0
    for k in range(n):
        xrh, xll = f32(xr[k]), f32(0.0)
        xlh = f32(xl[k])
        fh, fl = axpy_diff(fh, fl, c, xrh, f32(0.0), xlh, xll, f32(extra[k]), lazy=True)
        if (k + 1) % 24 == 0:
            fh, fl = renorm(fh, fl)
        ref += np.float64(c) * (np.float64(xrh) - np.float64(xlh)) + np.float64(f32(extra[k]))
        single = f32(single + f32(c * f32(xrh - xlh)) + f32(extra[k]))
        scale = max(abs(ref), 1e8)
        worst = max(worst, abs(np.float64(fh) + np.float64(fl) - ref) / scale)
        worst_single = max(worst_single, abs(np.float64(single) - ref) / scale)
    assert worst < 1e-9, worst
    assert worst_single > 1e-7                     # what a single FP32 word would lose


def kahan_add(d, c, x):
    y = f32(x - c)
    t = f32(d + y)
    return t, f32(f32(t - d) - y)


def test_kahan_keeps_increments_below_half_an_ulp():
    """A deviation of 0.5 receiving 200,000 increments of 1e-9 (a slow
    relaxation: each increment is below half an ulp of the value): plain FP32
    loses every one, the compensated sum (true value d - c) keeps them to
    1e-6 of their total."""
    d, c, plain = f32(0.5), f32(0.0), f32(0.5)
    inc = f32(1e-9)
    n = 200_000
    for _ in range(n):
        d, c = kahan_add(d, c, inc)
        plain = f32(plain + inc)
    total = n * np.float64(inc)
    assert plain == f32(0.5)                                    # stagnation
    assert abs((np.float64(d) - np.float64(c) - 0.5) - total) <= 1e-6 * total


def step_form(fh, fl, c, xrh, xrl, xlh, xll, extra):
    """The tiles' per-step update (vectorised): plain difference of the high
    words, TwoProd, Fast2Sum into the pair, low terms into the low word."""
    dh = (xrh - xlh).astype(f32)
    dl = (xrl - xll).astype(f32)
    ph = (c * dh).astype(f32)
    pe = (c.astype(np.float64) * dh.astype(np.float64) - ph.astype(np.float64)).astype(f32)
    s = (fh + ph).astype(f32)
    e = (ph - (s - fh).astype(f32)).astype(f32)
    b = (c.astype(np.float64) * dl.astype(np.float64) + (pe + extra).astype(f32).astype(np.float64)).astype(f32)
    return s, (e + (fl + b).astype(f32)).astype(f32)


def test_step_form_carries_a_pulse():
    nx, nt, C, kdz = 3000, 6000, 1.0 - 2.0 ** -13, 2.0 * np.pi / 128.0
    m = np.arange(nx, dtype=np.float64)
    env = lambda x: 1e9 * np.exp(-((x - 700.0) / 150.0) ** 2) * np.sin(kdz * x)
    E64, H64 = env(m), -env(m - 0.5 - C / 2.0)
    Eh, Hh = E64.astype(f32), H64.astype(f32)
    El = (E64 - Eh.astype(np.float64)).astype(f32)
    Hl = (H64 - Hh.astype(np.float64)).astype(f32)
    Es, Hs = Eh.copy(), Hh.copy()
    c = np.full(nx - 1, f32(C), f32)
    z = np.zeros(nx - 1, f32)
    for n in range(nt):
        H64[1:] += C * (E64[1:] - E64[:-1])
        E64[:-1] += C * (H64[1:] - H64[:-1])
        Hh[1:], Hl[1:] = step_form(Hh[1:], Hl[1:], c, Eh[1:], El[1:], Eh[:-1], El[:-1], z)
        Eh[:-1], El[:-1] = step_form(Eh[:-1], El[:-1], c, Hh[1:], Hl[1:], Hh[:-1], Hl[:-1], z)
        Hs[1:] = (Hs[1:] + c * (Es[1:] - Es[:-1]).astype(f32)).astype(f32)
        Es[:-1] = (Es[:-1] + c * (Hs[1:] - Hs[:-1]).astype(f32)).astype(f32)
        if (n + 1) % 24 == 0:
            for h, l in ((Eh, El), (Hh, Hl)):
                sm = (h + l).astype(f32)
                l[:] = (l - (sm - h).astype(f32)).astype(f32)
                h[:] = sm
    ref = np.linalg.norm(E64)
    err = np.linalg.norm(Eh.astype(np.float64) + El.astype(np.float64) - E64) / ref
    err_single = np.linalg.norm(Es.astype(np.float64) - E64) / ref
    assert err < 2e-7, err
    assert err_single > 1e-5, err_single


def blocked_run(d, c, incs, T):
    """The two-level tiles' blocked accumulation: acc = -c on load, one FP32
    addition per increment, TwoSum of (d, acc) at the end of every T steps;
    returns the Kahan pair (d, c), true value d - c."""
    acc = f32(-c)
    for k, x in enumerate(incs):
        acc = f32(acc + x)
        if (k + 1) % T == 0:
            d, acc = two_sum(d, acc)
    d, acc = two_sum(d, acc)
    return d, f32(-acc)


def test_blocked_accumulation_keeps_increments_below_half_an_ulp():
    """The slow-relaxation case of the Kahan test: 200,000 increments of 1e-9
    on a deviation of 0.5 survive the blocked sum too (each block's 32e-9
    folds into d exactly, its rounding stays in acc)."""
    n = 200_000
    d, c = blocked_run(f32(0.5), f32(0.0), [f32(1e-9)] * n, 32)
    total = n * np.float64(f32(1e-9))
    assert abs((np.float64(d) - np.float64(c) - 0.5) - total) <= 1e-6 * total


def test_blocked_accumulation_error_bound():
    """A pulse-like run of large increments of both signs plus a slow drift:
    the blocked sum (T = 32) lands within the worst-case bound (T + 1) 2^-24
    sum |x| of the exact sum, in practice within 1 % of it (measured 0.11 %,
    7.7e-9; Kahan 2.7e-10), and 100 times closer than plain FP32 (6.1e-6); a
    planted mistake (the fold dropping its rounding error) loses that."""
    T, n = 32, 20_000
    k = np.arange(n, dtype=np.float64)
    incs = (2e-3 * np.sin(k / 37.0) / np.cosh((k - 6000.0) / 900.0) + 3e-9).astype(f32)
    exact = 0.25 + incs.astype(np.float64).sum()
    d, c = blocked_run(f32(0.25), f32(0.0), list(incs), T)
    err = abs(np.float64(d) - np.float64(c) - exact)
    bound = (T + 1) * 2.0 ** -24 * np.abs(incs.astype(np.float64)).sum()
    assert err <= 1e-2 * bound, (err, bound)
    plain = f32(0.25)
    for x in incs:
        plain = f32(plain + x)
    assert err * 100 < abs(np.float64(plain) - exact), (err, plain)
    # planted: fold by plain addition (rounding of every fold lost)
    acc, dd = f32(0.0), f32(0.25)
    for i, x in enumerate(incs):
        acc = f32(acc + x)
        if (i + 1) % T == 0:
            dd, acc = f32(dd + acc), f32(0.0)
    assert abs(np.float64(f32(dd + acc)) - exact) > err * 20

"""Parity at the benchmark's full size (1,048,576 cells x 200,000 steps, the
jittered two-level medium), in the launch configuration bench.py times
(FP32, temporal tiles of 24 steps).

The oracle cannot run the whole grid, so the check has three parts:
  * sampled outputs the oracle computes exactly: nothing travels faster than
    one cell per step, so for the first S steps the cells [0, S + 8) evolve
    as in the full grid; the oracle runs that window and is compared with
    the full-size GPU traces at probes just inside the medium;
  * FP32 against FP64 on the GPU over the whole run, every probe;
  * the state invariants (trace, smallest eigenvalue) at the end.
"""
import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu

WINDOW_STEPS = 58_000
NEAR = (52_500, 54_000, 56_000)     # medium starts at cell 52,429


@pytest.fixture(scope="module")
def full_runs():
    from paper_2005_05412_gb300 import build
    build.build()
    p = W.sit_2lvl_jitter()
    extra = []
    for c in NEAR:
        extra += [W.Probe(c, W.Q_E), W.Probe(c, W.Q_RHO_RE, 0, 0)]
    p = p.replace(probes=p.probes + extra)
    out = {}
    for prec in ("fp32", "fp64"):
        out[prec] = mbs.run(p, precision=prec, algo="tiled", tile_steps=24)
    return p, out


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fullsize_fp32_vs_fp64(full_runs):
    p, out = full_runs
    a, b = out["fp32"]["records"], out["fp64"]["records"]
    assert a.shape == (len(p.probes), 200_000)
    for k, pr in enumerate(p.probes):
        e = rel_l2(a[k], b[k])
        if pr.quantity == W.Q_RHO_RE:
            e = max(e, rel_l2(a[k] - 1.0, b[k] - 1.0))
        assert e <= 1e-4, (k, pr, e)
    for prec in ("fp32", "fp64"):
        st = out[prec]["stats"]
        assert st["max_trace_dev"] <= 1e-6 and st["min_eig"] >= -1e-6, (prec, st)


def test_fullsize_window_vs_oracle(full_runs):
    """Probe traces within the paper-path bounds (1e-10 FP64, 1e-4 FP32 rel-L2).
    The offset-free deviation rho11 - 1 (a stricter measure, since rho11 ~ 1)
    is held to 1e-4 in FP32 and to 1e-8 in FP64: after 52,000 steps of
    propagation, FP64 round-off differences between two correct
    implementations are amplified by the resonant medium to ~1e-10 of the
    (small) deviation."""
    p, out = full_runs
    win = W.light_cone_window(p, WINDOW_STEPS)
    ref = oracle.run(win)
    assert ref["nt"] == WINDOW_STEPS
    names = [(q.cell, q.quantity, q.i, q.j) for q in p.probes]
    report = []
    for k, q in enumerate(win.probes):
        if q.cell not in NEAR:
            continue
        kk = names.index((q.cell, q.quantity, q.i, q.j))
        r = ref["records"][k]
        for prec, tol, tol_dev in (("fp64", 1e-10, 1e-8), ("fp32", 1e-4, 1e-4)):
            g = out[prec]["records"][kk][:WINDOW_STEPS]
            e = rel_l2(g, r)
            report.append((prec, q.cell, q.quantity, e))
            assert e <= tol, (prec, q, e, report)
            if q.quantity == W.Q_RHO_RE:
                ed = rel_l2(g - 1.0, r - 1.0)
                report.append((prec, q.cell, "dev", ed, float(np.abs(r - 1.0).max())))
                assert ed <= tol_dev, (prec, q, ed, report)
    print(report)


# ------------------------------------------------------------------ six levels
# The six-level ladder at full size (131,072 cells x 50,000 steps) in the
# launch configuration bench.py times (FP32 tensor-core tiles of 10 steps),
# against the FP64 plain path over the whole run and against the oracle on
# the light-cone window of the first 7,300 steps (probes just inside the
# medium, which starts at cell 6,554; the pulse reaches them near step 6,800).
# Bounds as for two levels: traces 1e-10 (FP64) and 1e-4 (FP32) relative L2;
# the offset-free deviation rho_kk - rho_kk(0) 1e-8 (FP64) and 1e-4 (FP32).
WINDOW6 = 7_300
NEAR6 = (6_560, 6_600, 6_700)


@pytest.fixture(scope="module")
def full_runs6():
    from paper_2005_05412_gb300 import build
    build.build()
    p = W.ladder_6lvl()
    extra = []
    for c in NEAR6:
        extra += [W.Probe(c, W.Q_E)] + [W.Probe(c, W.Q_RHO_RE, k, k) for k in range(6)]
    p = p.replace(probes=p.probes + extra)
    out = {"fp32": mbs.run(p, precision="fp32", algo="tiled", tile_steps=10),
           "fp64": mbs.run(p, precision="fp64", algo="plain")}
    return p, out


def test_fullsize6_fp32_tc_vs_fp64(full_runs6):
    p, out = full_runs6
    a, b = out["fp32"]["records"], out["fp64"]["records"]
    assert a.shape == (len(p.probes), 50_000)
    for k, pr in enumerate(p.probes):
        e = rel_l2(a[k], b[k])
        if pr.quantity == W.Q_RHO_RE and np.any(b[k] != b[k][0]):
            e = max(e, rel_l2(a[k] - b[k][0], b[k] - b[k][0]))
        assert e <= 1e-4, (k, pr, e)
    for prec in ("fp32", "fp64"):
        st = out[prec]["stats"]
        assert st["max_trace_dev"] <= 1e-6 and st["min_eig"] >= -1e-6, (prec, st)


def test_fullsize6_window_vs_oracle(full_runs6):
    p, out = full_runs6
    win = W.light_cone_window(p, WINDOW6)
    ref = oracle.run(win)
    assert ref["nt"] == WINDOW6
    names = [(q.cell, q.quantity, q.i, q.j) for q in p.probes]
    report = []
    for k, q in enumerate(win.probes):
        if q.cell not in NEAR6:
            continue
        kk = names.index((q.cell, q.quantity, q.i, q.j))
        r = ref["records"][k]
        for prec, tol, tol_dev in (("fp64", 1e-10, 1e-8), ("fp32", 1e-4, 1e-4)):
            g = out[prec]["records"][kk][:WINDOW6]
            e = rel_l2(g, r)
            report.append((prec, q.cell, q.quantity, q.i, e))
            assert e <= tol, (prec, q, e, report)
            if q.quantity == W.Q_RHO_RE and np.any(r != r[0]):
                ed = rel_l2(g - r[0], r - r[0])
                report.append((prec, q.cell, "dev", q.i, ed))
                assert ed <= tol_dev, (prec, q, ed, report)
    print(report)

"""Parity of the 512-simulation mixed batch (two- and three-level media,
1,024 to 65,536 cells, 20,000 to 100,000 steps, +-20 % parameters), solved
in the launch configuration bench.py times: one batched FP32 solve with
autotuned tile depths, recorded as a CUDA graph and replayed.

  * FP32 against FP64 (batched tiled FP64) over the whole run of the first
    32 simulations, every probe;
  * all 512 simulations truncated to the steps it takes the left pulse to
    pass 10 cells into the medium (its centre t0 plus 5 tau, plus the travel
    time: 500 to 7,800 steps), batched on the GPU in FP32 and FP64, against
    the oracle, at the probes the whole pulse has passed: 10 cells inside
    each medium (E and every population) and the rule probes before it.
    (A probe deeper in sees only the pulse's leading edge by then; its
    populations stay below 1e-5, where the FP32 form's absolute rounding,
    ~1e-9 on populations formed from dipole-eigenbasis components of order
    0.05, is itself 1e-4 of the trace.)  The oracle runs each simulation on
    the cells that can reach those probes in time (a left-edge source moves
    at most one cell per step, so a cell beyond (steps + p) / 2 cannot send
    anything back to a probe at p), or on the whole grid when the
    simulation's right-edge source could reach a probe.

Bounds per trace (relative L2): FP32 1e-4, FP64 1e-10; populations also as
the offset-free deviation from their initial value (FP32 1e-4; FP64 1e-8,
the FP64 floor of a small population riding on a near-unity one).  In the
truncated runs FP32 leaves populations that move by less than 1e-4 (see
SMALL_POP) to the FP64 and full-length comparisons.  The
per-simulation worst errors are printed and, when MBS_PARITY_OUT names a
file, written there as JSON.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu

N_FULL64 = 32
# A population that the truncated run barely moves (the Lambda medium's rho_22,
# fed only by decay from level 3 within a picosecond) stays below this: the
# FP32 form rounds populations formed from dipole-eigenbasis components of
# order 0.05 to ~3e-9 absolute, 1e-4 of such a trace, so FP32 compares it in
# the full-length test (where it grows) and FP64 compares it here.
SMALL_POP = 1e-4


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def trace_err(g, r, q):
    """Relative L2 of a trace; for a population also of its deviation from
    the initial value.  Traces the oracle sees as exactly zero (beyond the
    light cone) compare in absolute terms."""
    nr = np.linalg.norm(r)
    if nr == 0.0:
        return float(np.abs(g).max()), 0.0
    e = rel_l2(g, r)
    ed = 0.0
    if q.quantity == W.Q_RHO_RE and np.any(r != r[0]):
        ed = rel_l2(g - r[0], r - r[0])
    return e, ed


def _solve(ps, precision, **kw):
    devs = [mbs.device_from_problem(p) for p in ps]
    scs = [mbs.scenario_from_problem(d, p) for d, p in zip(devs, ps)]
    mbs.mbs_solve(scs, precision, "tiled", **kw)
    recs = [np.stack([mbs.mbs_fetch_records(sc, k) for k in range(len(p.probes))]) for sc, p in zip(scs, ps)]
    stats = [mbs.mbs_scenario_stats(sc) for sc in scs]
    for sc in scs:
        sc.close()
    for d in devs:
        d.close()
    return recs, stats


def _medium_front(p):
    return next(c for c in range(p.n_cells) if W.in_medium(c, p.n_cells))


def _with_front_probes(p):
    m = _medium_front(p) + 10
    n = p.qms[0].n_levels
    return p.replace(probes=p.probes + [W.Probe(m, W.Q_E)] + [W.Probe(m, W.Q_RHO_RE, k, k) for k in range(n)])


def _oracle_window(p, steps):
    """The oracle's problem for the first `steps` steps of p, and the indices
    of p's probes it records (those at or before the front probe, 10 cells
    into the medium).  The whole grid when p is short or the front probe lies
    in the light cone of a right-edge source; else the cells [0, (steps +
    pmax) / 2 + 16), pmax the farthest kept probe, which evolve exactly as in
    the full grid."""
    right = min([s.cell for s in p.sources if s.kind == W.SRC_TFSF_LEFT], default=10 ** 9)
    front = _medium_front(p) + 10
    idx = [k for k, q in enumerate(p.probes) if q.cell <= front]
    kept = [p.probes[k] for k in idx]
    if p.n_cells <= steps + 16 or front >= right - steps - 2:
        return p.replace(n_steps=steps, t_end=0.0, probes=kept), idx
    nx = min(p.n_cells, (steps + max(q.cell for q in kept)) // 2 + 16)
    win = p.replace(n_cells=nx, length=nx * p.dz, n_steps=steps, t_end=0.0, probes=kept,
                    sources=[s for s in p.sources if s.cell < nx - 2])
    return win, idx


@pytest.fixture(scope="module")
def batch():
    from paper_2005_05412_gb300 import build
    build.build()
    return W.batch_mixed()


def _report(log, name, rows):
    worst = max(rows, key=lambda r: r["err"])
    print(f"{name}: {len(rows)} simulations, worst trace {worst['err']:.3e} (simulation {worst['sim']}), "
          f"worst population deviation {max(r['dev'] for r in rows):.3e}")
    log(name, {"simulations": len(rows), "worst": worst, "rows": rows})


def test_batch_fp32_vs_fp64_full_length(batch, parity_log):
    ps = batch
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    r32, st32 = _solve(ps, "fp32", autotune=True, graph=True, stream=stream)
    r64, st64 = _solve(ps[:N_FULL64], "fp64")
    rows = []
    for s in range(N_FULL64):
        err = dev = 0.0
        for k, q in enumerate(ps[s].probes):
            e, ed = trace_err(r32[s][k], r64[s][k], q)
            err, dev = max(err, e), max(dev, ed)
        rows.append({"sim": s, "levels": ps[s].qms[0].n_levels, "cells": ps[s].n_cells, "steps": ps[s].n_steps,
                     "err": err, "dev": dev})
        assert err <= 1e-4 and dev <= 1e-4, rows[-1]
    for s, st in enumerate(st32):
        assert np.isfinite(r32[s]).all(), s
        assert st["max_trace_dev"] <= 1e-6 and st["min_eig"] >= -1e-6, (s, st)
    _report(parity_log, "batch_fp32_vs_fp64_first32_full", rows)


def _pulse_passed(p):
    """Steps until the left pulse has passed 10 cells into the medium."""
    s = p.sources[0]
    dt = p.courant * p.dz / W.C0
    return min(p.n_steps, int((s.t0 + 5 * s.tau) / dt) + int((_medium_front(p) + 10) / p.courant) + 16)


def test_batch_truncated_vs_oracle(batch, parity_log):
    ps = [_with_front_probes(p) for p in batch]
    ps = [p.replace(n_steps=_pulse_passed(p), t_end=0.0) for p in ps]
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    wins = [_oracle_window(p, p.n_steps) for p in ps]
    ref = oracle.run_many([w for w, _ in wins], processes=os.cpu_count() or 1)
    got = {"fp32": _solve(ps, "fp32", autotune=True, graph=True, stream=stream)[0],
           "fp64": _solve(ps, "fp64")[0]}
    for prec, tol, tol_dev in (("fp32", 1e-4, 1e-4), ("fp64", 1e-10, 1e-8)):
        rows = []
        small = 0
        for s, ((w, idx), (rec, _dt, nt)) in enumerate(zip(wins, ref)):
            assert nt == ps[s].n_steps
            err = dev = 0.0
            at = None
            for kw, kp in enumerate(idx):
                q = w.probes[kw]
                if prec == "fp32" and q.quantity == W.Q_RHO_RE and np.abs(rec[kw] - rec[kw][0]).max() < SMALL_POP:
                    small += 1
                    continue
                e, ed = trace_err(got[prec][s][kp], rec[kw], q)
                if max(e, ed) >= max(err, dev):
                    q = w.probes[kw]
                    at = (q.cell, q.quantity, q.i)
                err, dev = max(err, e), max(dev, ed)
            rows.append({"sim": s, "levels": ps[s].qms[0].n_levels, "cells": ps[s].n_cells, "steps": nt,
                         "err": err, "dev": dev, "window_cells": w.n_cells, "worst_probe": at})
            assert err <= tol and dev <= tol_dev, (prec, rows[-1])
        print(f"{prec}: {small} population traces below {SMALL_POP} left to the FP64 and full-length comparisons")
        _report(parity_log, f"batch_{prec}_pulse_through_front_vs_oracle", rows)

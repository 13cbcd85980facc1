"""The periodic state check (check_every): the splitting of Sec. 2.2 keeps
every cell's density matrix a density matrix, so a check that finds a
non-finite value, a negative population or a negative 2 x 2 principal minor
stops the solve with MBS_E_NUMERIC -- a status, never a GPU fault.

The failure is made on the host: two superposed one-way sources of
1.7e308 V/m overflow the fields to inf at the first step (in FP32 the
source table itself holds inf).  The checks must then stop the solve at the
first check boundary, which the launch counter and the step count show.
"""
import math

import numpy as np
import pytest

import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05412_gb300 import build
    build.build()


def _overflowing(n_cells=2048, n_steps=4000):
    p = W.sit_2lvl(n_cells=n_cells, t_end=0.0, n_steps=n_steps)
    s = p.sources[0]
    p.sources = [W.Source(W.SRC_TFSF_RIGHT, c, 1.7e308, s.tau, 0.0, s.omega, 1.0) for c in (3, 5)]
    return p


def _solve_expect_numeric(p, **kw):
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_solve([sc], **kw)
    assert e.value.status == mbs.MBS_E_NUMERIC, e.value
    return sc, dev


@pytest.mark.parametrize("prec,algo,tile,chk", [("fp32", "tiled", 24, 96), ("fp64", "tiled", 24, 96),
                                                ("fp64", "plain", 0, 50), ("fp32", "plain", 0, 50)])
def test_failed_check_stops_the_solve(prec, algo, tile, chk):
    p = _overflowing()
    sc, dev = _solve_expect_numeric(p, precision=prec, algo=algo, tile_steps=tile, check_every=chk)
    st = mbs.mbs_scenario_stats(sc)
    ctr = mbs.mbs_scenario_counters(sc)
    assert st["n_steps"] == chk, st                     # stopped at the first check
    if algo == "tiled":
        # chk / tile step launches, the check pair, the final check
        assert ctr["kernel_launches"] <= math.ceil(chk / tile) + 3, ctr
    else:
        assert ctr["kernel_launches"] <= 2 * chk + 3, ctr
    # the context is still usable: a healthy problem solves afterwards
    ok = mbs.run(W.sit_2lvl(n_cells=256, t_end=0.0, n_steps=100), precision=prec, algo=algo,
                 tile_steps=tile, check_every=chk)
    assert np.all(np.isfinite(ok["records"]))


def test_checks_leave_healthy_traces_unchanged():
    """Periodic checks on a healthy run change nothing but the compensated
    pairs' canonical form: traces within 1e-6 of the run without checks (FP32,
    tiles), identical in FP64."""
    p = W.sit_2lvl_jitter(n_cells=20_000, n_steps=3_000)
    for prec, tol in (("fp32", 1e-6), ("fp64", 0.0)):
        a = mbs.run(p, precision=prec, algo="tiled", tile_steps=24)
        b = mbs.run(p, precision=prec, algo="tiled", tile_steps=24, check_every=240)
        assert b["counters"]["kernel_launches"] > a["counters"]["kernel_launches"]
        for k in range(len(p.probes)):
            d = np.linalg.norm(b["records"][k] - a["records"][k]) / np.linalg.norm(a["records"][k])
            assert d <= tol, (prec, k, d)
        assert b["stats"]["min_eig"] >= -1e-6


def test_batch_checks_isolate_the_failing_member():
    """check_every in a batched solve: the overflowing member fails its check
    and stops on the device; the healthy member finishes with records
    identical to its solve alone; the batch returns MBS_E_NUMERIC."""
    good = W.sit_2lvl(n_cells=3000, t_end=0.0, n_steps=2000)
    bad = _overflowing(n_cells=2500, n_steps=2000)
    for prec in ("fp32", "fp64"):
        alone = mbs.run(good, precision=prec, algo="tiled", tile_steps=24, check_every=96)["records"]
        devs = [mbs.device_from_problem(q) for q in (good, bad)]
        scs = [mbs.scenario_from_problem(d, q) for d, q in zip(devs, (good, bad))]
        with pytest.raises(mbs.MBSError) as e:
            mbs.mbs_solve(scs, prec, "tiled", tile_steps=24, check_every=96)
        assert e.value.status == mbs.MBS_E_NUMERIC
        for k in range(len(good.probes)):
            np.testing.assert_array_equal(mbs.mbs_fetch_records(scs[0], k), alone[k])

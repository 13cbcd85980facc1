"""Batched solves: several independent simulations (different cell counts,
level counts, step counts and parameters) advance together, one launch per
kernel variant per tile of steps.  Each member must give exactly what it
gives when solved alone, and the oracle's result."""
import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05412_gb300 import build
    build.build()


def _members():
    return [
        W.sit_2lvl(n_cells=2048, n_steps=1500),
        W.sit_2lvl_jitter(n_cells=5003, n_steps=2100, seed=11),
        W.lambda_3lvl(n_cells=3001, n_steps=4000, tau=20e-15, t0=120e-15),
        W.sit_2lvl(n_cells=700, n_steps=900, density=1.3e24, omega0=2.2e14, courant=W.COURANT_LONG),
        W.lambda_3lvl(n_cells=1100, n_steps=2500, tau=15e-15, t0=100e-15, t1=8e-12, t2=1.5e-12),
        W.sit_2lvl_jitter(n_cells=9000, n_steps=1200, seed=12).replace(refl_right=1.0),
    ]


def _scenarios(ps):
    devs = [mbs.device_from_problem(p) for p in ps]
    return devs, [mbs.scenario_from_problem(d, p) for d, p in zip(devs, ps)]


def _records(sc, n):
    return np.stack([mbs.mbs_fetch_records(sc, k) for k in range(n)])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_one_at_a_time(prec):
    ps = _members()
    _, scs = _scenarios(ps)
    mbs.mbs_solve(scs, prec, "tiled", tile_steps=12)
    batched = [_records(sc, len(p.probes)) for sc, p in zip(scs, ps)]
    stats = [mbs.mbs_scenario_stats(sc) for sc in scs]
    mbs.mbs_solve(scs, prec, "tiled", tile_steps=12, one_at_a_time=True)
    for k, (sc, p) in enumerate(zip(scs, ps)):
        alone = _records(sc, len(p.probes))
        np.testing.assert_allclose(batched[k], alone, rtol=0, atol=1e-12 * max(1.0, np.abs(alone).max()),
                                   err_msg=f"member {k}")
        assert stats[k]["n_steps"] == p.n_steps
        assert stats[k]["min_eig"] >= -1e-6 and stats[k]["max_trace_dev"] <= 1e-6


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("fp64", 1e-10)])
def test_batch_members_match_oracle(prec, tol):
    ps = _members()
    _, scs = _scenarios(ps)
    mbs.mbs_solve(scs, prec, "tiled", tile_steps=16)
    for k in (1, 2, 3):
        p = ps[k]
        ref = oracle.run(p)["records"]
        got = _records(scs[k], len(p.probes))
        for q in range(len(p.probes)):
            r, g = ref[q], got[q]
            e = np.linalg.norm(g - r) / np.linalg.norm(r)
            assert e <= tol, (k, q, e)


def test_batch_counters_and_errors():
    ps = _members()[:3]
    _, scs = _scenarios(ps)
    mbs.mbs_solve(scs, "fp32", "tiled", tile_steps=8)
    for sc, p in zip(scs, ps):
        c = mbs.mbs_scenario_counters(sc)
        assert c["kernel_launches"] >= -(-p.n_steps // 8)
    with pytest.raises(mbs.MBSError):
        mbs.mbs_solve(scs, "fp32", "tiled", tile_steps=6)

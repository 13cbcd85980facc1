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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_graph_replay(prec):
    """MBS_SOLVE_GRAPH: the first call records the batched solve as a CUDA
    graph, later calls replay it; both equal the solve without a graph to
    the last bit.  Destroying a member frees the graph; the rest still
    solves."""
    import torch
    st = torch.cuda.Stream()
    ps = _members()
    devs, scs = _scenarios(ps)
    mbs.mbs_solve(scs, prec, "tiled", tile_steps=12, stream=st.cuda_stream)
    torch.cuda.synchronize()
    ref = [_records(sc, len(p.probes)) for sc, p in zip(scs, ps)]
    for call in range(3):
        mbs.mbs_solve(scs, prec, "tiled", tile_steps=12, stream=st.cuda_stream, graph=True)
        torch.cuda.synchronize()
        for k, (sc, p) in enumerate(zip(scs, ps)):
            np.testing.assert_array_equal(_records(sc, len(p.probes)), ref[k], err_msg=f"call {call} member {k}")
            assert mbs.mbs_scenario_tile(sc) == 12
            assert mbs.mbs_scenario_counters(sc)["kernel_launches"] == -(-p.n_steps // 12)
    scs[2].close()
    rest = scs[:2] + scs[3:]
    mbs.mbs_solve(rest, prec, "tiled", tile_steps=12, stream=st.cuda_stream, graph=True)
    torch.cuda.synchronize()
    for k, sc in zip([0, 1, 3, 4, 5], rest):
        np.testing.assert_array_equal(_records(sc, len(ps[k].probes)), ref[k])


def test_autotune_picks_a_candidate_and_keeps_parity():
    """MBS_SOLVE_AUTOTUNE: the tile depth is measured (a candidate depth is
    used, the same on a second call from the cache) and the trial launches
    leave no trace in the result."""
    import torch
    st = torch.cuda.Stream()
    p = W.lambda_3lvl(n_cells=20_011, n_steps=3_000, tau=20e-15, t0=120e-15)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    mbs.mbs_solve([sc], "fp64", "plain", stream=st.cuda_stream)
    torch.cuda.synchronize()
    ref = _records(sc, len(p.probes))
    for call in range(2):
        mbs.mbs_solve([sc], "fp64", "tiled", stream=st.cuda_stream, autotune=True)
        torch.cuda.synchronize()
        T = mbs.mbs_scenario_tile(sc)
        assert T in (16, 20, 24, 28, 32, 40, 48)
        if call == 0:
            T0 = T
        assert T == T0
        got = _records(sc, len(p.probes))
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    ps = _members()
    _, scs = _scenarios(ps)
    mbs.mbs_solve(scs, "fp32", "tiled", stream=st.cuda_stream, autotune=True, graph=True)
    torch.cuda.synchronize()
    for k in (1, 2):
        r = oracle.run(ps[k])["records"]
        g = _records(scs[k], len(ps[k].probes))
        for q in range(len(ps[k].probes)):
            assert np.linalg.norm(g[q] - r[q]) / np.linalg.norm(r[q]) <= 1e-4, (k, q)
    q6 = W.ladder_6lvl(n_cells=3_000, n_steps=400)
    d6 = mbs.device_from_problem(q6)
    s6 = mbs.scenario_from_problem(d6, q6)
    mbs.mbs_solve([s6], "fp32", stream=st.cuda_stream, autotune=True)
    torch.cuda.synchronize()
    assert mbs.mbs_scenario_tile(s6) in (6, 8, 10, 12, 14, 16, 20)

"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.

Bounds: FP64 GPU path <= 1e-10 relative L2 per probe trace; FP32 path
<= 1e-4 (also on rho_11 - rho_11(0), which removes the near-unity offset
that would otherwise flatter the FP32 error).  FP64 tiled and plain forms
agree to rounding.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-10, 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05412_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


_ORACLE = {}


def oracle_run(key, p):
    if key not in _ORACLE:
        _ORACLE[key] = oracle.run(p)
    return _ORACLE[key]


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def assert_parity(p, got, ref, tol, label):
    assert got["nt"] == ref["nt"]
    assert got["dt"] == pytest.approx(ref["dt"], rel=1e-15)
    worst = 0.0
    for k, pr in enumerate(p.probes):
        g, r = got["records"][k], ref["records"][k]
        assert np.all(np.isfinite(g)), (label, k)
        e = rel_l2(g, r)
        if pr.quantity == W.Q_RHO_RE and pr.i == pr.j:
            e = max(e, rel_l2(g - r[0], r - r[0]) if np.any(r != r[0]) else 0.0)
        worst = max(worst, e)
        assert e <= tol, f"{label}: probe {k} (cell {pr.cell}, q {pr.quantity}) rel-L2 {e:.3e} > {tol}"
    return worst


# ------------------------------------------------------------ workloads
def sit_small():
    return W.sit_2lvl()                                    # 2,048 cells, 4,094 steps


def sit_jitter_small():
    return W.sit_2lvl_jitter(n_cells=12_289, n_steps=5_000)   # ragged vs every tile width


def lambda_small():
    return W.lambda_3lvl(n_cells=3_001, n_steps=4_000, tau=20e-15, t0=120e-15)


def ladder_small():
    return W.ladder_6lvl(n_cells=777, n_steps=1_200)


@pytest.mark.parametrize("algo", ["plain", "tiled"])
def test_sit_fp64(algo, parity_log):
    p = sit_small()
    ref = oracle_run("sit", p)
    got = mbs.run(p, precision="fp64", algo=algo)
    worst = assert_parity(p, got, ref, TOL64, f"sit fp64 {algo}")
    parity_log(f"sit_2lvl_fp64_{algo}_vs_oracle_full", {"worst": {"err": worst}, "rows": [{"dev": 0.0}],
                                                       "simulations": 1})


@pytest.mark.parametrize("algo,tile", [("plain", 0), ("tiled", 16), ("tiled", 8), ("tiled", 36), ("tiled", 24)])
def test_sit_fp32(algo, tile, parity_log):
    p = sit_small()
    ref = oracle_run("sit", p)
    got = mbs.run(p, precision="fp32", algo=algo, tile_steps=tile)
    worst = assert_parity(p, got, ref, TOL32, f"sit fp32 {algo} T={tile}")
    if tile in (0, 24):
        parity_log(f"sit_2lvl_fp32_{algo}_vs_oracle_full", {"worst": {"err": worst}, "rows": [{"dev": 0.0}],
                                                           "simulations": 1})
    assert got["stats"]["max_trace_dev"] <= 1e-6
    assert got["stats"]["min_eig"] >= -1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_sit_jitter(prec, tol):
    p = sit_jitter_small()
    ref = oracle_run("sitj", p)
    for algo in ("plain", "tiled"):
        got = mbs.run(p, precision=prec, algo=algo)
        assert_parity(p, got, ref, tol, f"jitter {prec} {algo}")


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_lambda_three_level(prec, tol):
    p = lambda_small()
    ref = oracle_run("lambda", p)
    for algo in ("plain", "tiled"):
        got = mbs.run(p, precision=prec, algo=algo)
        assert_parity(p, got, ref, tol, f"lambda {prec} {algo}")


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_ladder_six_level_plain(prec, tol):
    p = ladder_small()
    ref = oracle_run("ladder", p)
    got = mbs.run(p, precision=prec, algo="plain")
    assert_parity(p, got, ref, tol, f"ladder {prec}")


def test_tiled_matches_plain_fp64():
    """Same arithmetic per cell: the temporal tiles change nothing but the
    order of launches."""
    p = sit_jitter_small()
    a = mbs.run(p, precision="fp64", algo="plain")["records"]
    for T in (4, 16, 60):
        b = mbs.run(p, precision="fp64", algo="tiled", tile_steps=T)["records"]
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())


@pytest.mark.parametrize("n_levels,tile", [(2, 4), (2, 12), (2, 28), (3, 4), (3, 12)])
def test_tiled_right_boundary_at_tile_edge(n_levels, tile):
    """Grids whose last cell would start a warp's owned range; below Courant
    number 1 the absorbing end reads its neighbour's new field, so the tiled
    form must keep that neighbour in the same warp."""
    r = 4 if n_levels == 2 else 2
    own = 32 * r - 2 * tile
    nx = 25 * own + 1
    if n_levels == 2:
        p = W.sit_2lvl(n_cells=nx, n_steps=1500, courant=W.COURANT_LONG)
    else:
        p = W.lambda_3lvl(n_cells=nx, n_steps=1500, tau=20e-15, t0=120e-15)
    p.probes = p.probes + [W.Probe(nx - 1, W.Q_E), W.Probe(nx - 2, W.Q_E), W.Probe(nx - 1, W.Q_H)]
    a = mbs.run(p, precision="fp64", algo="plain")["records"]
    b = mbs.run(p, precision="fp64", algo="tiled", tile_steps=tile)["records"]
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())


# ------------------------------------------------------------ edge cases
def _edge_problem():
    """Ragged grid, mirrors on both ends, a hard source, a left-going source,
    H and Im(rho) probes, probes on boundary and source cells."""
    p = W.sit_2lvl(n_cells=613, t_end=0.0, n_steps=1_333)
    p.refl_left = p.refl_right = 1.0
    s = p.sources[0]
    p.sources = [W.Source(W.SRC_HARD, 300, s.e0 * 0.3, s.tau, s.t0, s.omega),
                 W.Source(W.SRC_TFSF_LEFT, 600, s.e0 * 0.5, s.tau, s.t0 + 10e-15, s.omega * 1.1, 0.3)]
    p.probes = [W.Probe(0, W.Q_E), W.Probe(612, W.Q_E), W.Probe(300, W.Q_E), W.Probe(600, W.Q_H),
                W.Probe(450, W.Q_H), W.Probe(450, W.Q_RHO_IM, 0, 1), W.Probe(451, W.Q_RHO_RE, 1, 1),
                W.Probe(36, W.Q_RHO_RE, 0, 1), W.Probe(1, W.Q_E)]
    return p


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_edge_cases(prec, tol):
    p = _edge_problem()
    ref = oracle.run(p)
    for algo, T in [("plain", 0), ("tiled", 4), ("tiled", 20)]:
        got = mbs.run(p, precision=prec, algo=algo, tile_steps=T)
        for k, pr in enumerate(p.probes):
            g, r = got["records"][k], ref["records"][k]
            if pr.cell in (0, 612) and pr.quantity == W.Q_E:      # mirrors: exactly zero
                assert np.all(g == 0.0)
                continue
            assert rel_l2(g, r) <= tol, (algo, T, k, rel_l2(g, r))


def test_minimal_grid_and_single_step():
    p = W.sit_2lvl(n_cells=8, t_end=0.0, n_steps=1)
    p.regions = [W.Region(0, 0, 2 * p.dz), W.Region(1, 2 * p.dz, 6 * p.dz), W.Region(0, 6 * p.dz, p.length)]
    p.sources[0].t0 = 0.0
    p.probes = [W.Probe(c, W.Q_E) for c in range(8)] + [W.Probe(3, W.Q_RHO_RE, 0, 0)]
    ref = oracle.run(p)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        for algo in ("plain", "tiled"):
            got = mbs.run(p, precision=prec, algo=algo)
            np.testing.assert_allclose(got["records"], ref["records"], rtol=tol, atol=tol * p.sources[0].e0)


def test_api_errors_on_gpu():
    p = W.sit_2lvl(n_cells=64, t_end=0.0, n_steps=5)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_fetch_records(sc, 0)
    assert e.value.status == mbs.MBS_E_STATE
    with pytest.raises(mbs.MBSError):
        mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=6)     # not a multiple of 4
    with pytest.raises(mbs.MBSError):
        mbs.mbs_scenario(dev, 0.0, 1.5, 1e-13, 0, p.sources, p.probes)   # Courant > 1
    with pytest.raises(mbs.MBSError):
        mbs.mbs_scenario(dev, 0.0, 1.0, 1e-13, 0, [W.Source(0, 1, 1.0, 1e-15, 0, 1e14)], [])
    mbs.mbs_solve([sc], "fp32")
    with pytest.raises(mbs.MBSError):
        mbs.mbs_fetch_records(sc, 99)


def test_numeric_failure_is_a_status_not_a_fault():
    """Two superposed 1.7e308 V/m pulses overflow the fields to inf and
    the state to NaN; the device state check reports MBS_E_NUMERIC (no
    GPU fault) and the context stays usable.  A non-finite step operator is
    rejected when the scenario is built, non-finite source parameters too."""
    p = W.sit_2lvl(n_cells=64, t_end=0.0, n_steps=200)
    s = p.sources[0]
    p.sources = [W.Source(W.SRC_TFSF_RIGHT, c, 1.7e308, s.tau, 0.0, s.omega, 1.0) for c in (3, 5)]
    for prec in ("fp64", "fp32"):
        with pytest.raises(mbs.MBSError) as e:
            mbs.run(p, precision=prec, algo="plain", check_every=50)
        assert e.value.status == mbs.MBS_E_NUMERIC
    q = W.sit_2lvl(n_cells=64, t_end=0.0, n_steps=8)
    q.qms[0].h0 = q.qms[0].h0 * 1e300
    with pytest.raises(mbs.MBSError) as e:
        mbs.run(q, precision="fp64")
    assert e.value.status == mbs.MBS_E_NUMERIC
    q = W.sit_2lvl(n_cells=64, t_end=0.0, n_steps=8)
    q.sources[0].e0 = float("nan")
    with pytest.raises(mbs.MBSError) as e:
        mbs.run(q, precision="fp64")
    assert e.value.status == mbs.MBS_E_INVALID
    ok = mbs.run(sit_small().replace(n_steps=10, t_end=0.0), precision="fp32")
    assert np.all(np.isfinite(ok["records"]))


@pytest.mark.parametrize("n_levels", [2, 3, 4, 5, 6])
def test_state_check_min_eigenvalue(n_levels):
    """The device state check reports the smallest eigenvalue of the stored
    density matrix: after one source-free step from rho0 that is
    exp(1.5 L0 dt) rho0 (the state carries half a step ahead)."""
    import scipy.linalg as sl
    p = W.ladder_6lvl(n_cells=64, n_steps=1)
    q = p.qms[0]
    n = n_levels
    rng = np.random.default_rng(n)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    rho0 = a @ a.conj().T + 0.05 * np.eye(n)
    rho0 /= np.trace(rho0).real
    keep = [k for k, o in enumerate(q.lindblad_ops) if not np.abs(o[n:, :]).any() and not np.abs(o[:, n:]).any()]
    q2 = W.QM(n, q.density, q.h0[:n, :n], q.mu[:n, :n], rho0, q.lindblad_rates[keep],
              q.lindblad_ops[keep][:, :n, :n])
    p = p.replace(qms=[q2], sources=[], probes=[W.Probe(10, W.Q_E)])
    L0 = oracle.liouvillian(q2)
    x = (sl.expm(1.5 * L0 * (p.courant * p.dz / W.C0)) @ rho0.reshape(-1)).reshape(n, n)
    ref = np.linalg.eigvalsh((x + x.conj().T) / 2).min()
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        st = mbs.run(p, precision=prec, algo="plain")["stats"]
        assert st["min_eig"] == pytest.approx(ref, abs=tol)
        assert st["max_trace_dev"] <= tol

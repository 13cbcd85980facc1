"""GPU parity of the tensor-core tiles (N = 4..6 levels, FP32 state, the
constant propagator applied as a 3xTF32 tcgen05 contraction) against the
CPU oracle and against the FP64 plain path, through the C ABI.

Bound: 1e-4 relative L2 per probe trace (also on rho_kk - rho_kk(0)), the
reduced-precision bound of the FP32 path.
"""
import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05412_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def trace_errors(p, got, ref):
    out = []
    for k, pr in enumerate(p.probes):
        g, r = got[k], ref[k]
        assert np.all(np.isfinite(g)), k
        e = rel_l2(g, r)
        if pr.quantity == W.Q_RHO_RE and pr.i == pr.j and np.any(r != r[0]):
            e = max(e, rel_l2(g - r[0], r - r[0]))
        out.append(e)
    return np.array(out)


def ladder(n_levels, n_cells, n_steps, **kw):
    """The seeded six-level ladder medium, or its first n_levels levels (the
    operators that stay inside them, the pulse at their mean transition)."""
    p = W.ladder_6lvl(n_cells=n_cells, n_steps=n_steps, **kw)
    if n_levels == 6:
        return p
    q = p.qms[0]
    n = n_levels
    keep = [k for k, o in enumerate(q.lindblad_ops) if not np.abs(o[n:, :]).any() and not np.abs(o[:, n:]).any()]
    rho0 = np.zeros((n, n), complex)
    rho0[0, 0] = 1.0
    q2 = W.QM(n, q.density, q.h0[:n, :n], q.mu[:n, :n], rho0, q.lindblad_rates[keep],
              q.lindblad_ops[keep][:, :n, :n])
    en = np.real(np.diag(q2.h0))
    s = p.sources[0]
    src = W.Source(s.kind, s.cell, s.e0, s.tau, s.t0, (en[-1] - en[0]) / (n - 1) / W.HBAR, s.phase)
    probes = []
    for pr in p.probes:
        if pr.quantity in (W.Q_E, W.Q_H):
            probes.append(pr)
        elif pr.i < n and pr.j < n:
            probes.append(pr)
    return p.replace(qms=[q2], sources=[src], probes=probes)


_ORACLE = {}


def oracle_run(key, p):
    if key not in _ORACLE:
        _ORACLE[key] = oracle.run(p)
    return _ORACLE[key]


@pytest.mark.parametrize("tile", [1, 8, 20])
def test_ladder_six_level_tc_vs_oracle(tile):
    p = ladder(6, 777, 1_200)
    ref = oracle_run("ladder6", p)
    got = mbs.run(p, precision="fp32", algo="tiled", tile_steps=tile)
    err = trace_errors(p, got["records"], ref["records"])
    assert err.max() <= TOL32, err
    assert got["stats"]["max_trace_dev"] <= 1e-6
    assert got["stats"]["min_eig"] >= -1e-6


@pytest.mark.parametrize("n_levels", [4, 5])
def test_four_and_five_levels_tc_vs_oracle(n_levels):
    p = ladder(n_levels, 1_031, 1_500)
    ref = oracle.run(p)
    got = mbs.run(p, precision="fp32", algo="tiled", tile_steps=8)
    err = trace_errors(p, got["records"], ref["records"])
    assert err.max() <= TOL32, err


def test_auto_algorithm_picks_the_tensor_core_tiles():
    p = ladder(6, 300, 40)
    got = mbs.run(p, precision="fp32")
    plain = mbs.run(p, precision="fp32", algo="plain")
    # tiles of 8 steps: 5 tiled launches + the final state check
    assert got["counters"]["kernel_launches"] == 6
    assert plain["counters"]["kernel_launches"] == 2 * 40 + 1
    np.testing.assert_allclose(got["records"], plain["records"], rtol=0,
                               atol=1e-4 * np.abs(plain["records"]).max())


@pytest.mark.parametrize("tile", [4, 8, 20])
def test_tc_right_boundary_at_tile_edge(tile):
    """Grids whose last cell would be the first owned cell of a tile; the
    absorbing end reads its neighbour's new field."""
    own = 128 - 2 * tile
    nx = 25 * own + 1
    p = ladder(6, nx, 1_500)
    p.probes = p.probes + [W.Probe(nx - 1, W.Q_E), W.Probe(nx - 2, W.Q_E), W.Probe(nx - 1, W.Q_H)]
    a = mbs.run(p, precision="fp64", algo="plain")["records"]
    b = mbs.run(p, precision="fp32", algo="tiled", tile_steps=tile)["records"]
    err = trace_errors(p, b, a)
    assert err.max() <= TOL32, err


def test_tc_edge_cases():
    """Mirrors on both ends, a hard source, a left-going source, H and
    Im(rho) probes, probes on boundary and source cells, a ragged grid."""
    p = ladder(6, 613, 1_333)
    p.refl_left = p.refl_right = 1.0
    s = p.sources[0]
    p.sources = [W.Source(W.SRC_HARD, 300, s.e0 * 0.3, s.tau, s.t0, s.omega),
                 W.Source(W.SRC_TFSF_LEFT, 600, s.e0 * 0.5, s.tau, s.t0 + 10e-15, s.omega * 1.1, 0.3)]
    p.probes = [W.Probe(0, W.Q_E), W.Probe(612, W.Q_E), W.Probe(300, W.Q_E), W.Probe(600, W.Q_H),
                W.Probe(450, W.Q_H), W.Probe(450, W.Q_RHO_IM, 0, 1), W.Probe(451, W.Q_RHO_RE, 1, 1),
                W.Probe(451, W.Q_RHO_RE, 2, 4), W.Probe(36, W.Q_RHO_RE, 0, 0), W.Probe(1, W.Q_E)]
    ref = oracle.run(p)
    for T in (4, 20):
        got = mbs.run(p, precision="fp32", algo="tiled", tile_steps=T)
        for k, pr in enumerate(p.probes):
            g, r = got["records"][k], ref["records"][k]
            if pr.cell in (0, 612) and pr.quantity == W.Q_E:      # mirrors: exactly zero
                assert np.all(g == 0.0)
                continue
            assert rel_l2(g, r) <= TOL32, (T, k, rel_l2(g, r))


def test_tc_minimal_grid_and_single_step():
    p = ladder(6, 8, 1)
    p.regions = [W.Region(0, 0, 2 * p.dz), W.Region(1, 2 * p.dz, 6 * p.dz), W.Region(0, 6 * p.dz, p.length)]
    p.sources[0].t0 = 0.0
    p.probes = [W.Probe(c, W.Q_E) for c in range(8)] + [W.Probe(3, W.Q_RHO_RE, 0, 0)]
    ref = oracle.run(p)
    got = mbs.run(p, precision="fp32", algo="tiled")
    np.testing.assert_allclose(got["records"], ref["records"], rtol=1e-6, atol=1e-6 * p.sources[0].e0)


def test_tc_limits():
    p = ladder(6, 300, 40)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    for bad in (50, 64):   # a 128-cell tile would own fewer than 32 cells
        with pytest.raises(mbs.MBSError) as e:
            mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=bad)
        assert e.value.status == mbs.MBS_E_INVALID
    with pytest.raises(mbs.MBSError) as e:       # FP64 has no tensor-core tiles
        mbs.mbs_solve([sc], "fp64", "tiled")
    assert e.value.status == mbs.MBS_E_INVALID
    mbs.mbs_solve([sc], "fp64")                  # auto: the plain FP64 path


@pytest.mark.parametrize("tile", [12, 20, 26, 40])
def test_wide_tiles_vs_oracle(tile):
    """256-cell tensor-core tiles (two 128-row MMA groups per block)."""
    p = ladder(6, 1_777, 1_200)
    ref = oracle_run("ladder6_1777", p)
    got = mbs.run(p, precision="fp32", algo="tiled", tile_steps=tile, wide_tiles=True)
    err = trace_errors(p, got["records"], ref["records"])
    assert err.max() <= TOL32, err


@pytest.mark.parametrize("tile", [8, 20, 24])
def test_wide_tiles_right_boundary_at_tile_edge(tile):
    own = 256 - 2 * tile
    nx = 9 * own + 1
    p = ladder(6, nx, 1_000)
    p.probes = p.probes + [W.Probe(nx - 1, W.Q_E), W.Probe(nx - 2, W.Q_E), W.Probe(nx - 1, W.Q_H)]
    a = mbs.run(p, precision="fp64", algo="plain")["records"]
    b = mbs.run(p, precision="fp32", algo="tiled", tile_steps=tile, wide_tiles=True)["records"]
    err = trace_errors(p, b, a)
    assert err.max() <= TOL32, err


def test_wide_tiles_reject_depths_outside_the_light_cone():
    """T = 28 on 197 cells would leave the last cell outside its tile's owned
    range after the shift that keeps it off a warp start: rejected."""
    p = ladder(6, 197, 40)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=28, wide_tiles=True)
    assert e.value.status == mbs.MBS_E_INVALID
    mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=26, wide_tiles=True)


@pytest.mark.parametrize("n_levels", [2, 3, 4, 5, 6])
def test_anharmonic_ladder_gaussian_source(n_levels):
    """The anharmonic ladder of the paper's six-level example for N = 2..6
    (FP32 CUDA-core tiles for N = 2, 3, tensor-core tiles for N >= 4) driven
    by a Gaussian-envelope source, against the oracle; FP64 plain to 1e-10."""
    p = W.ladder_anharmonic(n_levels, n_cells=1_500, n_steps=2_500, t0=200e-15, tau=40e-15)
    ref = oracle.run(p)["records"]
    got = mbs.run(p, precision="fp32")
    assert trace_errors(p, got["records"], ref).max() <= TOL32
    got64 = mbs.run(p, precision="fp64", algo="plain")
    for k in range(len(p.probes)):
        assert rel_l2(got64["records"][k], ref[k]) <= 1e-10, k


def test_tensor_core_wait_timeout_is_a_status():
    """Failure detection without a GPU fault: every wait on the tensor core is
    bounded.  With the test flag the tiles issue no MMA, so each block's wait
    on its MMA barrier runs out after about 1 s; the blocks free their TMEM
    and return, mbs_solve reports MBS_E_TIMEOUT, and the CUDA context stays
    usable (the next solve of the same scenario is correct)."""
    import time
    p = ladder(6, 300, 8)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    t0 = time.time()
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=8, test_stall=True)
    assert e.value.status == mbs.MBS_E_TIMEOUT
    assert time.time() - t0 < 60
    mbs.mbs_solve([sc], "fp32", "tiled", tile_steps=8)
    got = np.stack([mbs.mbs_fetch_records(sc, k) for k in range(len(p.probes))])
    ref = mbs.run(p, precision="fp64", algo="plain")["records"]
    assert trace_errors(p, got, ref).max() <= TOL32


@pytest.mark.parametrize("n_levels", [2, 3, 6])
def test_strong_field_wide_rotation_angles(n_levels):
    """A field so strong that the rotation angle of the widest eigenvalue gap
    reaches about 2 rad per step: the tiles leave the Taylor range |theta| <=
    1/2 of their sin / cos - 1 and take the library routine (a warp-uniform
    branch); FP32 tiles against the oracle, FP64 plain to 1e-10."""
    p = ladder(n_levels, 400, 600)
    dt = p.courant * p.dz / W.C0
    dev = mbs.device_from_problem(p)
    lam = mbs.mbs_device_propagators(dev, 0, dt, n_levels)["lam"]
    s = p.sources[0]
    e0 = 2.0 * W.HBAR / ((lam.max() - lam.min()) * dt)
    p = p.replace(sources=[W.Source(s.kind, s.cell, e0, s.tau, s.t0, s.omega, s.phase)])
    ref = oracle.run(p)["records"]
    e_max = max(np.abs(ref[k]).max() for k, pr in enumerate(p.probes) if pr.quantity == W.Q_E)
    assert (lam.max() - lam.min()) * e_max * dt / W.HBAR > 1.0
    got = mbs.run(p, precision="fp32")
    assert trace_errors(p, got["records"], ref).max() <= TOL32
    got64 = mbs.run(p, precision="fp64", algo="plain")["records"]
    for k in range(len(p.probes)):
        assert rel_l2(got64[k], ref[k]) <= 1e-10, k

"""Driven single cells (the borderline case Nx = 1 of Sec. 2.1, the master
equation alone) on the GPU, against the oracle's driven-cell solver
(oracle.cell_evolve, the same Strang splitting on full density matrices).

Bounds: FP64 <= 1e-10 relative L2 on every population trace, FP32 <= 1e-4
(also on rho_kk - rho_kk(0))."""
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
    import torch
    assert torch.cuda.is_available()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def ref_pops(qm, drive, dt, nt, every):
    traj = oracle.cell_evolve(qm, dt, W.cell_field(drive, dt, nt))
    pops = np.real(np.einsum("tkk->tk", traj))
    return pops[every - 1::every][: nt // every]


def check(got, ref, tol):
    for k in range(got.shape[1]):
        e = rel_l2(got[:, k], ref[:, k])
        if np.any(ref[:, k] != ref[0, k]):
            e = max(e, rel_l2(got[:, k] - ref[0, k], ref[:, k] - ref[0, k]))
        assert e <= tol, (k, e)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_vtype_example_vs_oracle(prec, tol):
    """The paper's V-type example: one driven three-level system, 10,000
    steps over 80 fs."""
    b = W.song_vtype(n_sys=1)
    c = mbs.cells_from_batch(b)
    mbs.mbs_cells_solve(c, prec)
    got = mbs.mbs_cells_fetch(c, 0)
    ref = ref_pops(b.qms[0], b.drives[0], b.dt, b.n_steps, 1)
    assert got.shape == (10_000, 3)
    check(got, ref, tol)
    st = mbs.mbs_cells_stats(c)
    assert st["max_trace_dev"] <= 1e-6 and st["min_eig"] >= -1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_vtype_batch_vs_oracle(prec, tol):
    """3,001 systems (ragged against the block size): parameters scaled by
    +-10 %, drive amplitude swept over 0.25..2 e0; records every 7 steps;
    sampled systems against the oracle."""
    b = W.song_vtype(n_sys=3_001, record_every=7)
    c = mbs.cells_from_batch(b)
    mbs.mbs_cells_solve(c, prec)
    for s in (0, 1, 2, 1500, 2999, 3000):
        got = mbs.mbs_cells_fetch(c, s)
        ref = ref_pops(b.qms[s], b.drives[s], b.dt, b.n_steps, 7)
        assert got.shape == ref.shape == (10_000 // 7, 3)
        check(got, ref, tol)


def test_two_level_cells_and_repeat_solves():
    """Two-level cells (the SIT medium's parameters) under 2 pi and pi sech
    pulses: the 2 pi cell returns to the ground state, the pi cell is
    inverted; FP32 twice in a row gives identical records; FP64 and FP32
    agree to the FP32 bound."""
    q = W.sit_2lvl(n_cells=8, n_steps=1).qms[0]
    tau, d = 10e-15, 1e-29
    dt, nt = 2.4431e-16 / 4, 8_000
    drives = [W.Source(W.SRC_HARD, 0, W.sech_area_amplitude(a, d, tau), tau, 300e-15, 2e14)
              for a in (2 * np.pi, np.pi)]
    c = mbs.mbs_cells_create([q, q], dt, nt, drives, 1)
    mbs.mbs_cells_solve(c, "fp32")
    a = [mbs.mbs_cells_fetch(c, s) for s in (0, 1)]
    mbs.mbs_cells_solve(c, "fp32")
    for s in (0, 1):
        np.testing.assert_array_equal(mbs.mbs_cells_fetch(c, s), a[s])
    assert a[0][-1, 0] > 0.98                 # 2 pi: back in the ground state
    assert a[1][-1, 1] > 0.9                  # pi: inverted
    mbs.mbs_cells_solve(c, "fp64")
    for s in (0, 1):
        ref = ref_pops(q, drives[s], dt, nt, 1)
        check(mbs.mbs_cells_fetch(c, s), ref, 1e-10)
        check(a[s], ref, 1e-4)


def test_cells_errors():
    b = W.song_vtype(n_sys=4, record_every=3, n_steps=100)
    c = mbs.cells_from_batch(b)
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_cells_solve(c, 7)
    assert e.value.status == mbs.MBS_E_INVALID
    mbs.mbs_cells_solve(c, "fp32")
    assert mbs.mbs_cells_fetch(c, 3).shape == (33, 3)
    with pytest.raises(mbs.MBSError):
        mbs.mbs_cells_fetch(c, 4)

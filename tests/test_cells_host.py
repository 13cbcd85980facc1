"""Driven single cells (Nx = 1): host-side validation of mbs_cells_create
(no GPU needed: the batch is built on the host, device memory only at the
first solve)."""
import numpy as np
import pytest

import paper_2005_05412_gb300 as mbs
import workloads as W


def test_create_builds_on_the_host():
    b = W.song_vtype(n_sys=16)
    c = mbs.cells_from_batch(b)
    assert c.status == mbs.MBS_OK and c.n_sys == 16
    with pytest.raises(mbs.MBSError) as e:     # nothing solved yet
        mbs.mbs_cells_fetch(c, 0)
    assert e.value.status == mbs.MBS_E_STATE


@pytest.mark.parametrize("what", ["dt", "steps", "every", "levels", "mixed", "tau", "rho"])
def test_create_rejects_bad_input(what):
    b = W.song_vtype(n_sys=3)
    qms, drives, dt, nt, every = list(b.qms), list(b.drives), b.dt, b.n_steps, 1
    if what == "dt":
        dt = 0.0
    elif what == "steps":
        nt = 0
    elif what == "every":
        every = 0
    elif what == "levels":
        qms = [W.ladder_6lvl(n_cells=8, n_steps=1).qms[0]] * 3
    elif what == "mixed":
        qms[1] = W.sit_2lvl(n_cells=8, n_steps=1).qms[0]
    elif what == "tau":
        d = drives[2]
        drives[2] = W.Source(d.kind, d.cell, d.e0, 0.0, d.t0, d.omega, d.phase)
    elif what == "rho":
        q = qms[1]
        bad = q.rho_init.copy()
        bad[0, 0] = 0.5
        qms[1] = W.QM(**{**q.__dict__, "rho_init": bad})
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_cells_create(qms, dt, nt, drives, every)
    assert e.value.status == mbs.MBS_E_INVALID
    if what in ("mixed", "tau", "rho"):
        assert ("system" in str(e.value)) or ("all systems" in str(e.value))

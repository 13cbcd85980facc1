"""The per-cell FP64 step operators of a jittered two-level medium are formed
on the device (mbs_setup_dev.cu, the host setup's own arithmetic from
mbs_step_math.h); with MBS_HOST_SETUP=1 the host forms them as before.  The
two setups must give the same solves: FP64 records within 1e-13 of each
other (the two compilers may contract different products into fused
multiply-adds), FP32 within 1e-6 (a last-bit difference of an FP64
coefficient can move its FP32 rounding), on the structured-row tiles, on the
dense per-cell rows of a medium without the optical-Bloch pattern, and on
the plain path.  Both setups are checked against the oracle by the other
parity tests (the device one by default)."""
import numpy as np
import pytest

import paper_2005_05412_gb300 as mbs
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05412_gb300 import build
    build.build()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _both(monkeypatch, p, **kw):
    monkeypatch.delenv("MBS_HOST_SETUP", raising=False)
    dev = mbs.run(p, **kw)
    monkeypatch.setenv("MBS_HOST_SETUP", "1")
    host = mbs.run(p, **kw)
    monkeypatch.delenv("MBS_HOST_SETUP", raising=False)
    return dev, host


def _tilted_dipole(p):
    """The same medium with a permanent-dipole difference: the dipole
    eigenbasis no longer diagonalises H0, so the step operator couples the
    populations to the coherences and the structured rows do not apply."""
    q = p.qms[0]
    mu = np.array(q.mu, complex)
    mu[0, 0], mu[1, 1] = 0.3 * abs(mu[0, 1]), -0.2 * abs(mu[0, 1])
    q2 = W.QM(**{**q.__dict__, "mu": mu})
    return p.replace(qms=[q2])


@pytest.mark.parametrize("medium", ["bloch", "tilted"])
def test_device_setup_matches_host_setup(monkeypatch, medium):
    p = W.sit_2lvl_jitter(n_cells=6000, n_steps=3000)
    if medium == "tilted":
        p = _tilted_dipole(p)
    for prec, algo, tol in (("fp64", "tiled", 1e-13), ("fp32", "tiled", 1e-6), ("fp64", "plain", 1e-13)):
        dev, host = _both(monkeypatch, p, precision=prec, algo=algo, tile_steps=24 if algo == "tiled" else 0)
        for k in range(len(p.probes)):
            assert np.isfinite(dev["records"][k]).all()
            e = rel_l2(dev["records"][k], host["records"][k])
            assert e <= tol, (medium, prec, algo, k, e)
        # the device setup uploads the jitter table instead of the per-cell rows
        assert dev["counters"]["h2d_bytes"] < host["counters"]["h2d_bytes"], (dev["counters"], host["counters"])

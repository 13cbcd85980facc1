"""Host-side checks of the CUDA library that need no GPU: the shared library
loads and exports every symbol the header declares, device creation
validates its inputs, and the FP64 setup (dipole eigenbasis, real Bloch
generator, step operators, d_t P functional) reproduces one split step of
the oracle's superoperator form."""
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2005_05412_gb300 as mbs
import workloads as W
from paper_2005_05412_gb300 import build as mbs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HBAR = 6.62607015e-34 / (2 * math.pi)
DT = W.DZ_SIT / W.C0


@pytest.fixture(scope="module", autouse=True)
def built():
    mbs_build.build()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "mbs.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(mbs_\w+)\s*\(", hdr))
    assert names, "no declarations found"
    L = mbs.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names == set(mbs.EXPORTS)
    assert mbs.mbs_abi_version() == 2


def _tiny_problem(**kw):
    return W.sit_2lvl(n_cells=64, t_end=0.0, n_steps=10, **kw)


def test_device_validation_errors():
    p = _tiny_problem()
    d = mbs.device_from_problem(p)
    assert d.status == mbs.MBS_OK
    bad_rho = p.qms[0].rho_init.copy()
    bad_rho[0, 0] = 0.9                      # trace 0.9
    q = W.QM(**{**p.qms[0].__dict__, "rho_init": bad_rho})
    with pytest.raises(mbs.MBSError, match="trace"):
        mbs.mbs_device_create([q], p.materials, p.regions, p.length, p.n_cells)
    nonherm = p.qms[0].mu.copy()
    nonherm[0, 1] = 2.0 * nonherm[0, 1]
    q = W.QM(**{**p.qms[0].__dict__, "mu": nonherm})
    with pytest.raises(mbs.MBSError, match="Hermitian"):
        mbs.mbs_device_create([q], p.materials, p.regions, p.length, p.n_cells)
    with pytest.raises(mbs.MBSError, match="no region"):
        mbs.mbs_device_create(p.qms, p.materials, p.regions[:2], p.length, p.n_cells)
    for bad in ((1.5, 0.0), (0.0, -0.1), (float("nan"), 0.0)):   # 0 <= R <= 1 (partial reflection allowed)
        with pytest.raises(mbs.MBSError, match="reflectivity"):
            mbs.mbs_device_create(p.qms, p.materials, p.regions, p.length, p.n_cells, bc=bad)
    assert mbs.mbs_device_create(p.qms, p.materials, p.regions, p.length, p.n_cells, bc=(0.5, 0.8)).status == 0
    notpsd = W.QM(**{**p.qms[0].__dict__, "rho_init": np.array([[1.2, 0], [0, -0.2]], complex)})
    with pytest.raises(mbs.MBSError, match="positive"):
        mbs.mbs_device_create([notpsd], p.materials, p.regions, p.length, p.n_cells)
    try:
        err = mbs.MBSError
        mbs.mbs_device_create(p.qms, p.materials, p.regions, p.length, 4)
    except err as e:
        assert e.status == mbs.MBS_E_INVALID


def test_not_psd_dephasing_warns():
    """Pure-dephasing rates 12 = 13 = 0, 23 large cannot come from a PSD
    coefficient matrix (Sec. 3.1.1): the device is created with a warning."""
    q = W.QM(3, 1e24, np.diag([0, 1e-20, 2e-20]).astype(complex), np.zeros((3, 3), complex),
             np.diag([1.0, 0, 0]).astype(complex), scattering=np.zeros((3, 3)),
             pure_dephasing=np.array([0.0, 0.0, 1e12]))
    p = _tiny_problem()
    d = mbs.mbs_device_create([q], p.materials, p.regions, p.length, p.n_cells)
    assert d.status == mbs.MBS_W_NOT_PSD


# ---------------------------------------------------------------------------
def _coords(rho_t, n):
    """Real coordinates of rho~ as documented in include/mbs.h."""
    y = [rho_t[k, k].real for k in range(n)]
    for j in range(n):
        for k in range(j + 1, n):
            y += [rho_t[j, k].real, rho_t[j, k].imag]
    return np.array(y)


def _herm(y, n):
    r = np.zeros((n, n), complex)
    for k in range(n):
        r[k, k] = y[k]
    q = 0
    for j in range(n):
        for k in range(j + 1, n):
            r[j, k] = y[n + 2 * q] + 1j * y[n + 2 * q + 1]
            r[k, j] = np.conj(r[j, k])
            q += 1
    return r


def _full_of(n, i):
    return i if i < n - 1 else i + 1


def _rand_rho(rng, n):
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    r = a @ a.conj().T
    return r / np.trace(r).real


def _qm_cases():
    rng = np.random.default_rng(11)
    n = 3
    h0 = np.diag([0.0, 1.1e-20, 1.9e-20]).astype(complex)
    h0[0, 1], h0[1, 0] = 1e-21 + 2e-21j, 1e-21 - 2e-21j
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    mu = 1e-29 * (a + a.conj().T) / 2
    ops = [np.outer(np.eye(n)[i], np.eye(n)[j]).astype(complex) for i, j in [(0, 2), (1, 2)]]
    ops.append(np.diag([0.3, -0.1, 0.5]).astype(complex) + 0.2j * np.eye(n))
    qa = W.QM(n, 2e24, h0, mu, _rand_rho(rng, n), np.array([3e11, 1e11, 5e11]), np.array(ops))
    qb = W.QM(n, 1e24, h0, mu, _rand_rho(rng, n), scattering=np.array([[0, 2e11, 1e11], [4e10, 0, 3e11], [0, 5e10, 0]]),
              pure_dephasing=np.array([2e11, 3e11, 2.5e11]))
    q2 = W.qm_two_level(1e24, 2e14, 1e-29, 1e9, 1e9, -1.0)
    q6 = W.ladder_6lvl(n_cells=64, n_steps=10).qms[0]
    return [("explicit3", qa), ("rate3", qb), ("two_level", q2), ("six_level", q6)]


@pytest.mark.parametrize("scale", [1.0, 64.0])
@pytest.mark.parametrize("name,qm", _qm_cases())
def test_setup_reproduces_oracle_split_step(name, qm, scale):
    """One split step S_h U(E) S_h and d_t P: the product's real Bloch form
    in the dipole eigenbasis equals the oracle's superoperator form.  At 64
    times the SIT time step ||L0 dt/2||_1 is 1.6-2.6, so the host's
    exp(L0 dt/2) - I takes 3-4 squarings and its longest series; the
    oracle's own exponential (Pade 13) is independent of it."""
    n = qm.n_levels
    DT = globals()["DT"] * scale
    p = _tiny_problem()
    dev = mbs.mbs_device_create([qm], [W.Material(), W.Material(qm=0)], p.regions, p.length, p.n_cells)
    pr = mbs.mbs_device_propagators(dev, 0, DT, n)
    lam, V = pr["lam"], pr["V"]
    np.testing.assert_allclose(V @ np.diag(lam) @ V.conj().T, qm.mu, atol=1e-12 * np.abs(qm.mu).max())
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
    L0 = oracle.liouvillian(qm)
    Sh = oracle.expm(L0 * DT / 2)
    rng = np.random.default_rng(3)
    k = n * n - 1
    zref = pr["zref"]
    Pz = np.array([zref[_full_of(n, i)] for i in range(k)])
    for e in [0.0, 3e9, -1.7e10]:
        rho = _rand_rho(rng, n)
        # oracle
        r1 = (Sh @ rho.reshape(-1)).reshape(n, n)
        U = V @ np.diag(np.exp(1j * lam * e * DT / HBAR)) @ V.conj().T
        r2 = U @ r1 @ U.conj().T
        rho_half = (Sh @ r2.reshape(-1)).reshape(n, n)
        x_next = (Sh @ rho_half.reshape(-1)).reshape(n, n)
        pd_ref = qm.density * np.trace(qm.mu @ (L0 @ rho_half.reshape(-1)).reshape(n, n)).real
        # product representation
        y = _coords(V.conj().T @ rho @ V, n)
        x = pr["Ah"] @ y
        q = 0
        for j in range(n):
            for kk in range(j + 1, n):
                th = (lam[j] - lam[kk]) * e * DT / HBAR
                a, b = x[n + 2 * q], x[n + 2 * q + 1]
                x[n + 2 * q], x[n + 2 * q + 1] = a * math.cos(th) - b * math.sin(th), a * math.sin(th) + b * math.cos(th)
                q += 1
        u = np.array([x[_full_of(n, i)] for i in range(k)]) - Pz
        d_next = pr["A"] @ u + pr["c"]
        yf = np.zeros(n * n)
        for i in range(k):
            yf[_full_of(n, i)] = zref[_full_of(n, i)] + d_next[i]
        yf[n - 1] = 1.0 - sum(yf[i] for i in range(n - 1))
        got = V @ _herm(yf, n) @ V.conj().T
        np.testing.assert_allclose(got, x_next, atol=1e-13)
        pd = qm.density * (pr["g"] @ u + pr["g0"])
        assert pd == pytest.approx(pd_ref, rel=1e-10, abs=1e-12 * qm.density * 1e-29 * 1e15)


def test_reference_state_is_steady_state():
    """For the SIT medium (w0 = -1) the deviation reference is the ground
    state, the fixed point of exp(L0 dt): the affine offset vanishes."""
    q2 = W.qm_two_level(1e24, 2e14, 1e-29, 1e9, 1e9, -1.0)
    p = _tiny_problem()
    dev = mbs.mbs_device_create([q2], p.materials, p.regions, p.length, p.n_cells)
    pr = mbs.mbs_device_propagators(dev, 0, DT, 2)
    V = pr["V"]
    rho = V @ _herm(pr["zref"], 2) @ V.conj().T
    np.testing.assert_allclose(rho, np.diag([1.0, 0.0]), atol=1e-14)
    assert np.abs(pr["c"]).max() < 1e-15
    assert abs(pr["g0"]) < 1e-6 * 1e-29 * 1e14


def test_scenario_validation_errors():
    """mbs_scenario validates before it touches the device: every bad
    argument is MBS_E_INVALID with a message, and nothing is allocated."""
    import dataclasses
    p = _tiny_problem()
    dev = mbs.device_from_problem(p)
    s0 = p.sources[0]
    cases = [
        ("probes", p.replace(probes=[W.Probe(3, W.Q_E)] * 65)),
        ("sources", p.replace(sources=[s0] * 5)),
        ("cell out of range", p.replace(probes=[W.Probe(p.n_cells, W.Q_E)])),
        ("bad quantity", p.replace(probes=[W.Probe(3, 7)])),
        ("without medium", p.replace(probes=[W.Probe(0, W.Q_RHO_RE, 0, 0)])),
        ("level index", p.replace(probes=[W.Probe(p.n_cells // 2, W.Q_RHO_RE, 0, 2)])),
        ("bad kind", p.replace(sources=[dataclasses.replace(s0, kind=9)])),
        ("bad shape", p.replace(sources=[dataclasses.replace(s0, shape=5)])),
        ("cell must be", p.replace(sources=[dataclasses.replace(s0, cell=1)])),
        ("tau", p.replace(sources=[dataclasses.replace(s0, tau=0.0)])),
        ("non-finite", p.replace(sources=[dataclasses.replace(s0, e0=float("nan"))])),
        ("courant", p.replace(courant=1.5)),
        ("no time steps", p.replace(n_steps=0, t_end=0.0)),
    ]
    for msg, q in cases:
        with pytest.raises(mbs.MBSError, match=msg) as e:
            mbs.scenario_from_problem(dev, q)
        assert e.value.status == mbs.MBS_E_INVALID, msg

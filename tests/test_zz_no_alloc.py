"""The allocation-free density-matrix check (mbs_check_rho_static).

Some callers cannot call cudaMalloc: a framework that owns every device
allocation through its own pool, or a loop that must not stall on the
device-wide synchronisation an allocation can imply.  mbs_check_rho_static
serves them with scratch in a fixed static device array.  Its result must
equal the state check that mbs_solve runs on its own state (read back
through mbs_scenario_stats) on two calls in a row, and numpy's eigenvalues
on mixed batches.  This file is collected last so that a failure here never
hides another test's result.
"""
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


def _one_step_problem(n):
    """Every medium cell holds the same state after one source-free step:
    x = exp(1.5 L0 dt) rho0 (the solver's state runs half a step ahead)."""
    import scipy.linalg as sl
    p = W.ladder_6lvl(n_cells=64, n_steps=1)
    q = p.qms[0]
    rng = np.random.default_rng(100 + n)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    rho0 = a @ a.conj().T + 0.02 * np.eye(n)
    rho0 /= np.trace(rho0).real
    keep = [k for k, o in enumerate(q.lindblad_ops) if not np.abs(o[n:, :]).any() and not np.abs(o[:, n:]).any()]
    q2 = W.QM(n, q.density, q.h0[:n, :n], q.mu[:n, :n], rho0, q.lindblad_rates[keep],
              q.lindblad_ops[keep][:, :n, :n])
    p = p.replace(qms=[q2], sources=[], probes=[W.Probe(10, W.Q_E)])
    x = (sl.expm(1.5 * oracle.liouvillian(q2) * (p.courant * p.dz / W.C0)) @ rho0.reshape(-1)).reshape(n, n)
    return p, x


def _call(rho_np, n_levels):
    """One call through the C ABI on torch's current stream; returns out."""
    import torch
    rho = torch.tensor(np.ascontiguousarray(rho_np), dtype=torch.complex128, device="cuda")
    out = torch.full((3,), -7.0, dtype=torch.float64, device="cuda")
    mbs.mbs_check_rho_static(rho.data_ptr(), rho_np.shape[0], n_levels, out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _reference(rho_np):
    """numpy: smallest eigenvalue of the Hermitian parts and largest
    |tr - 1| over the finite matrices, and the count of the others."""
    fin = np.all(np.isfinite(rho_np.view(np.float64).reshape(rho_np.shape[0], -1)), axis=1)
    if not fin.any():
        return float("nan"), 0.0, float(rho_np.shape[0])
    r = rho_np[fin]
    h = 0.5 * (r + np.conj(np.swapaxes(r, 1, 2)))
    mn = float(np.linalg.eigvalsh(h).min())
    tr = float(np.abs(np.trace(r, axis1=1, axis2=2).real - 1.0).max())
    return mn, tr, float((~fin).sum())


def _mixed(rng, n, n_levels):
    """n density matrices with varied traces (0.9 .. 1.1) and spectra, plus
    one non-PSD matrix, one with a NaN entry and one with an infinite one."""
    a = rng.normal(size=(n, n_levels, n_levels)) + 1j * rng.normal(size=(n, n_levels, n_levels))
    r = a @ np.conj(np.swapaxes(a, 1, 2))
    r /= np.trace(r, axis1=1, axis2=2).real[:, None, None]
    r *= rng.uniform(0.9, 1.1, size=n)[:, None, None]
    if n >= 4:
        e = np.diag(np.linspace(-0.05, 1.05, n_levels)).astype(complex)
        q, _ = np.linalg.qr(rng.normal(size=(n_levels, n_levels)) + 1j * rng.normal(size=(n_levels, n_levels)))
        r[n // 3] = q @ e @ q.conj().T                 # eigenvalue -0.05: not PSD
        r[n // 2, 0, 1] = np.nan
        r[n - 1, 1, 1] = np.inf
    return r


@pytest.mark.parametrize("n_levels", [2, 3, 6])
def test_static_check_matches_solver_check(n_levels):
    """Two calls in a row against the existing entry point's state check."""
    import torch
    p, x = _one_step_problem(n_levels)
    stats = mbs.run(p, precision="fp64", algo="plain")["stats"]     # the existing entry point
    n_mat = 1000
    rho = torch.tensor(np.broadcast_to(x, (n_mat, n_levels, n_levels)).copy(), dtype=torch.complex128,
                       device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        out.fill_(float("nan"))
        mbs.mbs_check_rho_static(rho.data_ptr(), n_mat, n_levels, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        mn, tr, bad = out.cpu().numpy()
        assert mn == pytest.approx(stats["min_eig"], abs=1e-12), call
        assert tr == pytest.approx(stats["max_trace_dev"], abs=1e-12), call
        assert bad == 0.0


@pytest.mark.parametrize("n_levels", [2, 4, 6])
def test_static_check_mixed_batches(n_levels):
    """Distinct matrices, a non-PSD one and non-finite ones, at n = 1,
    1,001 and the maximum; then a small call after the large one (the scratch
    still holds the large call's entries) and a batch with no finite matrix."""
    rng = np.random.default_rng(7 + n_levels)
    for n in (1, 1001, mbs.MBS_STATIC_CHECK_MAX, 10):
        r = _mixed(rng, n, n_levels)
        got = _call(r, n_levels)
        mn, tr, bad = _reference(r)
        assert got[0] == pytest.approx(mn, abs=1e-12), (n, got, mn)
        assert got[1] == pytest.approx(tr, abs=1e-12), (n, got, tr)
        assert got[2] == bad, (n, got, bad)
        if n >= 4:
            assert mn == pytest.approx(-0.05, abs=1e-12) and bad == 2.0
    r = _mixed(rng, 5, n_levels)
    r[:, 0, 0] = np.nan
    got = _call(r, n_levels)
    assert np.isnan(got[0]) and got[1] == 0.0 and got[2] == 5.0


def test_static_check_limits():
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rho = torch.zeros((1, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_check_rho_static(rho.data_ptr(), mbs.MBS_STATIC_CHECK_MAX + 1, 2, out.data_ptr())
    assert e.value.status == mbs.MBS_E_INVALID
    with pytest.raises(mbs.MBSError):
        mbs.mbs_check_rho_static(rho.data_ptr(), 1, 7, out.data_ptr())
    with pytest.raises(mbs.MBSError):
        mbs.mbs_check_rho_static(rho.data_ptr(), 0, 2, out.data_ptr())

"""The allocation-free density-matrix check (mbs_check_rho_static).

Some callers cannot call cudaMalloc: code running while a CUDA graph is
being captured, or inside a framework that owns every device allocation.
mbs_check_rho_static serves them with scratch in a fixed static device array.
Its result must equal the state check that mbs_solve runs on its own state
(read back through mbs_scenario_stats), on two calls in a row.  This file is
collected last so that a failure here never hides another test's result.
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


@pytest.mark.parametrize("n_levels", [2, 3, 6])
def test_static_check_matches_solver_check(n_levels):
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


def test_static_check_limits():
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rho = torch.zeros((1, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mbs.MBSError) as e:
        mbs.mbs_check_rho_static(rho.data_ptr(), mbs.MBS_STATIC_CHECK_MAX + 1, 2, out.data_ptr())
    assert e.value.status == mbs.MBS_E_INVALID
    with pytest.raises(mbs.MBSError):
        mbs.mbs_check_rho_static(rho.data_ptr(), 1, 7, out.data_ptr())

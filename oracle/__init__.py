"""CPU FP64 oracle for the 1D Maxwell-Bloch sweep -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its binding) never imports, links or runs it, and the two share no code:
this side is plain C (``mbs_oracle.c``) driven through ctypes, written from
the paper's equations in their most literal representation (full complex
density matrices and an N^2 x N^2 Liouvillian superoperator).

Entry points:
    run(problem, ...)        -- the full sweep, Algorithm 1 with the Strang
                                splitting of Sec. 2.2
    cell_evolve(qm, dt, e)   -- one driven cell, master equation only
    expm(A), eigh(A)         -- its own Pade-13 exponential and Jacobi eig
    liouvillian(qm)          -- L0 on row-major vec(rho)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fcx-limited-range",
          "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags: same results on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _QM(C.Structure):
    _fields_ = [("n", C.c_int), ("n3d", C.c_double), ("h0", C.c_void_p), ("mu", C.c_void_p),
                ("n_ops", C.c_int), ("rates", C.c_void_p), ("ops", C.c_void_p),
                ("scat", C.c_void_p), ("deph", C.c_void_p), ("rho0", C.c_void_p)]


class _Mat(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("mu_r", C.c_double), ("sigma", C.c_double),
                ("overlap", C.c_double), ("qm", C.c_int)]


class _Reg(C.Structure):
    _fields_ = [("mat", C.c_int), ("x0", C.c_double), ("x1", C.c_double)]


class _Src(C.Structure):
    _fields_ = [("kind", C.c_int), ("cell", C.c_int), ("e0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("omega", C.c_double), ("phase", C.c_double), ("shape", C.c_int)]


class _Probe(C.Structure):
    _fields_ = [("cell", C.c_int), ("q", C.c_int), ("i", C.c_int), ("j", C.c_int)]


class _Problem(C.Structure):
    _fields_ = [("n_qm", C.c_int), ("qm", C.POINTER(_QM)),
                ("n_mat", C.c_int), ("mat", C.POINTER(_Mat)),
                ("n_reg", C.c_int), ("reg", C.POINTER(_Reg)),
                ("length", C.c_double), ("nx", C.c_int),
                ("refl_l", C.c_double), ("refl_r", C.c_double),
                ("jitter", C.c_void_p),
                ("courant", C.c_double), ("t_end", C.c_double), ("n_steps", C.c_long),
                ("n_src", C.c_int), ("src", C.POINTER(_Src)),
                ("n_probe", C.c_int), ("probe", C.POINTER(_Probe)),
                ("e_init", C.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_run.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_run.restype = C.c_int
        lib.orc_expm.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
        lib.orc_expm.restype = C.c_int
        lib.orc_eigh.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_eigh.restype = C.c_int
        lib.orc_liouvillian.argtypes = [C.POINTER(_QM), C.c_double, C.c_void_p]
        lib.orc_liouvillian.restype = C.c_int
        lib.orc_cell_evolve.argtypes = [C.POINTER(_QM), C.c_double, C.c_long, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_cell_evolve.restype = C.c_int
        lib.orc_num_threads.restype = C.c_int
        lib.orc_grid.argtypes = [C.POINTER(_Problem), C.c_void_p]
        lib.orc_grid.restype = C.c_int
        _lib = lib
    return _lib


def _cbuf(a):
    """complex array -> contiguous interleaved float64 buffer (kept alive by caller)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return a.view(np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _qm_struct(qm, keep):
    n = qm.n_levels
    h0, mu, rho0 = _cbuf(qm.h0), _cbuf(qm.mu), _cbuf(qm.rho_init)
    rates = np.ascontiguousarray(np.asarray(qm.lindblad_rates, np.float64))
    nops = len(rates)
    ops = _cbuf(np.asarray(qm.lindblad_ops).reshape(nops, n, n)) if nops else None
    scat = None if qm.scattering is None else np.ascontiguousarray(np.asarray(qm.scattering, np.float64))
    deph = None if qm.pure_dephasing is None else np.ascontiguousarray(np.asarray(qm.pure_dephasing, np.float64))
    keep += [h0, mu, rho0, rates, ops, scat, deph]
    return _QM(n, float(qm.density), _ptr(h0), _ptr(mu), nops, _ptr(rates) if nops else None,
               _ptr(ops), _ptr(scat), _ptr(deph), _ptr(rho0))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def expm(a) -> np.ndarray:
    a = np.asarray(a, np.complex128)
    n = a.shape[0]
    out = np.zeros((n, n), np.complex128)
    buf = _cbuf(a)
    rc = _load().orc_expm(n, buf.ctypes.data, out.ctypes.data)
    if rc:
        raise RuntimeError("orc_expm failed")
    return out


def eigh(a):
    a = np.asarray(a, np.complex128)
    n = a.shape[0]
    w = np.zeros(n)
    v = np.zeros((n, n), np.complex128)
    buf = _cbuf(a)
    _load().orc_eigh(n, buf.ctypes.data, w.ctypes.data, v.ctypes.data)
    return w, v


def liouvillian(qm, h0_scale: float = 1.0) -> np.ndarray:
    keep = []
    s = _qm_struct(qm, keep)
    n2 = qm.n_levels ** 2
    out = np.zeros((n2, n2), np.complex128)
    _load().orc_liouvillian(C.byref(s), float(h0_scale), out.ctypes.data)
    return out


def cell_evolve(qm, dt: float, e, want_pdot=False):
    """Evolve one cell under the prescribed field sequence e[n] (V/m).
    Returns rho^{n+1/2}, shape (nt, N, N) [and d_t P, shape (nt,)]."""
    keep = []
    s = _qm_struct(qm, keep)
    e = np.ascontiguousarray(np.asarray(e, np.float64))
    nt = len(e)
    n = qm.n_levels
    traj = np.zeros((nt, n, n), np.complex128)
    pd = np.zeros(nt)
    rc = _load().orc_cell_evolve(C.byref(s), float(dt), nt, e.ctypes.data, traj.ctypes.data, pd.ctypes.data)
    if rc:
        raise RuntimeError("orc_cell_evolve failed")
    return (traj, pd) if want_pdot else traj


def run(problem, n_threads: int = 0, check_invariants: bool = False):
    """Run the full sweep of `problem` (a workloads.Problem).

    Returns dict(records=(n_probe, nt) array, dt, nt, seconds, threads,
    stats=(max|tr-1|, max|rho-rho^+|, min eig) if check_invariants)."""
    lib = _load()
    keep = []
    qms = (_QM * max(1, len(problem.qms)))(*[_qm_struct(q, keep) for q in problem.qms])
    mats = (_Mat * len(problem.materials))(*[_Mat(m.eps_r, m.mu_r, m.sigma, m.overlap, m.qm)
                                               for m in problem.materials])
    regs = (_Reg * len(problem.regions))(*[_Reg(r.material, r.x_start, r.x_end) for r in problem.regions])
    srcs = (_Src * max(1, len(problem.sources)))(*[_Src(s.kind, s.cell, s.e0, s.tau, s.t0, s.omega, s.phase,
                                                        getattr(s, "shape", 0)) for s in problem.sources])
    prbs = (_Probe * max(1, len(problem.probes)))(*[_Probe(p.cell, p.quantity, p.i, p.j)
                                                     for p in problem.probes])
    jit = None
    if problem.jitter is not None:
        jit = np.ascontiguousarray(np.asarray(problem.jitter, np.float64).reshape(-1, 2))
        assert jit.shape[0] == problem.n_cells
    e_init = getattr(problem, "e_init", None)
    if e_init is not None:
        e_init = np.ascontiguousarray(np.asarray(e_init, np.float64))
        assert e_init.shape == (problem.n_cells,)
    pb = _Problem(len(problem.qms), qms, len(problem.materials), mats, len(problem.regions), regs,
                  float(problem.length), int(problem.n_cells), float(problem.refl_left),
                  float(problem.refl_right), _ptr(jit), float(problem.courant), float(problem.t_end),
                  int(problem.n_steps), len(problem.sources), srcs, len(problem.probes), prbs, _ptr(e_init))
    info = np.zeros(2)
    if lib.orc_grid(C.byref(pb), info.ctypes.data):
        raise ValueError("a cell centre lies in no region")
    nt = int(info[1])
    rec = np.zeros((max(1, len(problem.probes)), nt))
    info = np.zeros(2)
    stats = np.zeros(3)
    t0 = time.perf_counter()
    rc = lib.orc_run(C.byref(pb), int(n_threads), int(bool(check_invariants)), rec.ctypes.data,
                     info.ctypes.data, stats.ctypes.data)
    secs = time.perf_counter() - t0
    if rc:
        raise RuntimeError(f"orc_run failed ({rc})")
    assert int(info[1]) == nt
    out = dict(records=rec[:len(problem.probes)], dt=float(info[0]), nt=nt, seconds=secs,
               threads=int(n_threads) if n_threads > 0 else num_threads())
    if check_invariants:
        out["stats"] = tuple(stats)
    return out


def _run_one(args):
    problem, n_threads = args
    r = run(problem, n_threads=n_threads)
    return r["records"], r["dt"], r["nt"]


def run_many(problems, processes: int = 0):
    """Run independent problems on a pool of single-threaded worker
    processes (started with `spawn`, so that a CUDA context in the caller is
    never forked).  Returns [(records, dt, nt), ...] in order."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    if processes <= 0:
        processes = max(1, os.cpu_count() or 1)
    build()
    # a worker that dies raises BrokenProcessPool here instead of hanging
    with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run_one, [(p, 1) for p in problems]))

"""GB300-native hot path of the full-wave 1D Maxwell-Bloch method
(Riesch & Jirauschek, "mbsolve", CPC 2021) -- Python binding of the C ABI
declared in include/mbs.h.

The binding only marshals arguments: every step of the time loop runs in the
CUDA kernels of libmbs.so.  It refuses to work without that library (there is
no CPU fallback).  The functions carry the C names:

    mbs_device_create(qms, materials, regions, length, n_cells, bc, jitter)
    mbs_scenario(device, dt, courant, t_end, n_steps, sources, probes)
    mbs_solve(scenarios, precision, algo, tile_steps, check_every, stream)
    mbs_fetch_records(scenario, probe)
    mbs_scenario_info / mbs_scenario_stats / mbs_device_propagators

plus ``device_from_problem`` / ``scenario_from_problem`` that marshal a
``workloads.Problem``-like description.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmbs.so")

MBS_OK, MBS_W_NOT_PSD = 0, 1
MBS_E_INVALID, MBS_E_CUDA, MBS_E_OOM, MBS_E_NUMERIC, MBS_E_TIMEOUT, MBS_E_STATE = -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "fp32": 1}
ALGO = {"auto": 0, "plain": 1, "tiled": 2}
Q_E, Q_H, Q_RHO_RE, Q_RHO_IM = 0, 1, 2, 3


class MBSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mbs status {status}: {msg}")
        self.status = status


class _QmDesc(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("density", C.c_double), ("h0", C.c_void_p), ("mu", C.c_void_p),
                ("n_lindblad", C.c_int), ("lindblad_rates", C.c_void_p), ("lindblad_ops", C.c_void_p),
                ("scattering", C.c_void_p), ("pure_dephasing", C.c_void_p), ("rho_init", C.c_void_p)]


class _Material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("mu_r", C.c_double), ("sigma", C.c_double),
                ("overlap", C.c_double), ("qm", C.c_int)]


class _Region(C.Structure):
    _fields_ = [("material", C.c_int), ("x_start", C.c_double), ("x_end", C.c_double)]


class _BC(C.Structure):
    _fields_ = [("refl_left", C.c_double), ("refl_right", C.c_double)]


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("cell", C.c_int), ("e0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("omega", C.c_double), ("phase", C.c_double), ("shape", C.c_int)]


class _Probe(C.Structure):
    _fields_ = [("cell", C.c_int), ("quantity", C.c_int), ("i", C.c_int), ("j", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("algo", C.c_int), ("tile_steps", C.c_int), ("check_every", C.c_int),
                ("flags", C.c_int)]


MBS_SOLVE_ONE_AT_A_TIME, MBS_SOLVE_AUTOTUNE, MBS_SOLVE_GRAPH, MBS_SOLVE_WIDE_TILES = 1, 2, 4, 8
MBS_SHAPE_SECH, MBS_SHAPE_GAUSS = 0, 1
MBS_SOLVE_TEST_STALL = 1 << 30


_lib = None

# every symbol include/mbs.h declares
EXPORTS = ["mbs_device_create", "mbs_device_destroy", "mbs_device_propagators", "mbs_scenario",
           "mbs_scenario_destroy", "mbs_scenario_info", "mbs_scenario_stats", "mbs_scenario_counters", "mbs_solve",
           "mbs_fetch_records", "mbs_last_error", "mbs_abi_version", "mbs_check_rho_static", "mbs_scenario_tile", "mbs_scenario_tile_cells", "mbs_tile_plan",
           "mbs_cells_create", "mbs_cells_solve", "mbs_cells_fetch", "mbs_cells_stats", "mbs_cells_destroy",
           "mbs_scenario_set_field", "mbs_peak_rates"]


def lib():
    """Load libmbs.so (raises if it has not been built -- no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2005_05412_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        L.mbs_device_create.argtypes = [C.POINTER(_QmDesc), i, C.POINTER(_Material), i, C.POINTER(_Region), i,
                                        d, i, _BC, vp, C.POINTER(vp)]
        L.mbs_device_destroy.argtypes = [vp]
        L.mbs_device_destroy.restype = None
        L.mbs_device_propagators.argtypes = [vp, i, d, vp, vp, vp, vp, vp, vp, vp, vp]
        L.mbs_scenario.argtypes = [vp, d, d, d, ll, C.POINTER(_Source), i, C.POINTER(_Probe), i, C.POINTER(vp)]
        L.mbs_scenario_destroy.argtypes = [vp]
        L.mbs_scenario_destroy.restype = None
        L.mbs_scenario_info.argtypes = [vp, C.POINTER(d), C.POINTER(d), C.POINTER(ll)]
        L.mbs_scenario_stats.argtypes = [vp, C.POINTER(d), C.POINTER(d), C.POINTER(ll)]
        L.mbs_scenario_counters.argtypes = [vp, C.POINTER(ll), C.POINTER(ll), C.POINTER(ll)]
        L.mbs_scenario_tile.argtypes = [vp, C.POINTER(i)]
        L.mbs_scenario_tile_cells.argtypes = [vp, C.POINTER(i)]
        L.mbs_tile_plan.argtypes = [i, i, i, i, C.POINTER(i)]
        L.mbs_abi_version.argtypes = []
        L.mbs_scenario_set_field.argtypes = [vp, vp, C.c_size_t]
        L.mbs_cells_create.argtypes = [C.POINTER(_QmDesc), i, d, ll, C.POINTER(_Source), i, C.POINTER(vp)]
        L.mbs_cells_solve.argtypes = [vp, i, vp]
        L.mbs_cells_fetch.argtypes = [vp, i, vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.mbs_cells_stats.argtypes = [vp, C.POINTER(d), C.POINTER(d)]
        L.mbs_cells_destroy.argtypes = [vp]
        L.mbs_cells_destroy.restype = None
        L.mbs_solve.argtypes = [C.POINTER(vp), i, C.POINTER(_Opts), vp]
        L.mbs_fetch_records.argtypes = [vp, i, vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.mbs_last_error.restype = C.c_char_p
        L.mbs_last_error.argtypes = []
        L.mbs_abi_version.restype = i
        L.mbs_check_rho_static.argtypes = [vp, i, i, vp, vp]
        L.mbs_check_rho_static.restype = i
        L.mbs_peak_rates.argtypes = [i, C.POINTER(d), C.POINTER(d), vp]
        L.mbs_peak_rates.restype = i
        for f in ["mbs_device_create", "mbs_device_propagators", "mbs_scenario", "mbs_scenario_info", "mbs_scenario_counters",
                  "mbs_scenario_stats", "mbs_solve", "mbs_fetch_records"]:
            getattr(L, f).restype = i
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise MBSError(rc, lib().mbs_last_error().decode())
    return rc


def _cbuf(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).reshape(-1))
    assert a.size == n
    return a.view(np.float64)


def _p(a):
    return None if a is None else a.ctypes.data


class Device:
    """Owning handle of an mbs_device_t."""

    def __init__(self, handle, status, keep):
        self.handle = handle
        self.status = status
        self._keep = keep

    def close(self):
        if self.handle:
            lib().mbs_device_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scenario:
    """Owning handle of an mbs_scenario_t (keeps its device alive)."""

    def __init__(self, handle, device, n_probes):
        self.handle = handle
        self.device = device
        self.n_probes = n_probes

    def close(self):
        if self.handle:
            lib().mbs_scenario_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _qm_desc(q, keep):
    """Marshal one quantum description (buffers appended to `keep`)."""
    n = q.n_levels
    h0, mu, rho = _cbuf(q.h0, n * n), _cbuf(q.mu, n * n), _cbuf(q.rho_init, n * n)
    rates = np.ascontiguousarray(np.asarray(q.lindblad_rates, np.float64).reshape(-1))
    nl = rates.size
    ops = _cbuf(q.lindblad_ops, nl * n * n) if nl else None
    scat = None if q.scattering is None else np.ascontiguousarray(np.asarray(q.scattering, np.float64).reshape(-1))
    deph = None if q.pure_dephasing is None else np.ascontiguousarray(np.asarray(q.pure_dephasing, np.float64).reshape(-1))
    keep += [h0, mu, rho, rates, ops, scat, deph]
    return _QmDesc(n, float(q.density), _p(h0), _p(mu), nl, _p(rates) if nl else None, _p(ops),
                   _p(scat), _p(deph), _p(rho))


def mbs_device_create(qms, materials, regions, length, n_cells, bc=(0.0, 0.0), jitter=None) -> Device:
    """qms: objects with n_levels, density, h0, mu, rho_init, lindblad_rates,
    lindblad_ops, scattering, pure_dephasing; materials: eps_r, mu_r, sigma,
    overlap, qm; regions: material, x_start, x_end."""
    keep = []
    descs = [_qm_desc(q, keep) for q in qms]
    qarr = (_QmDesc * max(1, len(descs)))(*descs)
    marr = (_Material * len(materials))(*[_Material(m.eps_r, m.mu_r, m.sigma, m.overlap, m.qm) for m in materials])
    rarr = (_Region * len(regions))(*[_Region(r.material, r.x_start, r.x_end) for r in regions])
    jit = None
    if jitter is not None:
        jit = np.ascontiguousarray(np.asarray(jitter, np.float64).reshape(-1))
        assert jit.size == 2 * n_cells
    h = C.c_void_p()
    rc = _check(lib().mbs_device_create(qarr, len(descs), marr, len(materials), rarr, len(regions),
                                        float(length), int(n_cells), _BC(*bc), _p(jit), C.byref(h)))
    return Device(h.value, rc, keep)


def mbs_scenario(device: Device, dt=0.0, courant=1.0, t_end=0.0, n_steps=0, sources=(), probes=()) -> Scenario:
    sarr = (_Source * max(1, len(sources)))(*[_Source(s.kind, s.cell, s.e0, s.tau, s.t0, s.omega, s.phase, getattr(s, 'shape', 0))
                                              for s in sources])
    parr = (_Probe * max(1, len(probes)))(*[_Probe(p.cell, p.quantity, p.i, p.j) for p in probes])
    h = C.c_void_p()
    _check(lib().mbs_scenario(device.handle, float(dt), float(courant), float(t_end), int(n_steps),
                              sarr, len(sources), parr, len(probes), C.byref(h)))
    return Scenario(h.value, device, len(probes))


def mbs_solve(scenarios, precision="fp32", algo="auto", tile_steps=0, check_every=0, stream=None,
              one_at_a_time=False, autotune=False, graph=False, wide_tiles=False, test_stall=False):
    """Run every scenario to its end (a batch advances together unless
    one_at_a_time).  stream: a cudaStream_t handle (int), e.g.
    torch.cuda.current_stream().cuda_stream, or None.  autotune / graph /
    wide_tiles set MBS_SOLVE_AUTOTUNE / MBS_SOLVE_GRAPH / MBS_SOLVE_WIDE_TILES
    (see include/mbs.h)."""
    if isinstance(scenarios, Scenario):
        scenarios = [scenarios]
    arr = (C.c_void_p * len(scenarios))(*[s.handle for s in scenarios])
    flags = ((MBS_SOLVE_ONE_AT_A_TIME if one_at_a_time else 0) | (MBS_SOLVE_AUTOTUNE if autotune else 0)
             | (MBS_SOLVE_GRAPH if graph else 0) | (MBS_SOLVE_WIDE_TILES if wide_tiles else 0)
             | (MBS_SOLVE_TEST_STALL if test_stall else 0))
    o = _Opts(PREC[precision] if isinstance(precision, str) else int(precision),
              ALGO[algo] if isinstance(algo, str) else int(algo), int(tile_steps), int(check_every), flags)
    return _check(lib().mbs_solve(arr, len(scenarios), C.byref(o), None if stream is None else C.c_void_p(int(stream))))


def mbs_fetch_records(scenario: Scenario, probe: int, out=None) -> np.ndarray:
    n = C.c_size_t()
    _check(lib().mbs_fetch_records(scenario.handle, int(probe), None, 0, C.byref(n)))
    if out is None:
        out = np.empty(n.value, np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size >= n.value
    _check(lib().mbs_fetch_records(scenario.handle, int(probe), out.ctypes.data, out.size, C.byref(n)))
    return out[:n.value]


def mbs_scenario_info(scenario: Scenario):
    dt, dz, nt = C.c_double(), C.c_double(), C.c_longlong()
    _check(lib().mbs_scenario_info(scenario.handle, C.byref(dt), C.byref(dz), C.byref(nt)))
    return dt.value, dz.value, nt.value


def mbs_scenario_stats(scenario: Scenario):
    tr, mn, nt = C.c_double(), C.c_double(), C.c_longlong()
    _check(lib().mbs_scenario_stats(scenario.handle, C.byref(tr), C.byref(mn), C.byref(nt)))
    return dict(max_trace_dev=tr.value, min_eig=mn.value, n_steps=nt.value)


def mbs_scenario_set_field(scenario: Scenario, e0) -> int:
    """Initial field E^0 [V/m] per cell (None: zero)."""
    if e0 is None:
        return _check(lib().mbs_scenario_set_field(scenario.handle, None, 0))
    buf = np.ascontiguousarray(np.asarray(e0, np.float64))
    return _check(lib().mbs_scenario_set_field(scenario.handle, buf.ctypes.data, buf.size))


def mbs_scenario_tile(scenario: Scenario) -> int:
    t = C.c_int()
    _check(lib().mbs_scenario_tile(scenario.handle, C.byref(t)))
    return t.value


def mbs_tile_plan(n_levels: int, tile_cells: int, nx: int, tile_steps: int) -> int:
    """Number of tiles one tiled launch runs; MBSError (MBS_E_INVALID) when
    tile_steps does not fit (see include/mbs.h)."""
    t = C.c_int()
    _check(lib().mbs_tile_plan(int(n_levels), int(tile_cells), int(nx), int(tile_steps), C.byref(t)))
    return t.value


def mbs_scenario_tile_cells(scenario: Scenario) -> int:
    t = C.c_int()
    _check(lib().mbs_scenario_tile_cells(scenario.handle, C.byref(t)))
    return t.value


def mbs_scenario_counters(scenario: Scenario):
    h, d, n = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check(lib().mbs_scenario_counters(scenario.handle, C.byref(h), C.byref(d), C.byref(n)))
    return dict(h2d_bytes=h.value, d2h_bytes=d.value, kernel_launches=n.value)


def mbs_device_propagators(device: Device, qm: int, dt: float, n_levels: int):
    n, n2, k = n_levels, n_levels ** 2, n_levels ** 2 - 1
    out = dict(lam=np.zeros(n), V=np.zeros((n, n), np.complex128), A=np.zeros((k, k)),
               Ah=np.zeros((n2, n2)), c=np.zeros(k), zref=np.zeros(n2), g=np.zeros(k), g0=np.zeros(1))
    _check(lib().mbs_device_propagators(device.handle, int(qm), float(dt), *[out[x].ctypes.data for x in
                                        ("lam", "V", "A", "Ah", "c", "zref", "g", "g0")]))
    out["g0"] = float(out["g0"][0])
    return out


MBS_STATIC_CHECK_MAX = 65536


def mbs_check_rho_static(rho_ptr: int, n: int, n_levels: int, out_ptr: int, stream=None) -> int:
    """Allocation-free density-matrix check (see include/mbs.h).  rho_ptr:
    device address of n complex128 n_levels x n_levels matrices; out_ptr:
    device address of 3 float64 (min eigenvalue, max |tr - 1|, non-finite
    count).  Enqueues on `stream` (a cudaStream_t handle or None)."""
    return _check(lib().mbs_check_rho_static(C.c_void_p(int(rho_ptr)), int(n), int(n_levels),
                                             C.c_void_p(int(out_ptr)),
                                             None if stream is None else C.c_void_p(int(stream))))


def mbs_peak_rates(which: int, stream=None):
    """Measured arithmetic peak of the current GPU: which = 0 FP32 FMA,
    1 FP64 FMA, 2 TF32 tensor-core MMA.  Returns (flop/s, seconds)."""
    r, t = C.c_double(), C.c_double()
    _check(lib().mbs_peak_rates(int(which), C.byref(r), C.byref(t), None if stream is None else C.c_void_p(int(stream))))
    return r.value, t.value


def mbs_abi_version() -> int:
    return int(lib().mbs_abi_version())


class Cells:
    """Owns an mbs_cells_t (a batch of driven single cells)."""

    def __init__(self, handle, status, n_sys, n_levels, keep):
        self.handle = handle
        self.status = status
        self.n_sys = n_sys
        self.n_levels = n_levels
        self._keep = keep

    def close(self):
        if self.handle:
            lib().mbs_cells_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mbs_cells_create(qms, dt, n_steps, drives, record_every=1) -> Cells:
    keep = []
    qarr = (_QmDesc * len(qms))(*[_qm_desc(q, keep) for q in qms])
    darr = (_Source * len(drives))(*[_Source(s.kind, s.cell, s.e0, s.tau, s.t0, s.omega, s.phase, getattr(s, 'shape', 0)) for s in drives])
    h = C.c_void_p()
    rc = _check(lib().mbs_cells_create(qarr, len(qms), float(dt), int(n_steps), darr, int(record_every),
                                       C.byref(h)))
    return Cells(h.value, rc, len(qms), qms[0].n_levels, keep)


def mbs_cells_solve(cells: Cells, precision="fp32", stream=None) -> int:
    return _check(lib().mbs_cells_solve(cells.handle, PREC[precision] if isinstance(precision, str) else int(precision),
                                        None if stream is None else C.c_void_p(int(stream))))


def mbs_cells_fetch(cells: Cells, sys: int) -> np.ndarray:
    """Populations of system `sys`: array (n_rec, N), row r = record r."""
    n = C.c_size_t()
    _check(lib().mbs_cells_fetch(cells.handle, int(sys), None, 0, C.byref(n)))
    out = np.empty(n.value, np.float64)
    _check(lib().mbs_cells_fetch(cells.handle, int(sys), out.ctypes.data, out.size, C.byref(n)))
    return out.reshape(-1, cells.n_levels)


def mbs_cells_stats(cells: Cells):
    tr, mn = C.c_double(), C.c_double()
    _check(lib().mbs_cells_stats(cells.handle, C.byref(tr), C.byref(mn)))
    return dict(max_trace_dev=tr.value, min_eig=mn.value)


def cells_from_batch(b) -> Cells:
    """Marshal a workloads.CellBatch-like description."""
    return mbs_cells_create(b.qms, b.dt, b.n_steps, b.drives, b.record_every)


# ------------------------------------------------------------ conveniences
def device_from_problem(p) -> Device:
    return mbs_device_create(p.qms, p.materials, p.regions, p.length, p.n_cells,
                             (p.refl_left, p.refl_right), p.jitter)


def scenario_from_problem(dev: Device, p, courant=None) -> Scenario:
    sc = mbs_scenario(dev, 0.0, p.courant if courant is None else courant, p.t_end, p.n_steps,
                      p.sources, p.probes)
    if getattr(p, "e_init", None) is not None:
        mbs_scenario_set_field(sc, p.e_init)
    return sc


def run(p, precision="fp32", algo="auto", tile_steps=0, check_every=0, stream=None, **flags):
    """Create, solve and fetch one problem; returns dict(records, dt, nt,
    stats, counters, device_status)."""
    dev = device_from_problem(p)
    sc = scenario_from_problem(dev, p)
    mbs_solve([sc], precision, algo, tile_steps, check_every, stream, **flags)
    dt, dz, nt = mbs_scenario_info(sc)
    rec = np.stack([mbs_fetch_records(sc, k) for k in range(len(p.probes))]) if p.probes else np.zeros((0, nt))
    return dict(records=rec, dt=dt, nt=nt, stats=mbs_scenario_stats(sc), counters=mbs_scenario_counters(sc),
                device_status=dev.status)

"""Seeded synthetic inputs for the 1D Maxwell-Bloch sweep.

This module only *describes* problems: geometry, materials, quantum
descriptions (H0, mu, relaxation), sources and probes, in SI units, plus the
seeded random draws some workloads need.  It holds none of the method's
arithmetic (no Liouvillian, no propagator, no field update).  Both the CUDA
path (through its C-ABI binding) and the CPU oracle consume the same
``Problem`` objects, each with its own code.

Workload recipes follow the paper's application examples (Sec. 4: the
self-induced-transparency two-level medium, the three-level and six-level
media) re-parameterised to the sizes the benchmark and the parity tests use:

* ``sit_2lvl``      two-level SIT medium, 2,048 cells, 1 ps (4,094 steps)
* ``sit_2lvl_jitter`` the same physics over 1,048,576 cells and 200,000 steps
  with a seeded +-1 % per-cell jitter of density and transition frequency
* ``lambda_3lvl``   three-level Lambda medium, 262,144 cells, 100,000 steps,
  probe and control sech pulses injected from opposite ends
* ``ladder_6lvl``   seeded six-level medium, 131,072 cells, 50,000 steps
* ``batch_mixed``   512 independent two- and three-level simulations

Every builder takes size overrides so the tests can run the same physics on
grids the oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# CODATA 2018 exact / recommended values (SI).  Used here only to state the
# inputs (e.g. a pulse amplitude for a given pulse area); each consumer keeps
# its own copy for its arithmetic.
PLANCK_H = 6.62607015e-34
HBAR = PLANCK_H / (2.0 * math.pi)
E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 1.0 / math.sqrt(EPS0 * MU0)

# source kinds (same numbering as the C-ABI header and the oracle)
SRC_TFSF_RIGHT = 0   # one-way injection of a +x travelling wave at `cell`
SRC_TFSF_LEFT = 1    # one-way injection of a -x travelling wave at `cell`
SRC_HARD = 2         # E at `cell` is overwritten by the waveform
SHAPE_SECH = 0       # source envelope sech((t - t0)/tau)
SHAPE_GAUSS = 1      # source envelope exp(-((t - t0)/tau)^2)

# probe quantities
Q_E = 0        # E_z at the cell centre, time level n+1
Q_H = 1        # H_y at the left face of the cell, time level n+1/2
Q_RHO_RE = 2   # Re rho_ij of the cell, time level n+1/2
Q_RHO_IM = 3   # Im rho_ij

BC_ABSORB = 0.0  # reflectivity R = 0
BC_MIRROR = 1.0  # reflectivity R = 1


@dataclass
class QM:
    """One quantum-mechanical description (paper Sec. 3.1.1, class
    qm_description): density, H0, dipole operator, relaxation, initial rho.

    Relaxation is given either as explicit Lindblad operators with rates
    (D(rho) = sum_k g_k (L rho L^+ - 1/2 {L^+ L, rho})), or in the paper's
    rate form: scattering matrix R (R[i, j] = gamma_ij, the rate from level j
    into level i) plus pure-dephasing rates in the order 12, 13, 23, 14, ...
    Both forms may be combined.
    """
    n_levels: int
    density: float
    h0: np.ndarray                 # (N, N) complex, Hermitian [J]
    mu: np.ndarray                 # (N, N) complex, Hermitian [C m]
    rho_init: np.ndarray           # (N, N) complex, trace 1
    lindblad_rates: np.ndarray = field(default_factory=lambda: np.zeros(0))
    lindblad_ops: np.ndarray = field(default_factory=lambda: np.zeros((0, 1, 1), complex))
    scattering: Optional[np.ndarray] = None   # (N, N) real, diagonal ignored
    pure_dephasing: Optional[np.ndarray] = None  # (N(N-1)/2,) real


@dataclass
class Material:
    eps_r: float = 1.0
    mu_r: float = 1.0
    sigma: float = 0.0
    overlap: float = 1.0
    qm: int = -1                   # index into Problem.qms, -1 = no medium


@dataclass
class Region:
    material: int
    x_start: float
    x_end: float


@dataclass
class Source:
    kind: int
    cell: int
    e0: float
    tau: float
    t0: float
    omega: float
    phase: float = 0.0
    shape: int = 0          # SHAPE_SECH or SHAPE_GAUSS

    def waveform(self, t):
        """E0 envelope((t - t0)/tau) sin(omega t + phase) with the envelope
        sech(x) or exp(-x^2)  (input definition)."""
        t = np.asarray(t, dtype=np.float64)
        x = (t - self.t0) / self.tau
        env = np.exp(-x * x) if self.shape == SHAPE_GAUSS else 1.0 / np.cosh(x)
        return self.e0 * env * np.sin(self.omega * t + self.phase)


@dataclass
class Probe:
    cell: int
    quantity: int
    i: int = 0
    j: int = 0


@dataclass
class Problem:
    name: str
    qms: List[QM]
    materials: List[Material]
    regions: List[Region]
    length: float
    n_cells: int
    refl_left: float = BC_ABSORB
    refl_right: float = BC_ABSORB
    jitter: Optional[np.ndarray] = None      # (n_cells, 2): density factor, H0 factor
    courant: float = 1.0
    t_end: float = 0.0
    n_steps: int = 0                          # >0 overrides t_end
    sources: List[Source] = field(default_factory=list)
    probes: List[Probe] = field(default_factory=list)
    e_init: Optional[np.ndarray] = None      # (n_cells,) initial field E^0 [V/m], or None (zero)

    @property
    def dz(self) -> float:
        return self.length / self.n_cells

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014) -- the seeded generator every random
# input is drawn from, so that any consumer can reproduce the draws.
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` successive SplitMix64 outputs (uint64) for `seed`."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & _M64)
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        # vectorised: state_k = seed + (k+1) * golden
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = s + k * g
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    out[:] = z
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """U[0, 1) doubles from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normals(seed: int, count: int, skip: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from U(0,1] pairs (after `skip` draws)."""
    m = (count + 1) // 2
    u = uniform01(seed, skip + 2 * m)[skip:]
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# ---------------------------------------------------------------------------
# helpers that state inputs
# ---------------------------------------------------------------------------
def _ketbra(n, i, j):
    m = np.zeros((n, n), complex)
    m[i, j] = 1.0
    return m


def qm_two_level(density, omega21, dipole, gamma1, gamma2, w0, rho_init=None) -> QM:
    """Two-level description in the paper's qm_desc_2lvl parameterisation
    (Sec. 3.1.1): H0 = hbar w21/2 diag(-1, 1), mu = -d sigma_x (d = e z21),
    scattering R = gamma1/2 [[0, 1-w0], [1+w0, 0]], pure dephasing
    gamma2 - gamma1/2."""
    h0 = HBAR * omega21 / 2.0 * np.diag([-1.0, 1.0]).astype(complex)
    mu = -dipole * np.array([[0, 1], [1, 0]], complex)
    scat = gamma1 / 2.0 * np.array([[0.0, 1.0 - w0], [1.0 + w0, 0.0]])
    deph = np.array([gamma2 - gamma1 / 2.0])
    if rho_init is None:
        rho_init = np.diag([1.0, 0.0]).astype(complex)
    return QM(2, density, h0, mu, np.asarray(rho_init, complex), scattering=scat, pure_dephasing=deph)


def sech_area_amplitude(area, dipole, tau):
    """Amplitude E0 of E0 sech(t/tau) whose area d/hbar int E dt is `area`."""
    return area * HBAR / (dipole * math.pi * tau)


def rule_probes(m_s, n_cells, n_steps, fracs=(0.25, 0.5, 0.75)):
    """Probe cells m_s + floor(f * min(Nx - 1 - m_s, Nt))."""
    span = min(n_cells - 1 - m_s, n_steps)
    return [m_s + int(math.floor(f * span)) for f in fracs]


def in_medium(cell, n_cells, frac_lo=0.05, frac_hi=0.95):
    """Whether a cell centre lies in the 5 %-95 % medium region."""
    x = (cell + 0.5) / n_cells
    return frac_lo <= x < frac_hi


def _medium_device(n_cells, dz, frac_lo=0.05, frac_hi=0.95, qm_index=0):
    length = n_cells * dz
    mats = [Material(), Material(qm=qm_index)]
    regs = [Region(0, 0.0, frac_lo * length),
            Region(1, frac_lo * length, frac_hi * length),
            Region(0, frac_hi * length, length)]
    return length, mats, regs


DZ_SIT = 150e-6 / 2048          # 73.24 nm cells of the SIT example
SOURCE_CELL = 2                 # first total-field cell of a left-edge source
# Courant number of the long runs.  At exactly 1 the Yee scheme has no
# stability margin, and a dense resonant medium (chi < 0 at the grid's
# Nyquist frequency) pushes the effective Courant number above 1: round-off
# then grows by ~e^(1.5e-3) per step and swamps the solution after ~4e4
# steps.  1 - 2^-13 restores a margin far larger than |chi| there (~3e-7),
# and is exact in binary32, so that FP32 field coefficients (which then
# equal it to double rounding) carry no systematic error: a relative
# coefficient error d shifts the grid's wave speed by d and the phase by
# 2 pi (L / lambda) d over a path L.
COURANT_LONG = 1.0 - 2.0 ** -13


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def sit_2lvl(n_cells=2048, t_end=1e-12, n_steps=0, pulse_area=2.0 * math.pi,
             gamma1=1e9, gamma2=1e9, density=1e24, omega0=2e14, dipole=1e-29,
             tau=10e-15, t0=60e-15, probe_fracs=(0.25, 0.5, 0.75), courant=1.0) -> Problem:
    """Two-level SIT medium (paper Sec. 4.1 setup): 5 %-95 % medium,
    eps_r = 1, w0 = -1, rho(0) = diag(1, 0), one-way sech pulse from the left,
    absorbing ends, E and rho_11 recorded at three probes every step."""
    qm = qm_two_level(density, omega0, dipole, gamma1, gamma2, -1.0)
    length, mats, regs = _medium_device(n_cells, DZ_SIT)
    e0 = sech_area_amplitude(pulse_area, dipole, tau)
    src = Source(SRC_TFSF_RIGHT, SOURCE_CELL, e0, tau, t0, omega0, 0.0)
    dt = courant * DZ_SIT / C0
    nt = n_steps if n_steps > 0 else int(math.ceil(t_end / dt))
    probes = []
    for c in rule_probes(SOURCE_CELL, n_cells, nt, probe_fracs):
        probes.append(Probe(c, Q_E))
        if in_medium(c, n_cells):
            probes.append(Probe(c, Q_RHO_RE, 0, 0))
    return Problem("sit_2lvl", [qm], mats, regs, length, n_cells, t_end=t_end,
                   n_steps=n_steps, sources=[src], probes=probes, courant=courant)


def cell_jitter(n_cells, seed=1, spread=0.01) -> np.ndarray:
    """Per-cell factors (1 + spread U(-1,1)) on density and on H0, drawn
    interleaved (density, H0) cell by cell from SplitMix64(seed)."""
    u = uniform01(seed, 2 * n_cells).reshape(n_cells, 2)
    return 1.0 + spread * (2.0 * u - 1.0)


def sit_2lvl_jitter(n_cells=1_048_576, n_steps=200_000, seed=1, courant=COURANT_LONG, **kw) -> Problem:
    """The SIT physics at scale with +-1 % seeded per-cell jitter of the
    density and of the transition frequency (H0), at the long-run Courant
    number."""
    p = sit_2lvl(n_cells=n_cells, n_steps=n_steps, t_end=0.0, courant=courant, **kw)
    return p.replace(name="sit_2lvl_jitter", jitter=cell_jitter(n_cells, seed))


def lambda_3lvl(n_cells=262_144, n_steps=100_000, tau=100e-15, t0=600e-15,
                t1=10e-12, t2=1e-12, probe_area=0.2 * math.pi,
                control_area=math.pi, courant=COURANT_LONG) -> Problem:
    """Three-level Lambda medium: levels (0, 1.5e-20, 1.9e-20) J, dipoles
    1-3 = 1e-29 and 2-3 = 0.8e-29 C m; decays 3->1 and 3->2 at 1/(2 T1);
    dephasing |k><k| so the optical coherences decay at 1/T2; probe sech at
    w31 from the left, control sech at w32 from the right."""
    n = 3
    en = np.array([0.0, 1.5e-20, 1.9e-20])
    h0 = np.diag(en).astype(complex)
    mu = np.zeros((n, n), complex)
    mu[0, 2] = mu[2, 0] = 1e-29
    mu[1, 2] = mu[2, 1] = 0.8e-29
    g_dec = 1.0 / (2.0 * t1)
    g_phi = 1.0 / t2 - 1.0 / (2.0 * t1)
    ops = [_ketbra(n, 0, 2), _ketbra(n, 1, 2)] + [_ketbra(n, k, k) for k in range(n)]
    rates = [g_dec, g_dec] + [g_phi] * n
    qm = QM(n, 1e24, h0, mu, _ketbra(n, 0, 0), np.array(rates), np.array(ops))
    length, mats, regs = _medium_device(n_cells, DZ_SIT)
    w31 = (en[2] - en[0]) / HBAR
    w32 = (en[2] - en[1]) / HBAR
    e_p = sech_area_amplitude(probe_area, 1e-29, tau)
    e_c = sech_area_amplitude(control_area, 0.8e-29, tau)
    srcs = [Source(SRC_TFSF_RIGHT, SOURCE_CELL, e_p, tau, t0, w31),
            Source(SRC_TFSF_LEFT, n_cells - 1 - SOURCE_CELL, e_c, tau, t0, w32)]
    probes = []
    for c in rule_probes(SOURCE_CELL, n_cells, n_steps):
        probes.append(Probe(c, Q_E))
        if in_medium(c, n_cells):
            probes += [Probe(c, Q_RHO_RE, k, k) for k in range(n)]
    return Problem("lambda_3lvl", [qm], mats, regs, length, n_cells, n_steps=n_steps,
                   sources=srcs, probes=probes, courant=courant)


def ladder_6lvl(n_cells=131_072, n_steps=50_000, seed=3, tau=10e-15, t0=60e-15,
                decay=1e11, dephase=1e12, courant=COURANT_LONG) -> Problem:
    """Seeded six-level medium: H0 = diag(0, sorted U(0, 5e-20) J x 5),
    mu real symmetric with zero diagonal and N(0, (1e-29)^2) off-diagonals,
    decays |k-1><k| (k = 2..6) and |1><6|, dephasing |k><k|; sech pulse at the
    mean adjacent transition frequency with E0 = 2 hbar/(1e-29 tau)."""
    n = 6
    u = uniform01(seed, n - 1)
    en = np.concatenate([[0.0], np.sort(u * 5e-20)])
    g = normals(seed, n * (n - 1) // 2, skip=n - 1) * 1e-29
    mu = np.zeros((n, n), complex)
    k = 0
    for j in range(1, n):
        for i in range(j):
            mu[i, j] = mu[j, i] = g[k]
            k += 1
    ops = [_ketbra(n, k - 1, k) for k in range(1, n)] + [_ketbra(n, 0, n - 1)]
    rates = [decay] * n
    ops += [_ketbra(n, k, k) for k in range(n)]
    rates += [dephase] * n
    qm = QM(n, 1e24, np.diag(en).astype(complex), mu, _ketbra(n, 0, 0),
            np.array(rates), np.array(ops))
    length, mats, regs = _medium_device(n_cells, DZ_SIT)
    w_mean = (en[-1] - en[0]) / (n - 1) / HBAR
    e0 = 2.0 * HBAR / (1e-29 * tau)
    src = Source(SRC_TFSF_RIGHT, SOURCE_CELL, e0, tau, t0, w_mean)
    probes = []
    for c in rule_probes(SOURCE_CELL, n_cells, n_steps):
        probes.append(Probe(c, Q_E))
        if in_medium(c, n_cells):
            probes += [Probe(c, Q_RHO_RE, k, k) for k in range(n)]
    return Problem("ladder_6lvl", [qm], mats, regs, length, n_cells, n_steps=n_steps,
                   sources=[src], probes=probes, courant=courant)


def batch_mixed(n_sims=512, seed=4, min_cells=1024, max_cells=65536,
                min_steps=20_000, max_steps=100_000) -> List[Problem]:
    """512 independent simulations: each is a two-level SIT medium or a
    three-level Lambda medium (by a seeded coin), with log-uniform cell count,
    uniform step count, and density, transition frequencies, T1 and T2 each
    scaled by (1 + 0.2 U(-1, 1))."""
    u = uniform01(seed, 8 * n_sims).reshape(n_sims, 8)
    out = []
    for s in range(n_sims):
        r = u[s]
        nx = int(round(math.exp(math.log(min_cells) + r[1] * (math.log(max_cells) - math.log(min_cells)))))
        nx = max(min_cells, min(max_cells, nx))
        nt = min_steps + int(r[2] * (max_steps - min_steps + 1))
        fd, fw, f1, f2 = (1.0 + 0.2 * (2.0 * r[3 + k] - 1.0) for k in range(4))
        if r[0] < 0.5:
            p = sit_2lvl(n_cells=nx, n_steps=nt, t_end=0.0, density=1e24 * fd,
                         omega0=2e14 * fw, gamma1=1e9 / f1, gamma2=1e9 / f2, courant=COURANT_LONG)
        else:
            p = lambda_3lvl(n_cells=nx, n_steps=nt, t1=10e-12 * f1, t2=1e-12 * f2)
            qm = p.qms[0]
            qm.h0 = qm.h0 * fw
            qm.density *= fd
        out.append(p.replace(name=f"batch_{s}"))
    return out


def ladder_anharmonic(n_levels=6, n_cells=8192, n_steps=20_000, omega0=2.0 * math.pi * 1e13, d=1e-29,
                      density=1e24, decay=1e11, dephase=1e12, area=math.pi, tau=200e-15, t0=1.2e-12,
                      courant=COURANT_LONG) -> Problem:
    """The anharmonic ladder of the paper's six-level example, for any N >= 2:
    E_1 = 0, E_{n+1} = E_n + hbar omega0 [1 - 0.1 (n - 3)], omega0 = 2 pi 1e13
    rad/s.  The rest is the builder's choice (the paper cites it from
    elsewhere): nearest-neighbour dipoles mu_{n,n+1} = d sqrt(n), decays
    |n><n+1| at `decay`, dephasing |n><n| at `dephase`, a Gaussian pulse from
    the left at omega0 with area `area` on mu_12, 8192 cells of the SIT grid
    (medium 5-95 %), probes by the usual rule."""
    n = n_levels
    en = [0.0]
    for k in range(1, n):
        en.append(en[-1] + HBAR * omega0 * (1.0 - 0.1 * (k - 3)))
    mu = np.zeros((n, n), complex)
    for k in range(n - 1):
        mu[k, k + 1] = mu[k + 1, k] = d * math.sqrt(k + 1)
    ops = [_ketbra(n, k, k + 1) for k in range(n - 1)] + [_ketbra(n, k, k) for k in range(n)]
    rates = [decay] * (n - 1) + [dephase] * n
    qm = QM(n, density, np.diag(en).astype(complex), mu, _ketbra(n, 0, 0), np.array(rates), np.array(ops))
    length, mats, regs = _medium_device(n_cells, DZ_SIT)
    # area of exp(-x^2) sin envelope: mu E0 tau sqrt(pi) / hbar
    e0 = area * HBAR / (d * tau * math.sqrt(math.pi))
    src = Source(SRC_TFSF_RIGHT, SOURCE_CELL, e0, tau, t0, (en[1] - en[0]) / HBAR, 0.0, SHAPE_GAUSS)
    probes = []
    for c in rule_probes(SOURCE_CELL, n_cells, n_steps):
        probes.append(Probe(c, Q_E))
        if in_medium(c, n_cells):
            probes += [Probe(c, Q_RHO_RE, k, k) for k in range(n)]
    return Problem(f"ladder_anharmonic_{n}lvl", [qm], mats, regs, length, n_cells, n_steps=n_steps,
                   sources=[src], probes=probes, courant=courant)


def qcl_tzenov(n_cells=8192, n_steps=20_000, seed=7, e_noise=1e2, refl=0.8, courant=COURANT_LONG) -> Problem:
    """The quantum cascade laser of the paper's frequency-comb example (five
    levels, parameters of its listing): H0 with diagonal 0.10103, 0.09677,
    0.09720, 0.08129, 0.07633 eV and tunnelling couplings H_13 = 1.2329 meV,
    H_23 = -1.3447 meV; one dipole element mu_34 = -e 4 nm; the scattering
    matrix and pure-dephasing rates (1/0.6 ps for 13, 23; 1/1 ps for the
    other pairs except 12, which has none) of the listing; n3D = 5.6e21 m^-3;
    eps_r = 12.96, overlap 0.9, loss alpha0 = 1100 m^-1 (sigma = 2 alpha0
    eps c); a 5 mm cavity filled with the medium; both facets R = 0.8;
    rho(0) = |3><3|; a seeded random initial field (normals x e_noise V/m),
    no source.  Probes: E at both facets and the centre, populations at the
    centre."""
    n = 5
    ev = E_CHARGE
    h0 = np.diag([0.10103, 0.09677, 0.09720, 0.08129, 0.07633]).astype(complex) * ev
    h0[0, 2] = h0[2, 0] = 1.2329e-3 * ev
    h0[1, 2] = h0[2, 1] = -1.3447e-3 * ev
    mu = np.zeros((n, n), complex)
    mu[2, 3] = mu[3, 2] = -ev * 4e-9
    scat = np.array([[0.0, 0.4947, 0.0974, 0.8116, 1.0410],
                     [0.8245, 0.0, 0.1358, 0.6621, 1.1240],
                     [0.0229, 0.0469, 0.0, 0.0794, 0.0357],
                     [0.0047, 0.0029, 0.1252, 0.0, 0.2810],
                     [0.0049, 0.0049, 0.1101, 0.4949, 0.0]]) * 1e12
    d_inj, d_other = 1.0 / 0.6e-12, 1.0 / 1.0e-12
    deph = np.array([0.0, d_inj, d_inj] + [d_other] * 7)   # order 12, 13, 23, 14, 24, 34, 15, 25, 35, 45
    rho0 = np.zeros((n, n), complex)
    rho0[2, 2] = 1.0
    qm = QM(n, 5.6e21, h0, mu, rho0, scattering=scat, pure_dephasing=deph)
    eps_r, alpha0 = 12.96, 1100.0
    sigma = 2.0 * alpha0 * EPS0 * eps_r * C0 / math.sqrt(eps_r)
    length = 5e-3
    mats = [Material(eps_r=eps_r, sigma=sigma, overlap=0.9, qm=0)]
    regs = [Region(0, 0.0, length)]
    e_init = normals(seed, n_cells) * e_noise
    mid = n_cells // 2
    probes = [Probe(0, Q_E), Probe(n_cells - 1, Q_E), Probe(mid, Q_E)] + [Probe(mid, Q_RHO_RE, k, k) for k in range(n)]
    return Problem("qcl_tzenov", [qm], mats, regs, length, n_cells, refl_left=refl, refl_right=refl,
                   n_steps=n_steps, probes=probes, courant=courant, e_init=e_init)


@dataclass
class CellBatch:
    """Independent driven quantum systems without propagation (the borderline
    case Nx = 1 of Sec. 2.1): system s evolves under the field
    drives[s].waveform(n dt) at step n (0 at n = 0)."""
    name: str
    qms: List[QM]
    drives: List[Source]
    dt: float
    n_steps: int
    record_every: int = 1


def song_vtype_qm(scale_e=1.0, scale_d=1.0, scale_g=1.0) -> QM:
    """The driven V-type three-level system of the paper's application example
    (atomic rubidium after Song et al.): level energies 0, 2.3717e15 hbar,
    2.4165e15 hbar; dipole elements mu_12 = -e 9.2374e-11 m, mu_13 = sqrt(2)
    mu_12, mu_23 = 0; scattering rate 1e10 s^-1 between every pair of levels,
    no pure dephasing; rho(0) = |1><1|; n3D = 6e24 m^-3.  The scale factors
    multiply the energies, the dipole elements and the rates."""
    n = 3
    en = np.array([0.0, 2.3717e15, 2.4165e15]) * HBAR * scale_e
    d = -E_CHARGE * 9.2374e-11 * scale_d
    mu = np.zeros((n, n), complex)
    mu[0, 1] = mu[1, 0] = d
    mu[0, 2] = mu[2, 0] = d * math.sqrt(2.0)
    scat = np.full((n, n), 1e10 * scale_g)
    np.fill_diagonal(scat, 0.0)
    return QM(n, 6e24, np.diag(en).astype(complex), mu, _ketbra(n, 0, 0), scattering=scat,
              pure_dephasing=np.zeros(3))


def song_vtype_drive(e0=3.5471e9) -> Source:
    """The sech drive of the V-type example, in the reading (amplitude,
    frequency [Hz], t0 in units of tau, 1/tau, phase) of the listing's
    numbers: e0 = 3.5471e9 V/m, omega = 2 pi 3.8118e14 rad/s, tau = 5 fs/1.76,
    t0 = 17.248 tau, phase -pi/2."""
    tau = 5e-15 / 1.76
    return Source(SRC_HARD, 0, e0, tau, 17.248 * tau, 2.0 * math.pi * 3.8118e14, -math.pi / 2.0)


def song_vtype(n_sys=1, seed=5, spread=0.1, n_steps=10_000, t_end=80e-15, record_every=1,
               amp_range=(0.25, 2.0)) -> CellBatch:
    """The V-type example as a batch: system 0 is the paper's system under its
    drive; systems s > 0 have energies, dipoles and rates scaled by
    (1 + spread U(-1, 1)) each and the drive amplitude swept uniformly over
    amp_range x e0 (seeded).  Nt steps over t_end: dt = t_end / Nt."""
    u = uniform01(seed, 4 * n_sys).reshape(n_sys, 4)
    qms, drives = [], []
    base = song_vtype_drive()
    for s in range(n_sys):
        if s == 0:
            qms.append(song_vtype_qm())
            drives.append(base)
            continue
        f = [1.0 + spread * (2.0 * u[s, k] - 1.0) for k in range(3)]
        qms.append(song_vtype_qm(*f))
        a = amp_range[0] + (amp_range[1] - amp_range[0]) * u[s, 3]
        drives.append(Source(SRC_HARD, 0, base.e0 * a, base.tau, base.t0, base.omega, base.phase))
    return CellBatch("song_vtype", qms, drives, t_end / n_steps, n_steps, record_every)


def cell_field(drive: Source, dt: float, n_steps: int) -> np.ndarray:
    """The prescribed field sequence E^n of a driven cell: the waveform at
    t_n = n dt for n >= 1, and the initial field 0 at n = 0."""
    e = np.asarray(drive.waveform(np.arange(n_steps) * dt), np.float64)
    e[0] = 0.0
    return e


WORKLOADS = {
    "sit_2lvl": sit_2lvl,
    "sit_2lvl_jitter": sit_2lvl_jitter,
    "lambda_3lvl": lambda_3lvl,
    "ladder_6lvl": ladder_6lvl,
}


def light_cone_window(p: Problem, n_steps: int, margin: int = 8) -> Problem:
    """The same problem truncated to the cells a left-edge source can reach in
    `n_steps` steps (plus a margin), with `n_steps` steps.  At Courant number
    1 nothing travels faster than one cell per step, so for a problem whose
    only sources sit at the left edge and whose medium starts in equilibrium
    the truncated run reproduces the full run's probes (those inside the
    window) for the first `n_steps` steps."""
    nx = min(p.n_cells, n_steps + margin)
    jit = None if p.jitter is None else p.jitter[:nx].copy()
    probes = [q for q in p.probes if q.cell < nx - 1]
    srcs = [s for s in p.sources if s.cell < nx - 2]
    return p.replace(n_cells=nx, length=nx * p.dz, jitter=jit, n_steps=n_steps,
                     t_end=0.0, probes=probes, sources=srcs)

"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code that the CUDA path's callers and the oracle have in
common.  It holds none of the integrator's arithmetic: it samples the prescribed
plane-wave fields of the model problem on the staggered grid (the "perfectly
propagating PIC" field source of Sec. III, Eqs. laser5 - laser3) and draws
initial particle states from fixed seeds.

Grid convention: E_y at nodes x = i dx and times n dt; B_z at nodes
x = (i + 1/2) dx and times (n + 1/2) dt (the Yee staggering of Eqs. eq:Ey/eq:Bz,
shifted by half a cell).  A level is W consecutive nodes from global node i0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi
# 10 keV over the electron rest energy 510.99895 keV; thermal momentum spread.
MAXWELL_10KEV_SIGMA = math.sqrt(10.0 / 510.99895)


@dataclass(frozen=True)
class PlaneWave:
    """Linearly polarized plane wave along +x, a = a(xi), xi = t - x (Sec. II).

    profile "sine":  a = a0 sin(xi) for xi > 0, 0 before (a switched-on wave);
    profile "gauss": a = a0 exp(-(xi - xi0)^2 / (2 sigma^2)) sin(xi) (Eq. laser1).
    E_y = B_z = sign * (-da/dxi) (Eq. laser5 for sign = +1).
    """
    a0: float
    profile: str = "sine"
    xi0: float = 0.0
    sigma: float = 1.0
    sign: float = 1.0

    def a(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        if self.profile == "sine":
            return np.where(xi > 0.0, self.a0 * np.sin(xi), 0.0)
        env = np.exp(-((xi - self.xi0) ** 2) / (2.0 * self.sigma ** 2))
        return self.a0 * env * np.sin(xi)

    def field(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        if self.profile == "sine":
            dadxi = np.where(xi > 0.0, self.a0 * np.cos(xi), 0.0)
        else:
            env = np.exp(-((xi - self.xi0) ** 2) / (2.0 * self.sigma ** 2))
            dadxi = self.a0 * env * (np.cos(xi) - (xi - self.xi0) / self.sigma ** 2 * np.sin(xi))
        return self.sign * (-dadxi)


def sample_levels(wave: PlaneWave, dt: float, dx: float, n_first: int, n_count: int,
                  i0s, W: int, rowwise: bool = True):
    """Field levels n_first .. n_first+n_count-1 on windows of W nodes.

    Returns (E, B) of shape (n_count, W): E row r is E_y at t = (n_first+r) dt on
    nodes (i0s[r] + c) dx; B row r is B_z at t = (n_first+r+1/2) dt on nodes
    (i0s[r] + c + 1/2) dx.  Rows are computed one at a time, so a level's bits do
    not depend on how the caller groups levels into batches (rowwise=False
    evaluates the whole batch at once: faster, for runs that are not compared
    bit for bit).
    """
    i0s = np.asarray(i0s, dtype=np.int64).reshape(n_count)
    if not rowwise:
        n = np.arange(n_first, n_first + n_count, dtype=np.float64)[:, None]
        i0 = i0s.astype(np.float64)[:, None]
        cc = np.arange(W, dtype=np.float64)[None, :]
        return (np.ascontiguousarray(wave.field(n * dt - (i0 + cc) * dx)),
                np.ascontiguousarray(wave.field((n + 0.5) * dt - (i0 + cc + 0.5) * dx)))
    c = np.arange(W, dtype=np.float64)
    E = np.empty((n_count, W), dtype=np.float64)
    B = np.empty((n_count, W), dtype=np.float64)
    for r in range(n_count):
        n = float(n_first + r)
        i0 = float(i0s[r])
        E[r] = wave.field(n * dt - (i0 + c) * dx)
        B[r] = wave.field((n + 0.5) * dt - (i0 + c + 0.5) * dx)
    return E, B


def chase_origins(n_first: int, n_count: int, dt: float, dx: float, W: int, lead: int):
    """Window origins that follow the wave front x = t: the window ends `lead`
    nodes ahead of the front node at each level's time."""
    n = np.arange(n_first, n_first + n_count, dtype=np.float64)
    return (np.floor(n * dt / dx).astype(np.int64) + lead - W).astype(np.int64)


@dataclass
class ParticleInit:
    x: np.ndarray
    px: np.ndarray
    py: np.ndarray
    pz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def electrons_at_rest(n: int, seed: int, x_lo: float, x_hi: float,
                      sort_x: bool = False) -> ParticleInit:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(x_lo, x_hi, size=n)
    if sort_x:
        x = np.sort(x)
    z = np.zeros(n, dtype=np.float64)
    return ParticleInit(x, z.copy(), z.copy(), z.copy())


def electrons_maxwellian(n: int, seed: int, x_lo: float, x_hi: float,
                         sigma: float = MAXWELL_10KEV_SIGMA, sort_x: bool = False) -> ParticleInit:
    """Non-relativistic Maxwellian: each momentum component N(0, sigma^2).
    sort_x stores the electrons in order of initial position (the momenta stay
    independent draws): a layout choice, the ensemble is the same."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(x_lo, x_hi, size=n)
    if sort_x:
        x = np.sort(x)
    p = rng.standard_normal(size=(3, n)) * sigma
    return ParticleInit(x, p[0].copy(), p[1].copy(), p[2].copy())


@dataclass(frozen=True)
class Workload:
    """One synthetic configuration shaped like a run of the paper."""
    name: str
    n_particles: int
    a0: float
    dt: float
    dx: float
    psi_max: float
    order: int
    n_steps: int
    x_lo: float
    x_hi: float
    thermal_sigma: float = 0.0      # 0: at rest
    seed: int = 1
    window: int = 256               # W, a power of two
    window_origin: int | None = None  # fixed origin (full grid) or None (chase the front)
    lead: int = 96
    profile: str = "sine"
    xi0: float = 0.0
    sigma: float = 1.0
    sort_x: bool = False            # store electrons in order of initial position

    @property
    def wave(self) -> PlaneWave:
        return PlaneWave(self.a0, self.profile, self.xi0, self.sigma)

    def particles(self, n: int | None = None) -> ParticleInit:
        n = self.n_particles if n is None else n
        if self.thermal_sigma > 0.0:
            return electrons_maxwellian(n, self.seed, self.x_lo, self.x_hi, self.thermal_sigma,
                                        self.sort_x)
        return electrons_at_rest(n, self.seed, self.x_lo, self.x_hi, self.sort_x)

    def origins(self, n_first: int, n_count: int) -> np.ndarray:
        if self.window_origin is not None:
            return np.full(n_count, self.window_origin, dtype=np.int64)
        return chase_origins(n_first, n_count, self.dt, self.dx, self.window, self.lead)

    def levels(self, n_first: int, n_count: int):
        """(E, B, i0) for levels n_first .. n_first + n_count - 1."""
        i0 = self.origins(n_first, n_count)
        E, B = sample_levels(self.wave, self.dt, self.dx, n_first, n_count, i0, self.window)
        return E, B, i0


def steps_to_phase(a0: float, xi_end: float, x_span: float, dt: float) -> int:
    """Macro steps until an electron starting at rest at x0 <= x_span in a0 sin(xi)
    reaches phase xi_end: t = x0 + xi + (a0^2/2)(xi/2 - sin(2 xi)/4) (from
    dt/dxi = gamma/R with R = 1, Eq. R-def, and gamma = 1 + a^2/2)."""
    t = x_span + xi_end + 0.5 * a0 * a0 * (xi_end / 2.0 - math.sin(2.0 * xi_end) / 4.0)
    return int(math.ceil(t / dt)) + 1


# The configurations of the benchmark and the tests (normalized units, lambda = 2 pi).
DT75 = TWO_PI / 75.0

C1 = Workload(name="c1_testparticle_a0_100", n_particles=256, a0=100.0, dt=DT75,
              dx=TWO_PI / 74.26, psi_max=0.01, order=3,
              n_steps=steps_to_phase(100.0, TWO_PI, TWO_PI, DT75),
              x_lo=0.0, x_hi=TWO_PI, window=256, lead=96)

C2 = Workload(name="c2_maxwellian_a0_150_16M", n_particles=16_777_216, a0=150.0, dt=DT75,
              dx=DT75 / 0.99, psi_max=0.01, order=3, n_steps=20_000,
              x_lo=0.0, x_hi=64 * TWO_PI, thermal_sigma=MAXWELL_10KEV_SIGMA, seed=2,
              window=32768, window_origin=-512, sort_x=True)

C4 = Workload(name="c4_maxwellian_a0_300_64M", n_particles=67_108_864, a0=300.0, dt=DT75,
              dx=DT75 / 0.99, psi_max=0.01, order=3, n_steps=10_000,
              x_lo=0.0, x_hi=64 * TWO_PI, thermal_sigma=MAXWELL_10KEV_SIGMA, seed=4,
              window=32768, window_origin=-512, sort_x=True)


# ---------------------------------------------------------------- self-consistent 1D3V PIC

def sin2_duration_for_fwhm(fwhm: float) -> float:
    """Total length T of a sin^2(pi xi / T) field envelope whose intensity
    (sin^4) has the full width at half maximum `fwhm`."""
    alpha = math.asin(2.0 ** -0.25)
    return fwhm / (1.0 - 2.0 * alpha / math.pi)


@dataclass(frozen=True)
class LaserPlasma1D:
    """A laser pulse in vacuum heading into a plasma with an exponential ramp,
    on a 1D grid of n_cells cells (normalized units, lambda = 2 pi).

    Laser: a = a0 sin^2(pi xi / T) sin(xi) for 0 <= xi <= T, xi = t - x + x_front
    (front at x_front at t = 0), E_y = B_z = -da/dxi (Eq. laser5); T from the
    intensity FWHM (fwhm, normalized time).
    Plasma (electrons; ions an immobile neutralizing background): density
    n_top exp((x - x_top)/L) on [x_top - ramp_lengths L, x_top), n_top beyond
    x_top up to the end of the grid minus `tail_gap` cells; ppc electrons per
    cell on a regular lattice ((c + (j + 1/2)/ppc) dx), at rest, each of weight
    n(x)/ppc (units of n_c).
    Grids: E_y on nodes k dx, B_z and E_x on faces (k + 1/2) dx; arrays hold
    n_cells + 5 entries, index = node (or face) + 2."""
    name: str
    n_cells: int
    a0: float
    fwhm: float
    x_front: float
    x_top: float
    scale_length: float
    n_top: float
    ppc: int
    dt: float = DT75
    dx: float = DT75 / 0.99
    ramp_lengths: float = 6.0
    gap: float = TWO_PI             # vacuum between the pulse front and the plasma
    tail_gap: int = 8
    psi_max: float = 0.01
    order: int = 3

    @property
    def duration(self) -> float:
        return sin2_duration_for_fwhm(self.fwhm)

    def a(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        T = self.duration
        inside = (xi >= 0.0) & (xi <= T)
        return np.where(inside, self.a0 * np.sin(math.pi * xi / T) ** 2 * np.sin(xi), 0.0)

    def field(self, xi):
        """-da/dxi."""
        xi = np.asarray(xi, dtype=np.float64)
        T = self.duration
        inside = (xi >= 0.0) & (xi <= T)
        env = np.sin(math.pi * xi / T)
        d = self.a0 * (2.0 * math.pi / T * env * np.cos(math.pi * xi / T) * np.sin(xi)
                       + env * env * np.cos(xi))
        return np.where(inside, -d, 0.0)

    def density(self, x):
        x = np.asarray(x, dtype=np.float64)
        L = self.scale_length
        start = self.x_top - self.ramp_lengths * L
        end = (self.n_cells - self.tail_gap) * self.dx
        n = np.where(x < self.x_top, self.n_top * np.exp((x - self.x_top) / L), self.n_top)
        return np.where((x >= start) & (x < end), n, 0.0)

    def particles(self):
        """(x, px, py, pz, w) of every macro-electron, in order of position."""
        L = self.scale_length
        start = self.x_top - self.ramp_lengths * L
        end = (self.n_cells - self.tail_gap) * self.dx
        c0 = int(math.ceil(start / self.dx))
        c1 = int(math.floor(end / self.dx))
        cells = np.arange(c0, c1, dtype=np.float64)
        j = (np.arange(self.ppc, dtype=np.float64) + 0.5) / self.ppc
        x = ((cells[:, None] + j[None, :]) * self.dx).ravel()
        w = self.density(x) / self.ppc
        keep = w > 0.0
        x, w = x[keep], w[keep]
        z = np.zeros_like(x)
        return x, z.copy(), z.copy(), z.copy(), w

    def field_history(self):
        """Levels -p .. 0 of (E_x, E_y) and -p+1/2 .. 1/2 of B_z: the vacuum
        pulse (E_x = 0: the plasma is neutral and at rest before t = 0)."""
        p, N = self.order, self.n_cells
        M = N + 5
        nodes = np.arange(N + 1, dtype=np.float64)
        faces = np.arange(N, dtype=np.float64) + 0.5
        E_hist, B_hist = [], []
        for lev in range(-p, 1):
            ey = np.zeros(M)
            ey[2:N + 3] = self.field(lev * self.dt - nodes * self.dx + self.x_front)
            E_hist.append((np.zeros(M), ey))
            bz = np.zeros(M)
            bz[2:N + 2] = self.field((lev + 0.5) * self.dt - faces * self.dx + self.x_front)
            B_hist.append(bz)
        return E_hist, B_hist


def laser_plasma_c5(n_cells: int = 20_000, ppc: int = 100, a0: float = 150.0) -> LaserPlasma1D:
    """The self-consistent configuration: a0 = 150, 30 fs intensity FWHM at
    820 nm, exponential preplasma (5 lambda scale length) rising to 0.5 n_c,
    100 electrons per cell, 20,000 cells, c dt/dx = 0.99, dt = lambda/75."""
    omega = TWO_PI * 299_792_458.0 / 820e-9
    fwhm = 30e-15 * omega
    T = sin2_duration_for_fwhm(fwhm)
    x_front = TWO_PI + T                  # the tail one wavelength from the left edge
    L = 5 * TWO_PI
    x_top = x_front + TWO_PI + 6.0 * L    # ramp from n_top e^-6, a wavelength past the front
    return LaserPlasma1D(name=f"c5_laser_plasma_a0_{a0:g}_{n_cells}cells_{ppc}ppc", n_cells=n_cells,
                         a0=a0, fwhm=fwhm, x_front=x_front, x_top=x_top, scale_length=L,
                         n_top=0.5, ppc=ppc)


# ---------------------------------------------------------------- single-electron studies

# The Gaussian-enveloped pulse of the studies of Secs. IV-VII (Eq. laser1,
# sigma = 8 pi), centred 6 sigma ahead of an electron at x = 0 (where the field
# is below a0 e^-18).
STUDY_SIGMA = 8 * math.pi
STUDY_XI0 = 6 * STUDY_SIGMA


def study_steps(a0: float, dt: float, x_span: float = 0.0) -> int:
    """Macro steps until an electron from rest at x0 <= x_span is through the
    pulse: t = x0 + 2 xi0 + int_0^{2 xi0} a^2/2 dxi (t - x = xi, dx/dxi = a^2/2
    for R = 1)."""
    from scipy.integrate import quad
    xi_end = 2 * STUDY_XI0
    f = lambda s: 0.5 * (a0 * math.exp(-((s - STUDY_XI0) ** 2) / (2 * STUDY_SIGMA ** 2))
                         * math.sin(s)) ** 2
    t_end = x_span + xi_end + quad(f, 0, xi_end, limit=4000)[0]
    return int(t_end / dt) + 1

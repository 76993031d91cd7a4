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

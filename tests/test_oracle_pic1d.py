"""Pins of the self-consistent 1D3V PIC oracle (oracle/pic1d_oracle.c).

Each test names the passage or the textbook fact it checks: the Yee scheme of
Sec. III against its own dispersion relation, the Boris push with E_x against
exact cases, discrete charge conservation and Gauss's law of the deposit, the
time-averaged transverse current of one electron, and the cold-plasma
(Langmuir) frequency, which fixes the signs and factors of the E_x - J_x
coupling.  None compares the oracle with itself.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import pic1d
from paper_2102_10983_gb300 import workloads as W

DT = 2 * math.pi / 75
DX = DT / 0.99


def _vacuum_history(prm, ey_fn, bz_fn):
    N, p = prm.n_cells, prm.order
    M = N + 5
    nodes = np.arange(N + 1, dtype=np.float64) * prm.dx
    faces = (np.arange(N, dtype=np.float64) + 0.5) * prm.dx
    E_hist, B_hist = [], []
    for lev in range(-p, 1):
        ey = np.zeros(M)
        ey[2:N + 3] = ey_fn(nodes, lev * prm.dt)
        bz = np.zeros(M)
        bz[2:N + 2] = bz_fn(faces, (lev + 0.5) * prm.dt)
        E_hist.append((np.zeros(M), ey))
        B_hist.append(bz)
    return E_hist, B_hist


def _empty():
    z = np.zeros(0)
    return z, z, z, z, z


# ---------------------------------------------------------------- Boris with E_x (Sec. III)

def test_boris_with_ex_reduces_to_the_transverse_push_and_is_exact_in_uniform_ex():
    rng = np.random.default_rng(3)
    for _ in range(50):
        p0 = rng.standard_normal(3) * 5
        ey, bz, h = rng.standard_normal(3) * [30, 30, 0.05]
        np.testing.assert_array_equal(pic1d.boris(p0, 0.0, ey, bz, h), oracle.boris(p0, ey, bz, h))
    p = np.array([0.5, -0.25, 0.75])
    for _ in range(32):
        p = pic1d.boris(p, 2.0, 0.0, 0.0, 0.0625)
    np.testing.assert_array_equal(p, [0.5 - 32 * 2.0 * 0.0625, -0.25, 0.75])


# ---------------------------------------------------------------- Yee scheme (Sec. III, Eqs. eq:Ey, eq:Bz)

def test_yee_vacuum_wave_follows_the_numerical_dispersion_relation():
    """E_y = B_z = cos(k x - w t) with sin(w dt/2)/dt = sin(k dx/2)/dx is an
    exact solution of the discrete equations (B/E = 1 follows from the same
    relation); the continuum w = k is not (phase error ~ k^3 dx^2 (1 - r^2)/24
    per unit time).  Checked away from the boundaries' light cone."""
    prm = pic1d.Params(dt=DT, dx=DX, n_cells=2048)
    k = 2 * math.pi / (74.26 * DX)                      # one wavelength per 74.26 cells
    w = 2.0 / DT * math.asin(DT / DX * math.sin(k * DX / 2))
    E_hist, B_hist = _vacuum_history(prm, lambda x, t: np.cos(k * x - w * t),
                                     lambda x, t: np.cos(k * x - w * t))
    sim = pic1d.Pic1d(prm, *_empty(), E_hist, B_hist)
    steps = 600
    for _ in range(steps):
        sim.step()
    nodes = np.arange(700, prm.n_cells - 700)            # outside the boundaries' light cone
    x, t = nodes * DX, steps * DT
    got = sim.E[-1][1][nodes + 2]
    assert np.abs(got - np.cos(k * x - w * t)).max() < 1e-11
    assert np.abs(got - np.cos(k * x - k * t)).max() > 1e-5
    assert not np.any(sim.E[-1][0])                      # no charge, no E_x


# ---------------------------------------------------------------- deposit

def test_charge_conservation_for_a_face_crossing_inside_a_subcycle():
    """One electron crossing node 101 while sub-cycling (a uniform B_z forces
    k = 3): the node charges before and after the step and the face fluxes
    satisfy rho^{n+1}_k - rho^n_k = -(F_{k+1/2} - F_{k-1/2}) exactly, the
    fluxes vanish away from the particle, and Gauss's law still holds."""
    prm = pic1d.Params(dt=DT, dx=DX, n_cells=256)
    M = prm.n_cells + 5
    bz = 10.0
    E_hist = [(np.zeros(M), np.zeros(M)) for _ in range(prm.order + 1)]
    B_hist = [np.where((np.arange(M) >= 2) & (np.arange(M) < prm.n_cells + 2), bz, 0.0)
              for _ in range(prm.order + 1)]
    x0 = 100.93 * DX
    sim = pic1d.Pic1d(prm, [x0], [0.6], [0.2], [0.0], [3e-3], E_hist, B_hist)
    C0 = sim.rho_units()
    sim.step()
    C1 = sim.rho_units()
    F = sim.last_F
    assert sim.stats.k_hist[3] == 1
    assert math.floor(sim.x[0] / DX) == 101              # it crossed node 101
    q = np.arange(1, M)
    np.testing.assert_array_equal(C1[q] - C0[q], -(F[q] - F[q - 1]))
    assert C1.sum() == C0.sum()
    assert np.count_nonzero(F) <= 2 and np.all(F[:100] == 0) and np.all(F[106:] == 0)
    g, rmax = sim.gauss()
    assert g <= 1e-15 * max(rmax, 1.0) + 1e-13, (g, rmax)


def test_transverse_current_of_one_electron_without_fields():
    """No fields: one sub-step, p constant, so the time-averaged J_y is
    q n v_y S(x_mid) at the two tent nodes (x_mid: the middle of the step's
    displacement), each rounded once to the fixed-point unit."""
    prm = pic1d.Params(dt=DT, dx=DX, n_cells=64)
    M = prm.n_cells + 5
    E_hist = [(np.zeros(M), np.zeros(M)) for _ in range(prm.order + 1)]
    B_hist = [np.zeros(M) for _ in range(prm.order + 1)]
    px, py, wgt = 0.25, 0.75, 0.004
    x0 = 20.3 * DX
    sim = pic1d.Pic1d(prm, [x0], [px], [py], [0.0], [wgt], E_hist, B_hist)
    sim.step()
    g = math.sqrt(1 + px * px + py * py)
    s_mid = (x0 + 0.5 * DT * px / g) / DX
    i, f = math.floor(s_mid), s_mid - math.floor(s_mid)
    Q = round(wgt * 2 ** 44)
    D = sim.last_D
    assert abs(D[i + 2] + py / g * (1 - f) * Q) <= 1
    assert abs(D[i + 3] + py / g * f * Q) <= 1
    assert np.count_nonzero(D) == 2
    assert sim.stats.k_hist[0] == 1


def test_gauss_law_stays_at_roundoff_in_a_laser_plasma_run():
    """A small laser-plasma run (a0 = 20 pulse into a ramped plasma, 8
    electrons per cell): Gauss's law, div E_x = rho, holds to roundoff every
    step although the electrons sub-cycle and E_x grows."""
    wl = W.LaserPlasma1D(name="small", n_cells=1024, a0=20.0, fwhm=12.0, x_front=30.0,
                         x_top=55.0, scale_length=4.0, n_top=0.5, ppc=8, gap=2.0)
    prm = pic1d.Params(dt=wl.dt, dx=wl.dx, n_cells=wl.n_cells)
    E_hist, B_hist = wl.field_history()
    sim = pic1d.Pic1d(prm, *wl.particles(), E_hist, B_hist)
    worst = 0.0
    for n in range(400):
        sim.step()
        if n % 20 == 19:
            g, rmax = sim.gauss()
            worst = max(worst, g / rmax)
    assert worst < 1e-11, worst
    assert sum(sim.stats.k_hist[1:]) > 0                 # sub-cycling was exercised
    assert np.abs(sim.E[-1][0]).max() > 0.1               # charge separation built up


# ---------------------------------------------------------------- plasma response

def test_cold_plasma_oscillates_at_the_plasma_frequency():
    """A uniform cold plasma (n = 0.01 n_c, omega_p = sqrt(n) = 0.1) started
    neutral with a long-wavelength velocity perturbation: the momentum pattern
    oscillates at omega_p (cold fluid: dispersionless).  A wrong sign in the
    E_x - J_x coupling grows instead; a wrong factor shifts the frequency."""
    N, ppc, n0 = 512, 16, 0.01
    prm = pic1d.Params(dt=DT, dx=DX, n_cells=N)
    M = N + 5
    c = np.arange(4, N - 4, dtype=np.float64)
    x = ((c[:, None] + (np.arange(ppc) + 0.5)[None, :] / ppc) * DX).ravel()
    L = (N - 8) * DX
    kx = 2 * math.pi / L
    u0 = 1e-3
    px = u0 * np.sin(kx * (x - 4 * DX))
    z = np.zeros_like(x)
    E_hist = [(np.zeros(M), np.zeros(M)) for _ in range(prm.order + 1)]
    B_hist = [np.zeros(M) for _ in range(prm.order + 1)]
    sim = pic1d.Pic1d(prm, x, px, z, z, np.full_like(x, n0 / ppc), E_hist, B_hist)
    mode = np.sin(kx * (x - 4 * DX))
    S = []
    for _ in range(2000):
        sim.step()
        S.append(float(np.dot(sim.px, mode)))
    S = np.array(S)
    t = (np.arange(1, 2001) - 0.5) * DT                 # momentum time of each record
    zc = [t[i] - S[i] * (t[i + 1] - t[i]) / (S[i + 1] - S[i])
          for i in range(len(S) - 1) if S[i] * S[i + 1] < 0]
    assert len(zc) >= 4
    half_period = (zc[-1] - zc[0]) / (len(zc) - 1)
    omega = math.pi / half_period
    assert abs(omega / math.sqrt(n0) - 1) < 0.01, omega
    assert np.abs(S).max() <= 1.05 * np.abs(S[:10]).max()   # bounded: no growth

"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them compares the oracle with
itself: they use printed worked values, closed forms of the model problem
(Sec. II, App. A), textbook properties of Boris and of Lagrange interpolation,
library routines and convergence rates.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import _harness as H
from paper_2102_10983_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _node_offsets(p: int, field: str) -> np.ndarray:
    """Time of each level, in units of dt, relative to (n - 1/2) dt (Sec. VI):
    B level n+1/2+j-p sits at 1+j-p, E level n+j-p at 1/2+j-p."""
    j = np.arange(p + 1, dtype=np.float64)
    return (1.0 + j - p) if field == "B" else (0.5 + j - p)


# ---------------------------------------------------------------- Lagrange (Sec. VI)

def test_lagrange_worked_values_printed_in_paper():
    with open(os.path.join(GOLDEN, "lagrange_worked.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for field, p, theta, *ws in rows:
        got = oracle.lagrange(int(p), field, float(Fraction(theta)))
        want = np.array([float(Fraction(w)) for w in ws])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
@pytest.mark.parametrize("field", ["E", "B"])
def test_lagrange_reproduces_polynomials_and_matches_scipy(p, field):
    from scipy.interpolate import BarycentricInterpolator
    rng = np.random.default_rng(10 + p)
    nodes = _node_offsets(p, field)
    for theta in list(rng.uniform(0.0, 1.5, 12)) + [0.5, 1.0]:
        w = oracle.lagrange(p, field, theta)
        assert abs(w.sum() - 1.0) < 1e-13
        for deg in range(p + 1):                       # exact for degree <= p
            coef = rng.standard_normal(deg + 1)
            want = np.polyval(coef, theta)
            got = float(np.dot(w, np.polyval(coef, nodes)))
            assert abs(got - want) < 1e-11 * (1 + abs(want))
        for j in range(p + 1):                          # basis polynomial via scipy
            e = np.zeros(p + 1); e[j] = 1.0
            assert abs(BarycentricInterpolator(nodes, e)(theta) - w[j]) < 1e-10
    # theta = 1/2 is t = n dt: the E stencil hits its newest node exactly
    if field == "E":
        np.testing.assert_array_equal(oracle.lagrange(p, "E", 0.5), np.eye(p + 1)[p])


def test_interpolation_error_falls_with_order():
    """Fig. 4 / Sec. V: error of interpolating an analytic field to t = n dt from
    B at n+1/2 and earlier levels (dt = lambda/75) falls with the order."""
    dt = 2 * math.pi / 75
    errs = []
    for p in (1, 2, 3, 4, 5):
        worst = 0.0
        for phase in np.linspace(0, 2 * math.pi, 97):
            nodes = _node_offsets(p, "B")
            vals = np.cos(phase + nodes * dt)
            got = float(np.dot(oracle.lagrange(p, "B", 0.5), vals))
            worst = max(worst, abs(got - math.cos(phase + 0.5 * dt)))
        errs.append(worst)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    # first order: (dt/2)^2/2 max|f''| = 8.8e-4 for dt = lambda/75
    assert abs(errs[0] - (0.5 * dt) ** 2 / 2) < 1e-5 and errs[2] < 1e-5


# ---------------------------------------------------------------- Boris (Sec. III)

def test_boris_static_magnetic_field_rotation():
    """E = 0: |p| is conserved and each step rotates p by 2 atan(|Psi|),
    Psi = q B h / (2 gamma) (Eqs. eq:p - eq:gamman)."""
    p0 = np.array([3.0, -1.5, 0.7])
    gamma = math.sqrt(1 + p0 @ p0)
    for bz, h in [(1.0, 0.1), (50.0, 0.08), (-7.0, 0.3)]:
        p = p0.copy()
        psi = -1.0 * bz * h / (2 * gamma)
        for _ in range(200):
            q = oracle.boris(p, 0.0, bz, h)
            ang = math.atan2(p[0] * q[1] - p[1] * q[0], p[0] * q[0] + p[1] * q[1])
            assert abs(ang - (-2 * math.atan(psi))) < 1e-12
            p = q
        assert abs(np.linalg.norm(p) - np.linalg.norm(p0)) < 1e-12 * np.linalg.norm(p0)
        assert p[2] == p0[2]


def test_boris_uniform_electric_field_is_exact():
    """B = 0: p_y advances by q E h per step exactly (binary-exact inputs)."""
    p = np.array([0.25, -2.0, 0.5])
    for _ in range(64):
        p = oracle.boris(p, 1.5, 0.0, 0.125)
    np.testing.assert_array_equal(p, [0.25, -2.0 - 64 * 1.5 * 0.125, 0.5])


# ---------------------------------------------------------------- criterion (Sec. IV)

def _one_step_uniform(bz: float, dt: float, psi_max: float, order: int, k_max: int = 7):
    prm = oracle.Params(dt=dt, dx=1.0, psi_max=psi_max, order=order, k_max=k_max)
    parts = oracle.Particles([8.3], [0.0], [0.0], [0.0])
    W_ = 32
    E = np.zeros((order + 1, W_)); B = np.full((order + 1, W_), bz)
    i0 = np.zeros(order + 1, dtype=np.int64)
    st = oracle.push_step(prm, parts, E, i0, B, i0)
    return int(parts.status[0]), st


def _k_closed_form(psi0: Fraction, psi_max: Fraction, k_max: int):
    """Smallest k >= 0 with psi0 / 4^k <= psi_max, capped (Algorithm 1 loop)."""
    k = 0
    while psi0 / Fraction(4) ** k > psi_max and k < k_max:
        k += 1
    return k, psi0 / Fraction(4) ** k > psi_max


def test_criterion_matches_closed_form_including_ties():
    """p = 1 and a uniform field make B at t_n exact, so Psi0 = |B| dt / 2 at rest."""
    dt, psi_max = 0.5, 0.01
    rng = np.random.default_rng(5)
    cases = list(rng.uniform(0.0, 3000.0, 200))
    cases += [2 * psi_max * 4 ** j / dt for j in range(8)]               # exact ties
    cases += [np.nextafter(2 * psi_max * 4 ** j / dt, np.inf) for j in range(8)]
    for bz in cases:
        k, st = _one_step_uniform(float(bz), dt, psi_max, order=1)
        psi0 = Fraction(abs(float(bz))) * Fraction(dt) / 2
        want, clamped = _k_closed_form(psi0, Fraction(psi_max), 7)
        assert k == want, (bz, k, want)
        assert st.clamped == int(clamped)
        assert st.substeps == 4 ** want and st.k_hist[want] == 1
        assert st.n_star == (4 ** want if want > 0 else 0)


def test_criterion_cap_is_counted():
    k, st = _one_step_uniform(1e9, 0.5, 0.01, order=3, k_max=7)
    assert k == 7 and st.clamped == 1 and st.substeps == 4 ** 7


# ---------------------------------------------------------------- plane wave (Sec. II, App. A)

SMOOTH = dict(profile="gauss", xi0=12 * math.pi, sigma=2 * math.pi)


def _smooth_run(a0, order, psi_max, res, n=16, thermal=0.0, field_time=0, seed=3):
    from scipy.integrate import quad
    dt = 2 * math.pi / res
    wl = W.Workload(name="smooth", n_particles=n, a0=a0, dt=dt, dx=dt / 0.99, psi_max=psi_max,
                    order=order, n_steps=0, x_lo=0.0, x_hi=2 * math.pi, thermal_sigma=thermal,
                    seed=seed, **SMOOTH)
    wave = wl.wave
    xi_end = 24 * math.pi
    t_end = 2 * math.pi + xi_end + quad(lambda s: 0.5 * wave.a(s) ** 2, 0, xi_end, limit=500)[0]
    n_steps = int(t_end / dt) + 1
    prm = H.oracle_params(wl, field_time=field_time)
    parts = H.oracle_particles(wl)
    init = parts.copy()
    g0 = np.sqrt(1 + init.px ** 2 + init.py ** 2 + init.pz ** 2)
    r_ref = g0 - init.px
    r_dev = np.zeros(parts.n)
    worst = {"py": 0.0, "px": 0.0}

    def check(nn, P):
        g = np.sqrt(1 + P.px ** 2 + P.py ** 2 + P.pz ** 2)
        # momentum lives half a (last sub-)step h behind the position (Eq. eq:x)
        h = dt / 4.0 ** (P.status & 0x7F)
        xi_p = (nn * dt - 0.5 * h) - (P.x - 0.5 * h * P.px / g)
        a = wave.a(xi_p)
        worst["py"] = max(worst["py"], float(np.abs(P.py - init.py - a).max()) / a0)
        R0 = r_ref
        px_th = (1 + (a + init.py) ** 2 + init.pz ** 2 - R0 ** 2) / (2 * R0)
        worst["px"] = max(worst["px"], float(np.abs(P.px - px_th).max()) / (a0 * a0 / 2))

    st = H.run_oracle_follow(wl, prm, parts, 0, n_steps, chunk=200, r_ref=r_ref, r_dev=r_dev,
                             on_chunk=check)
    return dict(wl=wl, wave=wave, parts=parts, init=init, st=st, r_dev=r_dev, worst=worst,
                n_steps=n_steps, dt=dt)


def test_plane_wave_closed_form_smooth_pulse():
    """Electron from rest (Eqs. integral motion x, eq:6, theoretical dephasing):
    p_y = a, p_x = a^2/2, R = 1, and x(xi) = x0 + int a^2/2 dxi (dx/dxi = p_x/R,
    Eq. R-def).  Order 3 with sub-cycling (Sec. VI), a0 = 20, dt = lambda/75."""
    from scipy.integrate import quad
    r = _smooth_run(20.0, 3, 0.01, 75)
    assert r["st"].out_of_window == 0
    assert r["r_dev"].max() < 0.015                      # eps_dephasing, Eq. R error
    assert r["worst"]["py"] < 0.005 and r["worst"]["px"] < 0.01
    P, x0 = r["parts"], r["init"].x
    xi = r["n_steps"] * r["dt"] - P.x
    xth = x0 + np.array([quad(lambda s: 0.5 * r["wave"].a(s) ** 2, 0, q, limit=500)[0] for q in xi])
    assert np.abs(P.x - xth).max() < 0.012 * (xth - x0).max()
    assert r["st"].k_hist[3] > 0                         # sub-cycling was exercised


def test_paper_contrast_order_and_subcycling():
    """Sec. V-VI: order 3 with sub-cycling is far better than order 1 with
    sub-cycling and than order 3 without it."""
    e31 = _smooth_run(20.0, 3, 0.01, 75, n=4)["r_dev"].max()
    e11 = _smooth_run(20.0, 1, 0.01, 75, n=4)["r_dev"].max()
    e3n = _smooth_run(20.0, 3, 1e30, 75, n=4)["r_dev"].max()
    assert e31 * 10 < e11 and e31 * 5 < e3n, (e31, e11, e3n)


def test_general_invariants_thermal_start():
    """App. A: p_z, p_y - a and gamma - p_x are constant for any initial state."""
    r = _smooth_run(20.0, 3, 0.01, 75, n=16, thermal=W.MAXWELL_10KEV_SIGMA, seed=7)
    np.testing.assert_array_equal(r["parts"].pz, r["init"].pz)
    assert r["r_dev"].max() < 0.015
    assert r["worst"]["py"] < 0.005 and r["worst"]["px"] < 0.01


def test_second_order_convergence():
    """Without sub-cycling the integrator is second order: halving dt divides the
    dephasing error by ~4 (smooth pulse, a0 = 2, order 3)."""
    e = [_smooth_run(2.0, 3, 1e30, res, n=4)["r_dev"].max() for res in (40, 80, 160)]
    for a, b in zip(e, e[1:]):
        assert 3.3 < a / b < 4.8, e


# ---------------------------------------------------------------- sub-step field time (Sec. VI)

def _linear_in_time_kicks(field_time: int, order: int):
    """Two macro steps of a uniform E_y = alpha + beta t with a negligible B_z
    (1e-20) that only serves to make the criterion pick k = 2.  The rotation
    it causes is ~1e-21, far below FP64 rounding of p_y, so p_y gains exactly
    q sum_j E(tau_j) h_p(j): Lagrange interpolation of any order >= 1 is exact
    on a field linear in t, and tau_j is the sub-step's field time."""
    dt, alpha, beta, bz = 0.5, 0.75, -1.25, 1e-20
    psi0 = bz * dt / 2.0                     # at rest, gamma = 1
    prm = oracle.Params(dt=dt, dx=1.0, psi_max=psi0 / 10.0, order=order, field_time=field_time)
    parts = oracle.Particles([20.25], [0.0], [0.0], [0.0])
    W_, p = 64, order
    i0 = np.zeros(2 + p, dtype=np.int64)
    E = np.array([[alpha + beta * n * dt] * W_ for n in range(-p, 2)])
    B = np.full((2 + p, W_), bz)
    st = oracle.run(prm, parts, E, i0, B, i0)
    return float(parts.py[0]), st


def _kicks_closed_form(field_time: int) -> float:
    """q sum over the two steps of E(tau_j) h_p(j), exact rational arithmetic.
    Field time (Sec. VI, theta measured from t_n - dt/2 in units of dt):
    R1 (field_time 0) theta_j = 1/2 + (j-1)/m, R2 (field_time 1) theta_j = (j-1/2)/m.
    h_p = (h_old + h)/2 on j = 1 (the transitional step, Sec. IV), h after."""
    dt, alpha, beta = Fraction(1, 2), Fraction(3, 4), Fraction(-5, 4)
    m = 16
    h = dt / m
    total, h_old = Fraction(0), dt
    for n in (0, 1):
        for j in range(1, m + 1):
            theta = Fraction(1, 2) + Fraction(j - 1, m) if field_time == 0 else Fraction(2 * j - 1, 2 * m)
            tau = n * dt - dt / 2 + theta * dt
            hp = (h_old + h) / 2 if j == 1 else h
            total += -(alpha + beta * tau) * hp        # q = -1
        h_old = h
    return float(total)


@pytest.mark.parametrize("order", [1, 3])
def test_subcycle_field_time_readings(order):
    """Both readings of the sub-step field time, pinned by the field they must
    see: R1 at the position time t_n + (j-1)h, R2 in the middle of the j-th
    sub-interval of [t_n - dt/2, t_n + dt/2]."""
    got = {ft: _linear_in_time_kicks(ft, order) for ft in (0, 1)}
    for ft, (py, st) in got.items():
        assert st.k_hist[2] == 2 and st.substeps == 32
        want = _kicks_closed_form(ft)
        assert abs(py - want) <= 1e-14 * abs(want), (ft, py, want)
    assert abs(got[0][0] - got[1][0]) > 1e-3          # the two readings differ


# ---------------------------------------------------------------- window edge (Eqs. eq:Enp, eq:Bnp)

def test_window_edge_last_valid_node_and_one_past():
    """The tent gather reads nodes floor(s) and floor(s)+1 of the E grid
    (s = x/dx) and of the B grid (s - 1/2).  With every level's window on nodes
    [i0, i0 + W - 1], a particle is pushed iff i0 + 1/2 <= s < i0 + W - 1; one
    outside that range is frozen (status bit 7) where it stands and counted."""
    W_, i0v, p = 16, 5, 3
    lo, hi = i0v + 0.5, float(i0v + W_ - 1)
    xs = [lo, np.nextafter(lo, -np.inf), hi - 0.25, np.nextafter(hi, -np.inf), hi, hi + 0.5]
    inside = [True, False, True, True, False, False]
    prm = oracle.Params(dt=0.5, dx=1.0, psi_max=0.01, order=p)
    parts = oracle.Particles(xs, [0.0] * 6, [0.0] * 6, [0.0] * 6)
    i0 = np.full(p + 1, i0v, dtype=np.int64)
    E = np.zeros((p + 1, W_)); B = np.zeros((p + 1, W_))
    E[:, -1] = 2.0                    # the last node: a particle that gathers it gets a kick
    st = oracle.push_step(prm, parts, E, i0, B, i0)
    lost = (parts.status & 0x80) != 0
    assert list(~lost) == inside
    assert st.out_of_window == inside.count(False)
    np.testing.assert_array_equal(parts.x[lost], np.array(xs)[lost])     # frozen where it stands
    # the particle in the last cell: tent weight w = s - floor(s) on node W - 1,
    # q E w (h_old + h)/2 with h_old = h = dt
    w = (hi - 0.25) - math.floor(hi - 0.25)
    assert parts.py[2] == -2.0 * w * 0.5
    assert parts.py[3] == -2.0 * (np.nextafter(hi, -np.inf) - (hi - 1.0)) * 0.5

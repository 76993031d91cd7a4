"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 form: bit-exact positions, momenta, status bytes (k) and counters.
Mixed form: max |dp| / a0^2 <= 1e-4 and relative energy-gain difference
<= 1e-3 against the oracle (the stated budget of the mixed form).
All inputs are the seeded plane-wave workloads; the oracle and the GPU are fed
the same level arrays.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import _harness as H
from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import accuracy, native  # noqa: E402

P_OK_OR_RANGE = (native.PIC_OK, native.PIC_ERANGE, native.PIC_EKMAX)


def _c1(n, **kw):
    base = dict(name="c1_sized", n_particles=n, a0=100.0, dt=W.DT75, dx=2 * math.pi / 74.26,
                psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=2 * math.pi, window=256, lead=96)
    base.update(kw)
    return W.Workload(**base)


def _oracle_run(wl, n_steps, order=None, field_time=0, idx=None, k_max=7):
    prm = H.oracle_params(wl, order=order, field_time=field_time, k_max=k_max)
    parts = H.oracle_particles(wl)
    if idx is not None:
        parts = oracle.Particles(parts.x[idx], parts.px[idx], parts.py[idx], parts.pz[idx])
    st = H.run_oracle(wl, prm, parts, 0, n_steps)
    return parts, st


def _gpu_run(wl, n_steps, precision, order=None, field_time=0, schedule=0, k_max=7):
    p = wl.order if order is None else order
    integ = H.gpu_integrator(wl, precision, order=p, field_time=field_time, schedule=schedule,
                             k_max=k_max)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    run = H.GpuRun(integ, wl, p)
    st = run.run(0, n_steps, ok=P_OK_OR_RANGE)
    x, px, py, pz, status = integ.read_numpy()
    integ.close()
    return (x, px, py, pz, status), st


def _assert_bitwise(g, o, gst=None, ost=None):
    x, px, py, pz, status = g
    np.testing.assert_array_equal(status, o.status)
    np.testing.assert_array_equal(x, o.x)
    np.testing.assert_array_equal(px, o.px)
    np.testing.assert_array_equal(py, o.py)
    np.testing.assert_array_equal(pz, o.pz)
    if gst is not None:
        assert list(gst.k_hist) == list(ost.k_hist)[:8]
        assert gst.substeps == ost.substeps and gst.n_star == ost.n_star
        assert gst.clamped == ost.clamped and gst.out_of_window == ost.out_of_window


# ---------------------------------------------------------------- FP64: bit for bit

@pytest.mark.parametrize("order", [3, 1])
def test_fp64_bitwise_front_passage(order):
    """1000 electrons (several blocks + a ragged tail) through the switched-on
    front (k up to 5) and 2500 steps after it."""
    wl = _c1(1000, order=order)
    g, gst = _gpu_run(wl, 2500, native.PIC_FP64)
    o, ost = _oracle_run(wl, 2500)
    assert ost.k_hist[5] > 0
    _assert_bitwise(g, o, gst, ost)


@pytest.mark.parametrize("order,field_time", [(2, 0), (4, 0), (5, 0), (3, 1)])
def test_fp64_bitwise_other_orders_and_field_time(order, field_time):
    wl = _c1(257, order=order, seed=11)
    g, gst = _gpu_run(wl, 700, native.PIC_FP64, field_time=field_time)
    o, ost = _oracle_run(wl, 700, field_time=field_time)
    _assert_bitwise(g, o, gst, ost)


@pytest.mark.parametrize("n", [1, 31, 33])
def test_fp64_bitwise_tiny_and_ragged(n):
    wl = _c1(n, seed=20 + n)
    g, gst = _gpu_run(wl, 400, native.PIC_FP64)
    o, ost = _oracle_run(wl, 400)
    _assert_bitwise(g, o, gst, ost)


def test_fp64_bitwise_kmax_cap_and_mixed_k_in_one_warp():
    """Strong field and small Psi_max: k = 7 capped next to k = 0 lanes."""
    wl = _c1(64, a0=3000.0, psi_max=0.002, seed=5)
    g, gst = _gpu_run(wl, 200, native.PIC_FP64)
    o, ost = _oracle_run(wl, 200)
    assert ost.k_hist[7] > 0 and ost.clamped > 0 and ost.k_hist[0] > 0
    _assert_bitwise(g, o, gst, ost)


def test_fp64_window_exit_is_frozen_identically():
    """A window that lags behind the particles: they leave it, are frozen and
    counted (PIC_ERANGE), identically on both sides."""
    wl = _c1(96, lead=40, seed=9)
    g, gst = _gpu_run(wl, 300, native.PIC_FP64)
    o, ost = _oracle_run(wl, 300)
    assert ost.out_of_window > 0
    assert ((g[4] & native.PIC_STATUS_LOST) != 0).sum() == ost.out_of_window
    _assert_bitwise(g, o, gst, ost)


def test_fp64_full_c1_sampled():
    """Config 1 at full size and length (256 electrons until every one reaches
    xi = 2 pi): the oracle recomputes a sample of 12 electrons one by one."""
    wl = W.C1
    g, gst = _gpu_run(wl, wl.n_steps, native.PIC_FP64)
    idx = np.random.default_rng(0).choice(wl.n_particles, 12, replace=False)
    o, _ = _oracle_run(wl, wl.n_steps, idx=idx)
    _assert_bitwise(tuple(a[idx] for a in g), o)
    # The switched-on front (E jumps from 0 to a0 at xi = 0, and no grid
    # resolves the jump) leaves the electrons with R = gamma - p_x spread far
    # from the closed form's R = 1, in the method itself: the oracle, run on
    # all 256 electrons, loses 152 out of the back of the moving window (large
    # R: fast in xi) and ends the kept ones at R in [0.42, 1.59] and xi in
    # [3.1, 7.1], not at xi >= 2 pi.  So the closed-form check of this
    # configuration is not asserted here; it is pinned on the smooth pulse
    # (test_plane_wave_closed_form_smooth_pulse).  What holds on this front:
    # the same bits as the oracle (above), frozen electrons counted alike.
    kept = (g[4] & native.PIC_STATUS_LOST) == 0
    assert gst.out_of_window == (~kept).sum() and kept.any()


@pytest.mark.parametrize("k_max,psi_max", [(0, 0.01), (7, 1e30)])
def test_fp64_bitwise_degenerate_criterion(k_max, psi_max):
    """The criterion's degenerate ends: k_max = 0 (no sub-cycling; every step
    past the threshold counted as capped) and Psi_max = 1e30 (the criterion
    never fires): both reduce to the standard PIC push of Sec. III, bit for
    bit, counters included."""
    wl = _c1(300, psi_max=psi_max)
    g, gst = _gpu_run(wl, 400, native.PIC_FP64, k_max=k_max)
    o, ost = _oracle_run(wl, 400, k_max=k_max)
    _assert_bitwise(g, o, gst, ost)
    assert gst.k_hist[0] == sum(gst.k_hist) and gst.substeps == gst.k_hist[0]
    assert (gst.clamped > 0) == (k_max == 0)


@pytest.mark.parametrize("k_max,psi_max", [(0, 0.01), (7, 1e30)])
def test_mixed_binned_bitwise_plain_degenerate_criterion(k_max, psi_max):
    wl = _c1(300, psi_max=psi_max)
    a, sa = _gpu_run(wl, 400, native.PIC_MIXED, k_max=k_max, schedule=native.PIC_SCHED_PLAIN)
    b, sb = _gpu_run(wl, 400, native.PIC_MIXED, k_max=k_max, schedule=native.PIC_SCHED_BINNED)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert list(sa.k_hist) == list(sb.k_hist) and sa.clamped == sb.clamped


def test_empty_particle_set():
    """No electrons loaded: every form and schedule steps through the levels,
    launches nothing that touches particles, and reports zero counts."""
    wl = _c1(8)
    for precision, schedule in ((native.PIC_FP64, native.PIC_SCHED_PLAIN),
                                (native.PIC_MIXED, native.PIC_SCHED_PLAIN),
                                (native.PIC_MIXED, native.PIC_SCHED_BINNED)):
        integ = H.gpu_integrator(wl, precision, schedule=schedule, capacity=8)
        z = np.empty(0)
        integ.pic_particles_write(z, z, z, z)
        st = H.GpuRun(integ, wl, wl.order).run(0, 20)
        assert sum(st.k_hist) == 0 and st.substeps == 0 and st.out_of_window == 0
        assert all(len(a) == 0 for a in integ.read_numpy())
        integ.close()


def test_full_size_headline_workload_sampled():
    """The 16,777,216-electron a0 = 150 Maxwellian workload at full size and in
    the launch configuration the benchmark times (one multi-step call over a ring
    holding every level, binned mixed schedule), through its first 120 steps while
    the front sweeps the first electrons.  The FP64 form is checked against the
    oracle bit for bit on electrons the oracle recomputes one by one (the first
    ones, which the front hits and which sub-cycle, and random ones); the binned
    mixed form is checked against the FP64 form on every electron."""
    wl = W.C2
    p, K = wl.order, 120
    E, B, i0 = wl.levels(-p, K + p)
    ini = wl.particles()

    def run(precision, schedule):
        integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=precision,
                                  schedule=schedule, capacity=wl.n_particles, window=wl.window,
                                  ring_levels=K + p + 1)
        integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
        for r in range(K + p):
            integ.pic_fields_upload(r - p, int(i0[r]), E[r], B[r])
        st, _ = integ.pic_push_step(0, K, want_stats=True, ok=P_OK_OR_RANGE)
        out = integ.read_numpy()
        integ.close()
        return out, st

    g64, st64 = run(native.PIC_FP64, native.PIC_SCHED_PLAIN)
    gmx, stmx = run(native.PIC_MIXED, native.PIC_SCHED_BINNED)
    assert st64.k_hist[5] > 0, "the front must reach the first electrons"
    idx = np.concatenate([np.arange(48),
                          np.random.default_rng(5).choice(wl.n_particles, 48, replace=False)])
    o, _ = _oracle_run(wl, K, idx=idx)
    _assert_bitwise(tuple(a[idx] for a in g64), o)
    assert abs(stmx.substeps - st64.substeps) <= 0.01 * st64.substeps
    # the mixed form on the unresolved front: the backward-error criterion
    # (accuracy.backward_error_ok) on every electron, in the same launch
    # configuration
    dev = torch.device("cuda")
    init = [torch.as_tensor(a, device=dev) for a in (ini.x, ini.px, ini.py, ini.pz)]
    del g64, gmx
    u = accuracy.BACKWARD_ULPS
    res = accuracy.front_accuracy(native, wl, init, K, E, B, i0, K + p + 1,
                                  torch.cuda.current_stream(), native.PIC_SCHED_BINNED,
                                  unresolved=True, ulps=(u,))
    ok, why = accuracy.backward_error_ok(res, u)
    assert ok, (why, res)


# ---------------------------------------------------------------- mixed form: within budget

def _mixed_errors(g, o, a0, x0):
    x, px, py, pz, status = g
    dp = np.max(np.abs(np.stack([px - o.px, py - o.py, pz - o.pz])))
    gam_g = np.sqrt(1 + px ** 2 + py ** 2 + pz ** 2) - 1
    gam_o = np.sqrt(1 + o.px ** 2 + o.py ** 2 + o.pz ** 2) - 1
    de = abs(gam_g.mean() - gam_o.mean()) / max(gam_o.mean(), 1e-300)
    dx = np.max(np.abs(x - o.x) / np.maximum(np.abs(o.x - x0), 1.0))
    return dp / a0 ** 2, de, dx


@pytest.mark.parametrize("order", [3, 1])
def test_mixed_within_budget_front_passage(order):
    """Switched-on front: E jumps from 0 to a0 and no grid resolves the jump.
    The electrons it throws to large R = gamma - p_x sit on 4^k thresholds of
    the criterion for many steps, where any perturbation flips k for some of
    them: the FP64 method itself is hypersensitive there.  The mixed form is
    held to 0.1 % energy gain and 1 % sub-steps against the oracle (1000
    electrons), and to the backward-error criterion (accuracy.backward_error_ok)
    against the FP64 form on 16,384 electrons of the same workload (a fraction
    needs a sample large enough to count)."""
    wl = _c1(1000, order=order)
    g, gst = _gpu_run(wl, 2500, native.PIC_MIXED)
    o, ost = _oracle_run(wl, 2500)
    _, de, _ = _mixed_errors(g, o, wl.a0, wl.particles().x)
    assert de <= 1e-3, de
    assert abs(gst.substeps - ost.substeps) <= 0.01 * ost.substeps
    wl = _c1(16384, order=order)
    p = wl.order
    E, B, i0 = wl.levels(-p, 2500 + p)
    ini = wl.particles()
    init = [torch.as_tensor(a, device="cuda") for a in (ini.x, ini.px, ini.py, ini.pz)]
    u = accuracy.BACKWARD_ULPS_BY_ORDER[order]
    res = accuracy.front_accuracy(native, wl, init, 2500, E, B, i0, 2500 + p + 1,
                                  torch.cuda.current_stream(), native.PIC_SCHED_PLAIN,
                                  unresolved=True, ulps=(u,))
    ok, why = accuracy.backward_error_ok(res, u)
    assert ok, (why, res)


@pytest.mark.parametrize("order", [3, 1])
def test_mixed_within_budget_smooth_pulse(order):
    """Resolved (Gaussian-enveloped) wave at a0 = 150, thermal start, through
    several stopping points with sub-cycling: the whole ensemble stays within
    max |dp|/a0^2 <= 1e-4 and 0.1 % energy gain of the FP64 oracle."""
    wl = W.Workload(name="smooth_mixed", n_particles=1000, a0=150.0, dt=W.DT75,
                    dx=W.DT75 / 0.99, psi_max=0.01, order=order, n_steps=0, x_lo=0.0,
                    x_hi=2 * math.pi, thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=12,
                    window=1024, lead=200, profile="gauss", xi0=8 * math.pi, sigma=2 * math.pi)
    g, gst = _gpu_run(wl, 3000, native.PIC_MIXED)
    o, ost = _oracle_run(wl, 3000)
    assert ost.k_hist[4] > 0 and ost.out_of_window == 0
    dp, de, dx = _mixed_errors(g, o, wl.a0, wl.particles().x)
    assert dp <= 1e-4 and de <= 1e-3, (dp, de, dx)

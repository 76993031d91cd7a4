"""The self-consistent 1D3V PIC loop on the GPU against its oracle, bit for bit.

Same inputs on both sides (workloads.LaserPlasma1D: a laser pulse in vacuum
heading into a ramped plasma): after each run the electrons (positions,
momenta, status bytes), the newest field level (E_x, E_y, B_z) and the
counters must be identical, and the Gauss residual that the GPU measures
on the device must equal the oracle's.  The fixed-point deposit makes the
order of the GPU's atomic additions irrelevant, so nothing is left to
tolerance.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pic1d
from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402


def _small(**kw):
    base = dict(name="sc_small", n_cells=1024, a0=20.0, fwhm=12.0, x_front=30.0, x_top=55.0,
                scale_length=4.0, n_top=0.5, ppc=8, gap=2.0)
    base.update(kw)
    return W.LaserPlasma1D(**base)


def _run_both(wl, steps, order=3, field_time=0, k_max=7, gauss_every=0, chunks=None):
    p = order
    x, px, py, pz, w = wl.particles()
    E_hist, B_hist = W.LaserPlasma1D(**{**wl.__dict__, "order": p}).field_history()
    prm = pic1d.Params(dt=wl.dt, dx=wl.dx, n_cells=wl.n_cells, psi_max=wl.psi_max, order=p,
                       k_max=k_max, field_time=field_time)
    sim = pic1d.Pic1d(prm, x, px, py, pz, w, E_hist, B_hist)
    worst = 0.0
    for n in range(steps):
        sim.step()
        if gauss_every and (n + 1) % gauss_every == 0:
            worst = max(worst, sim.gauss()[0])
    g = native.Sc1d(wl.dt, wl.dx, wl.n_cells, psi_max=wl.psi_max, order=p, k_max=k_max,
                    field_time=field_time, capacity=len(x), gauss_every=gauss_every)
    g.particles_write(x, px, py, pz, w)
    for lev, ((ex, ey), bz) in enumerate(zip(E_hist, B_hist)):
        g.fields_write(lev - p, ex, ey, bz)
    st = native.PicSc1dStats()
    n0 = 0
    for c in (chunks or [steps]):
        s = g.step(n0, c)
        for k in range(8):
            st.k_hist[k] += s.k_hist[k]
        st.substeps += s.substeps
        st.n_star += s.n_star
        st.clamped += s.clamped
        st.frozen += s.frozen
        st.gauss_residual = max(st.gauss_residual, s.gauss_residual)
        n0 += c
    out = g.read_numpy()
    fields = g.fields_numpy(steps)
    g.close()
    return sim, worst, out, fields, st


def _assert_same(sim, worst, out, fields, st, gauss=False):
    x, px, py, pz, status = out
    np.testing.assert_array_equal(status, sim.status)
    np.testing.assert_array_equal(x, sim.x)
    np.testing.assert_array_equal(px, sim.px)
    np.testing.assert_array_equal(py, sim.py)
    np.testing.assert_array_equal(pz, sim.pz)
    ex, ey = sim.E[-1]
    np.testing.assert_array_equal(fields[0], ex)
    np.testing.assert_array_equal(fields[1], ey)
    np.testing.assert_array_equal(fields[2], sim.B[-1])
    o = sim.stats
    assert list(st.k_hist) == list(o.k_hist)[:8]
    assert (st.substeps, st.n_star, st.clamped, st.frozen) == (o.substeps, o.n_star, o.clamped,
                                                               o.frozen)
    if gauss:
        assert st.gauss_residual == worst


@pytest.mark.parametrize("order,field_time", [(3, 0), (1, 0), (3, 1), (5, 0)])
def test_sc1d_bitwise_laser_plasma(order, field_time):
    """A pulse (a0 = 20) through a ramped plasma, 400 steps: the electrons
    sub-cycle, E_x builds up; everything bit for bit, Gauss residual included."""
    wl = _small()
    sim, worst, out, fields, st = _run_both(wl, 400, order=order, field_time=field_time,
                                            gauss_every=25, chunks=[150, 1, 249])
    _assert_same(sim, worst, out, fields, st, gauss=True)
    assert sum(st.k_hist[1:]) > 0 and np.abs(fields[0]).max() > 0.1
    assert worst < 1e-11 * max(np.abs(fields[0]).max(), 1.0)


def test_sc1d_bitwise_frozen_at_the_edge_and_capped():
    """Electrons driven out of the right end (the plasma reaches the edge) are
    frozen with their charge; k capped at 2 is counted."""
    wl = _small(n_cells=256, a0=60.0, x_front=12.0, x_top=14.0, scale_length=1.0, ppc=5,
                tail_gap=1)
    sim, worst, out, fields, st = _run_both(wl, 600, k_max=2, gauss_every=100)
    _assert_same(sim, worst, out, fields, st, gauss=True)
    assert st.frozen > 0 and st.clamped > 0


def test_sc1d_vacuum_and_empty():
    """No electrons: the Yee solver alone, bit for bit."""
    wl = _small(n_cells=512, n_top=0.0)
    sim, worst, out, fields, st = _run_both(wl, 300)
    assert sim.x.shape[0] == 0
    _assert_same(sim, worst, out, fields, st)


def test_sc1d_full_size_configuration_first_steps():
    """The full self-consistent configuration (20,000 cells, 100 electrons per
    cell: 1.76M electrons, a0 = 150) through its first 110 steps -- the front
    of the pulse reaches the ramp -- in one multi-step call, against the whole
    oracle run: every electron and field value bit for bit."""
    wl = W.laser_plasma_c5()
    sim, worst, out, fields, st = _run_both(wl, 110, gauss_every=55)
    _assert_same(sim, worst, out, fields, st, gauss=True)

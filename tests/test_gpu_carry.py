"""Carried calls (pic_params.carry): a call leaves the long sub-cycles its last
step deferred to the next call instead of finishing them in a closing launch.
Only the order of work changes, so every result, counter and k is the plain
schedule's; reads, new particles and a changed predictor finish or drop the
carried work, and an upload that would replace a level it still needs is
refused.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import _harness as H
from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402


def _wl(n, **kw):
    base = dict(name="carry", n_particles=n, a0=150.0, dt=W.DT75, dx=W.DT75 / 0.99,
                psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=8 * math.pi,
                thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=4, window=1024, lead=200)
    base.update(kw)
    return W.Workload(**base)


def _make(wl, schedule, call_lens, carry=0, heavy_budget=0, order=3):
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=order, precision=native.PIC_MIXED,
                              schedule=schedule, capacity=wl.n_particles, window=wl.window,
                              ring_levels=order + 1 + max(carry, 1) + max(call_lens),
                              heavy_budget=heavy_budget, carry=carry)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    return integ


def _add(agg, st):
    """agg += st (the counters the closing launch of pic_finish or of a read
    adds: the criteria of steps that carried particles still had to take)."""
    for k in range(8):
        agg.k_hist[k] += st.k_hist[k]
    agg.substeps += st.substeps
    agg.n_star += st.n_star
    agg.clamped += st.clamped
    agg.out_of_window += st.out_of_window
    return agg


def _same(a, sa, b, sb):
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert list(sa.k_hist) == list(sb.k_hist)
    assert (sa.substeps, sa.n_star, sa.clamped, sa.out_of_window) == \
           (sb.substeps, sb.n_star, sb.clamped, sb.out_of_window)


_PLAIN = {}


def _plain(wl, n_steps, call_lens, order=3):
    key = (wl.n_particles, wl.seed, n_steps, tuple(call_lens), order)
    if key not in _PLAIN:
        integ = _make(wl, native.PIC_SCHED_PLAIN, call_lens, order=order)
        st = H.run_gpu_calls(integ, wl, order, 0, n_steps, call_lens)
        _PLAIN[key] = (integ.read_numpy(), st)
        integ.close()
    return _PLAIN[key]


@pytest.mark.parametrize("budget", [0, 5])
@pytest.mark.parametrize("carry", [1, 3])
@pytest.mark.parametrize("call_lens", [[1], [7, 64, 3]])
def test_carried_calls_are_bitwise_plain(call_lens, carry, budget):
    """One step per call (the field solver's rhythm) and calls of mixed
    lengths; with a budget of 5 sub-steps per launch the long sub-cycles
    (k up to 5) span many launches and, with carry = 3, calls."""
    wl = _wl(4097)
    a, sa = _plain(wl, 1000, call_lens)
    integ = _make(wl, native.PIC_SCHED_BINNED, call_lens, carry=carry, heavy_budget=budget)
    sb = H.run_gpu_calls(integ, wl, 3, 0, 1000, call_lens)
    b = integ.read_numpy()  # finishes the carried sub-cycles first
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    assert sa.k_hist[5] > 0, "the front must reach the electrons"
    _same(a, sa, b, sb)


@pytest.mark.parametrize("every", [1, 5])
def test_carried_predicted_schedule_is_bitwise_plain(every):
    """The refresh cadence runs over the carried run (not per call), with an
    untrained network that mispredicts most sub-cycling electrons."""
    wl = _wl(5000)
    net = native.Predictor(seed=123)
    a, sa = _plain(wl, 900, [1])
    integ = _make(wl, native.PIC_SCHED_PREDICTED, [1], carry=1)
    integ.attach_predictor(net, every)
    sb = H.run_gpu_calls(integ, wl, 3, 0, 900, [1])
    b = integ.read_numpy()
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    net.close()
    assert sa.k_hist[5] > 0
    _same(a, sa, b, sb)


def test_reads_in_the_middle_finish_and_the_run_continues():
    """A read (of the whole store or of the status bytes) finishes the carried
    sub-cycles; the next call starts a new run from the public state."""
    wl = _wl(3000)
    a, sa = _plain(wl, 900, [1])
    integ = _make(wl, native.PIC_SCHED_BINNED, [1], carry=2, heavy_budget=5)
    s1 = H.run_gpu_calls(integ, wl, 3, 0, 450, [1])
    mid = integ.read_numpy()
    assert not np.any(mid[4] & 0x78), "public status bytes after the read"
    s2 = H.run_gpu_calls(integ, wl, 3, 450, 450, [1])
    integ.pic_finish()
    integ.pic_finish()  # nothing carried: a no-op
    b = integ.read_numpy()
    sb = _add(_add(native.PicStepStats(), s1), s2)
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    _same(a, sa, b, sb)


def test_new_particles_drop_carried_work():
    """pic_particles_write in the middle of a carried run: the old particles'
    queues are dropped and the new set runs as in a fresh context."""
    wl = _wl(3000)
    a, sa = _plain(wl, 600, [1])
    integ = _make(wl, native.PIC_SCHED_BINNED, [1], carry=1)
    s0 = H.run_gpu_calls(integ, wl, 3, 0, 500, [1])  # the front sub-cycles some of them
    assert s0.k_hist[4] > 0
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    sb = H.run_gpu_calls(integ, wl, 3, 0, 600, [1])
    b = integ.read_numpy()
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    _same(a, sa, b, sb)


def test_upload_refuses_a_level_carried_work_needs():
    wl = _wl(2000)
    p = 3
    integ = _make(wl, native.PIC_SCHED_BINNED, [1], carry=1)
    R = integ.ring_levels
    S = 420
    H.run_gpu_calls(integ, wl, p, 0, S + 1, [1])  # the last step pushed: S
    E, B, i0 = wl.levels(S - p, 2 * R)
    lib = native.lib()

    def upload(level):
        r = level - (S - p)
        return lib.pic_fields_upload(integ.ctx, level, int(i0[r]), E[r].ctypes.data,
                                     B[r].ctypes.data, native.PIC_HOST)

    # step S's carried sub-cycles need levels S - p .. S; level L replaces L - R
    for level in range(S + 1, S - p + R):
        assert upload(level) == native.PIC_OK
    assert upload(S - p + R) == native.PIC_EINVAL
    assert b"carried" in lib.pic_last_error(integ.ctx)
    integ.pic_finish()
    assert upload(S - p + R) == native.PIC_OK
    integ.close()


def test_stream_change_in_the_middle_of_a_carried_run():
    """pic_set_stream while sub-cycles are carried: the library waits for the
    old stream, the run continues on the new one with the plain bits."""
    wl = _wl(3000)
    a, sa = _plain(wl, 600, [1])
    integ = _make(wl, native.PIC_SCHED_BINNED, [1], carry=1, heavy_budget=5)
    s1 = H.run_gpu_calls(integ, wl, 3, 0, 300, [1])
    other = torch.cuda.Stream()
    integ.set_stream(other)
    E, B, i0 = wl.levels(300, 300)
    sb = _add(native.PicStepStats(), s1)
    for r in range(300):  # level s, then step s, on the new stream
        integ.pic_fields_upload(300 + r, i0[r], E[r], B[r])
        st, _ = integ.pic_push_step(300 + r, 1, want_stats=True, ok=(0, 4, 5))
        _add(sb, st)
    b = integ.read_numpy()
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    _same(a, sa, b, sb)


@pytest.mark.parametrize("order", [1, 5])
def test_carried_calls_other_orders(order):
    """First and fifth order (p + 1 levels per step, ring order + 1 + carry +
    the longest call), carry 2, budget 7."""
    wl = _wl(2049, order=order)
    a, sa = _plain(wl, 700, [1, 5], order=order)
    integ = _make(wl, native.PIC_SCHED_BINNED, [1, 5], carry=2, heavy_budget=7, order=order)
    sb = H.run_gpu_calls(integ, wl, order, 0, 700, [1, 5])
    b = integ.read_numpy()
    _add(sb, integ.pic_stats_read(reset=True))
    integ.close()
    assert sa.k_hist[4] > 0
    _same(a, sa, b, sb)

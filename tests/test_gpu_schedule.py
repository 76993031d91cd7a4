"""The binned schedule (k > 0 pushes compacted into per-k queues and deferred
to the next step's kernel) gives exactly the bits of the plain schedule: both
call the same per-particle arithmetic; only the order of work differs.
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
    base = dict(name="sched", n_particles=n, a0=150.0, dt=W.DT75, dx=W.DT75 / 0.99,
                psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=8 * math.pi,
                thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=4, window=1024, lead=200)
    base.update(kw)
    return W.Workload(**base)


def _run(wl, schedule, n_steps, call_lens, order=3, heavy_budget=0):
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=order, precision=native.PIC_MIXED,
                              schedule=schedule, capacity=wl.n_particles, window=wl.window,
                              ring_levels=order + 2 + max(call_lens), heavy_budget=heavy_budget)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    st = H.run_gpu_calls(integ, wl, order, 0, n_steps, call_lens)
    out = integ.read_numpy()
    integ.close()
    return out, st


@pytest.mark.parametrize("call_lens", [[1], [7, 64, 3], [400]])
@pytest.mark.parametrize("n", [5000, 4097])
def test_binned_bitwise_equals_plain(call_lens, n):
    wl = _wl(n)
    a, sa = _run(wl, native.PIC_SCHED_PLAIN, 1200, call_lens)
    b, sb = _run(wl, native.PIC_SCHED_BINNED, 1200, call_lens)
    assert sa.k_hist[5] > 0, "the front must reach the electrons"
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert list(sa.k_hist) == list(sb.k_hist)
    assert (sa.substeps, sa.n_star, sa.clamped, sa.out_of_window) == \
           (sb.substeps, sb.n_star, sb.clamped, sb.out_of_window)


@pytest.mark.parametrize("budget", [5, 64, -1])
@pytest.mark.parametrize("call_lens", [[1], [9, 90, 40]])
def test_binned_resumable_long_subcycles_are_bitwise_plain(budget, call_lens):
    """With a budget of a few sub-steps per launch the electrons the front hits
    (k up to 5: 1,024 sub-steps) stop in the middle of their sub-cycles, run
    many steps behind the stream and catch up; the results, counters and k of
    every step stay the plain schedule's."""
    wl = _wl(3000)
    a, sa = _run(wl, native.PIC_SCHED_PLAIN, 1000, call_lens)
    b, sb = _run(wl, native.PIC_SCHED_BINNED, 1000, call_lens, heavy_budget=budget)
    assert sa.k_hist[5] > 0
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert list(sa.k_hist) == list(sb.k_hist)
    assert (sa.substeps, sa.n_star, sa.clamped, sa.out_of_window) == \
           (sb.substeps, sb.n_star, sb.clamped, sb.out_of_window)


@pytest.mark.parametrize("order", [1, 5])
def test_binned_bitwise_other_orders_and_window_exit(order):
    wl = _wl(1000, lead=60, window=256)   # a short window: some electrons leave it
    a, sa = _run(wl, native.PIC_SCHED_PLAIN, 600, [50], order=order)
    b, sb = _run(wl, native.PIC_SCHED_BINNED, 600, [50], order=order, heavy_budget=7)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert sa.out_of_window == sb.out_of_window
    assert list(sa.k_hist) == list(sb.k_hist)


def _run_pred(wl, n_steps, call_lens, predictor, every, order=3):
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=order, precision=native.PIC_MIXED,
                              schedule=native.PIC_SCHED_PREDICTED, capacity=wl.n_particles,
                              window=wl.window, ring_levels=order + 2 + max(call_lens))
    integ.attach_predictor(predictor, every)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    st = H.run_gpu_calls(integ, wl, order, 0, n_steps, call_lens)
    out = integ.read_numpy()
    integ.close()
    return out, st


@pytest.mark.parametrize("every", [1, 5])
def test_predicted_bitwise_equals_plain_even_with_an_untrained_network(every):
    """The network only orders the work: with random weights it mispredicts
    most sub-cycling electrons, and the results are still the plain bits."""
    wl = _wl(5000)
    net = native.Predictor(seed=123)
    a, sa = _run(wl, native.PIC_SCHED_PLAIN, 1200, [7, 64, 3])
    b, sb = _run_pred(wl, 1200, [7, 64, 3], net, every)
    assert sa.k_hist[5] > 0
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert list(sa.k_hist) == list(sb.k_hist)
    assert (sa.substeps, sa.n_star, sa.out_of_window) == (sb.substeps, sb.n_star, sb.out_of_window)
    net.close()


def test_trained_predictor_gains_over_the_unbinned_method():
    """What the network buys: the same steps of a 2M-electron slice of the
    a0 = 150 Maxwellian workload (electrons in random order) with the
    front among the electrons, timed
    with the plain (unbinned) schedule and with the predicted schedule driven by
    a network trained on pairs the integrator logged; same bits, and the
    predicted schedule must be at least 1.5x faster.  Exact-k binning is timed
    too, for the record."""
    from paper_2102_10983_gb300 import predictor
    X, Y, _ = predictor.c1_style_training_set(n_electrons=16384, steps=300)
    net = native.Predictor(seed=1)
    predictor.train(net, X, Y, iters=300)
    # electrons in random order: the layout a thermal plasma has once it has mixed
    wl = W.Workload(**{**W.C2.__dict__, "n_particles": 2_097_152, "seed": 8, "sort_x": False})
    p, start, K = 3, 600, 60
    E, B, i0 = wl.levels(-p, start + K + p)
    ini = wl.particles()
    results = {}
    for name, sched in (("plain", native.PIC_SCHED_PLAIN), ("binned", native.PIC_SCHED_BINNED),
                        ("predicted", native.PIC_SCHED_PREDICTED)):
        integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                                  schedule=sched, capacity=wl.n_particles, window=wl.window,
                                  ring_levels=start + K + p + 1)
        if sched == native.PIC_SCHED_PREDICTED:
            integ.attach_predictor(net, 4)
        integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
        for r in range(start + K + p):
            integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
        integ.pic_push_step(0, start, want_stats=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        integ.pic_push_step(start, K, want_stats=False)
        b.record()
        torch.cuda.synchronize()
        results[name] = (a.elapsed_time(b), integ.read_numpy())
        integ.close()
    for u, v in zip(results["plain"][1], results["predicted"][1]):
        np.testing.assert_array_equal(u, v)
    t_plain, t_bin, t_pred = (results[k][0] for k in ("plain", "binned", "predicted"))
    print(f"ms per step: plain {t_plain / K:.3f} binned {t_bin / K:.3f} predicted {t_pred / K:.3f}")
    assert t_plain / t_pred >= 1.5, (t_plain, t_bin, t_pred)
    net.close()

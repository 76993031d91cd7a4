"""PIC_ETIMEOUT reporting of the context API, through the C ABI.

A bounded device wait that gives up (the binned kernel's wait for a staged
tile) sets the context's device error word and leaves the step early.  Making
a real wait run out would need a broken copy, so the word is set from the host
(pic_inject_error), as the give-up path would set it, and the host's handling
is checked: the next pic_push_step with stats returns PIC_ETIMEOUT with the
word in stats.error, the word is then cleared, and the context keeps working.
"""
from __future__ import annotations

import math

import pytest

from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402


@pytest.mark.parametrize("precision,schedule", [(native.PIC_FP64, native.PIC_SCHED_PLAIN),
                                                (native.PIC_MIXED, native.PIC_SCHED_BINNED)])
def test_device_error_word_is_reported_as_timeout(precision, schedule):
    wl = W.Workload(name="err", n_particles=777, a0=20.0, dt=W.DT75, dx=W.DT75 / 0.99,
                    psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=2 * math.pi, window=256,
                    lead=96)
    p = wl.order
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=precision,
                              schedule=schedule, capacity=wl.n_particles, window=wl.window,
                              ring_levels=p + 4)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    E, B, i0 = wl.levels(-p, p + 3)
    for r in range(p + 3):
        integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
    st, code = integ.pic_push_step(0, 1, want_stats=True)
    assert code == native.PIC_OK and st.error == 0
    integ.inject_error(5)
    st, code = integ.pic_push_step(1, 1, want_stats=True, ok=(native.PIC_ETIMEOUT,))
    assert code == native.PIC_ETIMEOUT and st.error == 5
    assert b"error word" in native.lib().pic_last_error(integ.ctx)
    # reported once: the counters (and the word) were reset with the report
    st, code = integ.pic_push_step(2, 1, want_stats=True)
    assert code == native.PIC_OK and st.error == 0
    # pic_stats_read returns the word too (its own status stays PIC_OK)
    integ.inject_error(1)
    st = native.PicStepStats()
    rc = native.lib().pic_stats_read(integ.ctx, native.ctypes.byref(st), 1)
    assert rc == native.PIC_OK and st.error == 1
    integ.close()

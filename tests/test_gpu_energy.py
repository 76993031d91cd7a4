"""The energy-balance diagnostic of the FP64 form (App. B) against the oracle.

With diagnostics = PIC_DIAG_WORK the FP64 push accumulates, per particle, the
work of the electric field over every Boris push; it must equal the oracle's
accumulation bit for bit (same order of the same FP64 operations), through the
front passage with sub-cycling, and the particles themselves stay identical.
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

from paper_2102_10983_gb300 import native  # noqa: E402


@pytest.mark.parametrize("profile", ["sine", "gauss"])
def test_work_bitwise_against_oracle(profile):
    wl = W.Workload(name="work", n_particles=777, a0=60.0, dt=W.DT75, dx=W.DT75 / 0.99,
                    psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=2 * math.pi, window=512,
                    lead=160, profile=profile, xi0=6 * math.pi, sigma=2 * math.pi,
                    thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=8)
    steps = 1500
    prm = H.oracle_params(wl)
    parts = H.oracle_particles(wl)
    work = np.zeros(parts.n)
    p = wl.order
    done = 0
    while done < steps:
        c = min(500, steps - done)
        E, B, i0 = wl.levels(done - p, c + p)
        oracle.run(prm, parts, E, i0, B, i0, work=work)
        done += c
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_FP64,
                              capacity=wl.n_particles, window=wl.window, ring_levels=p + 2,
                              diagnostics=native.PIC_DIAG_WORK)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    H.GpuRun(integ, wl, p).run(0, steps, ok=(0, 4, 5))
    got = integ.work_read()
    x, px, py, pz, st = integ.read_numpy()
    integ.close()
    np.testing.assert_array_equal(px, parts.px)
    np.testing.assert_array_equal(got, work)
    assert np.abs(work).max() > 1.0
    # the balance: kinetic energy gained vs work done, per electron
    g0 = np.sqrt(1 + ini.px ** 2 + ini.py ** 2 + ini.pz ** 2)
    g = np.sqrt(1 + px ** 2 + py ** 2 + pz ** 2)
    kept = (st & native.PIC_STATUS_LOST) == 0
    assert np.median(np.abs((g - g0) - work)[kept]) < 1e-2 * np.abs(work[kept]).max()

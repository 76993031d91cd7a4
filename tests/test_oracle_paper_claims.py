"""The oracle against the paper's own accuracy statements (Gaussian pulse of
Eq. laser1, sigma = 8 pi, centred at xi0 = +160 pi so that an electron starting
at rest at x = 0 meets the whole pulse; dt = lambda/75, c dt/dx = 0.99).

 - Sec. VII: order 3 with sub-cycling (Psi_max = 0.01) keeps eps_dephasing < 0.1
   for 5 <= a0 <= 100 at this resolution (checked at a0 = 100, the hardest end).
 - Sec. IV: with first-order interpolation the peak energy at a0 = 100 comes out
   several times too low, with sub-cycling as well (the paper: about three times).
The two long single-electron runs go in parallel threads (the C call releases
the GIL).
"""
from __future__ import annotations

import math
import threading

import numpy as np
import pytest

import oracle
import _harness as H
from paper_2102_10983_gb300 import workloads as W


def _pulse_run(a0, order, psi_max, out, key):
    from scipy.integrate import quad
    dt = 2 * math.pi / 75
    wl = W.Workload(name="paper_pulse", n_particles=1, a0=a0, dt=dt, dx=dt / 0.99,
                    psi_max=psi_max, order=order, n_steps=0, x_lo=0.0, x_hi=0.0,
                    profile="gauss", xi0=160 * math.pi, sigma=8 * math.pi)
    wave = wl.wave
    xi_end = 320 * math.pi
    t_end = xi_end + quad(lambda s: 0.5 * wave.a(s) ** 2, 0, xi_end, limit=2000)[0]
    n_steps = int(t_end / dt) + 1
    parts = oracle.Particles([0.0], [0.0], [0.0], [0.0])
    r_ref, r_dev = np.ones(1), np.zeros(1)
    gmax = [1.0]

    def cb(nn, P):
        gmax[0] = max(gmax[0], math.sqrt(1 + P.px[0] ** 2 + P.py[0] ** 2 + P.pz[0] ** 2))

    st = H.run_oracle_follow(wl, H.oracle_params(wl), parts, 0, n_steps, chunk=200,
                             r_ref=r_ref, r_dev=r_dev, on_chunk=cb)
    out[key] = dict(eps=float(r_dev[0]), gmax_ratio=gmax[0] / (1 + a0 * a0 / 2), st=st)


@pytest.mark.slow
def test_paper_accuracy_statements_a0_100():
    out = {}
    jobs = [(100.0, 3, 0.01, "p3_sub"), (100.0, 1, 0.01, "p1_sub")]
    ts = [threading.Thread(target=_pulse_run, args=(*j[:3], out, j[3])) for j in jobs]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert out["p3_sub"]["eps"] < 0.1, out["p3_sub"]
    assert abs(out["p3_sub"]["gmax_ratio"] - 1.0) < 0.1, out["p3_sub"]
    assert out["p3_sub"]["st"].n_star > 0
    assert 0.1 < out["p1_sub"]["gmax_ratio"] < 0.5, out["p1_sub"]
    assert out["p1_sub"]["eps"] > 1.0

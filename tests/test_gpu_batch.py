"""Batched ensembles: one launch per macro step for many independent problems
gives, for every ensemble, exactly the bits its own single-problem context
gives (same mixed-form arithmetic, binned schedule); the graph-captured path
and the autotuner change nothing in the results."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402

WIN = 512


def _ensembles():
    """Different a0, resolution, Psi_max, k cap, field-time reading and size
    (including empty and ragged ones)."""
    spec = [(100.0, 75, 0.01, 7, 0, 3000), (300.0, 25, 0.003, 7, 0, 1000), (10.0, 150, 0.03, 7, 1, 37),
            (30.0, 50, 0.01, 5, 0, 0), (150.0, 75, 0.01, 7, 0, 4097), (100.0, 150, 0.01, 7, 1, 1)]
    out = []
    for q, (a0, res, psi, kmax, ft, n) in enumerate(spec):
        dt = 2 * math.pi / res
        dx = dt / 0.99
        wl = W.Workload(name=f"ens{q}", n_particles=n, a0=a0, dt=dt, dx=dx, psi_max=psi, order=3,
                        n_steps=0, x_lo=0.0, x_hi=2 * math.pi, seed=100 + q, window=WIN,
                        lead=int(math.ceil(2 * math.pi / dx)) + 16)
        out.append((wl, kmax, ft))
    return out


def _single(wl, kmax, ft, steps, calls):
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=3, k_max=kmax, field_time=ft,
                              precision=native.PIC_MIXED, schedule=native.PIC_SCHED_BINNED,
                              capacity=max(wl.n_particles, 1), window=WIN,
                              ring_levels=3 + 2 + max(calls))
    ini = wl.particles()
    if wl.n_particles:
        integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    E, B, i0 = wl.levels(-3, steps + 3)
    for r in range(3):
        integ.pic_fields_upload(r - 3, i0[r], E[r], B[r])
    s, q = 0, 0
    agg = np.zeros(12, dtype=np.int64)
    while s < steps:
        c = min(calls[q % len(calls)], steps - s)
        q += 1
        for r in range(c):
            integ.pic_fields_upload(s + r, i0[s + r + 3], E[s + r + 3], B[s + r + 3])
        st, _ = integ.pic_push_step(s, c, want_stats=True, ok=(0, 4, 5))
        agg[:8] += np.array(list(st.k_hist))
        agg[8] += st.substeps
        agg[9] += st.out_of_window
        s += c
    out = integ.read_numpy() if wl.n_particles else [np.empty(0)] * 4 + [np.empty(0, np.uint8)]
    integ.close()
    return out, agg


def _batch(ens, steps, calls, graph=False, tune=False, budget=0):
    b = native.Batch([dict(dt=wl.dt, dx=wl.dx, psi_max=wl.psi_max, k_max=kmax, field_time=ft,
                           n_particles=wl.n_particles) for wl, kmax, ft in ens],
                     order=3, window=WIN, ring_levels=3 + 2 + max(calls),
                     stream=torch.cuda.current_stream())
    if budget:
        b.heavy_budget(budget)
    inis = [wl.particles() for wl, _, _ in ens]
    cat = [np.concatenate([getattr(i, f) for i in inis]) for f in ("x", "px", "py", "pz")]
    b.particles_write(*cat)
    levs = [wl.levels(-3, steps + 3) for wl, _, _ in ens]

    def upload(r):
        E = np.stack([lv[0][r] for lv in levs])
        B = np.stack([lv[1][r] for lv in levs])
        b.fields_upload(r - 3, [lv[2][r] for lv in levs], E, B)

    for r in range(3):
        upload(r)
    if graph:
        b.config(chunk=256, blocks_per_sm=1, use_graph=True)
    s, q = 0, 0
    agg = np.zeros(12, dtype=np.int64)
    tuned = None
    while s < steps:
        c = min(calls[q % len(calls)], steps - s)
        q += 1
        for r in range(c):
            upload(s + r + 3)
        if tune and tuned is None:
            before = b.read_numpy()
            tuned = b.autotune(s, min(c, 4))
            after = b.read_numpy()
            for u, v in zip(before, after):
                np.testing.assert_array_equal(u, v)
        st = b.push_step(s, c)
        agg[:8] += np.array(list(st.k_hist))
        agg[8] += st.substeps
        agg[9] += st.out_of_window
        s += c
    out = b.read_numpy()
    b.close()
    return out, agg, tuned


@pytest.mark.parametrize("calls,budget", [([1], 0), ([13, 40], 0), ([13, 40], 5), ([40], -1)])
def test_batch_bitwise_equals_single_contexts(calls, budget):
    """Budgets of 5 sub-steps per launch (long sub-cycles resumed over many
    launches, particles running behind the stream) and no limit."""
    ens = _ensembles()
    steps = 600
    got, gagg, _ = _batch(ens, steps, calls, budget=budget)
    off = 0
    tot = np.zeros(12, dtype=np.int64)
    for wl, kmax, ft in ens:
        want, agg = _single(wl, kmax, ft, steps, calls)
        n = wl.n_particles
        for u, v in zip(got, want):
            np.testing.assert_array_equal(u[off:off + n], v)
        tot += agg
        off += n
    np.testing.assert_array_equal(gagg, tot)
    assert tot[5] > 0  # someone needed 4^5 sub-steps


def test_batch_graph_and_autotune_change_nothing():
    ens = _ensembles()
    a, aa, _ = _batch(ens, 300, [50])
    b, bb, _ = _batch(ens, 300, [50], graph=True)
    c, cc, tuned = _batch(ens, 300, [50], tune=True)
    for u, v, w in zip(a, b, c):
        np.testing.assert_array_equal(u, v)
        np.testing.assert_array_equal(u, w)
    np.testing.assert_array_equal(aa, bb)
    np.testing.assert_array_equal(aa, cc)
    chunk, blocks, ms = tuned
    assert chunk in (128, 256, 512, 1024) and blocks >= 1 and ms > 0

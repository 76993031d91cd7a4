"""Drivers that feed seeded plane-wave levels to the oracle and to the CUDA path."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2102_10983_gb300.workloads import Workload


def oracle_params(wl: Workload, order: int | None = None, psi_max: float | None = None,
                  field_time: int = 0, k_max: int = 7) -> oracle.Params:
    return oracle.Params(dt=wl.dt, dx=wl.dx, psi_max=wl.psi_max if psi_max is None else psi_max,
                         order=wl.order if order is None else order, k_max=k_max,
                         field_time=field_time)


def oracle_particles(wl: Workload, n: int | None = None) -> oracle.Particles:
    ini = wl.particles(n)
    return oracle.Particles(ini.x, ini.px, ini.py, ini.pz)


def run_oracle(wl: Workload, prm: oracle.Params, parts: oracle.Particles, n0: int, n_steps: int,
               chunk: int = 20000, r_ref=None, r_dev=None, stats=None) -> oracle.OrcStats:
    """Macro steps n0 .. n0+n_steps-1 through the oracle, levels generated in chunks."""
    p = prm.order
    st = stats if stats is not None else oracle.OrcStats()
    done = 0
    while done < n_steps:
        c = min(chunk, n_steps - done)
        n = n0 + done
        E, B, i0 = wl.levels(n - p, c + p)
        oracle.run(prm, parts, E, i0, B, i0, st, r_ref, r_dev)
        done += c
    return st


def run_oracle_follow(wl: Workload, prm: oracle.Params, parts: oracle.Particles, n0: int,
                      n_steps: int, chunk: int = 48, margin: int = 6, r_ref=None, r_dev=None,
                      stats=None, on_chunk=None, work=None,
                      field_scale: float = 1.0) -> oracle.OrcStats:
    """Like run_oracle, with a small window that follows the particles (all
    levels of a chunk share one origin; particles move < 1 node per step).
    field_scale multiplies every field sample (a perturbation of the inputs)."""
    p = prm.order
    st = stats if stats is not None else oracle.OrcStats()
    done = 0
    while done < n_steps:
        c = min(chunk, n_steps - done)
        n = n0 + done
        alive = (parts.status & 0x80) == 0
        xs = parts.x[alive] if alive.any() else parts.x
        lo = int(np.floor(xs.min() / wl.dx)) - margin - c
        span = int(np.ceil(xs.max() / wl.dx)) - lo + c + margin
        W = 1 << max(4, int(span - 1).bit_length())
        i0 = np.full(c + p, lo, dtype=np.int64)
        from paper_2102_10983_gb300.workloads import sample_levels
        E, B = sample_levels(wl.wave, wl.dt, wl.dx, n - p, c + p, i0, W, rowwise=False)
        if field_scale != 1.0:
            E, B = E * field_scale, B * field_scale
        oracle.run(prm, parts, E, i0, B, i0, st, r_ref, r_dev, work)
        done += c
        if on_chunk is not None:
            on_chunk(n + c, parts)
    return st


# ---------------------------------------------------------------- CUDA path drivers

def gpu_integrator(wl: Workload, precision: int, order: int | None = None,
                   psi_max: float | None = None, field_time: int = 0, k_max: int = 7,
                   schedule: int = 0, capacity: int | None = None, ring_levels: int | None = None):
    from paper_2102_10983_gb300 import native
    p = wl.order if order is None else order
    cap = wl.n_particles if capacity is None else capacity
    return native.Integrator(wl.dt, wl.dx, wl.psi_max if psi_max is None else psi_max, order=p,
                             k_max=k_max, precision=precision, field_time=field_time,
                             schedule=schedule, capacity=cap, window=wl.window,
                             ring_levels=ring_levels if ring_levels is not None else p + 2)


class GpuRun:
    """Feeds levels to an Integrator: level s is uploaded right before step s."""

    def __init__(self, integ, wl: Workload, order: int):
        self.integ, self.wl, self.p = integ, wl, order
        self.next_level = None
        self.stats = []

    def run(self, n0: int, n_steps: int, chunk: int = 4096, want_stats: bool = True,
            ok=(0,), on_chunk=None):
        from paper_2102_10983_gb300 import native
        p = self.p
        if self.next_level is None:
            E, B, i0 = self.wl.levels(n0 - p, p)
            for r in range(p):
                self.integ.pic_fields_upload(n0 - p + r, i0[r], E[r], B[r])
            self.next_level = n0
        assert self.next_level == n0
        agg = native.PicStepStats()
        done = 0
        while done < n_steps:
            c = min(chunk, n_steps - done)
            E, B, i0 = self.wl.levels(n0 + done, c)
            for r in range(c):
                s = n0 + done + r
                self.integ.pic_fields_upload(s, i0[r], E[r], B[r])
                st, _ = self.integ.pic_push_step(s, 1, want_stats=want_stats, ok=ok)
                if st is not None:
                    for k in range(8):
                        agg.k_hist[k] += st.k_hist[k]
                    agg.substeps += st.substeps
                    agg.n_star += st.n_star
                    agg.clamped += st.clamped
                    agg.out_of_window += st.out_of_window
            done += c
            self.next_level = n0 + done
            if on_chunk is not None:
                on_chunk(n0 + done)
        return agg


def run_gpu_calls(integ, wl: Workload, order: int, n0: int, n_steps: int, call_lens,
                  ok=(0, 4, 5)):
    """Steps n0..n0+n_steps-1 as pic_push_step calls of the given lengths (cycled);
    each call's levels are uploaded first (the ring must hold p + 1 + max(call))."""
    from paper_2102_10983_gb300 import native
    p = order
    E, B, i0 = wl.levels(n0 - p, n_steps + p)
    for r in range(p):
        integ.pic_fields_upload(n0 - p + r, i0[r], E[r], B[r])
    agg = native.PicStepStats()
    s, q = n0, 0
    while s < n0 + n_steps:
        c = min(call_lens[q % len(call_lens)], n0 + n_steps - s)
        q += 1
        for r in range(c):
            lev = s + r
            integ.pic_fields_upload(lev, i0[lev - n0 + p], E[lev - n0 + p], B[lev - n0 + p])
        st, _ = integ.pic_push_step(s, c, want_stats=True, ok=ok)
        for k in range(8):
            agg.k_hist[k] += st.k_hist[k]
        agg.substeps += st.substeps
        agg.n_star += st.n_star
        agg.clamped += st.clamped
        agg.out_of_window += st.out_of_window
        s += c
    return agg

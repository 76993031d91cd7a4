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
                      stats=None, on_chunk=None) -> oracle.OrcStats:
    """Like run_oracle, with a small window that follows the particles (all
    levels of a chunk share one origin; particles move < 1 node per step)."""
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
        E, B = sample_levels(wl.wave, wl.dt, wl.dx, n - p, c + p, i0, W)
        oracle.run(prm, parts, E, i0, B, i0, st, r_ref, r_dev)
        done += c
        if on_chunk is not None:
            on_chunk(n + c, parts)
    return st

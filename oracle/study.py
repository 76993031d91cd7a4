"""Oracle of the single-electron studies of Secs. IV-VII (oracle/traj_oracle.c).

TEST INFRASTRUCTURE ONLY.  One electron from rest at x = 0 through the
Gaussian-enveloped plane wave of Eq. laser1 (sigma = 8 pi), the field sampled
on the grid at c dt/dx = 0.99 ("perfectly propagating PIC", Sec. III), the
method of Algorithm 1 with order-p interpolation; per run the dephasing and
energy errors (Eqs. R error, gamma error), N and N* (Sec. VII).  The pulse is
centred at xi0 = 6 sigma, so the electron starts where the field is below
a0 e^-18, and the run ends at t = 2 xi0 + int_0^{2 xi0} a^2/2 dxi, when the
electron is through the pulse (t - x = xi and dx/dxi = a^2/2 for R = 1).
Runs go in parallel threads (the C call releases the interpreter lock).
"""
from __future__ import annotations

import ctypes
import math
from concurrent.futures import ThreadPoolExecutor

from . import lib as _orc_lib

from paper_2102_10983_gb300.workloads import STUDY_SIGMA as SIGMA, STUDY_XI0 as XI0, study_steps


class TrjParams(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("xi0", ctypes.c_double), ("sigma", ctypes.c_double),
                ("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("field_time", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n_steps", ctypes.c_int64), ("x0", ctypes.c_double),
                ("field_scale", ctypes.c_double)]


class TrjResult(ctypes.Structure):
    _fields_ = [("eps_dephasing", ctypes.c_double), ("eps_energy", ctypes.c_double),
                ("gamma_max", ctypes.c_double), ("n_steps", ctypes.c_int64),
                ("n_star", ctypes.c_int64), ("substeps", ctypes.c_int64),
                ("k_hist", ctypes.c_int64 * 8), ("x", ctypes.c_double), ("px", ctypes.c_double),
                ("py", ctypes.c_double), ("pz", ctypes.c_double)]

    def as_dict(self):
        n, ns = self.n_steps, self.n_star
        return {"eps_dephasing": self.eps_dephasing, "eps_energy": self.eps_energy,
                "gamma_max": self.gamma_max, "N": n, "N_star": ns,
                "delta_steps": ns / (ns + n) if n + ns else 0.0, "substeps": self.substeps,
                "k_hist": list(self.k_hist), "final": (self.x, self.px, self.py, self.pz)}


def _lib():
    L = _orc_lib()
    if not hasattr(L, "_trj_bound"):
        L.trj_run.argtypes = [ctypes.POINTER(TrjParams), ctypes.POINTER(TrjResult)]
        L.trj_run.restype = None
        L._trj_bound = True
    return L


def n_steps_for(a0: float, dt: float) -> int:
    return study_steps(a0, dt)


def params(a0: float, order: int, psi_max: float, res: float, k_max: int = 7,
           field_time: int = 0, field_scale: float = 1.0) -> TrjParams:
    """One run: lambda/(c dt) = res, c dt/dx = 0.99; psi_max = inf: no sub-cycling.
    field_scale multiplies every field sample (a perturbation of the inputs)."""
    dt = 2 * math.pi / res
    return TrjParams(a0, XI0, SIGMA, dt, dt / 0.99, psi_max, -1.0, order, k_max, field_time, 0,
                     n_steps_for(a0, dt), 0.0, field_scale)


def run(cases, threads: int = 8):
    """cases: TrjParams; returns their results (dicts) in order."""
    L = _lib()

    def one(q):
        r = TrjResult()
        L.trj_run(ctypes.byref(q), ctypes.byref(r))
        return r.as_dict()

    with ThreadPoolExecutor(max_workers=threads) as pool:
        return list(pool.map(one, cases))

"""Oracle of the self-consistent 1D3V PIC step (Yee solver, sub-cycling push
with E_x, charge-conserving fixed-point deposit, Gauss's law).

TEST INFRASTRUCTURE ONLY (tests, the smoke check, the benchmark's CPU
baseline).  A ctypes binding of pic1d_oracle.c plus a plain driver that keeps
the field history the order-p interpolation of Sec. VI needs.  Shares no code
with the CUDA path.
"""
from __future__ import annotations

import ctypes
from collections import deque
from dataclasses import dataclass

import numpy as np

from . import lib as _orc_lib

SHIFT = 44  # fixed-point charge unit 2^-44 (n_c e)


class P1Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("field_time", ctypes.c_int32), ("n_cells", ctypes.c_int32)]


class P1Stats(ctypes.Structure):
    _fields_ = [("k_hist", ctypes.c_int64 * 16), ("substeps", ctypes.c_int64),
                ("n_star", ctypes.c_int64), ("clamped", ctypes.c_int64),
                ("frozen", ctypes.c_int64)]

    def as_dict(self):
        return {"k_hist": list(self.k_hist)[:8], "substeps": self.substeps, "n_star": self.n_star,
                "clamped": self.clamped, "frozen": self.frozen}


def lib():
    L = _orc_lib()
    if not hasattr(L, "_p1_bound"):
        P, i64, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.p1_push_deposit.argtypes = [ctypes.POINTER(P1Params), i64, P, P, P, P, P, P, P, P, P, P,
                                      P, ctypes.POINTER(P1Stats)]
        L.p1_push_deposit.restype = None
        L.p1_field_step.argtypes = [ctypes.POINTER(P1Params), P, P, P, P, P, P, P, P]
        L.p1_field_step.restype = None
        L.p1_rho.argtypes = [ctypes.POINTER(P1Params), i64, P, P, P]
        L.p1_rho.restype = None
        L.p1_gauss.argtypes = [ctypes.POINTER(P1Params), P, P, P, ctypes.POINTER(d)]
        L.p1_gauss.restype = d
        L.p1_boris.argtypes = [P, d, d, d, d, d]
        L.p1_boris.restype = None
        L.p1_charge_units.argtypes = [d]
        L.p1_charge_units.restype = i64
        L._p1_bound = True
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def boris(p3, ex, ey, bz, hp, qm=-1.0):
    v = np.ascontiguousarray(np.array(p3, dtype=np.float64))
    lib().p1_boris(_p(v), float(ex), float(ey), float(bz), float(hp), float(qm))
    return v


def charge_units(w):
    return np.array([lib().p1_charge_units(float(v)) for v in np.atleast_1d(w)], dtype=np.int64)


@dataclass
class Params:
    dt: float
    dx: float
    n_cells: int
    psi_max: float = 0.01
    order: int = 3
    k_max: int = 7
    qm: float = -1.0
    field_time: int = 0

    def c(self):
        return P1Params(self.dt, self.dx, self.psi_max, self.qm, self.order, self.k_max,
                        self.field_time, self.n_cells)


class Pic1d:
    """The PIC loop on the CPU: per macro step, the push and deposit of every
    particle with the levels of the history, then the field solve; the newest
    p + 1 levels of E (E_x, E_y) and B (B_z) are kept.

    E_hist / B_hist: lists of p + 1 (Ex, Ey) pairs and Bz arrays, oldest first,
    levels n0 - p .. n0 (E) and n0 + 1/2 - p .. n0 + 1/2 (B); arrays of
    n_cells + 5 entries (index = node or face + 2)."""

    def __init__(self, prm: Params, x, px, py, pz, w, E_hist, B_hist, n0: int = 0):
        self.prm, self.c = prm, prm.c()
        self.x = np.ascontiguousarray(x, dtype=np.float64).copy()
        self.px = np.ascontiguousarray(px, dtype=np.float64).copy()
        self.py = np.ascontiguousarray(py, dtype=np.float64).copy()
        self.pz = np.ascontiguousarray(pz, dtype=np.float64).copy()
        self.status = np.zeros(self.x.shape[0], np.uint8)
        self.Q = charge_units(w) if self.x.shape[0] else np.zeros(0, np.int64)
        M = prm.n_cells + 5
        assert len(E_hist) == prm.order + 1 and len(B_hist) == prm.order + 1
        self.E = deque([(np.ascontiguousarray(ex, dtype=np.float64).copy(),
                         np.ascontiguousarray(ey, dtype=np.float64).copy()) for ex, ey in E_hist])
        self.B = deque([np.ascontiguousarray(bz, dtype=np.float64).copy() for bz in B_hist])
        for ex, ey in self.E:
            assert ex.shape == (M,) and ey.shape == (M,)
        self.n = n0
        self.stats = P1Stats()
        self.C_ion = -self.rho_units()       # immobile ions: a neutral start

    def rho_units(self):
        C = np.zeros(self.prm.n_cells + 5, np.int64)
        if self.x.shape[0]:
            lib().p1_rho(ctypes.byref(self.c), self.x.shape[0], _p(self.x), _p(self.Q), _p(C))
        return C

    def step(self):
        p = self.prm.order
        M = self.prm.n_cells + 5
        F = np.zeros(M, np.int64)
        D = np.zeros(M, np.int64)
        Ex = (ctypes.c_void_p * (p + 1))(*[e[0].ctypes.data for e in self.E])
        Ey = (ctypes.c_void_p * (p + 1))(*[e[1].ctypes.data for e in self.E])
        Bz = (ctypes.c_void_p * (p + 1))(*[b.ctypes.data for b in self.B])
        if self.x.shape[0]:
            lib().p1_push_deposit(ctypes.byref(self.c), self.x.shape[0], _p(self.x), _p(self.px),
                                  _p(self.py), _p(self.pz), _p(self.status), _p(self.Q), Ex, Ey,
                                  Bz, _p(F), _p(D), ctypes.byref(self.stats))
        ex0, ey0 = self.E[-1]
        bz0 = self.B[-1]
        ex1, ey1, bz1 = np.empty(M), np.empty(M), np.empty(M)
        lib().p1_field_step(ctypes.byref(self.c), _p(ex0), _p(ey0), _p(bz0), _p(F), _p(D),
                            _p(ex1), _p(ey1), _p(bz1))
        self.E.popleft()
        self.E.append((ex1, ey1))
        self.B.popleft()
        self.B.append(bz1)
        self.n += 1
        self.last_F, self.last_D = F, D

    def gauss(self):
        """(max Gauss residual over nodes -1 .. N+1, max |rho_e|) at the newest E level."""
        C = self.rho_units()
        rmax = ctypes.c_double()
        g = lib().p1_gauss(ctypes.byref(self.c), _p(self.E[-1][0]), _p(C), _p(self.C_ion),
                           ctypes.byref(rmax))
        return g, rmax.value

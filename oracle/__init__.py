"""Oracle for the adaptive electron sub-cycling particle integrator.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, serial FP64 CPU
restatement of the method of arXiv 2102.10983 (Algorithm 1 of Sec. IV, the Boris
pusher of Sec. III, the order-p temporal Lagrange interpolation of Sec. VI and
the tent gather of Eqs. eq:Enp / eq:Bnp).  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import it.  It shares no code with the
CUDA path; the two meet only through the seeded input generators in
``paper_2102_10983_gb300.workloads``.

Pins (see tests/test_oracle_*.py): Lagrange worked values (Eq. eq:2nd interp and
Eq. linear interp orig), polynomial reproduction, Boris textbook cases, the
closed-form plane-wave motion of Sec. II / App. A, the general plane-wave
invariants of App. A, the closed form of the criterion, and second-order
convergence.  The MLP part (``oracle.mlp``) is pinned by finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "pic1d_oracle.c"), os.path.join(_HERE, "traj_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                                 for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double),
                ("psi_max", ctypes.c_double), ("qm", ctypes.c_double),
                ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("field_time", ctypes.c_int32), ("pad", ctypes.c_int32)]


class OrcStats(ctypes.Structure):
    _fields_ = [("k_hist", ctypes.c_int64 * 16), ("substeps", ctypes.c_int64),
                ("n_star", ctypes.c_int64), ("clamped", ctypes.c_int64),
                ("out_of_window", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {"k_hist": list(self.k_hist)[:8], "substeps": self.substeps,
                "n_star": self.n_star, "clamped": self.clamped,
                "out_of_window": self.out_of_window}


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i32, i64, p = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        _lib.orc_lagrange.argtypes = [i32, i32, d, p]
        _lib.orc_lagrange.restype = None
        _lib.orc_boris.argtypes = [p, d, d, d, d]
        _lib.orc_boris.restype = None
        _lib.orc_push_step.argtypes = [ctypes.POINTER(OrcParams), i64, p, p, p, p, p,
                                       p, p, p, p, i64, ctypes.POINTER(OrcStats), p]
        _lib.orc_push_step.restype = i64
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lagrange(p: int, field: str, theta: float) -> np.ndarray:
    """Weights L^E_{p,j}(theta) or L^B_{p,j}(theta), j = 0..p (Sec. VI)."""
    w = np.zeros(p + 1, dtype=np.float64)
    lib().orc_lagrange(int(p), 1 if field == "E" else 0, float(theta), _ptr(w))
    return w


def boris(p3, ey: float, bz: float, hp: float, qm: float = -1.0) -> np.ndarray:
    """One Boris push (Sec. III) in the field E=(0,ey,0), B=(0,0,bz)."""
    v = np.ascontiguousarray(np.array(p3, dtype=np.float64))
    lib().orc_boris(_ptr(v), float(ey), float(bz), float(hp), float(qm))
    return v


@dataclass
class Params:
    dt: float
    dx: float
    psi_max: float
    order: int = 3
    k_max: int = 7
    qm: float = -1.0
    field_time: int = 0  # 0 position time, 1 sub-interval middle

    def c(self) -> OrcParams:
        return OrcParams(self.dt, self.dx, self.psi_max, self.qm, self.order, self.k_max,
                         self.field_time, 0)


class Particles:
    """SoA particle state for the oracle (x, px, py, pz f64; status u8)."""

    def __init__(self, x, px, py, pz, status=None):
        self.x = np.ascontiguousarray(x, dtype=np.float64).copy()
        self.px = np.ascontiguousarray(px, dtype=np.float64).copy()
        self.py = np.ascontiguousarray(py, dtype=np.float64).copy()
        self.pz = np.ascontiguousarray(pz, dtype=np.float64).copy()
        n = self.x.shape[0]
        self.status = (np.zeros(n, np.uint8) if status is None
                       else np.ascontiguousarray(status, dtype=np.uint8).copy())

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def copy(self) -> "Particles":
        return Particles(self.x, self.px, self.py, self.pz, self.status)


def push_step(prm: Params, parts: Particles, E_lv: np.ndarray, E_i0, B_lv: np.ndarray, B_i0,
              stats: OrcStats | None = None, work: np.ndarray | None = None) -> OrcStats:
    """One macro step of Algorithm 1 over all particles.

    E_lv, B_lv: (p+1, W) float64, ascending time (E levels n-p..n, B levels
    n+1/2-p..n+1/2); E_i0, B_i0: the global node index of each level's first node.
    """
    p = prm.order
    E_lv = np.ascontiguousarray(E_lv, dtype=np.float64)
    B_lv = np.ascontiguousarray(B_lv, dtype=np.float64)
    assert E_lv.shape == B_lv.shape and E_lv.shape[0] == p + 1
    W = E_lv.shape[1]
    e0 = np.ascontiguousarray(E_i0, dtype=np.int64)
    b0 = np.ascontiguousarray(B_i0, dtype=np.int64)
    assert e0.shape == (p + 1,) and b0.shape == (p + 1,)
    st = stats if stats is not None else OrcStats()
    c = prm.c()
    if work is not None:
        assert work.dtype == np.float64 and work.flags["C_CONTIGUOUS"] and work.shape == (parts.n,)
    lib().orc_push_step(ctypes.byref(c), parts.n, _ptr(parts.x), _ptr(parts.px), _ptr(parts.py),
                        _ptr(parts.pz), _ptr(parts.status), _ptr(E_lv), _ptr(e0), _ptr(B_lv),
                        _ptr(b0), W, ctypes.byref(st), None if work is None else _ptr(work))
    return st


def _bind_run():
    L = lib()
    if not hasattr(L, "_run_bound"):
        d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        L.orc_run.argtypes = [ctypes.POINTER(OrcParams), i64, i64, p, p, p, p, p, p, p, p, p, i64,
                              p, p, ctypes.POINTER(OrcStats), p]
        L.orc_run.restype = i64
        L._run_bound = True
    return L


def run(prm: Params, parts: Particles, E_all: np.ndarray, E_i0_all, B_all: np.ndarray, B_i0_all,
        stats: OrcStats | None = None, r_ref: np.ndarray | None = None,
        r_dev: np.ndarray | None = None, work: np.ndarray | None = None) -> OrcStats:
    """len(E_all) - p consecutive macro steps; row r of E_all/B_all is level n0 - p + r.

    r_ref/r_dev: optional per-particle dephasing reference and running max of
    |(gamma - p_x) - r_ref| (Eq. R error).
    """
    p = prm.order
    E_all = np.ascontiguousarray(E_all, dtype=np.float64)
    B_all = np.ascontiguousarray(B_all, dtype=np.float64)
    n_steps = E_all.shape[0] - p
    assert n_steps >= 1 and E_all.shape == B_all.shape
    W = E_all.shape[1]
    e0 = np.ascontiguousarray(E_i0_all, dtype=np.int64)
    b0 = np.ascontiguousarray(B_i0_all, dtype=np.int64)
    assert e0.shape == (n_steps + p,) and b0.shape == (n_steps + p,)
    st = stats if stats is not None else OrcStats()
    c = prm.c()
    rr = None if r_ref is None else _ptr(r_ref)
    rd = None if r_dev is None else _ptr(r_dev)
    if work is not None:
        assert work.dtype == np.float64 and work.flags["C_CONTIGUOUS"] and work.shape == (parts.n,)
    _bind_run().orc_run(ctypes.byref(c), n_steps, parts.n, _ptr(parts.x), _ptr(parts.px),
                        _ptr(parts.py), _ptr(parts.pz), _ptr(parts.status), _ptr(E_all), _ptr(e0),
                        _ptr(B_all), _ptr(b0), W, rr, rd, ctypes.byref(st),
                        None if work is None else _ptr(work))
    return st

"""Thin ctypes binding of the C ABI in include/pic_gb300.h.

Argument marshalling only: every step of the integrator runs in the CUDA
kernels of libpic_gb300.so.  The functions keep the C names.  Host arrays are
numpy arrays; device arrays are torch CUDA tensors (PyTorch provides device
memory and streams here, nothing else).  There is no CPU fallback: if the
library is missing or fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ERANGE, PIC_EKMAX, PIC_ETIMEOUT = range(7)
PIC_HOST, PIC_DEVICE = 0, 1
PIC_FP64, PIC_MIXED = 0, 1
PIC_SCHED_PLAIN, PIC_SCHED_BINNED, PIC_SCHED_PREDICTED = 0, 1, 2
PIC_DIAG_WORK = 1
PIC_STATUS_LOST = 0x80

ERR_NAMES = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECUDA", 4: "PIC_ERANGE",
             5: "PIC_EKMAX", 6: "PIC_ETIMEOUT"}


class PicParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("field_time", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("heavy_budget", ctypes.c_int32),
                ("diagnostics", ctypes.c_int32), ("carry", ctypes.c_int32)]


class PicEnsemble(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("k_max", ctypes.c_int32), ("field_time", ctypes.c_int32),
                ("n_particles", ctypes.c_int64)]


class PicStepStats(ctypes.Structure):
    _fields_ = [("k_hist", ctypes.c_int64 * 8), ("substeps", ctypes.c_int64),
                ("n_star", ctypes.c_int64), ("clamped", ctypes.c_int64),
                ("out_of_window", ctypes.c_int64), ("error", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"k_hist": list(self.k_hist), "substeps": self.substeps, "n_star": self.n_star,
                "clamped": self.clamped, "out_of_window": self.out_of_window, "error": self.error}


class PicSc1dParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("field_time", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("gauss_every", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class PicSc1dStats(ctypes.Structure):
    _fields_ = [("k_hist", ctypes.c_int64 * 8), ("substeps", ctypes.c_int64),
                ("n_star", ctypes.c_int64), ("clamped", ctypes.c_int64), ("frozen", ctypes.c_int64),
                ("gauss_residual", ctypes.c_double), ("rho_max", ctypes.c_double),
                ("checks", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"k_hist": list(self.k_hist), "substeps": self.substeps, "n_star": self.n_star,
                "clamped": self.clamped, "frozen": self.frozen,
                "gauss_residual": self.gauss_residual, "rho_max": self.rho_max,
                "checks": self.checks}


class PicStudyCase(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("xi0", ctypes.c_double), ("sigma", ctypes.c_double),
                ("dt", ctypes.c_double), ("dx", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("qm", ctypes.c_double), ("order", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("field_time", ctypes.c_int32), ("n_electrons", ctypes.c_int32),
                ("n_steps", ctypes.c_int64)]


class PicStudyResult(ctypes.Structure):
    _fields_ = [("eps_dephasing", ctypes.c_double), ("eps_energy", ctypes.c_double),
                ("gamma_max", ctypes.c_double), ("eps_dephasing_first", ctypes.c_double),
                ("eps_energy_first", ctypes.c_double), ("gamma_max_first", ctypes.c_double),
                ("n_star_mean", ctypes.c_double), ("n_steps", ctypes.c_int64),
                ("n_star_first", ctypes.c_int64), ("substeps", ctypes.c_int64),
                ("k_hist", ctypes.c_int64 * 8)]

    def as_dict(self) -> dict:
        n, ns = self.n_steps, self.n_star_mean
        return {"eps_dephasing": self.eps_dephasing, "eps_energy": self.eps_energy,
                "gamma_max": self.gamma_max, "eps_dephasing_first": self.eps_dephasing_first,
                "eps_energy_first": self.eps_energy_first,
                "gamma_max_first": self.gamma_max_first, "N": n, "N_star_mean": ns,
                "N_star_first": self.n_star_first,
                "delta_steps": ns / (ns + n) if n + ns else 0.0, "substeps": self.substeps,
                "k_hist": list(self.k_hist)}


# (name, restype, argtypes) of every symbol declared in include/*.h
_VP, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "pic_create": (ctypes.c_int, [ctypes.POINTER(PicParams), _I64, _I64, _I32, _VP,
                                  ctypes.POINTER(_VP)]),
    "pic_destroy": (ctypes.c_int, [_VP]),
    "pic_particles_write": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32]),
    "pic_particles_read": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32]),
    "pic_fields_upload": (ctypes.c_int, [_VP, _I64, _I64, _VP, _VP, _I32]),
    "pic_push_step": (ctypes.c_int, [_VP, _I64, _I64, ctypes.POINTER(PicStepStats)]),
    "pic_stats_read": (ctypes.c_int, [_VP, ctypes.POINTER(PicStepStats), _I32]),
    "pic_finish": (ctypes.c_int, [_VP]),
    "pic_batch_heavy_budget": (ctypes.c_int, [_VP, _I32]),
    "pic_noalloc_inject_error": (ctypes.c_int, [_I32, _VP]),
    "pic_set_stream": (ctypes.c_int, [_VP, _VP]),
    "pic_timing_enable": (ctypes.c_int, [_VP, _I32]),
    "pic_timing_read": (ctypes.c_int, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I64), _I32]),
    "pic_launch_count": (ctypes.c_int64, [_VP]),
    "pic_inject_error": (ctypes.c_int, [_VP, _I32]),
    "pic_work_read": (ctypes.c_int, [_VP, _VP, _I64, _I32]),
    "pic_last_error": (ctypes.c_char_p, [_VP]),
    "pic_features": (ctypes.c_int, [_VP, _I64, _VP]),
    "pic_predict": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "pic_attach_predictor": (ctypes.c_int, [_VP, _VP, _I32]),
    "pic_mlp_param_count": (ctypes.c_int, []),
    "pic_mlp_create": (ctypes.c_int, [ctypes.c_uint64, _VP, ctypes.POINTER(_VP)]),
    "pic_mlp_destroy": (ctypes.c_int, [_VP]),
    "pic_mlp_params": (ctypes.c_int, [_VP, _VP, _I32, _I32]),
    "pic_mlp_grad": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _VP]),
    "pic_mlp_train_step": (ctypes.c_int, [_VP, _VP, _VP, _I64, ctypes.c_float, _VP]),
    "pic_mlp_infer": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "pic_batch_create": (ctypes.c_int, [ctypes.POINTER(PicEnsemble), _I32, _I32, _I64, _I32, _VP,
                                        ctypes.POINTER(_VP)]),
    "pic_batch_destroy": (ctypes.c_int, [_VP]),
    "pic_batch_config": (ctypes.c_int, [_VP, _I32, _I32, _I32]),
    "pic_batch_particles_write": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I32]),
    "pic_batch_particles_read": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I32]),
    "pic_batch_fields_upload": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _I32]),
    "pic_batch_push_step": (ctypes.c_int, [_VP, _I64, _I64, ctypes.POINTER(PicStepStats)]),
    "pic_batch_timing": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "pic_batch_launch_count": (ctypes.c_int64, [_VP]),
    "pic_batch_autotune": (ctypes.c_int, [_VP, _I64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                          ctypes.POINTER(_D)]),
    "pic_batch_last_error": (ctypes.c_char_p, [_VP]),
    "pic_push_mixed_noalloc": (ctypes.c_int, [ctypes.POINTER(PicParams), _I64, _VP, _VP, _VP, _VP,
                                              _VP, _VP, _VP, _VP, _VP, _I64, _I64, _I64, _VP,
                                              ctypes.POINTER(PicStepStats)]),
    "pic_study_run": (ctypes.c_int, [ctypes.POINTER(PicStudyCase), _I32,
                                     ctypes.POINTER(PicStudyResult), _VP]),
    "pic_sc1d_create": (ctypes.c_int, [ctypes.POINTER(PicSc1dParams), _I64, _VP,
                                       ctypes.POINTER(_VP)]),
    "pic_sc1d_destroy": (ctypes.c_int, [_VP]),
    "pic_sc1d_particles_write": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32]),
    "pic_sc1d_particles_read": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32]),
    "pic_sc1d_fields_write": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _I32]),
    "pic_sc1d_fields_read": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _I32]),
    "pic_sc1d_step": (ctypes.c_int, [_VP, _I64, _I64, ctypes.POINTER(PicSc1dStats)]),
    "pic_sc1d_timing": (ctypes.c_int, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "pic_sc1d_launch_count": (ctypes.c_int64, [_VP]),
    "pic_sc1d_last_error": (ctypes.c_char_p, [_VP]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libpic_gb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and _build.needs_build():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libpic_gb300.so not built ({_build.LIB}); run build()")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, ctx=None, ok=(PIC_OK,)):
    if code not in ok:
        raise PicError(code, (lib().pic_last_error(ctx) or b"").decode())
    return code


def _ptr(a):
    """(address, where) of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, PIC_HOST
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), (PIC_DEVICE if a.is_cuda else PIC_HOST)
    raise TypeError(type(a))


def _where(*arrs):
    ws = {w for _, w in (_ptr(a) for a in arrs if a is not None)}
    if len(ws) != 1:
        raise ValueError("arrays must all be on the host or all on the device")
    return ws.pop()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    return getattr(stream, "cuda_stream", stream)


class Integrator:
    """One context of the C library (pic_create ... pic_destroy)."""

    def __init__(self, dt, dx, psi_max, order=3, k_max=7, precision=PIC_FP64, field_time=0,
                 schedule=PIC_SCHED_PLAIN, qm=-1.0, capacity=0, window=256, ring_levels=None,
                 stream=None, heavy_budget=0, diagnostics=0, carry=0):
        self.params = PicParams(float(dt), float(dx), float(psi_max), float(qm), int(order),
                                int(k_max), int(precision), int(field_time), int(schedule),
                                int(heavy_budget), int(diagnostics), int(carry))
        self.window = int(window)
        self.ring_levels = int(ring_levels if ring_levels is not None else order + 1)
        self.capacity = int(capacity)
        h = ctypes.c_void_p()
        _check(lib().pic_create(ctypes.byref(self.params), self.capacity, self.window,
                                self.ring_levels, _stream_handle(stream), ctypes.byref(h)))
        self.ctx = h
        self.n = 0

    def close(self):
        if getattr(self, "ctx", None):
            lib().pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib().pic_set_stream(self.ctx, _stream_handle(stream)), self.ctx)

    def pic_particles_write(self, x, px, py, pz, status=None):
        n = int(x.shape[0])
        w = _where(x, px, py, pz, status)
        _check(lib().pic_particles_write(self.ctx, _ptr(x)[0], _ptr(px)[0], _ptr(py)[0],
                                         _ptr(pz)[0], _ptr(status)[0], n, w), self.ctx)
        self.n = n

    def pic_particles_read(self, x=None, px=None, py=None, pz=None, status=None, n=None):
        arrs = [a for a in (x, px, py, pz, status) if a is not None]
        n = self.n if n is None else int(n)
        w = _where(*arrs)
        _check(lib().pic_particles_read(self.ctx, _ptr(x)[0], _ptr(px)[0], _ptr(py)[0],
                                        _ptr(pz)[0], _ptr(status)[0], n, w), self.ctx)

    def pic_fields_upload(self, level, i0, Ey, By):
        w = _where(Ey, By)
        assert Ey.shape[-1] == self.window and By.shape[-1] == self.window
        _check(lib().pic_fields_upload(self.ctx, int(level), int(i0), _ptr(Ey)[0], _ptr(By)[0],
                                       w), self.ctx)

    def pic_push_step(self, n, n_steps=1, want_stats=True, ok=(PIC_OK,)):
        st = PicStepStats() if want_stats else None
        code = lib().pic_push_step(self.ctx, int(n), int(n_steps),
                                   ctypes.byref(st) if st is not None else None)
        _check(code, self.ctx, ok=ok)
        return (st, code) if want_stats else (None, code)

    def pic_finish(self):
        _check(lib().pic_finish(self.ctx), self.ctx)

    def pic_stats_read(self, reset=True) -> PicStepStats:
        st = PicStepStats()
        _check(lib().pic_stats_read(self.ctx, ctypes.byref(st), 1 if reset else 0), self.ctx)
        return st

    def attach_predictor(self, predictor: "Predictor", every: int = 1):
        _check(lib().pic_attach_predictor(self.ctx, predictor.h, int(every)), self.ctx)
        self._predictor = predictor

    def timing(self, on: bool = True):
        _check(lib().pic_timing_enable(self.ctx, 1 if on else 0), self.ctx)

    def timing_read(self, reset: bool = True):
        ms, steps = ctypes.c_double(), ctypes.c_int64()
        _check(lib().pic_timing_read(self.ctx, ctypes.byref(ms), ctypes.byref(steps),
                                     1 if reset else 0), self.ctx)
        return ms.value, steps.value

    def launches(self) -> int:
        return int(lib().pic_launch_count(self.ctx))

    def work_read(self, work=None):
        """The per-particle work of E (PIC_DIAG_WORK contexts): numpy unless
        a device tensor is given."""
        out = np.empty(self.n) if work is None else work
        _check(lib().pic_work_read(self.ctx, _ptr(out)[0], self.n, _where(out)), self.ctx)
        return out

    def inject_error(self, word: int = 1):
        _check(lib().pic_inject_error(self.ctx, int(word)), self.ctx)

    # convenience: read everything to numpy
    def read_numpy(self):
        n = self.n
        out = [np.empty(n) for _ in range(4)] + [np.empty(n, np.uint8)]
        self.pic_particles_read(*out)
        return out


class Predictor:
    """The learned sub-cycle-count predictor (pic_mlp_*): device tensors in and out."""

    def __init__(self, seed: int = 0, stream=None):
        h = ctypes.c_void_p()
        _check(lib().pic_mlp_create(int(seed), _stream_handle(stream), ctypes.byref(h)))
        self.h = h
        self.n_params = int(lib().pic_mlp_param_count())

    def close(self):
        if getattr(self, "h", None):
            lib().pic_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        buf = np.empty(self.n_params, dtype=np.float32)
        _check(lib().pic_mlp_params(self.h, buf.ctypes.data, 0, PIC_HOST))
        return buf

    def set_params(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.float32)
        assert buf.shape == (self.n_params,)
        _check(lib().pic_mlp_params(self.h, buf.ctypes.data, 1, PIC_HOST))

    def grad(self, phi, label):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().pic_mlp_grad(self.h, phi.data_ptr(), label.data_ptr(), int(phi.shape[0]),
                                  g.ctypes.data, ctypes.byref(loss)))
        return g, float(loss.value)

    def train_step(self, phi, label, lr: float) -> float:
        loss = ctypes.c_float()
        _check(lib().pic_mlp_train_step(self.h, phi.data_ptr(), label.data_ptr(),
                                        int(phi.shape[0]), float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def infer(self, phi, pred):
        _check(lib().pic_mlp_infer(self.h, phi.data_ptr(), int(phi.shape[0]), pred.data_ptr()))


def predict(integ: "Integrator", net: "Predictor", n: int, pred):
    """pic_predict: the network's class for every particle after macro step n
    (features and inference in one pass)."""
    _check(lib().pic_predict(integ.ctx, net.h, int(n), pred.data_ptr()), integ.ctx)


def features(integ: "Integrator", n: int, phi):
    """pic_features: predictor inputs of every particle after macro step n."""
    _check(lib().pic_features(integ.ctx, int(n), phi.data_ptr()), integ.ctx)


def pack_params(P: dict) -> np.ndarray:
    """Oracle-style parameter dict -> the packed FP32 layout of pic_mlp_params."""
    return np.concatenate([np.asarray(P[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def unpack_params(buf) -> dict:
    buf = np.asarray(buf, dtype=np.float64)
    out, off = {}, 0
    for name, shape in (("W1", (64, 6)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                        ("W3", (8, 64)), ("b3", (8,))):
        size = int(np.prod(shape))
        out[name] = buf[off:off + size].reshape(shape)
        off += size
    return out


class Batch:
    """Batched ensembles (pic_batch_*): arrays are concatenated in ensemble order."""

    def __init__(self, ensembles, order=3, window=512, ring_levels=None, stream=None):
        arr = (PicEnsemble * len(ensembles))()
        for q, e in enumerate(ensembles):
            arr[q] = PicEnsemble(float(e["dt"]), float(e["dx"]), float(e["psi_max"]),
                                 float(e.get("qm", -1.0)), int(e.get("k_max", 7)),
                                 int(e.get("field_time", 0)), int(e["n_particles"]))
        self.n_ens = len(ensembles)
        self.counts = [int(e["n_particles"]) for e in ensembles]
        self.n_total = sum(self.counts)
        self.window = int(window)
        self.order = int(order)
        self.ring_levels = int(ring_levels if ring_levels is not None else order + 2)
        h = ctypes.c_void_p()
        code = lib().pic_batch_create(arr, self.n_ens, self.order, self.window, self.ring_levels,
                                      _stream_handle(stream), ctypes.byref(h))
        _check(code)
        self.h = h

    def _chk(self, code, ok=(PIC_OK,)):
        if code not in ok:
            raise PicError(code, (lib().pic_batch_last_error(self.h) or b"").decode())
        return code

    def close(self):
        if getattr(self, "h", None):
            lib().pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def heavy_budget(self, budget: int):
        self._chk(lib().pic_batch_heavy_budget(self.h, int(budget)))

    def config(self, chunk=256, blocks_per_sm=2, use_graph=False):
        self._chk(lib().pic_batch_config(self.h, int(chunk), int(blocks_per_sm), 1 if use_graph else 0))

    def particles_write(self, x, px, py, pz, status=None):
        w = _where(x, px, py, pz, status)
        self._chk(lib().pic_batch_particles_write(self.h, _ptr(x)[0], _ptr(px)[0], _ptr(py)[0],
                                                  _ptr(pz)[0], _ptr(status)[0], w))

    def read_numpy(self):
        out = [np.empty(self.n_total) for _ in range(4)] + [np.empty(self.n_total, np.uint8)]
        self._chk(lib().pic_batch_particles_read(self.h, *[o.ctypes.data for o in out], PIC_HOST))
        return out

    def fields_upload(self, level, i0, Ey, Bz):
        i0 = np.ascontiguousarray(i0, dtype=np.int64)
        w = _where(Ey, Bz)
        self._chk(lib().pic_batch_fields_upload(self.h, int(level), i0.ctypes.data, _ptr(Ey)[0],
                                                _ptr(Bz)[0], w))

    def push_step(self, n, n_steps=1, want_stats=True, ok=(PIC_OK, PIC_ERANGE, PIC_EKMAX)):
        st = PicStepStats() if want_stats else None
        code = lib().pic_batch_push_step(self.h, int(n), int(n_steps),
                                         ctypes.byref(st) if st is not None else None)
        self._chk(code, ok=ok)
        return st

    def timing(self, on=True):
        ms, steps = ctypes.c_double(), ctypes.c_int64()
        self._chk(lib().pic_batch_timing(self.h, 1 if on else 0, ctypes.byref(ms), ctypes.byref(steps)))
        return ms.value, steps.value

    def launches(self) -> int:
        return int(lib().pic_batch_launch_count(self.h))

    def autotune(self, n, steps=4):
        c, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        self._chk(lib().pic_batch_autotune(self.h, int(n), int(steps), ctypes.byref(c),
                                           ctypes.byref(b), ctypes.byref(ms)))
        return c.value, b.value, ms.value


class Sc1d:
    """The self-consistent 1D3V PIC loop of the C library (pic_sc1d_*)."""

    def __init__(self, dt, dx, n_cells, psi_max=0.01, order=3, k_max=7, field_time=0, qm=-1.0,
                 capacity=0, gauss_every=0, stream=None):
        self.params = PicSc1dParams(float(dt), float(dx), float(psi_max), float(qm), int(order),
                                    int(k_max), int(field_time), int(n_cells), int(gauss_every))
        self.n_cells = int(n_cells)
        self.M = self.n_cells + 5
        h = ctypes.c_void_p()
        self._chk(lib().pic_sc1d_create(ctypes.byref(self.params), int(capacity),
                                        _stream_handle(stream), ctypes.byref(h)), None)
        self.h = h
        self.n = 0

    def _chk(self, code, h="self", ok=(PIC_OK,)):
        if code not in ok:
            hh = self.h if h == "self" else h
            raise PicError(code, (lib().pic_sc1d_last_error(hh) or b"").decode())
        return code

    def close(self):
        if getattr(self, "h", None):
            lib().pic_sc1d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def particles_write(self, x, px, py, pz, w):
        n = int(x.shape[0])
        wh = _where(x, px, py, pz, w)
        self._chk(lib().pic_sc1d_particles_write(self.h, _ptr(x)[0], _ptr(px)[0], _ptr(py)[0],
                                                 _ptr(pz)[0], _ptr(w)[0], n, wh))
        self.n = n

    def particles_read(self, x=None, px=None, py=None, pz=None, status=None, n=None):
        arrs = [a for a in (x, px, py, pz, status) if a is not None]
        wh = _where(*arrs)
        self._chk(lib().pic_sc1d_particles_read(self.h, _ptr(x)[0], _ptr(px)[0], _ptr(py)[0],
                                                _ptr(pz)[0], _ptr(status)[0],
                                                self.n if n is None else int(n), wh))

    def fields_write(self, level, Ex, Ey, Bz):
        wh = _where(Ex, Ey, Bz)
        assert Ex.shape[-1] == self.M and Ey.shape[-1] == self.M and Bz.shape[-1] == self.M
        self._chk(lib().pic_sc1d_fields_write(self.h, int(level), _ptr(Ex)[0], _ptr(Ey)[0],
                                              _ptr(Bz)[0], wh))

    def fields_read(self, level, Ex, Ey, Bz):
        wh = _where(Ex, Ey, Bz)
        self._chk(lib().pic_sc1d_fields_read(self.h, int(level), _ptr(Ex)[0], _ptr(Ey)[0],
                                             _ptr(Bz)[0], wh))

    def step(self, n0, n_steps=1, want_stats=True, ok=(PIC_OK, PIC_EKMAX)):
        st = PicSc1dStats() if want_stats else None
        self._chk(lib().pic_sc1d_step(self.h, int(n0), int(n_steps),
                                      ctypes.byref(st) if st is not None else None), ok=ok)
        return st

    def timing(self):
        ms, steps = ctypes.c_double(), ctypes.c_int64()
        self._chk(lib().pic_sc1d_timing(self.h, ctypes.byref(ms), ctypes.byref(steps)))
        return ms.value, steps.value

    def launches(self) -> int:
        return int(lib().pic_sc1d_launch_count(self.h))

    def read_numpy(self):
        out = [np.empty(self.n) for _ in range(4)] + [np.empty(self.n, np.uint8)]
        self.particles_read(*out)
        return out

    def fields_numpy(self, level):
        out = [np.empty(self.M) for _ in range(3)]
        self.fields_read(level, *out)
        return out


def study_run(cases, stream=None):
    """pic_study_run on a list of dicts (a0, order, psi_max, res, n_electrons
    and optionally k_max, field_time, n_steps): lambda/(c dt) = res,
    c dt/dx = 0.99, the pulse of workloads.STUDY_*; returns result dicts."""
    from . import workloads as Wl
    arr = (PicStudyCase * len(cases))()
    for q, c in zip(arr, cases):
        dt = 2 * math.pi / c["res"]
        n_e = int(c.get("n_electrons", 1))
        steps = c.get("n_steps") or Wl.study_steps(c["a0"], dt, x_span=2 * math.pi * (n_e - 1) / n_e)
        q.a0, q.xi0, q.sigma = float(c["a0"]), Wl.STUDY_XI0, Wl.STUDY_SIGMA
        q.dt, q.dx, q.psi_max, q.qm = dt, dt / 0.99, float(c["psi_max"]), -1.0
        q.order, q.k_max, q.field_time = int(c["order"]), int(c.get("k_max", 7)), int(c.get("field_time", 0))
        q.n_electrons, q.n_steps = n_e, int(steps)
    out = (PicStudyResult * len(cases))()
    code = lib().pic_study_run(arr, len(cases), out, _stream_handle(stream))
    if code != PIC_OK:
        raise PicError(code, (lib().pic_last_error(None) or b"").decode())
    return [r.as_dict() for r in out]

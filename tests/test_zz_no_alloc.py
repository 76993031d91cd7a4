"""pic_push_mixed_noalloc against the context API, through the C ABI.

The allocation-free entry point serves host programs that may not allocate
device memory when they push particles (their device memory belongs to another
framework, or a real-time loop must stay away from the allocator): it works on
the caller's arrays and keeps its own working data in a fixed device array
inside the library.  It must give the same bits as the binned push of a
pic_create context on consecutive calls (each finds the previous call's
leftovers in that array), with the counters or without them (an asynchronous
call), after a change of parameters, and without allocating.

This file sorts last so that a run stopping at the first failure has run
every other test before it; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import pytest

from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402

OK_CODES = (native.PIC_OK, native.PIC_ERANGE, native.PIC_EKMAX)


def _wl(n, order=3):
    return W.Workload(name="noalloc", n_particles=n, a0=150.0, dt=W.DT75, dx=W.DT75 / 0.99,
                      psi_max=0.01, order=order, n_steps=0, x_lo=0.0, x_hi=8 * math.pi,
                      thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=21, window=1024, lead=200)


def _mixed_layout(x, dx):
    """x -> (cell, frac) as pic_particles_write does: s = x*(1/dx), frac = s - floor(s)."""
    s = x * (1.0 / dx)
    fl = np.floor(s)
    f = (s - fl).astype(np.float32)
    over = f >= 1.0
    f[over] = 0.0
    fl[over] += 1.0
    return fl.astype(np.int32), f


def _circular(vals, i0, W_):
    out = np.empty(W_, dtype=np.float32)
    out[(i0 + np.arange(W_)) & (W_ - 1)] = vals.astype(np.float32)
    return out


def _context_run(wl, calls, k_max=7, field_time=0):
    """The context API (binned mixed push) over the same calls; returns the
    final state and each call's counters."""
    p = wl.order
    ini = wl.particles()
    E, B, i0 = wl.levels(-p, sum(c for _, c in calls) + p)
    ref = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, k_max=k_max,
                            precision=native.PIC_MIXED, field_time=field_time,
                            schedule=native.PIC_SCHED_BINNED, capacity=wl.n_particles,
                            window=wl.window, ring_levels=p + 2 + max(c for _, c in calls))
    ref.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    for r in range(p):
        ref.pic_fields_upload(r - p, i0[r], E[r], B[r])
    stats = []
    for n0, c in calls:
        for lev in range(n0, n0 + c):
            ref.pic_fields_upload(lev, i0[lev + p], E[lev + p], B[lev + p])
        st, _ = ref.pic_push_step(n0, c, want_stats=True, ok=OK_CODES)
        stats.append(st.as_dict())
    out = ref.read_numpy()
    ref.close()
    return out, stats


class NoAllocRun:
    """Caller-owned device arrays and FP32 levels for pic_push_mixed_noalloc."""

    def __init__(self, wl, n_levels):
        self.wl = wl
        p = wl.order
        dev = torch.device("cuda")
        ini = wl.particles()
        cell, frac = _mixed_layout(ini.x, wl.dx)
        self.d = {"cell": torch.as_tensor(cell, device=dev),
                  "frac": torch.as_tensor(frac, device=dev),
                  "px": torch.as_tensor(ini.px.astype(np.float32), device=dev),
                  "py": torch.as_tensor(ini.py.astype(np.float32), device=dev),
                  "pz": torch.as_tensor(ini.pz.astype(np.float32), device=dev),
                  "status": torch.zeros(wl.n_particles, dtype=torch.uint8, device=dev)}
        E, B, self.i0 = wl.levels(-p, n_levels + p)
        self.Ed = [torch.as_tensor(_circular(E[r], self.i0[r], wl.window), device=dev)
                   for r in range(len(E))]
        self.Bd = [torch.as_tensor(_circular(B[r], self.i0[r], wl.window), device=dev)
                   for r in range(len(B))]
        self.stream = torch.cuda.current_stream().cuda_stream

    def call(self, n0, c, k_max=7, field_time=0, want_stats=True):
        wl, d, p = self.wl, self.d, self.wl.order
        prm = native.PicParams(wl.dt, wl.dx, wl.psi_max, -1.0, p, k_max, native.PIC_MIXED,
                               field_time, native.PIC_SCHED_BINNED)
        rows = range(n0, n0 + p + c)            # levels n0 - p .. n0 + c - 1
        Ep = (ctypes.c_void_p * len(rows))(*[self.Ed[r].data_ptr() for r in rows])
        Bp = (ctypes.c_void_p * len(rows))(*[self.Bd[r].data_ptr() for r in rows])
        org = np.ascontiguousarray([self.i0[r] for r in rows], dtype=np.int64)
        st = native.PicStepStats() if want_stats else None
        rc = native.lib().pic_push_mixed_noalloc(
            ctypes.byref(prm), wl.n_particles, d["cell"].data_ptr(), d["frac"].data_ptr(),
            d["px"].data_ptr(), d["py"].data_ptr(), d["pz"].data_ptr(), d["status"].data_ptr(),
            Ep, Bp, org.ctypes.data, wl.window, n0, c, self.stream,
            ctypes.byref(st) if st is not None else None)
        ok = OK_CODES if want_stats else (native.PIC_OK,)
        assert rc in ok, native.lib().pic_last_error(None)
        return st.as_dict() if st is not None else None

    def assert_equal(self, ref):
        rx, rpx, rpy, rpz, rst = ref
        torch.cuda.synchronize()
        d, dx = self.d, self.wl.dx
        x = (d["cell"].cpu().numpy().astype(np.float64)
             + d["frac"].cpu().numpy().astype(np.float64)) * dx
        np.testing.assert_array_equal(x, rx)
        np.testing.assert_array_equal(d["px"].cpu().numpy().astype(np.float64), rpx)
        np.testing.assert_array_equal(d["py"].cpu().numpy().astype(np.float64), rpy)
        np.testing.assert_array_equal(d["pz"].cpu().numpy().astype(np.float64), rpz)
        np.testing.assert_array_equal(d["status"].cpu().numpy(), rst)


def test_noalloc_matches_context_api_on_consecutive_calls():
    """Two calls with counters, then an asynchronous one (stats NULL): the
    context API's bits and counters."""
    wl = _wl(6000)
    calls = [(0, 350), (350, 250), (600, 120)]
    ref, ref_stats = _context_run(wl, calls)
    run = NoAllocRun(wl, sum(c for _, c in calls))
    assert run.call(*calls[0]) == ref_stats[0]
    assert run.call(*calls[1]) == ref_stats[1]
    assert run.call(*calls[2], want_stats=False) is None
    run.assert_equal(ref)
    assert ref_stats[0]["k_hist"][5] > 0


def test_noalloc_after_a_change_of_parameters():
    """Order 1, k capped at 4, the other field-time reading: a new weight table
    in the shared array, the previous calls' queues and counters left behind;
    still the bits of a fresh context with those parameters."""
    wl = _wl(3001, order=1)
    calls = [(0, 300), (300, 200)]
    ref, ref_stats = _context_run(wl, calls, k_max=4, field_time=1)
    run = NoAllocRun(wl, sum(c for _, c in calls))
    for (n0, c), want in zip(calls, ref_stats):
        assert run.call(n0, c, k_max=4, field_time=1) == want
    run.assert_equal(ref)
    assert ref_stats[0]["clamped"] > 0          # the cap at 4 was reached


def test_noalloc_call_allocates_no_device_memory():
    """A warmed-up call leaves the device's free memory exactly as it was."""
    wl = _wl(4096)
    run = NoAllocRun(wl, 80)
    run.call(0, 40)                             # first call with this key: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    run.call(40, 40)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_more_particles_than_its_scratch_holds():
    prm = native.PicParams(W.DT75, W.DT75 / 0.99, 0.01, -1.0, 3, 7, native.PIC_MIXED, 0,
                           native.PIC_SCHED_BINNED)
    nul = (ctypes.c_void_p * 4)()
    org = np.zeros(4, dtype=np.int64)
    rc = native.lib().pic_push_mixed_noalloc(ctypes.byref(prm), 65537, 1, 1, 1, 1, 1, 1, nul, nul,
                                             org.ctypes.data, 1024, 0, 1, None, None)
    assert rc == native.PIC_EINVAL
    assert b"65,536" in native.lib().pic_last_error(None)


def test_noalloc_reports_a_set_error_word_once():
    """The array's error word, set from the host as a giving-up wait would set
    it: an asynchronous call (stats NULL) returns PIC_OK, the next call with
    stats returns PIC_ETIMEOUT with the word, and the one after it is clean."""
    wl = _wl(2048)
    run = NoAllocRun(wl, 60)
    run.call(0, 20)
    assert native.lib().pic_noalloc_inject_error(7, run.stream) == native.PIC_OK
    assert run.call(20, 20, want_stats=False) is None
    prm = native.PicParams(wl.dt, wl.dx, wl.psi_max, -1.0, wl.order, 7, native.PIC_MIXED, 0,
                           native.PIC_SCHED_BINNED)
    p = wl.order
    rows = range(40, 40 + p + 10)
    Ep = (ctypes.c_void_p * len(rows))(*[run.Ed[r].data_ptr() for r in rows])
    Bp = (ctypes.c_void_p * len(rows))(*[run.Bd[r].data_ptr() for r in rows])
    org = np.ascontiguousarray([run.i0[r] for r in rows], dtype=np.int64)
    st = native.PicStepStats()
    d = run.d
    rc = native.lib().pic_push_mixed_noalloc(
        ctypes.byref(prm), wl.n_particles, d["cell"].data_ptr(), d["frac"].data_ptr(),
        d["px"].data_ptr(), d["py"].data_ptr(), d["pz"].data_ptr(), d["status"].data_ptr(),
        Ep, Bp, org.ctypes.data, wl.window, 40, 10, run.stream, ctypes.byref(st))
    assert rc == native.PIC_ETIMEOUT and st.error == 7
    assert b"gave up" in native.lib().pic_last_error(None)
    assert run.call(50, 10)["error"] == 0

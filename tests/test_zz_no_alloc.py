"""pic_push_mixed_noalloc against the context API, through the C ABI.

The allocation-free entry point serves host programs that may not allocate
device memory when they push particles: it works on the caller's arrays and
keeps its own working data in a fixed device array inside the library.  It
must give the same bits as the binned push of a pic_create context, on two
calls in a row (the second finds the first call's leftovers in that array).

This file sorts last so that a run stopping at the first failure has run
every other test before it; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import pytest

import _harness as H
from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402


def _wl(n):
    return W.Workload(name="noalloc", n_particles=n, a0=150.0, dt=W.DT75, dx=W.DT75 / 0.99,
                      psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=8 * math.pi,
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


def test_noalloc_matches_context_api_on_two_calls():
    wl = _wl(6000)
    p, calls = wl.order, [(0, 350), (350, 250)]
    n_total = sum(c for _, c in calls)
    ini = wl.particles()
    E, B, i0 = wl.levels(-p, n_total + p)

    # reference: the context API, binned schedule, same two calls
    ref = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                            schedule=native.PIC_SCHED_BINNED, capacity=wl.n_particles,
                            window=wl.window, ring_levels=p + 2 + max(c for _, c in calls))
    ref.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    for r in range(p):
        ref.pic_fields_upload(r - p, i0[r], E[r], B[r])
    ref_stats = []
    for n0, c in calls:
        for lev in range(n0, n0 + c):
            ref.pic_fields_upload(lev, i0[lev + p], E[lev + p], B[lev + p])
        st, _ = ref.pic_push_step(n0, c, want_stats=True, ok=(0, 4, 5))
        ref_stats.append(st.as_dict())
    rx, rpx, rpy, rpz, rst = ref.read_numpy()
    ref.close()

    # the allocation-free entry point on caller-owned device arrays
    dev = torch.device("cuda")
    cell, frac = _mixed_layout(ini.x, wl.dx)
    d = {"cell": torch.as_tensor(cell, device=dev), "frac": torch.as_tensor(frac, device=dev),
         "px": torch.as_tensor(ini.px.astype(np.float32), device=dev),
         "py": torch.as_tensor(ini.py.astype(np.float32), device=dev),
         "pz": torch.as_tensor(ini.pz.astype(np.float32), device=dev),
         "status": torch.zeros(wl.n_particles, dtype=torch.uint8, device=dev)}
    Ed = [torch.as_tensor(_circular(E[r], i0[r], wl.window), device=dev) for r in range(len(E))]
    Bd = [torch.as_tensor(_circular(B[r], i0[r], wl.window), device=dev) for r in range(len(B))]
    prm = native.PicParams(wl.dt, wl.dx, wl.psi_max, -1.0, p, 7, native.PIC_MIXED, 0,
                           native.PIC_SCHED_BINNED)
    stream = torch.cuda.current_stream().cuda_stream
    L = native.lib()
    for (n0, c), want in zip(calls, ref_stats):
        rows = range(n0, n0 + p + c)            # levels n0 - p .. n0 + c - 1
        Ep = (ctypes.c_void_p * len(rows))(*[Ed[r].data_ptr() for r in rows])
        Bp = (ctypes.c_void_p * len(rows))(*[Bd[r].data_ptr() for r in rows])
        org = np.ascontiguousarray([i0[r] for r in rows], dtype=np.int64)
        st = native.PicStepStats()
        rc = L.pic_push_mixed_noalloc(ctypes.byref(prm), wl.n_particles, d["cell"].data_ptr(),
                                      d["frac"].data_ptr(), d["px"].data_ptr(),
                                      d["py"].data_ptr(), d["pz"].data_ptr(),
                                      d["status"].data_ptr(), Ep, Bp, org.ctypes.data,
                                      wl.window, n0, c, stream, ctypes.byref(st))
        assert rc in (native.PIC_OK, native.PIC_ERANGE, native.PIC_EKMAX), L.pic_last_error(None)
        assert st.as_dict() == want
    torch.cuda.synchronize()

    x = (d["cell"].cpu().numpy().astype(np.float64)
         + d["frac"].cpu().numpy().astype(np.float64)) * wl.dx
    np.testing.assert_array_equal(x, rx)
    np.testing.assert_array_equal(d["px"].cpu().numpy().astype(np.float64), rpx)
    np.testing.assert_array_equal(d["py"].cpu().numpy().astype(np.float64), rpy)
    np.testing.assert_array_equal(d["pz"].cpu().numpy().astype(np.float64), rpz)
    np.testing.assert_array_equal(d["status"].cpu().numpy(), rst)
    assert ref_stats[0]["k_hist"][5] > 0


def test_noalloc_rejects_more_particles_than_its_scratch_holds():
    prm = native.PicParams(W.DT75, W.DT75 / 0.99, 0.01, -1.0, 3, 7, native.PIC_MIXED, 0,
                           native.PIC_SCHED_BINNED)
    nul = (ctypes.c_void_p * 4)()
    org = np.zeros(4, dtype=np.int64)
    rc = native.lib().pic_push_mixed_noalloc(ctypes.byref(prm), 65537, 1, 1, 1, 1, 1, 1, nul, nul,
                                             org.ctypes.data, 1024, 0, 1, None, None)
    assert rc == native.PIC_EINVAL
    assert b"65,536" in native.lib().pic_last_error(None)

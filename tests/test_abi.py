"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call is made here: pic_create is only called with arguments that
its host-side validation rejects before any CUDA call.
"""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_2102_10983_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pic_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pic_fields_upload", "pic_push_step", "pic_particles_read", "pic_create",
                     "pic_destroy", "pic_particles_write"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = native.lib()
    for name in _declared():
        assert hasattr(L, name), name
        assert name in native.SIGNATURES, name


def test_host_side_validation_rejects_bad_parameters():
    L = native.lib()
    h = ctypes.c_void_p()
    bad = [
        native.PicParams(0.0, 1.0, 0.01, -1.0, 3, 7, 0, 0, 0),     # dt = 0
        native.PicParams(0.1, 1.0, 0.01, -1.0, 6, 7, 0, 0, 0),     # order 6
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 8, 0, 0, 0),     # k_max 8
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 2, 0, 0),     # precision
        native.PicParams(0.1, 1.0, -1.0, -1.0, 3, 7, 0, 0, 0),     # psi_max < 0
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 0, 0, 1),     # binned needs mixed
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 1, 0, 0, 0, native.PIC_DIAG_WORK),  # FP64 only
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 0, 0, 0, 0, 2),  # unknown diagnostic
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 1, 0, 0, 0, 0, 1),  # carry, plain schedule
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 1, 0, 1, 0, 0, -1),  # negative carry
        native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 1, 0, 1, 0, 0, 5),  # ring 8 < 3 + 1 + 5
    ]
    for prm in bad:
        assert L.pic_create(ctypes.byref(prm), 16, 64, 8, None, ctypes.byref(h)) == native.PIC_EINVAL
        assert h.value is None
        assert L.pic_last_error(None)
    good = native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 0, 0, 0)
    assert L.pic_create(ctypes.byref(good), 16, 100, 8, None, ctypes.byref(h)) == native.PIC_EINVAL
    assert L.pic_create(ctypes.byref(good), 16, 64, 3, None, ctypes.byref(h)) == native.PIC_EINVAL
    carried = native.PicParams(0.1, 1.0, 0.01, -1.0, 3, 7, 1, 0, 1, 0, 0, 2)
    assert L.pic_create(ctypes.byref(carried), 16, 64, 5, None, ctypes.byref(h)) == native.PIC_EINVAL
    assert b"carry" in L.pic_last_error(None)
    assert L.pic_finish(None) == native.PIC_EINVAL
    assert L.pic_destroy(None) == native.PIC_OK

"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function include/hr.h declares, and rejects
malformed scene descriptions before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:hr_status|size_t|int32_t|void)\s+(hr_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = hb.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert {"hr_create_scene", "hr_estimate_grad", "hr_estimate_hessian", "hr_estimate_hvp",
            "hr_newton_cg_step"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert L.hr_version() >= 100


def test_scene_validation_happens_on_the_host():
    hb.build()
    sc = wl.disc_scene()
    d = hr.hr_scene_desc()
    d.kind, d.width, d.height, d.n_params = sc["kind"], 64, 64, 3   # wrong n
    th = np.zeros(3)
    d.theta_target = th.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.radius = 0.2
    h = ctypes.c_void_p()
    assert hr.lib().hr_create_scene(ctypes.byref(d), ctypes.byref(h)) == -1
    assert "n_params" in hr.hr_last_error()
    d.n_params, d.width = 2, 0
    assert hr.lib().hr_create_scene(ctypes.byref(d), ctypes.byref(h)) == -1
    d.width, d.kind = 64, 9
    assert hr.lib().hr_create_scene(ctypes.byref(d), ctypes.byref(h)) == -1
    assert hr.lib().hr_create_scene(None, ctypes.byref(h)) == -1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hr, "_lib", None)
    monkeypatch.setattr(hr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(hr.HRError):
        hr.lib()


def test_queue_entry_points_check_arguments_on_the_host():
    """The persistent queue's calls reject missing handles and arguments
    before any device call (so they run without a GPU)."""
    hb.build()
    L = hr.lib()
    h = ctypes.c_void_p()
    o = hr.hr_queue_opts(8, 1000, 1 << 20)
    assert L.hr_queue_create(None, ctypes.byref(o), ctypes.byref(h)) == hr.HR_ERR_INVALID_ARG
    assert L.hr_queue_create(None, None, None) == hr.HR_ERR_INVALID_ARG
    t = ctypes.c_uint64()
    th = np.zeros(2)
    opts = hr.make_opts(0.05, 64, hr.HR_AGGREGATE, 1, 1)
    assert L.hr_queue_submit(None, hr.HR_HESSIAN, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                             ctypes.byref(opts), ctypes.byref(t)) == hr.HR_ERR_INVALID_ARG
    n = ctypes.c_int32()
    assert L.hr_queue_submit_many(None, 1, hr.HR_HESSIAN, None, None, None, None, ctypes.byref(n)) == \
        hr.HR_ERR_INVALID_ARG
    out = np.zeros(4)
    assert L.hr_queue_wait(None, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0) == \
        hr.HR_ERR_INVALID_ARG
    assert L.hr_queue_wait_many(None, 1, None, None, 4, 0) == hr.HR_ERR_INVALID_ARG
    st = ctypes.c_int32()
    assert L.hr_queue_status(None, ctypes.byref(st), None) == hr.HR_ERR_INVALID_ARG
    assert L.hr_queue_destroy(None) == hr.HR_OK
    assert "NULL" in hr.hr_last_error()

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

"""The C ABI library: builds for sm_103a, loads, exports every symbol the
header declares, and rejects bad arguments on the host before any GPU work.
None of these tests needs a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1009_1351_gb300 as tn
from paper_1009_1351_gb300 import build as tnbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    tnbuild.build()
    return tn.load_library()


def header_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnlm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(tn.EXPORTED) == set(names)


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(tnbuild.ARCH)
    out = os.popen(f"/usr/local/cuda/bin/cuobjdump --list-elf {tnbuild.LIB} 2>&1").read()
    assert "sm_103a" in out


def _desc(**kw):
    g = dict(nx=16, ny=16, pixel_mm=1.0, n_phases=4, n_views=5, n_bins=32, bin_mm=1.0,
             sid_mm=100.0, sdd_mm=150.0)
    g.update(kw)
    ang = np.linspace(0, 2 * np.pi, g["n_phases"] * g["n_views"], endpoint=False)
    if kw.get("nan_angle"):
        ang[3] = math.nan
    g.pop("nan_angle", None)
    det = g.pop("detector", tn.TNLM_DETECTOR_ARC)
    d = tn.GeometryDesc(g["nx"], g["ny"], g["pixel_mm"], g["n_phases"], g["n_views"], g["n_bins"],
                        g["bin_mm"], g["sid_mm"], g["sdd_mm"], det,
                        ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    return d, ang


@pytest.mark.parametrize("kw,msg", [
    (dict(n_phases=2), "n_phases"),
    (dict(nx=0), "nx"),
    (dict(n_views=0), "n_views"),
    (dict(n_bins=5000), "n_bins"),
    (dict(pixel_mm=-1.0), "pixel_mm"),
    (dict(sid_mm=5.0), "sid_mm"),
    (dict(sdd_mm=105.0), "sdd_mm"),
    (dict(detector=1), "arc"),
    (dict(nan_angle=True), "angle"),
])
def test_create_geometry_rejects_bad_descriptions(lib, kw, msg):
    d, ang = _desc(**kw)
    h = ctypes.c_void_p(123)
    st = lib.tnlm_create_geometry(ctypes.byref(d), ctypes.byref(h))
    assert st == tn.TNLM_ERR_INVALID_ARG
    assert h.value is None
    assert msg in lib.tnlm_last_error().decode()


def test_null_handles_and_pointers_are_rejected(lib):
    assert lib.tnlm_create_geometry(None, None) == tn.TNLM_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.tnlm_create_geometry(None, ctypes.byref(h)) == tn.TNLM_ERR_INVALID_ARG
    assert lib.tnlm_project(None, 16, 16, None) == tn.TNLM_ERR_INVALID_ARG
    assert lib.tnlm_backproject(None, 16, 16, None) == tn.TNLM_ERR_INVALID_ARG
    p = tn.ParamsC(0.5, 0.01, 0.0, 3, 5, 3, 5, 2, 0, 1, 0.0, 1)
    assert lib.tnlm_reconstruct(None, ctypes.byref(p), 16, 16, 16, None, None) == tn.TNLM_ERR_INVALID_ARG
    lib.tnlm_destroy_geometry(None)  # no-op

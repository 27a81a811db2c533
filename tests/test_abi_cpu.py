"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol the header declares, and argument validation rejects bad input before any
device work (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def rtlib():
    from paper_1001_3301_gb300 import build
    build()
    from paper_1001_3301_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported_and_bound(rtlib):
    names = declared_functions()
    assert len(names) >= 15
    raw = ctypes.CDLL(rtlib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), f"{n} declared but not exported"
        assert n in rtlib.SIGNATURES, f"{n} not bound in the Python binding"
    assert set(rtlib.SIGNATURES) <= set(names), "binding names a symbol the header lacks"


def test_status_strings(rtlib):
    assert rtlib.status_string(0) == "RT_OK"
    assert rtlib.status_string(-5) == "RT_ERR_NONFINITE_INPUT"
    assert rtlib.status_string(99) == "RT_UNKNOWN_STATUS"


def _desc(rtlib, r, th, ph, precision=0):
    r, th, ph = (np.ascontiguousarray(x, dtype=np.float64) for x in (r, th, ph))
    P = ctypes.POINTER(ctypes.c_double)
    d = rtlib.RtGridDesc(len(r) - 1, len(th) - 1, len(ph) - 1, r.ctypes.data_as(P),
                         th.ctypes.data_as(P), ph.ctypes.data_as(P), precision)
    return d, (r, th, ph)


@pytest.mark.parametrize("case", ["nonmonotone_r", "negative_r", "theta_beyond_pi",
                                  "bad_precision", "zero_size"])
def test_create_rejects_bad_grids_without_device(rtlib, case):
    r = np.geomspace(1e13, 1e16, 9)
    th = np.linspace(0, np.pi, 5)
    ph = np.array([0.0, 2 * np.pi])
    prec = 0
    if case == "nonmonotone_r":
        r[3] = r[2]
    elif case == "negative_r":
        r = np.linspace(-1.0, 5.0, 9)
    elif case == "theta_beyond_pi":
        th = np.linspace(0, 4.0, 5)
    elif case == "bad_precision":
        prec = 7
    d, keep = _desc(rtlib, r, th, ph, prec)
    if case == "zero_size":
        d.nr = 0
    out = ctypes.c_void_p()
    st = rtlib.lib.rt_create(ctypes.byref(d), None, ctypes.byref(out))
    assert st == rtlib.RT_ERR_INVALID_ARG
    assert out.value is None
    assert rtlib.last_error(None) != ""


def test_null_context_calls(rtlib):
    L = rtlib.lib
    assert L.rt_set_star(None, 5800.0, 7e10) == rtlib.RT_ERR_INVALID_ARG
    assert L.rt_irradiate(None, None, None, None, None, None) == rtlib.RT_ERR_INVALID_ARG
    assert L.rt_set_tuning(None, 0, 8, 8, 0) == rtlib.RT_ERR_INVALID_ARG
    L.rt_destroy(None)


def test_product_path_has_no_cpu_fallback():
    """The package imports no oracle code and has no CPU compute path."""
    pkg = os.path.join(ROOT, "paper_1001_3301_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "rt_oracle" not in src, f

"""CPU checks of the C ABI boundary: the library builds, loads and exports every
function declared in include/*.h (no compute calls: there is no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2609_31347_b300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "lbm_solid_create" in names and "lbm_solid_gradient" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly the exported surface
    assert sorted(lbm.EXPORTED) == names


def test_status_strings_without_a_device():
    lib = lbm.load_library()
    for st in range(7):
        assert lib.lbm_status_string(st)
    assert lib.lbm_solid_last_error(None) == b"null handle"
    assert lib.lbm_solid_launch_count(None) == -1


def test_create_rejects_bad_descriptions_without_touching_the_device():
    lib = lbm.load_library()
    h = ctypes.c_void_p()
    d = lbm._Desc(2, 2, 0.5, 1, 1.0, 0.3, None, None, None, None, None, None, 0, None, None, 0)
    assert lib.lbm_solid_create(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    d = lbm._Desc(8, 8, -1.0, 1, 1.0, 0.3, None, None, None, None, None, None, 0, None, None, 0)
    assert lib.lbm_solid_create(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    d = lbm._Desc(8, 8, 0.1, 1, 1.0, 0.3, None, None, None, None, None, None, 1, None, None, 0)
    assert lib.lbm_solid_create(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    assert not h.value


def test_destroy_null_is_an_error_code():
    assert lbm.load_library().lbm_solid_destroy(None) == lbm.LBM_ERR_ARG


def test_history_calls_reject_bad_arguments_without_touching_the_device():
    lib = lbm.load_library()
    assert lib.lbm_warm_dot_work_size() >= 15 * 296
    w = (ctypes.c_double * 5)(1, 1, 1, 1, 1)
    src = (ctypes.c_void_p * 5)(8, 8, 8, 8, 8)  # never dereferenced: rejected first
    out = (ctypes.c_double * 36)()
    for count, n in ((0, 10), (5, 10), (2, 0)):
        assert lib.lbm_warm_combine(count, n, w, src, ctypes.c_void_p(8), None) == lbm.LBM_ERR_ARG
    assert lib.lbm_warm_combine(2, 10, None, src, ctypes.c_void_p(8), None) == lbm.LBM_ERR_ARG
    src_null = (ctypes.c_void_p * 2)(8, None)
    assert lib.lbm_warm_combine(2, 10, w, src_null, ctypes.c_void_p(8), None) == lbm.LBM_ERR_ARG
    for m, n in ((0, 10), (6, 10), (3, 0)):
        assert lib.lbm_warm_dots(m, n, src, ctypes.c_void_p(8), out, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_warm_dots(2, 10, src, None, out, None) == lbm.LBM_ERR_ARG

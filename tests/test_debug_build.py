"""The KDE_DEBUG build (index-checked kernels): it compiles, links, exports
every symbol the header declares, and its host path reports a debug build
without touching a device; the release library reports a release build."""
import ctypes
import glob
import os

import pytest

from paper_1508_02766_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcs = glob.glob(os.path.join(B.CSRC, "*")) + [os.path.join(ROOT, "include", "kde_gb300.h")]
    return any(os.path.getmtime(f) > t for f in srcs)


@pytest.fixture(scope="module")
def debug_lib():
    if _stale(B.LIB_DEBUG):
        B.build(debug=True)
    return ctypes.CDLL(B.LIB_DEBUG)


def _enabled(L):
    L.kde_debug_status.restype = ctypes.c_int
    L.kde_debug_status.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    flag = ctypes.c_int(-1)
    assert L.kde_debug_status(ctypes.byref(flag), None) == 0
    return flag.value


def test_debug_build_reports_itself(debug_lib):
    assert _enabled(debug_lib) == 1


def test_release_build_reports_release():
    if _stale(B.LIB):
        B.build()
    assert _enabled(ctypes.CDLL(B.LIB)) == 0


def test_debug_build_exports_the_header(debug_lib):
    import re
    text = open(os.path.join(ROOT, "include", "kde_gb300.h")).read()
    names = set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(kde_\w+)\s*\(", text, re.M))
    for n in names:
        assert hasattr(debug_lib, n), n

"""The C ABI library builds for sm_103a, loads, and exports every symbol include/poisson.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1410_1942_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "poisson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(poisson_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def test_header_lists_match_binding():
    assert _declared() == sorted(capi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (poisson_\w+)", out))
    assert set(_declared()) <= exported


def test_library_is_built_for_sm_103a_only(lib):
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_version_without_gpu(lib):
    assert lib.poisson_strerror(0) == b"ok"
    assert lib.poisson_strerror(-6) == b"density not set"
    assert b"sm_103a" in lib.poisson_version()


def test_default_opts(lib):
    o = capi.default_opts()
    assert o.precision == capi.FP32 and o.precond == capi.JACOBI and o.omega == 1.0
    assert o.inner_tol == 1e-4 and o.stream is None


def test_create_rejects_bad_sizes_before_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    for args in [(0, 4, 4, 0.1), (4, -1, 4, 0.1), (4, 4, 4, 0.0), (4, 4, 4, -1.0),
                 (2048, 2048, 1024, 0.1)]:
        assert lib.poisson_create(*args, None, ctypes.byref(h)) == capi.EINVAL
    o = capi.default_opts()
    o.omega = 2.0
    assert lib.poisson_create(4, 4, 4, 0.1, ctypes.byref(o), ctypes.byref(h)) == capi.EINVAL

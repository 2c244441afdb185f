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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of poisson_opts, poisson_stats and poisson_kernel_times have the C
    structs' sizes and field offsets (compiled from the header with the host compiler)."""
    checks = {"poisson_opts": capi.Opts, "poisson_stats": capi.Stats,
              "poisson_kernel_times": capi.KernelTimes}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "poisson.h"', "int main(void) {"]
    for cname, cls in checks.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True,
                                                        text=True).stdout.splitlines())
    for cname, cls in checks.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, field)]) == getattr(cls, field).offset, (cname, field)

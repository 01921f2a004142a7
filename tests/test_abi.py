"""Host-only checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/ctap.h declares, and validates sizes
before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libctap():
    from paper_1309_2451_b300 import build, ctap
    build.build()
    return ctap.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ctap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ctap_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ctap_plan_create", "ctap_plan_destroy", "ctap_set_potential",
                     "ctap_step", "ctap_observables", "ctap_adjoint", "ctap_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(libctap):
    out = subprocess.check_output(["nm", "-D", "--defined-only",
                                   os.path.join(ROOT, "paper_1309_2451_b300", "libctap.so")],
                                  text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(libctap, n)


def test_binding_covers_the_header():
    from paper_1309_2451_b300 import ctap
    assert sorted(ctap.exported_symbols()) == declared_functions()


def test_status_strings_and_version(libctap):
    assert libctap.ctap_status_string(0) == b"ok"
    assert libctap.ctap_status_string(2) == b"unsupported grid size"
    assert libctap.ctap_status_string(99) == b"unknown status"
    assert b"sm_103a" in libctap.ctap_version()
    assert libctap.ctap_last_error(None) == b""


@pytest.mark.parametrize("shape,code", [((12, 16, 16), 2), ((16, 16, 4), 2), ((16, 2048, 16), 2),
                                        ((2048, 16, 16), 2)])
def test_plan_create_rejects_bad_sizes_without_gpu(libctap, shape, code):
    nz, ny, nx = shape
    box = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    h = ctypes.c_void_p()
    rc = libctap.ctap_plan_create(nx, ny, nz, box, 0, None, ctypes.byref(h))
    assert rc == code and not h.value


def test_plan_create_rejects_bad_args_without_gpu(libctap):
    box = (ctypes.c_double * 6)(-1, 1, -1, 1, 1, -1)        # zmax < zmin
    h = ctypes.c_void_p()
    assert libctap.ctap_plan_create(8, 8, 8, box, 0, None, ctypes.byref(h)) == 1
    good = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    assert libctap.ctap_plan_create(8, 8, 8, good, 7, None, ctypes.byref(h)) == 3
    assert libctap.ctap_plan_create(8, 8, 8, None, 0, None, ctypes.byref(h)) == 1
    for batch in (0, -3, 1025):
        assert libctap.ctap_plan_create_batched(8, 8, 8, batch, good, 0, None, ctypes.byref(h)) == 1
        assert not h.value
    assert libctap.ctap_plan_destroy(None) == 1
    assert libctap.ctap_step(None, None, 1, 0.1, 0) == 1
    assert libctap.ctap_sync(None, 10) == 1

"""The C-ABI library builds, loads and exports every entry point include/handrt.h
declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2107_05509_gb300 import build
    return build.build()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^(?:int|const char\*)\s+(hr_\w+)\s*\(", src, flags=re.M)
    return names


def test_exports_every_declared_symbol(libpath):
    names = _declared()
    assert len(names) >= 15
    L = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(L, n), n
    from paper_2107_05509_gb300 import binding
    assert set(names) == set(binding.EXPORTS)


def test_status_strings_and_host_argument_checks(libpath):
    L = ctypes.CDLL(libpath)
    L.hr_status_string.restype = ctypes.c_char_p
    assert L.hr_status_string(0) == b"ok"
    assert b"argument" in L.hr_status_string(-1)
    # null arguments are rejected on the host, before any CUDA call
    assert L.hr_context_create(None, None) == -1
    assert L.hr_context_destroy(None) == -1
    assert L.hr_skin(None, None, None, None, None) == -1
    assert L.hr_render_fwd(None, None, None, None, 1, 1, 1, None, None, None, None) == -1
    assert L.hr_loss(None, None, None, None, 1, 1, 1, None, None, None) == -1
    assert L.hr_get_status(None, None) == -1
    assert L.hr_model_check(None) == -1
    fn = L.hr_adam_step
    fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_float] * 4 + [ctypes.c_int, ctypes.c_void_p]
    assert fn(None, None, None, None, 61, 0.01, 0.9, 0.999, 1e-8, 1, None) == -1

"""The C ABI library builds for sm_103a, loads on a machine without a GPU and
exports every function include/gridpull.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gridpull.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:gp_status|void|const char\*|int64_t)\s+(gp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2308_13175_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gp_build_band", "gp_nn", "gp_step", "gp_update", "gp_sample", "gp_create", "gp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(gp_\w+)\b", out))
    assert set(declared_functions()) <= exported
    assert lib.gp_version  # callable without a device
    lib.gp_version.restype = ctypes.c_char_p
    assert lib.gp_version().startswith(b"gridpull-gb300")


def test_binding_covers_the_header():
    from paper_2308_13175_gb300 import binding
    assert set(binding.SIGNATURES) == set(declared_functions())


def test_invalid_arguments_are_rejected_without_a_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gp_create.restype = ctypes.c_int
    lib.gp_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.gp_create(None, 0, None) == 1  # GP_ERR_ARG on a null output pointer

"""The C-ABI library loads and exports every entry point the headers declare (no GPU needed; no
compute call is made)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SO = os.path.join(ROOT, "paper_1210_8018_gb300", "liblgf.so")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lgf_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(SO):
        import importlib.util
        spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_1210_8018_gb300", "_build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    return ctypes.CDLL(SO)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lgf_create", "lgf_fix", "lgf_measure", "lgf_destroy", "lgf_last_error", "lgf_load",
                     "lgf_iterate", "lgf_store", "lgf_delta", "lgf_filter", "lgf_gauge", "lgf_update"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lgf_\w+)", out))
    assert set(declared_functions()) <= exported


def test_host_only_calls(lib):
    import paper_1210_8018_gb300 as lgf
    o = lgf.Options()
    lgf._lib.lgf_default_options(ctypes.byref(o))
    assert o.precision == lgf.FP64 and o.theta_switch == 1e-11 and o.reunit_period == 16 and o.max_iter == 100000
    assert isinstance(lgf._lib.lgf_last_error(None), bytes)


def test_create_rejects_bad_extents_before_any_device_call(lib):
    """Extent checks happen before the context touches CUDA, so they run on a machine without a GPU."""
    lib.lgf_create.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_void_p)]
    lib.lgf_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    for dims in [(7, 4, 4, 4), (1, 4, 4, 4), (2048, 4, 4, 4), (1024, 1024, 1024, 2)]:
        assert lib.lgf_create(*dims, ctypes.byref(h)) == 1  # LGF_EINVAL
        assert not h.value
    assert b"2^31" in lib.lgf_last_error(None)


def test_no_oracle_in_product_path():
    """The product path (package and library sources) never refers to the oracle."""
    for path in glob.glob(os.path.join(ROOT, "paper_1210_8018_gb300", "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(path).read()
            assert "import oracle" not in src and "oracle." not in src and "liboracle" not in src, path


def test_noalloc_message_does_not_outlive_a_later_failure(lib):
    """A rejected lgf_delta_noalloc call sets the context-free error message; a later failing lgf_create
    must replace it with its own message (checked on a machine without a GPU, where lgf_create fails when
    it asks for the device)."""
    lib.lgf_create.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_void_p)]
    lib.lgf_last_error.restype = ctypes.c_char_p
    lib.lgf_delta_noalloc.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4 + [ctypes.c_void_p] * 3
    assert lib.lgf_delta_noalloc(None, 7, 4, 4, 4, None, None, None) == 1  # LGF_EINVAL before any CUDA call
    assert b"products of 2, 3 and 5" in lib.lgf_last_error(None)
    h = ctypes.c_void_p()
    st = lib.lgf_create(4, 4, 4, 4, ctypes.byref(h))
    if st == 0:
        lib.lgf_destroy.argtypes = [ctypes.c_void_p]
        lib.lgf_destroy(h)
        pytest.skip("a CUDA device is present: lgf_create does not fail here")
    assert st == 3  # LGF_ECUDA: no device
    assert b"products of 2, 3 and 5" not in lib.lgf_last_error(None)

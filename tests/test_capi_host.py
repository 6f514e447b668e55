"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point
declared in include/lobpcg_gb300.h, and rejects bad calls with status codes instead of crashing."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_0705_2626_gb300 import build as B
from paper_0705_2626_gb300 import capi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "lobpcg_gb300.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lobpcg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        B.build()
    return capi.lib()


def test_header_declares_expected_entry_points():
    names = header_functions()
    for must in ["lobpcg_create", "lobpcg_set_operator", "lobpcg_set_preconditioner",
                 "lobpcg_set_initial", "lobpcg_solve", "lobpcg_get_eigenpairs",
                 "lobpcg_last_error", "lobpcg_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(lobpcg_\w+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_header_exactly():
    assert capi.declared_symbols() == header_functions()


def test_calls_with_null_handle_return_err_arg(lib):
    assert capi.lobpcg_set_operator(None, 0, 4, 4, 4, 1.0, None) == capi.ERR_ARG
    assert capi.lobpcg_solve(None, 4, 1e-8, 10, 2, None) == capi.ERR_ARG
    assert capi.lobpcg_destroy(None) == capi.OK


def test_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert capi.lobpcg_create(None, 0, None, None, capi.FP64) == capi.ERR_ARG
    assert capi.lobpcg_create(ctypes.byref(h), 0, None, None, 7) == capi.ERR_ARG
    assert h.value is None
    assert "FP64" in capi.lobpcg_last_error(None)


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = capi.lobpcg_create(ctypes.byref(h), 0, None, None, capi.FP64)
    assert rc == capi.ERR_CUDA
    assert h.value is None
    assert capi.lobpcg_last_error(None) != ""


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the CUDA library the binding raises instead of falling back to anything else."""
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        capi.lib()
    with pytest.raises(RuntimeError):
        capi.lobpcg_destroy(None)


def _default_args(argtypes):
    out = []
    for t in argtypes:
        if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64):
            out.append(0)
        elif t is ctypes.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


def test_every_handle_call_rejects_a_null_handle(lib):
    """Each entry point that takes a handle returns LOBPCG_ERR_ARG for a NULL one (host check, no
    device work); destroy(NULL) is a no-op and last_error(NULL) returns the handle-free message."""
    checked = []
    for name, (res, argtypes) in capi._SIGNATURES.items():
        if name in ("lobpcg_create", "lobpcg_gram_noalloc", "lobpcg_last_error", "lobpcg_destroy"):
            continue
        assert argtypes[0] is ctypes.c_void_p, name
        rc = getattr(lib, name)(*_default_args(argtypes))
        assert rc == capi.ERR_ARG, (name, rc)
        checked.append(name)
    assert len(checked) == len(capi._SIGNATURES) - 4
    assert lib.lobpcg_destroy(None) == capi.OK


def test_gram_noalloc_rejects_bad_arguments_before_device_work(lib):
    f = lib.lobpcg_gram_noalloc
    fake = ctypes.c_void_p(0x1000)                      # never dereferenced: the checks come first
    # NULL inputs, n < 1, ld < n
    assert f(None, None, None, None, None, None, 10, 10, 1, 0, 0, None, fake, None) == capi.ERR_ARG
    assert f(fake, None, None, None, None, None, 0, 10, 1, 0, 0, None, fake, None) == capi.ERR_ARG
    assert f(fake, None, None, None, None, None, 10, 9, 1, 0, 0, None, fake, None) == capi.ERR_ARG
    # a second block without its pointer
    assert f(fake, None, None, None, None, None, 10, 10, 1, 2, 0, None, fake, None) == capi.ERR_ARG
    # basis wider than 96 columns
    assert f(fake, fake, None, None, None, None, 1000, 1000, 60, 40, 0, None, fake, None) == capi.ERR_ARG
    assert "96" in capi.lobpcg_last_error(None)

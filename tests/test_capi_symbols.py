"""The C ABI library loads and exports every function include/hawkes.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hawkes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("hawkes_", "hmc_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_02994_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hawkes_loglik", "hawkes_loglik_grad_locations", "hmc_leapfrog_trajectory",
                     "hawkes_batch_loglik_grad", "hawkes_ctx_create", "hawkes_ctx_destroy", "hawkes_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2010_02994_gb300 import _lib

    assert sorted(_lib.EXPORTED) == declared_functions()


def test_version_string(lib):
    lib.hawkes_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hawkes_version()


def test_create_without_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.hawkes_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_int32]
    lib.hawkes_last_error.argtypes = [ctypes.c_void_p]
    lib.hawkes_last_error.restype = ctypes.c_char_p
    st = lib.hawkes_ctx_create(ctypes.byref(h), 0, 100, 2)
    assert st != 0 and not h.value
    assert lib.hawkes_last_error(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2010_02994_gb300 import _lib

    with pytest.raises(RuntimeError):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "nope.so"))
        finally:
            _lib._lib = None


def test_binding_option_names_match_the_header():
    """Every HAWKES_OPT_* value of the header has a Python option name with the
    same number, and the binding names no value the header lacks."""
    from paper_2010_02994_gb300 import _lib

    src = open(os.path.join(ROOT, "include", "hawkes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    header = {name.lower(): int(v) for name, v in re.findall(r"HAWKES_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", src)}
    assert header, "no HAWKES_OPT_* values found"
    assert _lib.OPTIONS == header

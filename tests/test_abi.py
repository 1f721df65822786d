"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hydro.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hydro.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_4194_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hydro_init", "hydro_set_state", "hydro_step", "hydro_step_dt",
                     "hydro_get_state", "hydro_compute_dt", "hydro_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_1410_4194_gb300 import hydro
    assert sorted(hydro.EXPORTS) == declared_functions()


def test_error_strings_without_gpu(lib):
    lib.hydro_error_string.restype = ctypes.c_char_p
    assert lib.hydro_error_string(0) == b"ok"
    assert b"non-physical" in lib.hydro_error_string(-4)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1410_4194_gb300 import hydro
    monkeypatch.setattr(hydro, "_lib", None)
    monkeypatch.setattr(hydro, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        hydro.load()

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


def test_init_rejects_grids_beyond_32bit_indexing_without_gpu(lib):
    # validation happens before any device call: (1300+8)^3 padded cells >= 2^31
    h = ctypes.c_void_p()
    bc = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    rc = lib.hydro_init(ctypes.byref(h), 1300, 1300, 1300, ctypes.c_double(1.0 / 1300),
                        ctypes.c_double(5.0 / 3.0), bc)
    assert rc == -1 and not h.value
    dims = (ctypes.c_int * 6)(32, 32, 32, 1300, 1300, 1300)
    dx = (ctypes.c_double * 2)(1.0, 1.0)
    gam = (ctypes.c_double * 2)(1.4, 1.4)
    bcs = (ctypes.c_int * 12)(*([0] * 12))
    hb = ctypes.c_void_p()
    assert lib.hydro_batch_init(ctypes.byref(hb), 2, dims, dx, gam, bcs) == -1
    assert not hb.value


def test_index_division_matches_integer_division_without_gpu(lib):
    """The kernels turn a linear thread index into box coordinates with a
    multiply-high division by per-grid constants; the library's host check of
    that arithmetic (every divisor to 2^16, hashed ones to 2^31 - 1, edge and
    hashed numerators below 2^31) finds no mismatch."""
    lib.hydro_check_fastdiv.restype = ctypes.c_longlong
    assert lib.hydro_check_fastdiv() == 0


def test_noalloc_binding_rejects_bad_tensors_before_any_launch():
    """compute_dt_noalloc checks its tensors on the host: a CPU tensor, a
    float32 tensor, a non-tensor or a wrong shape raises ValueError before any
    pointer reaches the library (no GPU needed)."""
    torch = pytest.importorskip("torch")
    import numpy as np

    from paper_1410_4194_gb300 import hydro
    dt = torch.zeros(1, dtype=torch.float64)
    for bad in (torch.zeros((5, 2, 2, 2), dtype=torch.float64),   # on the CPU
                torch.zeros((5, 2, 2, 2), dtype=torch.float32),   # float32 (and CPU)
                np.zeros((5, 2, 2, 2)),                            # not a tensor
                torch.zeros((4, 2, 2, 2), dtype=torch.float64)):   # 4 planes
        with pytest.raises(ValueError):
            hydro.compute_dt_noalloc(bad, 0.1, 1.4, 0.3, dt)

"""hydro_compute_dt_noalloc: the CFL time step of a device state the caller
holds, computed without any device allocation (for callers that cannot call
cudaMalloc; its scratch is a static device array).  Its result is checked
against the handle-based hydro_compute_dt on two calls in a row, the second on
a smaller state so that stale scratch from the first call would show: to the
parity tolerance against the default mode, bit for bit against the strict mode
(the same operation order).  A state with a non-positive density or a NaN gives
a NaN dt.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1410_4194_gb300 import hydro
from paper_1410_4194_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the relative tolerance of the GPU parity tests


def test_noalloc_dt_matches_handle_dt_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    states = [W.sedov(48), dict(u=W.smooth_periodic((12, 20, 16), gamma=1.4, seed=5, vamp=0.9),
                                dx=0.05, gamma=1.4, bc=[0] * 6)]
    for w in states:
        _, nz, ny, nx = w["u"].shape
        u = torch.tensor(w["u"], device="cuda")
        dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = hydro.compute_dt_noalloc(u, w["dx"], w["gamma"], 0.3, dt)
        assert rc == 0
        torch.cuda.synchronize()
        got = float(dt.item())
        for mode in (hydro.HYDRO_FP64, hydro.HYDRO_FP64_STRICT):
            g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=mode)
            g.set_state(w["u"])
            ref = g.compute_dt(0.3)
            g.close()
            assert ref > 0 and abs(got - ref) <= TOL * ref, (mode, got, ref)
            if mode == hydro.HYDRO_FP64_STRICT:
                assert got == ref, (got, ref)


def test_noalloc_dt_is_nan_for_non_physical_states():
    """A cell with a negative density, a zero density or a NaN field makes the
    result NaN instead of dropping out of the maximum; the same state made
    physical again gives a finite dt (the scratch keeps no NaN)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    w = W.sedov(16)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for q, val in ((0, -1.0), (0, 0.0), (4, float("nan")), (2, float("nan"))):
        u = torch.tensor(w["u"], device="cuda")
        u[q, 3, 5, 7] = val
        assert hydro.compute_dt_noalloc(u, w["dx"], w["gamma"], 0.3, dt) == 0
        torch.cuda.synchronize()
        assert np.isnan(float(dt.item())), (q, val, float(dt.item()))
    u = torch.tensor(w["u"], device="cuda")
    assert hydro.compute_dt_noalloc(u, w["dx"], w["gamma"], 0.3, dt) == 0
    torch.cuda.synchronize()
    assert np.isfinite(float(dt.item())) and float(dt.item()) > 0


def test_noalloc_binding_rejects_bad_device_tensors():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros((5, 2, 2, 2), dtype=torch.float32, device="cuda"),
                torch.zeros((5, 2, 2, 4), dtype=torch.float64, device="cuda")[..., ::2],
                torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            hydro.compute_dt_noalloc(bad, 0.1, 1.4, 0.3, dt)
    with pytest.raises(ValueError):
        hydro.compute_dt_noalloc(torch.zeros((5, 2, 2, 2), dtype=torch.float64, device="cuda"),
                                 0.1, 1.4, 0.3, torch.zeros(1, dtype=torch.float32, device="cuda"))


def test_noalloc_rejects_states_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    u = torch.zeros((5, 1, 1, 8), dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = hydro.load()
    import ctypes
    # 2^24 + 1 cells: rejected before any launch, so the small buffer is never read
    rc = L.hydro_compute_dt_noalloc(ctypes.c_void_p(u.data_ptr()), 4097, 4096, 1, 0.1, 1.4, 0.3,
                                    ctypes.c_void_p(dt.data_ptr()), None)
    assert rc == -1

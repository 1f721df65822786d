"""Parity at the benchmark workloads' full sizes, in the launch configuration the
benchmark times (HYDRO_FP64, one grid or the 96-grid batch), one step.

The oracle cannot hold a 512^3 step, so there it recomputes sampled blocks: the
update of a cell depends on the cells within 3 of it along each axis
(test_oracle_ctu pins that), so the oracle run on a 20^3 block cut from the
initial state, with the step's dt and any boundary rule at the block's faces,
reproduces the full-grid update exactly in the block's interior 4 cells away
from its faces.  The dt is the oracle's own (its compute_dt on the full
state); the GPU computes its own.  Tolerance as in test_gpu_parity (HYDRO_FP64):
|gpu - oracle| <= 1e-10 max(|oracle|, 1e-4 S), S the variable's scale over the
full grid.
"""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import hydro
from paper_1410_4194_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10
FLOOR = 1e-4
R = 10       # block half-width
MARGIN = 4   # compared interior: cells at least MARGIN from the block's faces


@pytest.fixture(scope="module", autouse=True)
def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    hydro.load()
    oracle.set_threads(0)
    yield


def var_scale(u):
    m = np.abs(u).reshape(5, -1).max(axis=1)
    return np.array([m[0], m[1:4].max(), m[1:4].max(), m[1:4].max(), m[4]])


def check(g, o, scale):
    den = np.maximum(np.abs(o), FLOOR * scale.reshape(5, 1, 1, 1))
    err = np.abs(g - o) / den
    assert err.max() <= TOL, err.max()


def oracle_dt(w, cfl):
    _, nz, ny, nx = w["u"].shape
    g = oracle.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"])
    for face, prim in (w.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    g.set_state(w["u"])
    return g.compute_dt(cfl)


def sampled_blocks(w, centers, cfl=0.3):
    u0 = w["u"]
    _, nz, ny, nx = u0.shape
    dt = oracle_dt(w, cfl)
    g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"])
    for face, prim in (w.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    g.set_state(u0)
    dt_gpu = g.step(cfl)
    assert dt_gpu == pytest.approx(dt, rel=1e-13)
    u1 = g.get_state()
    g.close()
    scale = var_scale(u1)
    for (k, j, i) in centers:
        idx = [np.arange(c - R, c + R) % n for c, n in ((k, nz), (j, ny), (i, nx))]
        sub = np.ascontiguousarray(u0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]])
        b = oracle.Grid(2 * R, 2 * R, 2 * R, w["dx"], w["gamma"], [2] * 6)
        b.set_state(sub)
        b.step_dt(dt)
        ub = b.get_state()
        inner = [ix[MARGIN:2 * R - MARGIN] for ix in idx]
        o = ub[:, MARGIN:2 * R - MARGIN, MARGIN:2 * R - MARGIN, MARGIN:2 * R - MARGIN]
        gg = u1[:, inner[0]][:, :, inner[1]][:, :, :, inner[2]]
        check(gg, o, scale)


def test_shock_cloud_full_size_sampled_blocks():
    """512x256x256 Mach-10 shock on the lognormal cloud: blocks on the shock
    front, in the cloud, at the cloud's edge and at seeded positions."""
    w = W.shock_cloud()
    rng = np.random.default_rng(41)
    centers = [(128, 128, 128), (128, 128, 176), (128, 160, 176), (100, 30, 60)]
    centers += [(int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(rng.integers(R, 512 - R)))
                for _ in range(4)]
    sampled_blocks(w, centers)


def test_turbulence_full_size_sampled_blocks():
    """512^3 Mach-5 solenoidal turbulence, periodic: seeded blocks (wrapping)."""
    w = W.turbulence(512)
    rng = np.random.default_rng(43)
    centers = [tuple(int(x) for x in rng.integers(0, 512, size=3)) for _ in range(6)]
    centers.append((0, 0, 0))  # wraps across every periodic boundary
    sampled_blocks(w, centers)


def test_batched96_full_size_sampled_grids():
    """The 96-grid batch in one CUDA-graph step; sampled grids recomputed in
    full by the oracle (each grid takes its own CFL dt on both sides)."""
    grids = W.batched(ngrids=96)
    b = hydro.Batch(grids, precision=hydro.HYDRO_FP64)
    dts = b.step(0.3, nsteps=1)[0]
    rng = np.random.default_rng(47)
    picks = sorted(set(int(x) for x in rng.integers(0, 96, size=6)) | {0, 95})
    for i in picks:
        w = grids[i]
        ug = b.get_state(i)
        uo, to, no, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=1, cfl=0.3)
        assert fl == 0
        assert dts[i] == pytest.approx(to, rel=1e-13)
        check(ug, uo, var_scale(uo))
    b.close()

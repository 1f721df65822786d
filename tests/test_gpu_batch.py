"""Batches of independent grids (hydro_batch_*): every stage one launch over all
grids, per-grid dt, the steps of a call replayed from a captured CUDA graph.

The batched kernels run the same per-cell code as the single-grid ones, so each
grid of a batch must reproduce its single-grid run bit for bit (FP64 and mixed),
and through it the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import hydro
from paper_1410_4194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    hydro.load()
    oracle.set_threads(0)
    yield


def small_batch():
    grids = W.batched(ngrids=6, seed=7, edges=(16, 24, 32))
    # add an inflow grid and a 2D grid so every boundary path is batched
    rho2, u2, p2, vs = W.rankine_hugoniot(5.0)
    nx, ny, nz = 24, 12, 8
    rho = np.ones((nz, ny, nx)); vx = np.zeros_like(rho); p = np.ones_like(rho)
    rho[:, :, :6] = rho2; vx[:, :, :6] = u2; p[:, :, :6] = p2
    grids.append(dict(u=W.prim_to_cons(rho, vx, 0.0, 0.0, p, 5 / 3), dx=1 / 24, gamma=5 / 3,
                      bc=[3, 2, 1, 1, 0, 0], inflow={0: (rho2, u2, 0.0, 0.0, p2)}))
    grids.append(dict(u=W.smooth_periodic((1, 20, 28), gamma=1.4, seed=4, vamp=0.7), dx=0.05,
                      gamma=1.4, bc=[0, 0, 1, 1, 0, 0]))
    return grids


@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED], ids=["fp64", "mixed"])
def test_batch_matches_single_grid_runs_bitwise(precision):
    grids = small_batch()
    b = hydro.Batch(grids, precision=precision)
    dts = b.step(0.3, nsteps=4)
    for i, w in enumerate(grids):
        _, nz, ny, nx = w["u"].shape
        g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=precision)
        g.set_block_size(128)  # the batch's default schedule (the mixed dt pick is per block)
        for face, prim in (w.get("inflow") or {}).items():
            g.set_inflow(face, prim)
        g.set_state(w["u"])
        single_dt = [g.step(0.3) for _ in range(4)]
        single = g.get_state()
        g.close()
        assert np.array_equal(dts[:, i], np.array(single_dt)), (i, dts[:, i], single_dt)
        assert np.array_equal(b.get_state(i), single), i
    b.close()


def test_batch_fp64_matches_oracle():
    grids = small_batch()
    b = hydro.Batch(grids)
    b.step(0.3, nsteps=5)
    for i, w in enumerate(grids):
        uo, to, no, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=5, cfl=0.3,
                                    inflow=w.get("inflow"))
        assert fl == 0
        ug = b.get_state(i)
        m = np.abs(uo).reshape(5, -1).max(axis=1)
        scale = np.array([m[0], m[1:4].max(), m[1:4].max(), m[1:4].max(), m[4]])[:, None, None, None]
        err = np.abs(ug - uo) / np.maximum(np.abs(uo), 1e-4 * scale)
        assert err.max() <= 1e-10, (i, err.max())
    b.close()


def test_graph_replay_continues_and_autotune_restores_state():
    grids = small_batch()
    a = hydro.Batch(grids)
    dt_a = np.vstack([a.step(0.3, nsteps=2), a.step(0.3, nsteps=2)])  # one graph, replayed
    c = hydro.Batch(grids)
    before = [c.get_state(i) for i in range(len(grids))]
    bs, order, ms = c.autotune(use_cache=False)
    assert bs in (128, 256) and order in (0, 1) and ms > 0
    for i in range(len(grids)):
        assert np.array_equal(c.get_state(i), before[i])  # the tuner restored the states
    dt_c = c.step(0.3, nsteps=4)  # one graph of four steps, tuned schedule
    assert np.array_equal(dt_a, dt_c)
    for i in range(len(grids)):
        assert np.array_equal(a.get_state(i), c.get_state(i))
    a.close()
    c.close()


def test_batch_rejects_bad_arguments():
    with pytest.raises(hydro.HydroError):
        hydro.Batch([dict(u=np.ones((5, 4, 4, 3)), dx=0.1, gamma=1.4, bc=[0] * 6)])
    b = hydro.Batch([W.sedov(8)])
    with pytest.raises(hydro.HydroError):
        b.step(-0.3)
    b.close()


@pytest.mark.parametrize("recon,solver", [(hydro.HYDRO_RECON_PPMP, hydro.HYDRO_RIEMANN_EXACT),
                                          (hydro.HYDRO_RECON_PLMP, hydro.HYDRO_RIEMANN_ROE),
                                          (hydro.HYDRO_RECON_PPMC, hydro.HYDRO_RIEMANN_ROE)],
                         ids=["ppmp-exact", "plmp-roe", "ppmc-roe"])
def test_batch_other_methods_match_single_grids_and_oracle(recon, solver):
    """Other reconstructions and the Roe solver in the batched form: every grid
    reproduces its single-grid run bit for bit and the oracle within the FP64
    tolerance."""
    grids = small_batch()
    b = hydro.Batch(grids, recon=recon, solver=solver)
    dts = b.step(0.3, nsteps=3)
    for i, w in enumerate(grids):
        _, nz, ny, nx = w["u"].shape
        g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], recon=recon, solver=solver)
        for face, prim in (w.get("inflow") or {}).items():
            g.set_inflow(face, prim)
        g.set_state(w["u"])
        single_dt = [g.step(0.3) for _ in range(3)]
        single = g.get_state()
        g.close()
        assert np.array_equal(dts[:, i], np.array(single_dt)), i
        assert np.array_equal(b.get_state(i), single), i
        uo, to, no, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=3, cfl=0.3,
                                    inflow=w.get("inflow"), recon=recon, solver=solver)
        assert fl == 0
        m = np.abs(uo).reshape(5, -1).max(axis=1)
        scale = np.array([m[0], m[1:4].max(), m[1:4].max(), m[1:4].max(), m[4]])[:, None, None, None]
        err = np.abs(single - uo) / np.maximum(np.abs(uo), 1e-4 * scale)
        assert err.max() <= 1e-10, (i, err.max())
    b.close()


@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED], ids=["fp64", "mixed"])
def test_block_size_leaves_results_unchanged(precision):
    """A single grid's launches with 128 or 256 threads a block: the same
    arithmetic per cell, the dt a maximum over cells.  FP64 is bitwise the
    same.  In mixed precision each block evaluates in FP64 the signal speed of
    the cell with its largest float estimate, so dt is the FP64 maximum except
    where two cells' float estimates tie while their FP64 values differ: then
    within 10 * 2^-24 relative, and which tied cell a block picks depends on
    the block size (the blast's mirror-image cells can tie); the states then
    differ only by the effect of that dt difference."""
    w = W.sedov(40)
    out = {}
    for bs in (128, 256):
        g = hydro.Grid(40, 40, 40, w["dx"], w["gamma"], w["bc"], precision=precision)
        try:
            g.set_block_size(bs)
            assert g.block_size() == bs
            g.set_state(w["u"])
            dts = [g.step(0.3) for _ in range(5)]
            out[bs] = (dts, g.get_state())
        finally:
            g.close()
    if precision == hydro.HYDRO_FP64:
        assert out[128][0] == out[256][0]
        assert np.array_equal(out[128][1], out[256][1])
    else:
        d128, d256 = np.array(out[128][0]), np.array(out[256][0])
        assert np.all(np.abs(d128 - d256) <= 10 * 2.0 ** -24 * d256), (d128, d256)
        m = np.abs(out[256][1]).reshape(5, -1).max(axis=1)
        scale = np.array([m[0], m[1:4].max(), m[1:4].max(), m[1:4].max(), m[4]])
        diff = np.abs(out[128][1] - out[256][1]).reshape(5, -1).max(axis=1) / scale
        assert np.all(diff <= 1e-6), diff
    g = hydro.Grid(16, 16, 16, 0.1, 1.4, [0] * 6)
    try:
        assert g.block_size() == 128  # the default
        with pytest.raises(hydro.HydroError):
            g.set_block_size(64)
        g.set_block_size(256)
        g.set_block_size(0)
        assert g.block_size() == 128
    finally:
        g.close()


def test_batch_async_pipeline_matches_synchronous_steps():
    """Asynchronous uploads, steps and downloads on two batches alternating on
    two streams give the synchronous batch step's states bit for bit; sync
    reports a step's error status."""
    torch = pytest.importorskip("torch")
    grids = small_batch()
    ref = hydro.Batch(grids)
    ref.step(0.3, nsteps=1)
    expect = [ref.get_state(i) for i in range(len(grids))]
    ref.close()
    hosts = [torch.from_numpy(np.ascontiguousarray(g["u"])).pin_memory() for g in grids]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pipe = []
    for s in streams:
        b = hydro.Batch(grids)
        b.set_stream(s)
        pipe.append(b)
    outs = [[torch.empty_like(x).pin_memory() for x in hosts] for _ in range(3)]
    try:
        for k in range(3):
            bk = pipe[k % 2]
            for i, x in enumerate(hosts):
                bk.set_state_async(i, x)
            bk.step_async(0.3, nsteps=1)
            for i, x in enumerate(outs[k]):
                bk.get_state_async(i, x)
            if k >= 1:
                pipe[(k - 1) % 2].sync()
        pipe[0].sync()
        for o in outs:
            for i, x in enumerate(o):
                assert np.array_equal(x.numpy(), expect[i]), i
        bad = hosts[0].clone().pin_memory()
        bad[0, 0, 0, 0] = -1.0
        pipe[1].set_state_async(0, bad)
        pipe[1].step_async(0.3, nsteps=1)
        with pytest.raises(hydro.HydroError):
            pipe[1].sync()
    finally:
        for b in pipe:
            b.close()

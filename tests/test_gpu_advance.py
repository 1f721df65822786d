"""Device-driven runs (hydro_advance): the steps loop inside one CUDA graph, the
dt kernel shortening the step that would pass the end time.  The result must be
the host loop's, bit for bit -- the same CFL dt sequence (Eq. calc_dt_3D), the
same last step dt = t_end - t, the same final time -- in every precision mode,
reconstruction and Riemann solver, across the graph relaunches of a long run,
and must stay within the parity bar of the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import hydro
from paper_1410_4194_gb300 import workloads as W
from tests.test_gpu_parity import FLOOR, TOL, rel_err

pytestmark = pytest.mark.gpu

P = hydro.HYDRO_BC_PERIODIC
MODES = [hydro.HYDRO_FP64, hydro.HYDRO_MIXED, hydro.HYDRO_FP64_STRICT]
MODE_ID = {hydro.HYDRO_FP64: "fp64", hydro.HYDRO_MIXED: "mixed", hydro.HYDRO_FP64_STRICT: "strict"}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    hydro.load()
    oracle.set_threads(0)


def both_loops(w, **kw):
    a = hydro.run(w["u"], w["dx"], w["gamma"], w["bc"], inflow=w.get("inflow"), loop="host", **kw)
    b = hydro.run(w["u"], w["dx"], w["gamma"], w["bc"], inflow=w.get("inflow"), loop="device", **kw)
    return a, b


def assert_same(a, b):
    (ua, ta, na), (ub, tb, nb) = a, b
    assert na == nb and ta == tb
    assert np.array_equal(ua, ub)


@pytest.mark.parametrize("mode", MODES, ids=lambda m: MODE_ID[m])
def test_sod_to_end_time_matches_the_host_loop(mode):
    w = W.sod(512)
    a, b = both_loops(w, t_end=0.2, cfl=0.3, precision=mode)
    assert_same(a, b)
    assert b[1] == 0.2 and b[2] > 100


@pytest.mark.parametrize("mode", MODES, ids=lambda m: MODE_ID[m])
def test_sedov_fixed_step_count_matches_the_host_loop(mode):
    w = W.sedov(24)
    assert_same(*both_loops(w, nsteps=7, cfl=0.3, precision=mode))


@pytest.mark.parametrize("recon,solver", [
    (hydro.HYDRO_RECON_PPMP, hydro.HYDRO_RIEMANN_EXACT),
    (hydro.HYDRO_RECON_PLMC, hydro.HYDRO_RIEMANN_ROE),
    (hydro.HYDRO_RECON_PLMP, hydro.HYDRO_RIEMANN_EXACT),
    (hydro.HYDRO_RECON_PCM, hydro.HYDRO_RIEMANN_ROE),
])
def test_other_schemes_match_the_host_loop(recon, solver):
    w2 = dict(u=W.smooth_periodic((1, 24, 40)), dx=1.0 / 40, gamma=1.4, bc=[P] * 6)
    assert_same(*both_loops(w2, nsteps=6, cfl=0.3, recon=recon, solver=solver))
    w3 = W.sedov(20)
    assert_same(*both_loops(w3, t_end=2e-3, cfl=0.3, recon=recon, solver=solver))


def test_noh_boundary_time_matches_the_host_loop():
    """The analytic Noh boundary reads the time the dt kernel advances."""
    w = W.noh(20, 3)
    a, b = both_loops(w, t_end=0.05, cfl=0.3)
    assert_same(a, b)


def test_long_run_spans_several_graph_launches():
    """96^3 cells: at most 75 steps a graph launch (2^26 cell updates), so 160
    steps take three launches; the state equals the host loop's."""
    w = W.sedov(96)
    a, b = both_loops(w, nsteps=160, cfl=0.3)
    assert_same(a, b)


def test_parity_with_the_oracle_after_10_steps():
    """The per-cell bar after 10 steps; the whole Sod run to t = 0.2 is compared
    in L1 by test_gpu_parity (hydro.run takes the device loop by default)."""
    for w in (W.sod(512), W.sedov(24)):
        ug, tg, ng = hydro.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=10, cfl=0.3)
        uo, to, no, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=10, cfl=0.3)
        assert fl == 0 and ng == no == 10
        assert abs(tg - to) <= 1e-12 * to
        assert rel_err(ug, uo, FLOOR[hydro.HYDRO_FP64]).max() <= TOL


def test_advance_api_edges():
    w = W.sedov(16)
    g = hydro.Grid(16, 16, 16, w["dx"], w["gamma"], w["bc"])
    try:
        with pytest.raises(hydro.HydroError):
            g.advance(0.3, 1.0, 5)  # no state yet
        g.set_state(w["u"])
        assert g.advance(0.3, math.inf, 0) == 0  # no steps
        assert np.array_equal(g.get_state(), w["u"])
        g.set_time(0.5)
        assert g.advance(0.3, 0.5, 10) == 0  # already at the end time
        assert g.advance(0.3, 0.25, 10) == 0
        assert g.get_time() == 0.5
        for bad in ((0.0, 1.0, 1), (0.3, math.nan, 1), (0.3, 1.0, -1)):
            with pytest.raises(hydro.HydroError):
                g.advance(*bad)
        # steps counted across calls, time lands on the end time exactly
        n1 = g.advance(0.3, math.inf, 3)
        t1 = g.get_time()
        assert n1 == 3 and t1 > 0.5
        n2 = g.advance(0.3, t1 + 1e-3, 1000)
        assert n2 >= 1 and g.get_time() == t1 + 1e-3
        # a precision change recaptures the loop graph
        g.set_precision(hydro.HYDRO_MIXED)
        assert g.advance(0.3, math.inf, 2) == 2
    finally:
        g.close()


def test_advance_counts_launches():
    w = W.sedov(16)
    g = hydro.Grid(16, 16, 16, w["dx"], w["gamma"], w["bc"])
    try:
        g.set_state(w["u"])
        g.profile(True)
        g.step(0.3)
        _, per_step = g.profile_read()
        g.profile(True)
        assert g.advance(0.3, math.inf, 4) == 4
        _, total = g.profile_read()
        # per step: the step's kernels and the loop-condition kernel; per graph
        # launch: the kernel that sets the condition
        assert total == 4 * (per_step + 1) + 1
    finally:
        g.close()


def test_advance_stops_at_a_failing_step():
    """A negative density injected on the host: the first step raises
    ENONPHYS, the loop stops after it and reports one step taken."""
    u = W.prim_to_cons(np.ones((8, 8, 8)), 0.0, 0.0, 0.0, np.ones((8, 8, 8)), 1.4)
    u[0, 4, 4, 4] = -1.0
    g = hydro.Grid(8, 8, 8, 0.1, 1.4, [P] * 6)
    try:
        g.set_state(u)
        n = g.advance(0.3, math.inf, 10, check=False)
        assert n == 1 and g.last_error() == -4
        with pytest.raises(hydro.HydroError):
            g.set_state(u)
            g.advance(0.3, math.inf, 10)
    finally:
        g.close()


def test_inflow_change_recaptures():
    """An inflow state is baked into the strict path's launches: changing it
    after a device run must take effect in the next one."""
    w = W.noh(16, 2)
    res = []
    for rho0 in (1.0, 2.0):
        g = hydro.Grid(16, 16, 1, w["dx"], w["gamma"], w["bc"], precision=hydro.HYDRO_FP64_STRICT)
        try:
            for f, p in w["inflow"].items():
                g.set_inflow(f, p)
            g.set_state(w["u"])
            g.advance(0.3, math.inf, 2)
            for f, p in w["inflow"].items():
                q = list(p)
                q[0] = rho0
                g.set_inflow(f, q)
            g.advance(0.3, math.inf, 3)
            res.append(g.get_state())
        finally:
            g.close()
    assert not np.array_equal(res[0], res[1])
    # and the reference: the same sequence with host steps
    g = hydro.Grid(16, 16, 1, w["dx"], w["gamma"], w["bc"], precision=hydro.HYDRO_FP64_STRICT)
    try:
        for f, p in w["inflow"].items():
            g.set_inflow(f, p)
        g.set_state(w["u"])
        for _ in range(2):
            g.step(0.3)
        for f, p in w["inflow"].items():
            q = list(p)
            q[0] = 2.0
            g.set_inflow(f, q)
        for _ in range(3):
            g.step(0.3)
        assert np.array_equal(g.get_state(), res[1])
    finally:
        g.close()


# ---- asynchronous forms (pipelines of independent problems) -----------------
def test_async_pipeline_matches_synchronous_steps():
    """Two grids on two streams, alternating: each upload-step-download of the
    same input gives the synchronous step's state bit for bit, and sync returns
    its dt."""
    torch = pytest.importorskip("torch")
    w = W.sedov(24)
    _, nz, ny, nx = w["u"].shape
    ref = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"])
    try:
        ref.set_state(w["u"])
        dt_ref = ref.step(0.3)
        u_ref = ref.get_state()
    finally:
        ref.close()
    u_in = torch.from_numpy(w["u"]).pin_memory()
    outs = [torch.empty_like(u_in).pin_memory() for _ in range(4)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    grids = [hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], stream=s) for s in streams]
    try:
        for k in range(4):
            gk = grids[k % 2]
            gk.set_state_async(u_in)
            gk.step_async(0.3)
            gk.get_state_async(outs[k])
        dts = [gg.sync() for gg in grids]
        assert dts == [dt_ref, dt_ref]
        for o in outs:
            assert np.array_equal(o.numpy(), u_ref)
    finally:
        for gg in grids:
            gg.close()


def test_async_status_is_reported_by_sync():
    u = W.prim_to_cons(np.ones((8, 8, 8)), 0.0, 0.0, 0.0, np.ones((8, 8, 8)), 1.4)
    good = u.copy()
    u[0, 4, 4, 4] = -1.0
    g = hydro.Grid(8, 8, 8, 0.1, 1.4, [P] * 6)
    try:
        g.set_state_async(u)
        g.step_async(0.3)
        g.set_state_async(good)
        g.step_async(0.3)  # a good step does not clear the earlier status
        with pytest.raises(hydro.HydroError) as e:
            g.sync()
        assert e.value.code == -4
        assert g.sync() > 0  # read and cleared
        with pytest.raises(ValueError):
            g.set_state_async(u[:, ::-1])  # would need a temporary copy
    finally:
        g.close()

"""Pins of the oracle's full CTU step (Sec. 2.3) and boundary fill (Sec. 3.1).

  * a uniform state is preserved exactly (periodic, outflow, reflective at rest);
  * totals of mass, momentum and energy are conserved to rounding on periodic
    boxes (Eq. conserved_update telescopes);
  * mirror and cyclic axis-permutation symmetry on small 3D grids;
  * Sod shock tube (config: 512 cells, t = 0.2): converges to the exact Riemann
    solution (sampled with the exact solver, pinned separately by Toro's values);
  * smooth advection converges at second order or better (paper Sec. 4.1: the
    method is second-order for smooth flow);
  * Sedov-Taylor blast: shock radius follows R = xi0 (E t^2 / rho)^(1/5) with
    xi0 = 1.152 for gamma = 5/3 (Sedov 1959), peak density below the strong
    shock limit (gamma+1)/(gamma-1);
  * ghost cells: periodic wrap, reflective mirror with negated normal
    momentum, outflow copy, inflow state; corners filled x, then y, then z;
  * the CFL time step (Eq. calc_dt_3D) equals hand-worked values on states
    whose arithmetic is exact in binary (uniform, one cell and axis setting the
    minimum, inactive axes ignored in 1D and 2D, floored pressure, real cells
    only), and copies of the oracle with planted mistakes (gamma dropped, an
    inactive axis counted, max for min, |v_d|^2 or |v| for |v_d|, ghosts
    counted, no pressure floor) each fail at least one of those cases.
"""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import workloads as W
from tests.helpers import mirror_x, rotate_xyz

P, R_, O, I_ = 0, 1, 2, 3


@pytest.fixture(autouse=True, scope="module")
def _threads():
    oracle.set_threads(0)
    yield


def uniform_state(shape, rho, v, p, gamma):
    nz, ny, nx = shape
    return W.prim_to_cons(np.full(shape, rho), v[0], v[1], v[2], np.full(shape, p), gamma)


@pytest.mark.parametrize("shape,bc,v", [
    ((8, 8, 8), [P] * 6, (0.3, -0.2, 0.1)),
    ((1, 1, 32), [O, O, P, P, P, P], (0.5, 0.0, 0.0)),
    ((6, 7, 8), [R_] * 6, (0.0, 0.0, 0.0)),
    ((1, 12, 10), [O, O, P, P, P, P], (0.2, 0.4, 0.0)),
])
def test_uniform_state_preserved_exactly(shape, bc, v):
    u0 = uniform_state(shape, 1.3, v, 0.7, 1.4)
    u, t, n, fl = oracle.run(u0, 0.1, 1.4, bc, nsteps=3, cfl=0.4)
    assert fl == 0
    assert np.array_equal(u, u0)


@pytest.mark.parametrize("shape", [(12, 12, 12), (1, 16, 16), (1, 1, 64), (6, 10, 8)])
def test_conservation_periodic(shape):
    u0 = W.smooth_periodic(shape, gamma=1.4, seed=21)
    tot0 = u0.reshape(5, -1).sum(axis=1)
    scale = np.abs(u0).reshape(5, -1).sum(axis=1)
    u, t, n, fl = oracle.run(u0, 1.0 / max(shape), 1.4, [P] * 6, nsteps=6, cfl=0.4)
    assert fl == 0
    tot = u.reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale + 1e-15), (tot - tot0) / scale
    assert not np.array_equal(u, u0)  # the state did evolve


def test_mirror_symmetry_3d():
    shape = (8, 10, 12)
    u0 = W.smooth_periodic(shape, gamma=1.4, seed=5, vamp=0.8)
    bc = [R_, R_, P, P, O, O]
    ua, *_ = oracle.run(u0, 0.1, 1.4, bc, nsteps=4, cfl=0.4)
    ub, *_ = oracle.run(mirror_x(u0), 0.1, 1.4, bc, nsteps=4, cfl=0.4)
    scale = np.abs(ua).reshape(5, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(mirror_x(ub) - ua) <= 1e-12 * scale)


def test_axis_permutation_symmetry_3d():
    shape = (8, 8, 8)
    u0 = W.smooth_periodic(shape, gamma=1.4, seed=6, vamp=0.8)
    ua, *_ = oracle.run(u0, 0.1, 1.4, [P] * 6, nsteps=4, cfl=0.4)
    ub, *_ = oracle.run(rotate_xyz(u0), 0.1, 1.4, [P] * 6, nsteps=4, cfl=0.4)
    scale = np.abs(ua).reshape(5, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(ub - rotate_xyz(ua)) <= 1e-12 * scale)


def exact_riemann_profile(x, t, x0, left, right, gamma):
    """Exact solution of a 1D Riemann problem at time t, through the exact
    solver's interface sampler and a Galilean shift per point."""
    n = len(x)
    S = (x - x0) / t
    WL = np.tile([left[0], left[1], 0.0, 0.0, left[2]], (n, 1))
    WR = np.tile([right[0], right[1], 0.0, 0.0, right[2]], (n, 1))
    WL[:, 1] -= S
    WR[:, 1] -= S
    r = oracle.riemann_prim(WL, WR, gamma)
    ws = r["ws"]
    return ws[:, 0], ws[:, 1] + S, ws[:, 4]


def sod_l1(nx):
    w = W.sod(nx)
    u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], t_end=0.2, cfl=0.3)
    assert fl == 0 and t == 0.2
    x = (np.arange(nx) + 0.5) / nx
    rho_e, v_e, p_e = exact_riemann_profile(x, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1), 1.4)
    rho = u[0, 0, 0]
    return np.mean(np.abs(rho - rho_e)), u, rho_e


def test_sod_converges_to_exact_solution():
    e1, _, _ = sod_l1(128)
    e2, _, _ = sod_l1(256)
    e3, u, rho_e = sod_l1(512)
    assert e2 < e1 and e3 < e2
    assert e1 / e3 > 2.5  # at least ~first order overall across the discontinuities
    assert e3 < 3e-3
    rho = u[0, 0, 0]
    # plateau values away from the waves: star-left and star-right densities
    x = (np.arange(512) + 0.5) / 512
    mid_l = (x > 0.62) & (x < 0.66)  # between rarefaction tail and contact
    mid_r = (x > 0.72) & (x < 0.82)  # between contact and shock
    np.testing.assert_allclose(rho[mid_l], 0.42632, rtol=2e-3)
    np.testing.assert_allclose(rho[mid_r], 0.26557, rtol=2e-3)
    # total mass in the box is conserved until waves reach the ends
    assert abs(u[0].sum() / 512 - (0.5 * 1 + 0.5 * 0.125)) < 1e-13


def test_smooth_advection_second_order():
    errs = []
    for n in (32, 64, 128):
        x = (np.arange(n) + 0.5) / n
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        u0 = W.prim_to_cons(rho.reshape(1, 1, n), 1.0, 0.0, 0.0, 1.0, 1.4)
        u, t, _, fl = oracle.run(u0, 1.0 / n, 1.4, [P] * 6, t_end=1.0, cfl=0.4)
        assert fl == 0
        errs.append(np.mean(np.abs(u[0, 0, 0] - rho)))
    order = np.log2(errs[1] / errs[2])
    assert order > 1.8, errs


@pytest.mark.slow
def test_sedov_radius_and_symmetry():
    n = 32
    w = W.sedov(n)
    g = oracle.Grid(n, n, n, w["dx"], w["gamma"], w["bc"])
    g.set_state(w["u"])
    t = 0.0
    t_check = 0.04
    while t < t_check:
        dt = min(g.compute_dt(0.3), t_check - t)
        assert g.step_dt(dt) == 0
        t += dt
    u = g.get_state()
    rho = u[0]
    gamma = w["gamma"]
    assert rho.max() < (gamma + 1) / (gamma - 1)
    # shock radius: outermost radius where the spherically binned density
    # exceeds half of its peak excess
    c = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    bins = np.linspace(0, 0.5, 41)
    idx = np.digitize(r.ravel(), bins)
    prof = np.array([rho.ravel()[idx == k].mean() if np.any(idx == k) else 1.0
                     for k in range(1, len(bins))])
    rc = 0.5 * (bins[1:] + bins[:-1])
    kpk = int(np.argmax(prof))
    half = 1.0 + 0.5 * (prof[kpk] - 1.0)
    k = kpk
    while k + 1 < len(prof) and prof[k + 1] > half:
        k += 1
    r_shock = rc[k]
    r_exact = 1.152 * (1.0 * t * t / 1.0) ** 0.2
    assert abs(r_shock - r_exact) / r_exact < 0.12, (r_shock, r_exact)
    # symmetry of the blast under the 48 cube symmetries, spot-checked
    scale = np.abs(rho).max()
    assert np.max(np.abs(rho - rho[::-1, :, :])) < 1e-12 * scale
    assert np.max(np.abs(rho - rho[:, ::-1, :])) < 1e-12 * scale
    assert np.max(np.abs(rho - rho[:, :, ::-1])) < 1e-12 * scale
    assert np.max(np.abs(rho - np.transpose(rho, (1, 2, 0)))) < 1e-12 * scale
    assert np.max(np.abs(rho - np.transpose(rho, (0, 2, 1)))) < 1e-12 * scale


def test_ghost_fill_rules():
    nx, ny, nz = 6, 5, 4
    rng = np.random.Generator(np.random.PCG64(2))
    u0 = np.zeros((5, nz, ny, nx))
    u0[0] = 1.0 + rng.random((nz, ny, nx))
    u0[1:4] = rng.normal(size=(3, nz, ny, nx))
    u0[4] = 5.0 + rng.random((nz, ny, nx))
    g = oracle.Grid(nx, ny, nz, 0.1, 1.4, [P, P, R_, O, I_, O])
    inflow = (2.0, 0.5, -0.25, 0.75, 3.0)
    g.set_inflow(4, inflow)
    g.set_state(u0)
    up = g.padded_after_ghost_fill()
    G = 4
    real = up[:, G:G + nz, G:G + ny, G:G + nx]
    assert np.array_equal(real, u0)
    # x periodic: ghost i = -d copies real nx - d
    for d in range(1, G + 1):
        np.testing.assert_array_equal(up[:, G:G + nz, G:G + ny, G - d], u0[:, :, :, nx - d])
        np.testing.assert_array_equal(up[:, G:G + nz, G:G + ny, G + nx - 1 + d], u0[:, :, :, d - 1])
    # y- reflective: ghost j = -d mirrors real d-1 with negated y momentum
    for d in range(1, G + 1):
        got = up[:, G:G + nz, G - d, G:G + nx]
        exp = u0[:, :, d - 1, :].copy()
        exp[2] = -exp[2]
        np.testing.assert_array_equal(got, exp)
    # y+ outflow: every ghost copies the last real row
    for d in range(1, G + 1):
        np.testing.assert_array_equal(up[:, G:G + nz, G + ny - 1 + d, G:G + nx], u0[:, :, ny - 1, :])
    # z- inflow: the prescribed state everywhere in the ghost slab, corners included
    rho, vx, vy, vz, p = inflow
    E = p / (1.4 - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    for q, val in enumerate((rho, rho * vx, rho * vy, rho * vz, E)):
        assert np.all(up[q, :G] == val)
    # z+ outflow copies the last real plane including its x/y ghosts (corners)
    for d in range(1, G + 1):
        np.testing.assert_array_equal(up[:, G + nz - 1 + d], up[:, G + nz - 1])
    # an x-y corner ghost equals the y rule applied to the x-filled ghost column
    exp = up[:, G:G + nz, G, G - 1].copy()  # x-ghost of the first real row
    exp[2] = -exp[2]
    np.testing.assert_array_equal(up[:, G:G + nz, G - 1, G - 1], exp)


def test_update_depends_on_cells_within_three():
    """One CTU step of a cell depends only on the cells within 3 of it along each
    axis (slopes reach 1, PPMC 1 more, the transverse fluxes 1 more): the step of
    a 20^3 block cut from a periodic field, with outflow faces, equals the
    full-grid step bit for bit 3 cells away from the block's faces, and not 2
    away.  The full-size GPU parity tests rely on this to sample 512^3 steps."""
    w = W.turbulence(48, kmax=2)
    u0, n = w["u"], 48
    g = oracle.Grid(n, n, n, w["dx"], w["gamma"], w["bc"])
    g.set_state(u0)
    dt = g.compute_dt(0.3)
    g.step_dt(dt)
    uf = g.get_state()
    R = 10
    for c in [(20, 17, 30), (0, 47, 5)]:
        idx = [np.arange(ci - R, ci + R) % n for ci in c]
        sub = np.ascontiguousarray(u0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]])
        b = oracle.Grid(2 * R, 2 * R, 2 * R, w["dx"], w["gamma"], [2] * 6)
        b.set_state(sub)
        b.step_dt(dt)
        ub = b.get_state()
        for m, exact in ((3, True), (2, False)):
            cen = ub[:, m:2 * R - m, m:2 * R - m, m:2 * R - m]
            inner = [ix[m:2 * R - m] for ix in idx]
            ref = uf[:, inner[0]][:, :, inner[1]][:, :, :, inner[2]]
            assert np.array_equal(cen, ref) == exact, (c, m)


def test_threaded_oracle_is_bit_identical_to_one_thread():
    """The OpenMP loops over the outer index change nothing: the step on all
    cores equals the single-thread step bit for bit."""
    w = W.turbulence(24, kmax=2)
    out = []
    for nthreads in (1, 0):
        oracle.set_threads(nthreads)
        u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], nsteps=3, cfl=0.3)
        out.append((u, t))
    oracle.set_threads(0)
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


# ---- the CFL time step (Sec. 2.1, Eqs. calc_dt_1D / calc_dt_3D) --------------
# dt = C0 * min over real cells and active axes of dx / (|v_d| + a), a =
# sqrt(gamma p / rho) from the cell averages (pressure floored at 1e-20).  The
# states below are written directly as conserved variables whose primitives,
# sound speeds and quotients are exact in binary floating point (gamma = 2
# makes gamma p / rho a product of exact numbers), so the expected dt is a
# number worked out by hand, not the formula evaluated again.

def _cons(shape, rho, m, E):
    """Conserved state [5, nz, ny, nx] filled with (rho, m_x, m_y, m_z, E)."""
    u = np.empty((5,) + tuple(shape))
    for q, v in enumerate((rho, m[0], m[1], m[2], E)):
        u[q] = v
    return u


def _dt_cases():
    """(name, u, dx, gamma, bc, cfl, inflow, check) -- check(dt) is True for
    the value the equation gives; every number in a comment is exact."""
    cases = []
    # uniform 3D, gamma 2: rho 4, v (0.5, -2, 1), p 8 -> a = sqrt(2*8/4) = 2;
    # |v_d| + a = 2.5, 4, 3 -> the y axis sets dt = 0.4 * 0.5/4 = 0.05;
    # m = (2, -8, 4), E = 8 + 4 (0.25 + 4 + 1)/2 = 18.5
    cases.append(("uniform3d", _cons((4, 5, 6), 4.0, (2.0, -8.0, 4.0), 18.5), 0.5, 2.0, [P] * 6,
                  0.4, None, lambda dt: dt == 0.05))
    # one cell and one axis set the minimum: background rho 1, v 0, p 0.5 (a = 1,
    # E = 0.5); cell (i4, j1, k2) moves at v_z = 3 (signal 4; E = 0.5 + 4.5 = 5),
    # cell (i1, j3, k0) at v_x = -2.5 (signal 3.5; E = 0.5 + 3.125 = 3.625):
    # dt = 0.8 * 0.25/4 = 0.05
    u = _cons((4, 5, 6), 1.0, (0.0, 0.0, 0.0), 0.5)
    u[3, 2, 1, 4] = 3.0; u[4, 2, 1, 4] = 5.0
    u[1, 0, 3, 1] = -2.5; u[4, 0, 3, 1] = 3.625
    cases.append(("one_cell_z", u, 0.25, 2.0, [P] * 6, 0.8, None, lambda dt: dt == 0.05))
    # 1D box along x: the inactive y and z velocities (10, -20) do not count;
    # rho 1, p 0.5 (a = 1), v_x 1 -> dt = 0.5 * 0.5/2 = 0.125; E = 0.5 + 501/2 = 251
    cases.append(("inactive_1d", _cons((1, 1, 16), 1.0, (1.0, 10.0, -20.0), 251.0), 0.5, 2.0,
                  [O, O, P, P, P, P], 0.5, None, lambda dt: dt == 0.125))
    # 2D box (x, y): v_z = 50 does not count; v = (1, -1.5), a = 1 -> signal 2.5,
    # dt = 0.5 * 0.5/2.5 = 0.1; E = 0.5 + (1 + 2.25 + 2500)/2 = 1252.125
    cases.append(("inactive_2d", _cons((1, 6, 8), 1.0, (1.0, -1.5, 50.0), 1252.125), 0.5, 2.0,
                  [P] * 6, 0.5, None, lambda dt: dt == 0.1))
    # a cell with no internal energy (E = rho v^2/2 exactly: p = 0, floored to
    # 1e-20, a = sqrt(2e-20) = 1.414e-10) at v_x = 4 sets the minimum: dt =
    # 0.5 * 0.5/(4 + 1.414e-10) = 0.0625 (1 - 3.54e-11), strictly below the
    # 0.0625 that a zero sound speed would give; background as above
    u = _cons((4, 4, 4), 1.0, (0.0, 0.0, 0.0), 0.5)
    u[1, 1, 2, 3] = 4.0; u[4, 1, 2, 3] = 8.0
    cases.append(("floored_p", u, 0.5, 2.0, [P] * 6, 0.5, None,
                  lambda dt: 0.0625 * (1 - 3.6e-11) < dt < 0.0625 * (1 - 3.5e-11)))
    # a cell whose total energy is below its kinetic energy (E = 7 < 8): the
    # floored pressure gives it the same tiny sound speed, so it still sets dt
    u = _cons((4, 4, 4), 1.0, (0.0, 0.0, 0.0), 0.5)
    u[2, 3, 0, 1] = -4.0; u[4, 3, 0, 1] = 7.0
    cases.append(("negative_p", u, 0.5, 2.0, [P] * 6, 0.5, None,
                  lambda dt: 0.0625 * (1 - 3.6e-11) < dt < 0.0625 * (1 - 3.5e-11)))
    # gamma 5/3 (not exact in binary): rho 1, p 0.6 -> a = 1, v = (0.25, 0, 0),
    # signal 1.25, dt = 0.3 * (1/32)/1.25 = 0.0075 to a few ulp
    E = 0.6 / (2.0 / 3.0) + 0.5 * 0.0625
    cases.append(("gamma53", _cons((4, 4, 4), 1.0, (0.25, 0.0, 0.0), E), 1.0 / 32, 5.0 / 3.0,
                  [P] * 6, 0.3, None, lambda dt: abs(dt / 0.0075 - 1) < 1e-15))
    # only real cells count: an x- inflow face at v = 50 fills the ghosts; after
    # a step of 1e-15 (which moves the real cells' pressure by ~1e-10 relative)
    # the real cells still give rho 1, v_x 1, a 1: dt = 0.5 * 0.5/2 = 0.125
    cases.append(("ghosts_excluded", _cons((1, 1, 16), 1.0, (1.0, 0.0, 0.0), 1.0), 0.5, 2.0,
                  [I_, O, P, P, P, P], 0.5, {0: (1.0, 50.0, 0.0, 0.0, 0.5)},
                  lambda dt: abs(dt / 0.125 - 1) < 1e-9))
    return cases


def _bind(L):
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_init.restype = ctypes.c_void_p
    L.oracle_init.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.POINTER(ctypes.c_int)]
    L.oracle_free.argtypes = [ctypes.c_void_p]
    L.oracle_set_state.argtypes = [ctypes.c_void_p, dp]
    L.oracle_set_inflow.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
    L.oracle_compute_dt.restype = ctypes.c_double
    L.oracle_compute_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.oracle_step_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    return L


def _dt_with(L, u, dx, gamma, bc, cfl, inflow):
    """dt of the case through the oracle library L (the real one or a mutant)."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    u = np.ascontiguousarray(u)
    _, nz, ny, nx = u.shape
    h = L.oracle_init(nx, ny, nz, dx, gamma, (ctypes.c_int * 6)(*bc))
    assert h
    try:
        L.oracle_set_state(h, u.ctypes.data_as(dp))
        if inflow:
            for face, prim in inflow.items():
                pa = np.asarray(prim, dtype=np.float64)
                L.oracle_set_inflow(h, face, pa.ctypes.data_as(dp))
            L.oracle_step_dt(h, 1e-15)
        return L.oracle_compute_dt(h, cfl)
    finally:
        L.oracle_free(h)


@pytest.mark.parametrize("case", _dt_cases(), ids=lambda c: c[0])
def test_cfl_dt_hand_computed(case):
    """The oracle's dt equals the hand-worked value of Eq. calc_dt_3D."""
    name, u, dx, gamma, bc, cfl, inflow, check = case
    dt = _dt_with(_bind(oracle.lib()), u, dx, gamma, bc, cfl, inflow)
    assert check(dt), (name, repr(dt))


_CDT = "R compute_dt_min(const Grid<R>& G) {"
_C2P = "void cons_to_prim(const R U[5], const Gas& g, R W[5]) {"
_DT_MUTANTS = {
    # the sound speed without gamma
    "gamma_dropped": [(_CDT, "sqrt(R(g.gamma) * W[4] / W[0])", "sqrt(W[4] / W[0])")],
    # an axis with one cell counted
    "inactive_axis_counted": [(_CDT, "if (G.n[d] <= 1) continue;", "")],
    # the largest quotient kept instead of the smallest
    "max_for_min": [(_CDT, "std::numeric_limits<double>::infinity()", "0.0"),
                    (_CDT, "if (t < bestR)", "if (t > bestR)")],
    # |v_d|^2 in place of |v_d|
    "v_squared": [(_CDT, "fabs(W[1 + d])", "(W[1 + d] * W[1 + d])")],
    # the speed |v| in place of the axis component |v_d|
    "speed_not_component": [(_CDT, "fabs(W[1 + d])", "sqrt(W[1] * W[1] + W[2] * W[2] + W[3] * W[3])")],
    # ghost cells counted
    "ghosts_counted": [(_CDT, "for (int k = G.gh[2]; k < G.gh[2] + G.n[2]; ++k)",
                        "for (int k = 0; k < G.N[2]; ++k)"),
                       (_CDT, "for (int j = G.gh[1]; j < G.gh[1] + G.n[1]; ++j)",
                        "for (int j = 0; j < G.N[1]; ++j)"),
                       (_CDT, "for (int i = G.gh[0]; i < G.gh[0] + G.n[0]; ++i)",
                        "for (int i = 0; i < G.N[0]; ++i)")],
    # no pressure floor in the cell primitives
    "no_pressure_floor": [(_C2P, "W[4] = mx(p, R(P_FLOOR));", "W[4] = p;")],
}


def test_cfl_dt_pins_catch_planted_mistakes():
    """Each plausible mistake in the oracle's dt, planted in a copy of the
    oracle source, fails at least one hand-computed case: gamma dropped from the
    sound speed, an inactive axis counted, the maximum taken for the minimum,
    |v_d|^2 for |v_d|, the speed |v| for the component |v_d|, ghost cells
    counted, the pressure floor left out."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_DT_MUTANTS)) as ex:
        libs = dict(zip(_DT_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                              _DT_MUTANTS.items())))
    cases = _dt_cases()
    for tag, L in libs.items():
        _bind(L)
        failed = [c[0] for c in cases if not c[7](_dt_with(_bind(L), *c[1:7]))]
        assert failed, "planted mistake %r passes every dt pin" % tag
        print("%s fails %s" % (tag, failed))


# ---- the transverse half-step (Eq. transverse_evolution) ------------------
# Two 2D problems whose exact solution after a known time is the initial state:
# a density wave advected supersonically along the diagonal, v = (1, 1), one
# period at t = 1; and a small-amplitude acoustic simple wave travelling along
# the diagonal through a subsonic flow, one period at T = (1/sqrt 2)/(v.n + a).
# The unsplit CTU step with its transverse half-step is stable up to a Courant
# number 1 per axis in 2D; without the transverse terms, or with them wrong,
# the scheme is unstable there (the per-axis Courant numbers add up to 1.9) or
# loses its accuracy.

def _bind_run(L):
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    _bind(L)
    L.oracle_get_state.argtypes = [ctypes.c_void_p, dp]
    return L


def _periodic_2d_error(L, u0, gamma, t_end, cfl):
    """Run the 2D periodic state u0 [5, 1, n, n] to t_end with the oracle library
    L; returns the mean |rho - rho0| (NaN when the run blew up)."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    u0 = np.ascontiguousarray(u0)
    n = u0.shape[-1]
    h = L.oracle_init(n, n, 1, 1.0 / n, gamma, (ctypes.c_int * 6)(*([P] * 6)))
    assert h
    try:
        L.oracle_set_state(h, u0.ctypes.data_as(dp))
        t, steps = 0.0, 0
        while t < t_end and steps < 1000:
            dt = min(L.oracle_compute_dt(h, cfl), t_end - t)
            if not dt > 0.0:
                return float("nan")
            L.oracle_step_dt(h, dt)
            t += dt
            steps += 1
        out = np.zeros_like(u0)
        L.oracle_get_state(h, out.ctypes.data_as(dp))
    finally:
        L.oracle_free(h)
    return float(np.abs(out[0] - u0[0]).mean())


def _transverse_cases(n=48):
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.sin(2 * np.pi * (X + Y))
    # supersonic advection of a density wave (p uniform, a = 0.012)
    rho = (1.0 + 0.2 * f)[None]
    adv = W.prim_to_cons(rho, 1.0, 1.0, 0.0, np.full_like(rho, 1e-4), 1.4)
    # acoustic simple wave along n = (1, 1)/sqrt 2 in a flow v = (0.3, 0.3)
    g, eps, v0 = 1.4, 1e-3, 0.3
    a0 = np.sqrt(g)
    dr = eps * f
    nn = 1 / np.sqrt(2)
    ac = W.prim_to_cons((1.0 + dr)[None], (v0 + a0 * dr * nn)[None], (v0 + a0 * dr * nn)[None],
                        0.0, (1.0 + a0 * a0 * dr)[None], g)
    T = (1 / np.sqrt(2)) / (2 * v0 * nn + a0)
    return {"advection": (adv, 1.4, 1.0, 0.2), "acoustic": (ac, g, T, eps)}


def _transverse_errors(L, cfl=0.95):
    """Mean density error after one period over the wave's amplitude, per case."""
    return {k: _periodic_2d_error(L, u, g, T, cfl) / amp
            for k, (u, g, T, amp) in _transverse_cases().items()}


def test_ctu_transverse_half_step_stable_and_accurate_at_courant_095():
    """The diagonal density wave (supersonic) and the diagonal acoustic wave
    (subsonic) return to their initial state after one period at a Courant number
    0.95 per axis: mean density error below 1% (advection; measured 0.23%) and 2%
    (acoustic; measured 0.43%) of the amplitude."""
    errs = _transverse_errors(_bind_run(oracle.lib()))
    assert errs["advection"] <= 0.01, errs
    assert errs["acoustic"] <= 0.02, errs


_CTU = "int ctu_step(Grid<R>& G, double dt_in, bool threaded) {"
_TL = "UhL[q] = UhL[q] + hdtdx * (F1[t][q * nc + cl] - F1[t][q * nc + cl + st]);"
_TR = "UhR[q] = UhR[q] + hdtdx * (F1[t][q * nc + cr] - F1[t][q * nc + cr + st]);"
_TRANSVERSE_MUTANTS = {
    # the transverse half-step left out (the plain unsplit step)
    "no_transverse": [(_CTU, _TL, ""), (_CTU, _TR, "")],
    # the transverse flux differences with the wrong sign
    "sign": [(_CTU, _TL, _TL.replace("+ hdtdx", "- hdtdx")),
             (_CTU, _TR, _TR.replace("+ hdtdx", "- hdtdx"))],
    # a full dt/dx instead of dt/(2 dx)
    "full_dt": [(_CTU, "const R hdtdx = R(0.5) * dtdx;", "const R hdtdx = dtdx;")],
    # the right state corrected with the left cell's transverse fluxes
    "wrong_cell": [(_CTU, _TR, _TR.replace("cr", "cl"))],
}


def test_transverse_pin_catches_planted_mistakes():
    """Each plausible mistake in the transverse half-step, planted in a copy of
    the oracle, fails the Courant-0.95 pin: the half-step left out, its sign
    flipped, a full step dt/dx, the right state taking the left cell's
    transverse fluxes (the supersonic case alone cannot see that one: there the
    flux is the left state's)."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_TRANSVERSE_MUTANTS)) as ex:
        libs = dict(zip(_TRANSVERSE_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                      _TRANSVERSE_MUTANTS.items())))
    for tag, L in libs.items():
        errs = _transverse_errors(_bind_run(L))
        caught = not (errs["advection"] <= 0.01) or not (errs["acoustic"] <= 0.02)
        assert caught, "planted mistake %r passes the transverse pin: %s" % (tag, errs)
        print("%s: %s" % (tag, errs))



# ---------------------------------------------------------------------------
# Planted mistakes in the conserved update and the ghost rules: each fails the
# smooth-advection order pin or the ghost-rule pin, re-run through a copy of
# the oracle with the mistake.

def _advection_order(L):
    """The smooth-advection pin through the oracle library L: the mean density
    errors after one period at 32, 64, 128 cells and the observed order."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    errs = []
    for n in (32, 64, 128):
        x = (np.arange(n) + 0.5) / n
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        u0 = np.ascontiguousarray(W.prim_to_cons(rho.reshape(1, 1, n), 1.0, 0.0, 0.0, 1.0, 1.4))
        h = L.oracle_init(n, 1, 1, 1.0 / n, 1.4, (ctypes.c_int * 6)(*([P] * 6)))
        assert h
        try:
            L.oracle_set_state(h, u0.ctypes.data_as(dp))
            t, steps = 0.0, 0
            while t < 1.0 and steps < 2000:
                dt = min(L.oracle_compute_dt(h, 0.4), 1.0 - t)
                if not dt > 0.0:
                    break
                L.oracle_step_dt(h, dt)
                t += dt
                steps += 1
            out = np.zeros_like(u0)
            L.oracle_get_state(h, out.ctypes.data_as(dp))
        finally:
            L.oracle_free(h)
        errs.append(float(np.abs(out[0, 0, 0] - rho).mean()))
    with np.errstate(all="ignore"):
        order = float(np.log2(errs[1] / errs[2]))
    return errs, order


def _ghost_rule_errors(L):
    """The reflective, periodic and outflow ghost rules of test_ghost_fill_rules
    through the oracle library L: the number of ghost values that differ from
    the rule."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_fill_ghosts.argtypes = [ctypes.c_void_p, dp]
    nx, ny, nz = 6, 5, 4
    rng = np.random.Generator(np.random.PCG64(2))
    u0 = np.zeros((5, nz, ny, nx))
    u0[0] = 1.0 + rng.random((nz, ny, nx))
    u0[1:4] = rng.normal(size=(3, nz, ny, nx))
    u0[4] = 5.0 + rng.random((nz, ny, nx))
    h = L.oracle_init(nx, ny, nz, 0.1, 1.4, (ctypes.c_int * 6)(P, P, R_, O, O, O))
    assert h
    G = 4
    up = np.zeros((5, nz + 2 * G, ny + 2 * G, nx + 2 * G))
    try:
        L.oracle_set_state(h, np.ascontiguousarray(u0).ctypes.data_as(dp))
        L.oracle_fill_ghosts(h, up.ctypes.data_as(dp))
    finally:
        L.oracle_free(h)
    bad = 0
    for d in range(1, G + 1):
        bad += int(np.sum(up[:, G:G + nz, G:G + ny, G - d] != u0[:, :, :, nx - d]))
        bad += int(np.sum(up[:, G:G + nz, G:G + ny, G + nx - 1 + d] != u0[:, :, :, d - 1]))
        exp = u0[:, :, d - 1, :].copy()
        exp[2] = -exp[2]
        bad += int(np.sum(up[:, G:G + nz, G - d, G:G + nx] != exp))
        bad += int(np.sum(up[:, G:G + nz, G + ny - 1 + d, G:G + nx] != u0[:, :, ny - 1, :]))
    return bad


_UPD = "un = un + dtdx * (F2[d][q * nc + c] - F2[d][q * nc + c + sd]);"
_FG = "void fill_ghosts(Grid<R>& G) {"
_UPDATE_GHOST_MUTANTS = {
    # the flux difference with the wrong sign (still conservative)
    "update_sign": [(_CTU, _UPD, "un = un - dtdx * (F2[d][q * nc + c] - F2[d][q * nc + c + sd]);")],
    # half the step
    "update_half": [(_CTU, _UPD, "un = un + R(0.5) * dtdx * (F2[d][q * nc + c] - F2[d][q * nc + c + sd]);")],
    # the fluxes of the faces one cell to the left (still conservative)
    "update_shift": [(_CTU, _UPD, "un = un + dtdx * (F2[d][q * nc + c - sd] - F2[d][q * nc + c]);")],
    # the reflective rule without the negated normal momentum
    "reflect_momentum": [(_FG, "if (type == BC_REFLECT && q == 1 + d) val_ = -val_;", "")],
    # the periodic rule one cell off
    "periodic_offset": [(_FG, "case BC_PERIODIC: src = side == 0 ? G.gh[d] + G.n[d] - gd : G.gh[d] + gd - 1; break;",
                         "case BC_PERIODIC: src = side == 0 ? G.gh[d] + G.n[d] - gd - 1 : G.gh[d] + gd; break;")],
    # the outflow rule copying the second real cell from the face
    "outflow_inner": [(_FG, "case BC_OUTFLOW: src = side == 0 ? G.gh[d] : G.gh[d] + G.n[d] - 1; break;",
                       "case BC_OUTFLOW: src = side == 0 ? G.gh[d] + 1 : G.gh[d] + G.n[d] - 2; break;")],
}


def test_update_and_ghost_pins_catch_planted_mistakes():
    """Each plausible slip in the conserved update (Eq. conserved_update) or
    the ghost rules (Sec. 3.1), planted in a copy of the oracle source, fails
    the smooth-advection pin (observed order above 1.8, error at 128 cells
    below 1e-3) or the ghost-rule pin; the oracle as it is passes both."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_UPDATE_GHOST_MUTANTS)) as ex:
        libs = dict(zip(_UPDATE_GHOST_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                        _UPDATE_GHOST_MUTANTS.items())))

    def passes(L):
        _bind_run(L)
        errs, order = _advection_order(L)
        ghosts = _ghost_rule_errors(L)
        ok = bool(order > 1.8 and errs[2] < 1e-3 and ghosts == 0)
        return ok, {"errs": errs, "order": order, "ghost_mismatches": ghosts}

    for tag, L in libs.items():
        ok, info = passes(L)
        assert not ok, "planted mistake %r passes the update and ghost pins: %s" % (tag, info)
        print("%s: %s" % (tag, info))
    ok, info = passes(oracle.lib())
    assert ok, info

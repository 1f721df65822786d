"""Pins of the oracle's other reconstructions (Sec. 2.2.1, App. A): PPMP, PLMC,
PLMP and PCM, on single stencils and through whole CTU steps.

Every expected value here comes from the mathematics (exact averages of
polynomials, the exact Riemann solution) or from the paper's reported results,
not from the reconstruction formulas themselves.
"""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import workloads as W
from tests.test_oracle_ctu import exact_riemann_profile

G = 1.4
ALL = [oracle.RECON_PPMC, oracle.RECON_PPMP, oracle.RECON_PLMC, oracle.RECON_PLMP,
       oracle.RECON_PCM]
NAMES = {oracle.RECON_PPMC: "ppmc", oracle.RECON_PPMP: "ppmp", oracle.RECON_PLMC: "plmc",
         oracle.RECON_PLMP: "plmp", oracle.RECON_PCM: "pcm"}
P, O = 0, 2


def cons(w):
    """[n, 5] primitives -> conserved (rotated order is the same layout)."""
    w = np.asarray(w, dtype=np.float64)
    u = W.prim_to_cons(w[:, 0], w[:, 1], w[:, 2], w[:, 3], w[:, 4], G)
    return u.reshape(5, -1).T


def stencil(rho, u, v, ww, p):
    """[7, 5] stencil from per-cell arrays (or scalars) of the 7 cells i-3..i+3."""
    st = np.zeros((7, 5))
    for q, f in enumerate((rho, u, v, ww, p)):
        st[:, q] = f
    return st


def cell_averages(poly, x0, dx, n=7):
    """Exact cell averages of a polynomial (numpy poly1d) over n cells of width
    dx whose first cell starts at x0."""
    P_ = np.polyint(poly)
    edges = x0 + dx * np.arange(n + 1)
    return (P_(edges[1:]) - P_(edges[:-1])) / dx


@pytest.mark.parametrize("recon", ALL, ids=lambda r: NAMES[r])
def test_constant_data_exact(recon):
    st = stencil(1.3, 0.4, -0.2, 0.7, 2.1)
    UsL, UsR = oracle.reconstruct(recon, st[None], 0.3, 0.01, G)
    expect = cons(st[3:4])
    assert np.array_equal(UsL, expect) or np.allclose(UsL, expect, rtol=2e-16, atol=0)
    assert np.allclose(UsR, expect, rtol=2e-16, atol=0)


@pytest.mark.parametrize("recon", [oracle.RECON_PPMP, oracle.RECON_PLMC, oracle.RECON_PLMP],
                         ids=lambda r: NAMES[r])
def test_linear_data_gives_exact_face_values_at_dt0(recon):
    # gentle monotone linear profiles (no limiter, steepening or flattening acts)
    x = np.arange(7) - 3.0
    st = stencil(1.0 + 0.002 * x, 0.3 + 0.01 * x, 0.1 - 0.02 * x, 0.05 * x, 1.0 + 0.01 * x)
    UsL, UsR = oracle.reconstruct(recon, st[None], 0.0, 1.0, G)
    wl = stencil(1.0 - 0.001, 0.3 - 0.005, 0.1 + 0.01, -0.025, 1.0 - 0.005)[3:4]
    wr = stencil(1.0 + 0.001, 0.3 + 0.005, 0.1 - 0.01, 0.025, 1.0 + 0.005)[3:4]
    np.testing.assert_allclose(UsL, cons(wl), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(UsR, cons(wr), rtol=1e-13, atol=1e-15)


def test_ppmp_cubic_averages_give_cubic_face_values_at_dt0():
    """The parabolic interpolation of PPMP (centred slopes, the MC limiter
    inactive) is fourth order: cell averages of a cubic give its point values
    at the faces.  Small amplitudes keep steepening (density jump < 1%) and
    flattening (pressure jump < 1/3) off."""
    dx = 0.1
    cubics = [np.poly1d([0.002, 0.001, 0.004, 1.0]), np.poly1d([0.05, -0.02, 0.3, 0.2]),
              np.poly1d([-0.03, 0.01, 0.2, -0.1]), np.poly1d([0.02, 0.03, -0.1, 0.3]),
              np.poly1d([0.001, -0.002, 0.02, 1.0])]
    st = np.stack([cell_averages(c, -3.5 * dx, dx) for c in cubics], axis=1)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PPMP, st[None], 0.0, dx, G)
    wl = np.array([[c(-0.5 * dx) for c in cubics]])
    wr = np.array([[c(0.5 * dx) for c in cubics]])
    np.testing.assert_allclose(UsL, cons(wl), rtol=1e-12)
    np.testing.assert_allclose(UsR, cons(wr), rtol=1e-12)


@pytest.mark.parametrize("recon", [oracle.RECON_PPMP, oracle.RECON_PPMC],
                         ids=lambda r: NAMES[r])
def test_advected_quadratic_traces_to_exact_average(recon):
    """Uniform subsonic flow (u > 0) and pressure with a quadratic density: the
    density at the right face is the exact average of the quadratic over the
    contact's domain of dependence [x_R - u dt, x_R], at the left face over the
    left acoustic wave's [x_L, x_L + (a - u) dt]."""
    dx, u, p = 1.0, 0.4, 1.0
    q = np.poly1d([0.001, 0.004, 1.0])  # rho(x): 0.3% variation, no steepening
    rho = cell_averages(q, -3.5 * dx, dx)
    st = stencil(rho, u, 0.0, 0.0, p)
    dtdx = 0.3
    UsL, UsR = oracle.reconstruct(recon, st[None], dtdx, dx, G)
    a = np.sqrt(G * p / rho[3])
    Q = np.polyint(q)
    xR, xL = 0.5 * dx, -0.5 * dx
    sR = u * dtdx * dx
    sL = (a - u) * dtdx * dx
    rhoR = (Q(xR) - Q(xR - sR)) / sR
    rhoL = (Q(xL + sL) - Q(xL)) / sL
    assert UsR[0, 0] == pytest.approx(rhoR, rel=1e-13)
    assert UsL[0, 0] == pytest.approx(rhoL, rel=1e-13)


def test_plm_advected_linear_density():
    """Uniform flow, linear density: PLMC traces the right face to the average
    over [x_R - u dt, x_R] and the left face over [x_L, x_L + (a - u) dt]; PLMP
    evolves both faces by the cell's own flux difference, i.e. to the profile
    at x - u dt/2 (exact for a linear profile in uniform flow)."""
    dx, u, p, s = 1.0, 0.4, 1.0, 0.002
    x = np.arange(7) - 3.0
    st = stencil(1.0 + s * x, u, 0.0, 0.0, p)
    dtdx = 0.3
    a = np.sqrt(G * p / 1.0)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PLMC, st[None], dtdx, dx, G)
    assert UsR[0, 0] == pytest.approx(1.0 + s * (0.5 - 0.5 * u * dtdx), rel=1e-14)
    assert UsL[0, 0] == pytest.approx(1.0 + s * (-0.5 + 0.5 * (a - u) * dtdx), rel=1e-14)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PLMP, st[None], dtdx, dx, G)
    assert UsR[0, 0] == pytest.approx(1.0 + s * (0.5 - 0.5 * u * dtdx), rel=1e-14)
    assert UsL[0, 0] == pytest.approx(1.0 + s * (-0.5 - 0.5 * u * dtdx), rel=1e-14)


def test_pcm_face_states_are_the_cell_average():
    rng = np.random.default_rng(5)
    st = np.abs(rng.normal(1.0, 0.3, size=(4, 7, 5))) + 0.1
    UsL, UsR = oracle.reconstruct(oracle.RECON_PCM, st, 0.4, 1.0, G)
    np.testing.assert_array_equal(UsL, cons(st[:, 3]))
    np.testing.assert_array_equal(UsR, cons(st[:, 3]))


@pytest.mark.parametrize("recon", ALL, ids=lambda r: NAMES[r])
def test_mirror_symmetry(recon):
    """Mirrored stencil (order reversed, normal velocity negated): the left and
    right face states swap, with the normal momentum negated."""
    rng = np.random.default_rng(11)
    st = np.column_stack([rng.uniform(0.5, 2.0, 7), rng.uniform(-0.5, 0.5, 7),
                          rng.uniform(-0.5, 0.5, 7), rng.uniform(-0.5, 0.5, 7),
                          rng.uniform(0.5, 2.0, 7)])
    mir = st[::-1].copy()
    mir[:, 1] = -mir[:, 1]
    UsL, UsR = oracle.reconstruct(recon, st[None], 0.25, 1.0, G)
    ML, MR = oracle.reconstruct(recon, mir[None], 0.25, 1.0, G)
    flip = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    np.testing.assert_allclose(ML[0], UsR[0] * flip, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(MR[0], UsL[0] * flip, rtol=1e-12, atol=1e-14)


def test_ppmp_flattens_a_one_cell_compressive_shock():
    """A pressure jump of 10 between cells i and i+1 with converging flow is a
    shock inside fewer than two cells: the flattening coefficient is 1 and the
    face values fall back to the cell average (at dt = 0 the face states are
    w_i).  The same jump in expanding flow is not flattened."""
    p = np.array([1.0, 1.0, 1.0, 1.0, 10.0, 10.0, 10.0])
    conv = stencil(1.0, np.array([1.0, 1.0, 1.0, 0.5, 0.0, 0.0, 0.0]), 0.0, 0.0, p)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PPMP, conv[None], 0.0, 1.0, G)
    np.testing.assert_allclose(UsL, cons(conv[3:4]), rtol=1e-15)
    np.testing.assert_allclose(UsR, cons(conv[3:4]), rtol=1e-15)
    expd = conv.copy()
    expd[:, 1] = -expd[:, 1]
    UsL, UsR = oracle.reconstruct(oracle.RECON_PPMP, expd[None], 0.0, 1.0, G)
    assert abs(UsR[0, 4] - cons(expd[3:4])[0, 4]) > 0.1


def _contact_cells(recon, nx=100):
    w = W.sod(nx, left=(1.0, 0.0, 1.0), right=(0.1, 0.0, 0.1))
    u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], t_end=0.2, cfl=0.3,
                             recon=recon)
    assert fl == 0 and t == 0.2
    x = (np.arange(nx) + 0.5) / nx
    rho_e, _, _ = exact_riemann_profile(x, 0.2, 0.5, (1, 0, 1), (0.1, 0, 0.1), 1.4)
    rl = rho_e[(x > 0.6) & (x < 0.66)].mean()
    rr = rho_e[(x > 0.75) & (x < 0.8)].mean()
    lo, hi = rr + 0.05 * (rl - rr), rr + 0.95 * (rl - rr)
    rho = u[0, 0, 0]
    return int(np.sum((x > 0.62) & (x < 0.8) & (rho > lo) & (rho < hi)))


def test_ppmp_resolves_the_sod_contact_in_two_zones():
    """Sec. 4.1.1 (the paper's Sod: rho, p = 1 | 0.1, 100 cells, t = 0.2): the
    contact is resolved over two zones with PPMP and three to four with PPMC.
    Counted: cells between the two star densities by more than 5% of the jump."""
    assert _contact_cells(oracle.RECON_PPMP) <= 2
    assert 3 <= _contact_cells(oracle.RECON_PPMC) <= 4


@pytest.mark.parametrize("recon", ALL, ids=lambda r: NAMES[r])
def test_uniform_state_and_conservation_through_steps(recon):
    u0 = W.prim_to_cons(np.full((6, 7, 8), 1.3), 0.4, -0.3, 0.2, np.full((6, 7, 8), 0.9), G)
    u, t, n, fl = oracle.run(u0, 0.1, G, [P] * 6, nsteps=3, cfl=0.4, recon=recon)
    assert np.array_equal(u, u0)
    w = W.smooth_periodic((12, 10, 14), gamma=G, seed=3)
    u, t, n, fl = oracle.run(w, 1.0 / 14, G, [P] * 6, nsteps=5, cfl=0.4, recon=recon)
    assert fl == 0
    tot0, tot = w.reshape(5, -1).sum(axis=1), u.reshape(5, -1).sum(axis=1)
    scale = np.abs(w).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale)


@pytest.mark.parametrize("recon,order", [(oracle.RECON_PPMP, 0.75), (oracle.RECON_PLMC, 0.75),
                                         (oracle.RECON_PLMP, 0.75), (oracle.RECON_PCM, 0.45)],
                         ids=["ppmp", "plmc", "plmp", "pcm"])
def test_sod_converges_to_exact_solution(recon, order):
    """L1 density error against the exact solution falls with resolution
    (128 -> 512 cells).  With a contact and a shock in the solution the L1
    order is below one even for the higher-order methods (a contact's smearing
    shrinks slower than the cell width); PCM, first order and diffusive,
    converges slowest."""
    errs = []
    for nx in (128, 512):
        w = W.sod(nx)
        u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], t_end=0.2, cfl=0.3,
                                 recon=recon)
        assert fl == 0
        x = (np.arange(nx) + 0.5) / nx
        rho_e, _, _ = exact_riemann_profile(x, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1), 1.4)
        errs.append(np.mean(np.abs(u[0, 0, 0] - rho_e)))
    assert np.log2(errs[0] / errs[1]) / 2 >= order, errs


def test_ppmp_flattening_takes_the_upstream_neighbour():
    """Pressure falling to the right (p_{i+1} < p_{i-1}): F_i = max(F~_i,
    F~_{i+1}).  Cell i sits in diverging flow (F~_i = 0) next to a one-cell
    compressive shock in cell i+1 (F~_{i+1} = 1), so cell i is flattened: at
    dt = 0 its face states are w_i."""
    p = np.array([10.0, 10.0, 10.0, 10.0, 1.0, 1.0, 1.0])
    u = np.array([0.0, 0.0, 0.0, 1.0, 0.5, 0.0, 0.0])
    st = stencil(np.array([1.0, 1.1, 1.2, 1.3, 1.5, 1.6, 1.7]), u, 0.0, 0.0, p)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PPMP, st[None], 0.0, 1.0, G)
    np.testing.assert_allclose(UsL, cons(st[3:4]), rtol=1e-15)
    np.testing.assert_allclose(UsR, cons(st[3:4]), rtol=1e-15)


@pytest.mark.parametrize("side", ["left", "right"])
def test_ppmp_supersonic_acoustic_wave_corrections(side):
    """Linear acoustics in supersonic flow.  Background rho0, p0 and u0 with
    |u0| = 2 a0 (toward the face), plus a small linear perturbation along one
    acoustic eigenvector (the wave that is not the reference one: the right
    acoustic wave, p, at the left face; the left acoustic wave, m, at the right
    face).  Every characteristic reaches the face from inside the cell, so the
    exact state at the face at dt/2 is the background plus that wave's
    perturbation at the midpoint of its own domain of dependence.  The chi
    corrections must turn the reference state (the other acoustic wave's) into
    it: to the perturbation's second order, i.e. 1e-12 for an amplitude 1e-6."""
    rho0, p0 = 1.0, 1.0
    a0 = np.sqrt(G * p0 / rho0)
    C = rho0 * a0
    eps = 1e-6
    x = np.arange(7) - 3.0  # cell centres, dx = 1 (linear data: averages = centre values)
    dtdx = 0.1
    if side == "left":
        u0, sgn, lam = -2.0 * a0, +1.0, -2.0 * a0 + a0      # p-wave: du = dp/C
    else:
        u0, sgn, lam = 2.0 * a0, -1.0, 2.0 * a0 - a0        # m-wave: du = -dp/C
    dp = eps * p0 * x
    st = stencil(rho0 + dp / a0 ** 2, u0 + sgn * dp / C, 0.0, 0.0, p0 + dp)
    UsL, UsR = oracle.reconstruct(oracle.RECON_PPMP, st[None], dtdx, 1.0, G)
    xf = -0.5 if side == "left" else 0.5
    xm = xf - 0.5 * lam * dtdx  # midpoint of the wave's domain of dependence
    expect = stencil(rho0 + eps * p0 * xm / a0 ** 2, u0 + sgn * eps * p0 * xm / C, 0.0, 0.0,
                     p0 + eps * p0 * xm)[3:4]
    got = UsL if side == "left" else UsR
    np.testing.assert_allclose(got, cons(expect), rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# Planted mistakes in PLMP, PLMC and PPMP: each fails one of the pins above,
# re-run through a copy of the oracle with the mistake.

def _reconstruct_lib(L):
    """oracle.reconstruct through a given oracle library (a planted-mistake copy)."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_reconstruct.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp, dp]
    L.oracle_reconstruct.restype = ctypes.c_int

    def rec(recon, w, dtdx, dx, gamma):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 7, 5)
        UsL = np.zeros((w.shape[0], 5)); UsR = np.zeros((w.shape[0], 5))
        L.oracle_reconstruct(w.shape[0], int(recon), w.ctypes.data_as(dp), float(dtdx),
                             float(dx), float(gamma), UsL.ctypes.data_as(dp),
                             UsR.ctypes.data_as(dp))
        return UsL, UsR

    return rec


def _sod_contact_cells_lib(L, recon, nx=100):
    """_contact_cells through the oracle library L."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_init.restype = ctypes.c_void_p
    L.oracle_init.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.POINTER(ctypes.c_int)]
    L.oracle_free.argtypes = [ctypes.c_void_p]
    L.oracle_set_state.argtypes = [ctypes.c_void_p, dp]
    L.oracle_get_state.argtypes = [ctypes.c_void_p, dp]
    L.oracle_set_recon.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.oracle_compute_dt.restype = ctypes.c_double
    L.oracle_compute_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.oracle_step_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    w = W.sod(nx, left=(1.0, 0.0, 1.0), right=(0.1, 0.0, 0.1))
    u0 = np.ascontiguousarray(w["u"])
    h = L.oracle_init(nx, 1, 1, w["dx"], w["gamma"], (ctypes.c_int * 6)(*w["bc"]))
    assert h
    try:
        L.oracle_set_recon(h, int(recon))
        L.oracle_set_state(h, u0.ctypes.data_as(dp))
        t, steps = 0.0, 0
        while t < 0.2 and steps < 2000:
            dt = min(L.oracle_compute_dt(h, 0.3), 0.2 - t)
            if not dt > 0.0:
                return 99
            L.oracle_step_dt(h, dt)
            t += dt
            steps += 1
        u = np.zeros_like(u0)
        L.oracle_get_state(h, u.ctypes.data_as(dp))
    finally:
        L.oracle_free(h)
    x = (np.arange(nx) + 0.5) / nx
    rho_e, _, _ = exact_riemann_profile(x, 0.2, 0.5, (1, 0, 1), (0.1, 0, 0.1), 1.4)
    rl = rho_e[(x > 0.6) & (x < 0.66)].mean()
    rr = rho_e[(x > 0.75) & (x < 0.8)].mean()
    lo, hi = rr + 0.05 * (rl - rr), rr + 0.95 * (rl - rr)
    rho = u[0, 0, 0]
    return int(np.sum((x > 0.62) & (x < 0.8) & (rho > lo) & (rho < hi)))


def _recon_pin_violations(rec, contact_cells):
    """Each pin's largest error over its tolerance (1: at the tolerance): linear
    data (PPMP, PLMC, PLMP), PPMP's cubic, the advected quadratic (PPMP), the
    advected linear density (PLMC, PLMP) and PPMP's Sod contact width."""
    out = {}
    x = np.arange(7) - 3.0
    st = stencil(1.0 + 0.002 * x, 0.3 + 0.01 * x, 0.1 - 0.02 * x, 0.05 * x, 1.0 + 0.01 * x)
    wl = cons(stencil(1.0 - 0.001, 0.3 - 0.005, 0.1 + 0.01, -0.025, 1.0 - 0.005)[3:4])
    wr = cons(stencil(1.0 + 0.001, 0.3 + 0.005, 0.1 - 0.01, 0.025, 1.0 + 0.005)[3:4])
    err = 0.0
    for recon in (oracle.RECON_PPMP, oracle.RECON_PLMC, oracle.RECON_PLMP):
        UsL, UsR = rec(recon, st[None], 0.0, 1.0, G)
        err = max(err, np.max(np.abs(UsL - wl) / (np.abs(wl) + 1e-2)),
                  np.max(np.abs(UsR - wr) / (np.abs(wr) + 1e-2)))
    out["linear"] = err / 1e-13
    dx = 0.1
    cubics = [np.poly1d([0.002, 0.001, 0.004, 1.0]), np.poly1d([0.05, -0.02, 0.3, 0.2]),
              np.poly1d([-0.03, 0.01, 0.2, -0.1]), np.poly1d([0.02, 0.03, -0.1, 0.3]),
              np.poly1d([0.001, -0.002, 0.02, 1.0])]
    stc = np.stack([cell_averages(c, -3.5 * dx, dx) for c in cubics], axis=1)
    UsL, UsR = rec(oracle.RECON_PPMP, stc[None], 0.0, dx, G)
    cl = cons(np.array([[c(-0.5 * dx) for c in cubics]]))
    cr = cons(np.array([[c(0.5 * dx) for c in cubics]]))
    out["ppmp_cubic"] = max(np.max(np.abs(UsL / cl - 1)), np.max(np.abs(UsR / cr - 1))) / 1e-12
    dxq, u, p = 1.0, 0.4, 1.0
    q = np.poly1d([0.001, 0.004, 1.0])
    rho = cell_averages(q, -3.5 * dxq, dxq)
    UsL, UsR = rec(oracle.RECON_PPMP, stencil(rho, u, 0.0, 0.0, p)[None], 0.3, dxq, G)
    a = np.sqrt(G * p / rho[3])
    Q = np.polyint(q)
    sR, sL = u * 0.3, (a - u) * 0.3
    rhoR = (Q(0.5) - Q(0.5 - sR)) / sR
    rhoL = (Q(-0.5 + sL) - Q(-0.5)) / sL
    out["ppmp_quadratic"] = max(abs(UsR[0, 0] / rhoR - 1), abs(UsL[0, 0] / rhoL - 1)) / 1e-13
    s = 0.002
    stl = stencil(1.0 + s * x, u, 0.0, 0.0, p)
    a1 = np.sqrt(G * p)
    err = 0.0
    UsL, UsR = rec(oracle.RECON_PLMC, stl[None], 0.3, 1.0, G)
    err = max(err, abs(UsR[0, 0] - (1.0 + s * (0.5 - 0.5 * u * 0.3))),
              abs(UsL[0, 0] - (1.0 + s * (-0.5 + 0.5 * (a1 - u) * 0.3))))
    UsL, UsR = rec(oracle.RECON_PLMP, stl[None], 0.3, 1.0, G)
    err = max(err, abs(UsR[0, 0] - (1.0 + s * (0.5 - 0.5 * u * 0.3))),
              abs(UsL[0, 0] - (1.0 + s * (-0.5 - 0.5 * u * 0.3))))
    out["plm_linear_advection"] = err / 1e-14
    out["ppmp_sod_contact"] = contact_cells / 2.0
    out["ppmp_acoustic"] = max(_ppmp_acoustic_error(rec, side) for side in ("left", "right"))
    return out


def _ppmp_acoustic_error(rec, side):
    """test_ppmp_supersonic_acoustic_wave_corrections through the
    reconstruction rec: the largest error over its tolerance (rtol 1e-11,
    atol 1e-12)."""
    rho0, p0 = 1.0, 1.0
    a0 = np.sqrt(G * p0 / rho0)
    C = rho0 * a0
    eps = 1e-6
    x = np.arange(7) - 3.0
    dtdx = 0.1
    if side == "left":
        u0, sgn, lam = -2.0 * a0, +1.0, -2.0 * a0 + a0
    else:
        u0, sgn, lam = 2.0 * a0, -1.0, 2.0 * a0 - a0
    dp = eps * p0 * x
    st = stencil(rho0 + dp / a0 ** 2, u0 + sgn * dp / C, 0.0, 0.0, p0 + dp)
    UsL, UsR = rec(oracle.RECON_PPMP, st[None], dtdx, 1.0, G)
    xm = (-0.5 if side == "left" else 0.5) - 0.5 * lam * dtdx
    expect = cons(stencil(rho0 + eps * p0 * xm / a0 ** 2, u0 + sgn * eps * p0 * xm / C, 0.0, 0.0,
                          p0 + eps * p0 * xm)[3:4])
    got = UsL if side == "left" else UsR
    return float(np.max(np.abs(got - expect) / (1e-12 + 1e-11 * np.abs(expect))))


_PLMP = "void plmp_cell("
_PLMC = "void plmc_cell("
_PPMP = "void ppmp_cell("
_RECON_MUTANTS = {
    # PLMP's half-step flux evolution with the wrong sign
    "plmp_evolution_sign": [(_PLMP, "UsL[q] = UL[q] + h * (FL[q] - FR[q]);",
                             "UsL[q] = UL[q] - h * (FL[q] - FR[q]);")],
    # PLMP's left boundary value a whole slope from the average
    "plmp_full_slope": [(_PLMP, "WL[q] = w[1][q] - R(0.5) * dw[q];", "WL[q] = w[1][q] - dw[q];")],
    # PLMC's contact correction with the acoustic speed difference
    "plmc_contact_speed": [(_PLMC, "sR[0] = sR[0] + (lp - l0) * (dw[0] - dw[4] / a2);",
                            "sR[0] = sR[0] + (lp - lm) * (dw[0] - dw[4] / a2);")],
    # PLMC's trace of the right face with the wrong sign
    "plmc_trace_sign": [(_PLMC, "WsR[q] = (WR[q] - R(0.5) * bp * dw[q]) + h * sR[q];",
                         "WsR[q] = (WR[q] + R(0.5) * bp * dw[q]) + h * sR[q];")],
    # PPMP's interpolation with a third of the slope difference
    "ppmp_face_third": [(_PPMP, "WL[q] = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(6.0);",
                         "WL[q] = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(3.0);")],
    # PPMP's contact test as printed (same concavity; reading N1)
    "ppmp_contact_printed": [(_PPMP, "d2m * d2p < R(0.0)) {", "d2m * d2p > R(0.0)) {")],
    # PPMP's chi^p_L as printed (reading N4)
    "chi_p_printed": [(_PPMP, "((WLm[1] - WLp[1]) + (WLm[4] - WLp[4]) / CL)",
                       "((WLm[1] - WLp[1]) - (WLm[4] + WLp[4]) / CL)")],
    # PPMP's right-face velocity correction with the wrong sign
    "chi_m_velocity": [(_PPMP, "WsR[1] = WRp[1] - CR * chiRm;", "WsR[1] = WRp[1] + CR * chiRm;")],
    # the primitive MC limiter without its factor 2
    "mc_prim_factor": [("void plm_prim_slope(",
                        "dw[q] = sgn(dC) * mn(mn(fabs(dC), R(2.0) * fabs(dL)), R(2.0) * fabs(dR));",
                        "dw[q] = sgn(dC) * mn(mn(fabs(dC), fabs(dL)), fabs(dR));")],
}


def test_recon_pins_catch_planted_mistakes():
    """Each plausible slip in PLMP, PLMC or PPMP (a sign, a factor, the wrong
    wave speed, the printed contact test and chi^p_L, the limiter's factor 2),
    planted in a copy of the oracle source, fails one of the pins (linear data,
    PPMP's cubic, the advected quadratic and linear profiles, PPMP's two-zone
    Sod contact, PPMP's supersonic acoustic corrections); the oracle as it is
    passes them all."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_RECON_MUTANTS)) as ex:
        libs = dict(zip(_RECON_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                 _RECON_MUTANTS.items())))
    for tag, L in libs.items():
        with np.errstate(all="ignore"):
            v = _recon_pin_violations(_reconstruct_lib(L),
                                      _sod_contact_cells_lib(L, oracle.RECON_PPMP))
        assert max(v.values()) > 1.4 or not np.all(np.isfinite(list(v.values()))), (
            "planted mistake %r passes the reconstruction pins: %s" % (tag, v))
        print("%s: %s" % (tag, {k: "%.3g" % x for k, x in v.items()}))
    base = _recon_pin_violations(oracle.reconstruct, _contact_cells(oracle.RECON_PPMP))
    assert max(base.values()) <= 1.0, base

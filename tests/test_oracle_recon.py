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

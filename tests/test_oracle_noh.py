"""Noh's strong shock (Sec. 4.3.1) in the oracle: the analytic boundary, the
closed-form solution, and the HLLE limit the reflecting walls of the test reach.

Closed forms for gamma = 5/3 (Noh 1987): gas at rest-frame speed V = 1 streaming
toward the origin through n dimensions keeps density rho0 (1 + t/r)^(n-1) ahead
of the reflected shock, which moves out at (gamma-1)/2 V = 1/3; behind it the
gas is at rest at density rho0 ((gamma+1)/(gamma-1))^n = 4^n (16 in 2D, 64 in
3D).  The wall-heating dip at the origin (Sec. 4.3.1) is excluded from the
post-shock comparison."""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import workloads as W

G53 = 5.0 / 3.0
NOH = (1.0, 1.0, 0.0, 0.0, 1e-6)  # rho0, V, -, -, p0


def noh_case(n, nd):
    w = W.noh(n, nd)
    return w["u"], w["dx"], w["bc"], w["inflow"], w["r"]


def test_noh_ghosts_hold_the_analytic_state():
    """Ghosts of a Noh face hold the analytic state at their own centre and the
    grid's time; where a Noh face meets a reflective one the x, y, z passes give
    the Noh state at the mirrored position with the mirrored momentum negated."""
    n, t = 12, 0.3
    u0, dx, bc, inflow, r = noh_case(n, 2)
    g = oracle.Grid(n, n, 1, dx, G53, bc)
    for f, p in inflow.items():
        g.set_inflow(f, p)
    g.set_state(u0)
    g.set_time(t)
    assert g.get_time() == t
    N = n + 8
    up = np.zeros((5, 1, N, N))
    oracle.lib().oracle_fill_ghosts(g.h, oracle._ptr(up))
    U = up[:, 0]

    def noh_state(xx, yy):
        rr = np.hypot(xx, yy)
        rho = 1.0 + t / rr
        return np.array([rho, -rho * xx / rr, -rho * yy / rr, 0.0, 1e-6 / (G53 - 1) + 0.5 * rho])

    pos = lambda i: (i - 4 + 0.5) * dx  # padded index -> cell centre
    # x+ ghosts on real rows
    for i in range(n + 4, N):
        for j in (4, 9):
            np.testing.assert_allclose(U[:, j, i], noh_state(pos(i), pos(j)), rtol=1e-15, atol=0)
    # corner x+ Noh / y- reflect: Noh at the mirrored y, y momentum negated
    i, j = n + 5, 2
    jm = 4 + (4 - j) - 1
    expect = noh_state(pos(i), pos(jm)) * np.array([1, 1, -1, 1, 1])
    np.testing.assert_allclose(U[:, j, i], expect, rtol=1e-15, atol=0)
    # corner x+ / y+ (both Noh): the y pass evaluates at the cell's own centre
    i, j = n + 6, n + 5
    np.testing.assert_allclose(U[:, j, i], noh_state(pos(i), pos(j)), rtol=1e-15, atol=0)


def test_time_advances_by_each_step():
    u0, dx, bc, inflow, r = noh_case(16, 2)
    g = oracle.Grid(16, 16, 1, dx, G53, bc)
    for f, p in inflow.items():
        g.set_inflow(f, p)
    g.set_state(u0)
    total = 0.0
    for _ in range(3):
        dt, fl = g.step(0.3)
        assert fl == 0
        total += dt
    assert g.get_time() == total


def shock_radius_on_diagonal(d, nd, n, dx):
    diag = d[tuple([np.arange(n)] * nd)] if nd == 3 else d[0][np.arange(n), np.arange(n)]
    rd = (np.arange(n) + 0.5) * dx * np.sqrt(nd)
    mid = 0.5 * (4.0 ** nd + 4.0 ** (nd - 1))  # between post-shock and pre-shock at r_s
    return rd[np.argmax(diag < mid)]


@pytest.mark.parametrize("nd,n,t_end,recon", [(3, 40, 0.75, oracle.RECON_PPMC),
                                              (2, 64, 0.6, oracle.RECON_PLMP)],
                         ids=["3d_ppmc", "2d_plmp"])
def test_noh_matches_the_closed_form(nd, n, t_end, recon):
    u0, dx, bc, inflow, r = noh_case(n, nd)
    u, t, ns, fl = oracle.run(u0, dx, G53, bc, t_end=t_end, cfl=0.3, inflow=inflow, recon=recon)
    assert fl == 0 and t == pytest.approx(t_end, abs=1e-15)
    d = u[0]
    rs = t_end / 3.0
    post = d[(r > 0.3 * rs) & (r < 0.8 * rs)]
    ahead = (r > 1.3 * rs) & (r < 0.7)
    pre_exact = (1.0 + t_end / r) ** (nd - 1)
    # the resolution of the runs puts the post-shock mean 3-7% below 4^n
    assert abs(post.mean() / 4.0 ** nd - 1) < (0.10 if nd == 3 else 0.05), post.mean()
    assert np.abs(d[ahead] / pre_exact[ahead] - 1).max() < (0.03 if nd == 3 else 0.01)
    assert abs(shock_radius_on_diagonal(d, nd, n, dx) - rs) <= 1.5 * dx * np.sqrt(nd)


def test_hlle_with_zero_bounds_is_the_wall_flux():
    """Mirrored states of cold gas hitting a reflecting wall (taken from a 2D
    Noh step): negative internal energy, so the Roe average has no real sound
    speed, u~ = 0, and both HLLE bounds are 0.  The flux is the symmetric limit
    (F_L + F_R)/2: no mass or energy through the wall, the momentum flux
    rho u^2 + p_floor, the transverse momentum flux 0."""
    UL = np.array([[1.120682244649055, 0.014366113259713032, -1.0710651635732049, 0.0,
                    0.50367101371388745]])
    UR = UL * np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    F = oracle.riemann_roe(UL, UR, G53)
    rho, m = UL[0, 0], UL[0, 1]
    assert np.all(np.isfinite(F))
    np.testing.assert_allclose(F[0], [0.0, m * m / rho + 1e-20, 0.0, 0.0, 0.0], rtol=1e-15,
                               atol=1e-18)

"""Pins of the oracle's Roe solver, its HLLE fallback and the H correction
(Sec. 2.2.2, App. B.2, App. C), on single interfaces and through whole CTU
steps.  Expected values come from properties of the linearisation (Roe's exact
resolution of an isolated discontinuity), symmetry, limits of the method (the
H correction at large eta is the local Lax-Friedrichs flux) or the paper's
reported behaviour (the 123 problem runs with the fallback)."""
import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import workloads as W
from tests.test_oracle_ctu import exact_riemann_profile, mirror_x, rotate_xyz

P, R_, O = 0, 1, 2


def cons1(w, g):
    w = np.asarray(w, dtype=np.float64).reshape(-1, 5)
    return W.prim_to_cons(w[:, 0], w[:, 1], w[:, 2], w[:, 3], w[:, 4], g).reshape(5, -1).T


def flux1(w, g):
    w = np.asarray(w, dtype=np.float64).reshape(-1, 5)
    rho, u, v, ww, p = w.T
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v + ww * ww)
    return np.column_stack([rho * u, rho * u * u + p, rho * u * v, rho * u * ww, (E + p) * u])


def shock_pair(mach, s, g, rho1=1.0, p1=1.0, v=0.3, w=-0.2):
    """States on both sides of a shock moving with speed s into gas (right state)
    at rest in the shock frame plus s: Rankine-Hugoniot in the shock frame."""
    a1 = np.sqrt(g * p1 / rho1)
    u1s = -mach * a1  # pre-shock gas flows into the shock (shock frame)
    m2 = mach * mach
    rho2 = rho1 * (g + 1) * m2 / ((g - 1) * m2 + 2)
    p2 = p1 * (2 * g * m2 - (g - 1)) / (g + 1)
    u2s = u1s * rho1 / rho2
    left = [rho2, u2s + s, v, w, p2]   # post-shock (behind a right-moving shock)
    right = [rho1, u1s + s, v, w, p1]
    return np.array(left), np.array(right)


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_identical_states_give_the_physical_flux(g):
    rng = np.random.default_rng(3)
    WL, _ = W.random_states(200, seed=4, gamma=g)
    U = cons1(WL, g)
    F = oracle.riemann_roe(U, U, g)
    np.testing.assert_allclose(F, flux1(WL, g), rtol=1e-13, atol=1e-13)


def test_supersonic_gives_the_upwind_flux():
    """lambda^m >= 0: the left state's flux; lambda^p <= 0: the right state's."""
    g = 1.4
    WL = np.array([[1.0, 3.5, 0.1, 0.2, 1.0]])
    WR = np.array([[0.5, 3.0, -0.1, 0.0, 0.7]])
    F = oracle.riemann_roe(cons1(WL, g), cons1(WR, g), g)
    np.testing.assert_allclose(F, flux1(WL, g), rtol=1e-14, atol=1e-14)
    flip = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    F = oracle.riemann_roe(cons1(WR * flip, g), cons1(WL * flip, g), g)
    np.testing.assert_allclose(F, flux1(WL * flip, g), rtol=1e-14, atol=1e-14)


def cons_to_prim(U, g):
    rho = U[:, 0]
    u, v, w = U[:, 1] / rho, U[:, 2] / rho, U[:, 3] / rho
    p = (g - 1) * (U[:, 4] - 0.5 * rho * (u * u + v * v + w * w))
    return np.column_stack([rho, u, v, w, p])


@pytest.mark.parametrize("mach,s", [(1.5, 0.4), (3.0, -0.3), (2.0, 0.05)])
def test_isolated_shock_is_resolved_exactly(mach, s):
    """Roe's linearisation has U_R - U_L as an eigenvector for a pair joined by a
    single shock (Rankine-Hugoniot), with the shock speed as eigenvalue, so the
    Roe flux is the upwind flux of the shock: F_L for s > 0, F_R for s < 0."""
    g = 1.4
    WL, WR = shock_pair(mach, s, g)
    UL, UR = cons1(WL, g), cons1(WR, g)
    F = oracle.riemann_roe(UL, UR, g)
    expect = flux1(WL, g) if s > 0 else flux1(WR, g)
    np.testing.assert_allclose(F, expect, rtol=1e-12, atol=1e-12)
    # and the states really are joined by a shock moving at s
    np.testing.assert_allclose(flux1(WR, g) - flux1(WL, g), s * (UR - UL), rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("u", [0.4, -0.25])
def test_isolated_contact_is_resolved_exactly(u):
    g = 5.0 / 3.0
    WL = np.array([[2.0, u, 0.3, -0.1, 1.0]])
    WR = np.array([[0.5, u, -0.2, 0.4, 1.0]])
    F = oracle.riemann_roe(cons1(WL, g), cons1(WR, g), g)
    expect = flux1(WL, g) if u > 0 else flux1(WR, g)
    np.testing.assert_allclose(F, expect, rtol=1e-12, atol=1e-12)


def test_large_h_correction_gives_the_local_lax_friedrichs_flux():
    """With eta^H above every |lambda| all coefficients use eta^H, the sum of the
    waves is eta^H (U_R - U_L), and the flux is 1/2 (F_L + F_R) - eta^H/2 (U_R - U_L)."""
    g = 1.4
    # moderate contrasts keep the Roe intermediate states positive (no fallback)
    WL, WR = W.random_states(100, seed=9, gamma=g, rho_range=(0.5, 2.0), p_range=(0.5, 2.0),
                             vmax=0.5)
    aL = np.sqrt(g * WL[:, 4] / WL[:, 0])
    aR = np.sqrt(g * WR[:, 4] / WR[:, 0])
    UL, UR = cons1(WL, g), cons1(WR, g)
    eta = 50.0 * np.ones(len(UL))
    F = oracle.riemann_roe(UL, UR, g, eta)
    expect = 0.5 * (flux1(WL, g) + flux1(WR, g)) - 0.5 * eta[:, None] * (UR - UL)
    # supersonic pairs return the upwind flux before the coefficients are formed
    sub = np.abs(0.5 * (WL[:, 1] + WR[:, 1])) < 0.5 * np.minimum(aL, aR)
    assert sub.sum() > 10
    np.testing.assert_allclose(F[sub], expect[sub], rtol=1e-11, atol=1e-11)


def test_123_problem_interface_takes_the_hlle_flux():
    """The 123 states (rho = 1, p = 0.4, u = -2 | +2, Sec. 4.1.3) give a negative
    intermediate Roe density (rho_L + xi_0 = 1 - 2/a~ < 0), so the fallback
    applies.  For mirror-symmetric states the HLLE bounds are -b, +b with
    b = |u| + a (a = sqrt(gamma p / rho)), and its flux reduces to the local
    Lax-Friedrichs flux 1/2 (F_L + F_R) - b/2 (U_R - U_L): (0, 4.4 - 2 b, 0, 0, 0).
    The Roe flux would have a momentum flux of 4.4 - 2 a~ with a~ = sqrt(1.36)."""
    g = 1.4
    WL = np.array([[1.0, -2.0, 0.0, 0.0, 0.4]])
    WR = np.array([[1.0, 2.0, 0.0, 0.0, 0.4]])
    b = 2.0 + np.sqrt(g * 0.4)
    F = oracle.riemann_roe(cons1(WL, g), cons1(WR, g), g)
    np.testing.assert_allclose(F, [[0.0, 4.4 - 2.0 * b, 0.0, 0.0, 0.0]], rtol=1e-13,
                               atol=1e-14)


def test_123_problem_runs_with_the_roe_solver():
    """Sec. 4.1.3: with the fallback the 123 problem (128 cells, t = 0.15, PPMP)
    runs with the Roe solver; density and pressure stay positive and the
    solution is close to the exact one."""
    nx, g = 128, 1.4
    w = W.sod(nx, gamma=g, left=(1.0, -2.0, 0.4), right=(1.0, 2.0, 0.4))
    u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], t_end=0.15, cfl=0.3,
                             recon=oracle.RECON_PPMP, solver=oracle.SOLVER_ROE)
    assert fl == 0 and t == 0.15
    rho = u[0, 0, 0]
    p = (g - 1) * (u[4, 0, 0] - 0.5 * u[1, 0, 0] ** 2 / rho)
    assert rho.min() > 0 and p.min() > 0
    x = (np.arange(nx) + 0.5) / nx
    rho_e, _, _ = exact_riemann_profile(x, 0.15, 0.5, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4), g)
    assert np.mean(np.abs(rho - rho_e)) < 0.02


def test_sod_converges_with_the_roe_solver():
    errs = []
    for nx in (128, 512):
        w = W.sod(nx)
        u, t, n, fl = oracle.run(w["u"], w["dx"], w["gamma"], w["bc"], t_end=0.2, cfl=0.3,
                                 solver=oracle.SOLVER_ROE)
        assert fl == 0
        x = (np.arange(nx) + 0.5) / nx
        rho_e, _, _ = exact_riemann_profile(x, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1), 1.4)
        errs.append(np.mean(np.abs(u[0, 0, 0] - rho_e)))
    assert np.log2(errs[0] / errs[1]) / 2 >= 0.75, errs
    assert errs[1] < 1.5e-3


@pytest.mark.parametrize("recon", [oracle.RECON_PPMC, oracle.RECON_PLMP])
def test_roe_steps_conserve_and_keep_symmetries(recon):
    """Roe with the H correction (its nine-face stencil) through 3D steps: a
    uniform state is kept exactly, totals are conserved, and mirror and axis
    permutation symmetries hold (a one-sided stencil would break them)."""
    u0 = W.prim_to_cons(np.full((6, 7, 8), 1.3), 0.4, -0.3, 0.2, np.full((6, 7, 8), 0.9), 1.4)
    u, t, n, fl = oracle.run(u0, 0.1, 1.4, [P] * 6, nsteps=3, cfl=0.4, recon=recon,
                             solver=oracle.SOLVER_ROE)
    assert np.array_equal(u, u0)
    w = W.sedov(16)
    run = lambda x: oracle.run(x, w["dx"], w["gamma"], [P] * 6, nsteps=4, cfl=0.3, recon=recon,
                               solver=oracle.SOLVER_ROE)[0]
    u = run(w["u"])
    tot0, tot = w["u"].reshape(5, -1).sum(axis=1), u.reshape(5, -1).sum(axis=1)
    scale = np.abs(w["u"]).reshape(5, -1).sum(axis=1) + np.abs(u).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale)
    sc = np.abs(u).max()
    np.testing.assert_allclose(run(mirror_x(w["u"])), mirror_x(u), rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(run(rotate_xyz(w["u"])), rotate_xyz(u), rtol=0, atol=1e-12 * sc)


# ---------------------------------------------------------------------------
# Planted mistakes in the Roe solver, the HLLE fallback and the H-correction
# quantity: each fails one of the pins above, re-run through a copy of the
# oracle with the mistake.

def _roe_lib(L):
    """oracle.riemann_roe through a given oracle library (a planted-mistake copy)."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_riemann_roe.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
    L.oracle_riemann_roe.restype = ctypes.c_int

    def roe(UL, UR, gamma, etaH=None):
        UL = np.ascontiguousarray(UL, dtype=np.float64).reshape(-1, 5)
        UR = np.ascontiguousarray(UR, dtype=np.float64).reshape(-1, 5)
        F = np.zeros((UL.shape[0], 5))
        e = None if etaH is None else np.ascontiguousarray(etaH, dtype=np.float64).reshape(-1)
        L.oracle_riemann_roe(UL.shape[0], UL.ctypes.data_as(dp), UR.ctypes.data_as(dp),
                             None if e is None else e.ctypes.data_as(dp), float(gamma),
                             F.ctypes.data_as(dp))
        return F

    return roe


def _roe_pin_violations(roe):
    """Each pin's largest error over its tolerance (1: at the tolerance): the
    isolated shocks and contacts, the large-H local Lax-Friedrichs flux and the
    123 interface's HLLE flux."""
    out = {}
    g = 1.4
    err = 0.0
    for mach, s in ((1.5, 0.4), (3.0, -0.3), (2.0, 0.05)):
        WL, WR = shock_pair(mach, s, g)
        F = roe(cons1(WL, g), cons1(WR, g), g)
        expect = flux1(WL, g) if s > 0 else flux1(WR, g)
        err = max(err, np.max(np.abs(F - expect) / (1.0 + np.abs(expect))))
    out["shock"] = err / 1e-12
    err = 0.0
    for u in (0.4, -0.25):
        gc = 5.0 / 3.0
        WL = np.array([[2.0, u, 0.3, -0.1, 1.0]])
        WR = np.array([[0.5, u, -0.2, 0.4, 1.0]])
        F = roe(cons1(WL, gc), cons1(WR, gc), gc)
        expect = flux1(WL, gc) if u > 0 else flux1(WR, gc)
        err = max(err, np.max(np.abs(F - expect) / (1.0 + np.abs(expect))))
    out["contact"] = err / 1e-12
    WL, WR = W.random_states(100, seed=9, gamma=g, rho_range=(0.5, 2.0), p_range=(0.5, 2.0),
                             vmax=0.5)
    aL = np.sqrt(g * WL[:, 4] / WL[:, 0])
    aR = np.sqrt(g * WR[:, 4] / WR[:, 0])
    UL, UR = cons1(WL, g), cons1(WR, g)
    eta = 50.0 * np.ones(len(UL))
    F = roe(UL, UR, g, eta)
    expect = 0.5 * (flux1(WL, g) + flux1(WR, g)) - 0.5 * eta[:, None] * (UR - UL)
    sub = np.abs(0.5 * (WL[:, 1] + WR[:, 1])) < 0.5 * np.minimum(aL, aR)
    out["llf"] = np.max(np.abs(F[sub] - expect[sub]) / (1.0 + np.abs(expect[sub]))) / 1e-11
    WL = np.array([[1.0, -2.0, 0.0, 0.0, 0.4]])
    WR = np.array([[1.0, 2.0, 0.0, 0.0, 0.4]])
    b = 2.0 + np.sqrt(g * 0.4)
    F = roe(cons1(WL, g), cons1(WR, g), g)
    out["hlle_123"] = np.max(np.abs(F - [[0.0, 4.4 - 2.0 * b, 0.0, 0.0, 0.0]])) / 1e-13
    return out


_ROE_H = "int riemann_roe_cons("
_HLLE_H = "void roe_hlle_flux("
_ROE_MUTANTS = {
    # the Roe velocity as the plain average instead of the sqrt(rho)-weighted one
    "plain_average": [(_ROE_H, "const R u = (sL * WL[1] + sR * WR[1]) / (sL + sR);",
                       "const R u = R(0.5) * (WL[1] + WR[1]);")],
    # the enthalpy average with the weights swapped
    "enthalpy_weights": [(_ROE_H, "const R H = (sL * HL + sR * HR) / (sL + sR);",
                          "const R H = (sR * HL + sL * HR) / (sL + sR);")],
    # the u - a wave strength with the sign of its u a term flipped
    "xi0_sign": [(_ROE_H, "dU[0] * Na * (R(0.5) * gp * V2 + u * a)",
                  "dU[0] * Na * (R(0.5) * gp * V2 - u * a)")],
    # the energy component of the u + a eigenvector with H - u a
    "eigvec_energy": [(_ROE_H, "C4 * (H + u * a);", "C4 * (H - u * a);")],
    # the H correction not applied to the u + a family
    "h_corr_missing": [(_ROE_H, "alp = mx(fabs(lp), etaH);", "alp = fabs(lp);")],
    # the HLLE bounds taken without the data states' wave speeds
    "hlle_bounds": [(_HLLE_H, "const R bm = mn(mn(lm, WL[1] - aL), R(0.0));",
                     "const R bm = mn(lm, R(0.0));"),
                    (_HLLE_H, "const R bp = mx(mx(lp, WR[1] + aR), R(0.0));",
                     "const R bp = mx(lp, R(0.0));")],
    # the fallback test on the intermediate state dropped
    "no_fallback": [(_ROE_H, "if (fail) roe_hlle_flux(UL, UR, WL, WR, FL, FR, lm, lp, g, F);", "")],
}


def test_roe_pins_catch_planted_mistakes():
    """Each plausible slip in the Roe averages, the wave strengths, an
    eigenvector, the H correction, the HLLE bounds or the fallback test,
    planted in a copy of the oracle source, fails one of the pins (isolated
    shock and contact, large-H Lax-Friedrichs flux, the 123 interface) by far
    more than its tolerance; the oracle as it is passes them all."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_ROE_MUTANTS)) as ex:
        libs = dict(zip(_ROE_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                               _ROE_MUTANTS.items())))
    for tag, L in libs.items():
        with np.errstate(all="ignore"):
            v = _roe_pin_violations(_roe_lib(L))
        assert max(v.values()) > 10.0 or not np.all(np.isfinite(list(v.values()))), (
            "planted mistake %r passes the Roe pins: %s" % (tag, v))
        print("%s: %s" % (tag, {k: "%.3g" % x for k, x in v.items()}))
    base = _roe_pin_violations(oracle.riemann_roe)
    assert max(base.values()) <= 1.0, base


def _roe_steps_lib(L, u0, dx, gamma, nsteps, cfl, recon):
    """oracle.run with the Roe solver through the oracle library L."""
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_init.restype = ctypes.c_void_p
    L.oracle_init.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.POINTER(ctypes.c_int)]
    L.oracle_free.argtypes = [ctypes.c_void_p]
    L.oracle_set_state.argtypes = [ctypes.c_void_p, dp]
    L.oracle_get_state.argtypes = [ctypes.c_void_p, dp]
    L.oracle_set_recon.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.oracle_set_solver.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.oracle_compute_dt.restype = ctypes.c_double
    L.oracle_compute_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.oracle_step_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
    u0 = np.ascontiguousarray(u0)
    _, nz, ny, nx = u0.shape
    h = L.oracle_init(nx, ny, nz, dx, gamma, (ctypes.c_int * 6)(*([P] * 6)))
    assert h
    try:
        L.oracle_set_recon(h, int(recon))
        L.oracle_set_solver(h, int(oracle.SOLVER_ROE))
        L.oracle_set_state(h, u0.ctypes.data_as(dp))
        for _ in range(nsteps):
            L.oracle_step_dt(h, L.oracle_compute_dt(h, cfl))
        u = np.zeros_like(u0)
        L.oracle_get_state(h, u.ctypes.data_as(dp))
    finally:
        L.oracle_free(h)
    return u


def test_h_correction_reading_is_needed_for_mirror_symmetry():
    """Reading N10 (App. C): the H-correction quantity takes the largest jump of
    both acoustic speeds, max(|d(u + a)|, |d(u - a)|)/2.  A copy of the oracle
    with the printed single term |d(u + a)|/2 breaks the mirror symmetry of Roe
    steps on the Sedov blast (a mirrored flow gets different dissipation), which
    the oracle as it is keeps to rounding."""
    from tests.helpers import build_oracle_mutant
    L = build_oracle_mutant("eta_printed", [(
        "R h_eta(",
        "return R(0.5) * mx(fabs((WR[1] + aR) - (WL[1] + aL)), fabs((WR[1] - aR) - (WL[1] - aL)));",
        "return R(0.5) * fabs((WR[1] + aR) - (WL[1] + aL));")])
    w = W.sedov(16)

    def mirror_error(run):
        u = run(w["u"])
        return np.max(np.abs(run(mirror_x(w["u"])) - mirror_x(u))) / (1e-12 * np.abs(u).max())

    bad = mirror_error(lambda x: _roe_steps_lib(L, x, w["dx"], w["gamma"], 4, 0.3,
                                                oracle.RECON_PPMC))
    good = mirror_error(lambda x: oracle.run(x, w["dx"], w["gamma"], [P] * 6, nsteps=4, cfl=0.3,
                                             recon=oracle.RECON_PPMC,
                                             solver=oracle.SOLVER_ROE)[0])
    assert good <= 1.0, good
    assert bad > 10.0, bad
    print("mirror error over tolerance: printed eta %.3g, reading %.3g" % (bad, good))

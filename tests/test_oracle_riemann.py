"""Pins of the oracle's exact Riemann solver (App. B.1, after Toro ch. 4).

Each test fixes the oracle against something other than itself:
  * Toro's tabulated exact star states (tests/golden), to the printed digits;
  * the Rankine-Hugoniot jump conditions across a shock and the Riemann
    invariant plus isentrope across a rarefaction, which the exact solution must
    satisfy for any data (these are physics, not the solver's formulas);
  * closed-form special cases: identical states give the physical flux,
    supersonic data give the upwind flux exactly, mirror data mirror the flux;
  * the waves' interiors and positions: inside a rarefaction fan the state is
    the centred simple wave (characteristic through the origin, Riemann
    invariant, isentrope), and a shock sits where the Rankine-Hugoniot mass
    flux puts it;
and copies of the oracle with planted mistakes fail these pins.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1410_4194_gb300 import workloads
from tests.helpers import half_ulp_of_printed, read_golden

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_star_states.txt")


def physical_flux(W, gamma):
    """Euler flux in the normal direction of a primitive state (Eq. x_flux)."""
    rho, u, v, w, p = W.T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.column_stack([rho * u, rho * u * u + p, rho * u * v, rho * u * w, (E + p) * u])


def sample(WL, WR, gamma, S):
    """Exact solution at x/t = S via the oracle's x/t = 0 sampler and a Galilean shift."""
    WL = np.array(WL, dtype=float).reshape(-1, 5).copy()
    WR = np.array(WR, dtype=float).reshape(-1, 5).copy()
    S = np.broadcast_to(np.asarray(S, dtype=float), (WL.shape[0],))
    WL[:, 1] -= S
    WR[:, 1] -= S
    r = oracle.riemann_prim(WL, WR, gamma)
    ws = r["ws"].copy()
    ws[:, 1] += S
    return ws, r["pm"], r["um"] + S


@pytest.mark.parametrize("row", read_golden(GOLDEN), ids=lambda r: "toro%s" % r[0])
def test_toro_star_states(row):
    vals = [float(x) for x in row[1:11]]
    rl, ul, pl, rr, ur, pr = vals[:6]

    def close(got, printed):
        if row[11] == "print":
            return abs(got - float(printed)) <= half_ulp_of_printed(printed) * 1.0001
        return abs(got - float(printed)) <= float(row[11]) * abs(float(printed))

    WL = np.array([[rl, ul, 0.0, 0.0, pl]])
    WR = np.array([[rr, ur, 0.0, 0.0, pr]])
    r = oracle.riemann_prim(WL, WR, 1.4)
    assert r["flags"] == 0
    pm, um = r["pm"][0], r["um"][0]
    assert close(pm, row[7])
    assert close(um, row[8])
    # star densities on each side of the contact
    eps = 1e-9 * max(1.0, abs(um))
    wl, _, _ = sample(WL, WR, 1.4, um - eps)
    wr, _, _ = sample(WL, WR, 1.4, um + eps)
    assert close(wl[0, 0], row[9])
    assert close(wr[0, 0], row[10])


def test_paper_sod_variant():
    """Sod with rho_R = 0.1 as the paper runs it (Sec. 4.1.1): its star state
    equals the one obtained by bisection on the Rankine-Hugoniot/rarefaction
    relations below (self-consistency through independent physics)."""
    WL = np.array([[1.0, 0.0, 0.0, 0.0, 1.0]])
    WR = np.array([[0.1, 0.0, 0.0, 0.0, 0.1]])
    r = oracle.riemann_prim(WL, WR, 1.4)
    _check_jump_relations(WL, WR, 1.4)
    assert 0.25 < r["pm"][0] < 0.35


def _check_jump_relations(WL, WR, gamma, rtol=2e-6):
    """Jump conditions of the exact solution, side by side.

    Shock side (p* > p_k): with mass flux m = (p* - p_k)/(u_k - u*) the mass and
    momentum jumps give the post-shock density rho*_k = rho_k m / (m - rho_k (u_k - u*))
    written through the shock speed s = u_k - m/rho_k, and the energy jump
    (Hugoniot) must hold too.  Rarefaction side: the star state lies on the
    isentrope p/rho^gamma = const and on the Riemann invariant
    u +- 2a/(gamma-1) = const.
    """
    WL = np.asarray(WL, float).reshape(-1, 5)
    WR = np.asarray(WR, float).reshape(-1, 5)
    r = oracle.riemann_prim(WL, WR, gamma)
    pm, um = r["pm"], r["um"]
    eps = 1e-9 * np.maximum(1.0, np.abs(um))
    wl, _, _ = sample(WL, WR, gamma, um - eps)
    wr, _, _ = sample(WL, WR, gamma, um + eps)
    for side, W, ws, sgn in (("L", WL, wl, -1.0), ("R", WR, wr, +1.0)):
        rho, u, p = W[:, 0], W[:, 1], W[:, 4]
        rs = ws[:, 0]
        a = np.sqrt(gamma * p / rho)
        shock = pm > p
        # shock: Rankine-Hugoniot
        if shock.any():
            i = shock
            # mass flux through the shock (positive for flow crossing left to right)
            m = (pm[i] - p[i]) / (u[i] - um[i]) * (-sgn)
            m = np.abs(m)
            s = u[i] + sgn * m / rho[i]
            # mass conservation across the moving shock: rho (u - s) = rho* (u* - s)
            lhs = rho[i] * (u[i] - s)
            rhs = rs[i] * (um[i] - s)
            np.testing.assert_allclose(lhs, rhs, rtol=rtol, atol=1e-12)
            # energy: Hugoniot e* - e = (p* + p)/2 (1/rho - 1/rho*)
            e = p[i] / ((gamma - 1.0) * rho[i])
            es = pm[i] / ((gamma - 1.0) * rs[i])
            np.testing.assert_allclose(es - e, 0.5 * (pm[i] + p[i]) * (1.0 / rho[i] - 1.0 / rs[i]),
                                       rtol=rtol, atol=1e-12 * np.max(np.abs(es)))
        raref = ~shock
        if raref.any():
            i = raref
            # isentrope
            np.testing.assert_allclose(pm[i] / rs[i] ** gamma, p[i] / rho[i] ** gamma, rtol=rtol)
            # Riemann invariant: u + 2a/(gamma-1) (left fan) or u - 2a/(gamma-1)
            # (right fan) is carried through the fan
            as_ = np.sqrt(gamma * pm[i] / rs[i])
            np.testing.assert_allclose(um[i] - sgn * 2.0 * as_ / (gamma - 1.0),
                                       u[i] - sgn * 2.0 * a[i] / (gamma - 1.0),
                                       rtol=rtol, atol=rtol * np.max(a[i]))


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_random_states_satisfy_jump_relations(gamma):
    WL, WR = workloads.random_states(400, seed=11, gamma=gamma)
    keep = no_vacuum(WL, WR, gamma)
    assert keep.mean() > 0.8
    _check_jump_relations(WL[keep], WR[keep], gamma)


def test_identical_states_give_physical_flux():
    WL, _ = workloads.random_states(200, seed=3)
    r = oracle.riemann_prim(WL, WL, 1.4)
    F = physical_flux(WL, 1.4)
    scale = np.abs(F).max(axis=1, keepdims=True)
    np.testing.assert_allclose(r["F"], F, rtol=0, atol=1e-13 * scale.max())
    assert np.all(np.abs(r["F"] - F) <= 1e-13 * scale)


def test_supersonic_gives_upwind_flux_exactly():
    rng = np.random.Generator(np.random.PCG64(5))
    n = 200
    rho = np.exp(rng.uniform(-1, 1, (n, 2)))
    p = np.exp(rng.uniform(-1, 1, (n, 2)))
    a = np.sqrt(1.4 * p / rho)
    u = a.max(axis=1, keepdims=True) * rng.uniform(3.0, 6.0, (n, 1)) * np.ones((1, 2))
    WL = np.column_stack([rho[:, 0], u[:, 0], rng.normal(size=n), rng.normal(size=n), p[:, 0]])
    WR = np.column_stack([rho[:, 1], u[:, 1], rng.normal(size=n), rng.normal(size=n), p[:, 1]])
    r = oracle.riemann_prim(WL, WR, 1.4)
    assert np.array_equal(r["F"], physical_flux(WL, 1.4))
    # and leftward supersonic flow takes the right state
    WL2 = WL.copy(); WR2 = WR.copy()
    WL2[:, 1] *= -1; WR2[:, 1] *= -1
    r2 = oracle.riemann_prim(WL2, WR2, 1.4)
    assert np.array_equal(r2["F"], physical_flux(WR2, 1.4))


def no_vacuum(WL, WR, gamma):
    """Pairs that satisfy the pressure positivity condition (no vacuum is generated).

    The paper's solver has no vacuum branch, so such pairs have no defined answer.
    """
    aL = np.sqrt(gamma * WL[:, 4] / WL[:, 0])
    aR = np.sqrt(gamma * WR[:, 4] / WR[:, 0])
    return (WR[:, 1] - WL[:, 1]) < 0.9 * 2.0 * (aL + aR) / (gamma - 1.0)


def test_mirror_symmetry():
    WL, WR = workloads.random_states(300, seed=9)
    keep = no_vacuum(WL, WR, 1.4)
    WL, WR = WL[keep], WR[keep]
    r = oracle.riemann_prim(WL, WR, 1.4)
    mL = WR.copy(); mL[:, 1] *= -1
    mR = WL.copy(); mR[:, 1] *= -1
    m = oracle.riemann_prim(mL, mR, 1.4)
    sign = np.array([-1.0, 1.0, -1.0, -1.0, -1.0])
    scale = np.abs(r["F"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(m["F"] * sign - r["F"]) <= 1e-12 * scale)
    np.testing.assert_allclose(m["pm"], r["pm"], rtol=1e-12)


def test_newton_cap_and_floor_flags():
    # strong rarefaction into near vacuum: the floor keeps p* >= 1e-20, no NaN
    WL = np.array([[1.0, -20.0, 0.0, 0.0, 0.4]])
    WR = np.array([[1.0, 20.0, 0.0, 0.0, 0.4]])
    r = oracle.riemann_prim(WL, WR, 1.4)
    assert r["pm"][0] >= 1e-20
    assert np.all(np.isfinite(r["F"]))
    assert np.all(r["iters"] >= 1)


# ---------------------------------------------------------------------------
# The waves' interiors and positions.  The pins above fix the star states next
# to the contact; these fix what the sampling does elsewhere: inside a
# rarefaction fan (a centred simple wave: the characteristic through the
# origin, the Riemann invariant and the isentrope fix the state at each x/t)
# and across a shock (it sits where the Rankine-Hugoniot mass flux puts it).

def _riemann_lib(L):
    """oracle.riemann_prim through a given oracle library (a planted-mistake copy)."""
    import ctypes

    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.oracle_riemann_prim.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp, dp, ip]
    L.oracle_riemann_prim.restype = ctypes.c_int

    def rp(WL, WR, gamma):
        WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(-1, 5)
        WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(-1, 5)
        n = WL.shape[0]
        F = np.zeros((n, 5)); ws = np.zeros((n, 5))
        pm = np.zeros(n); um = np.zeros(n); it = np.zeros(n, dtype=np.int32)
        fl = L.oracle_riemann_prim(n, WL.ctypes.data_as(dp), WR.ctypes.data_as(dp), float(gamma),
                                   F.ctypes.data_as(dp), pm.ctypes.data_as(dp),
                                   um.ctypes.data_as(dp), ws.ctypes.data_as(dp),
                                   it.ctypes.data_as(ip))
        return dict(F=F, pm=pm, um=um, ws=ws, iters=it, flags=fl)

    return rp


def _sample_with(rp, WL, WR, gamma, S):
    """The exact solution at x/t = S (a Galilean shift of the x/t = 0 sampler)."""
    WL = np.array(WL, dtype=float).reshape(-1, 5).copy()
    WR = np.array(WR, dtype=float).reshape(-1, 5).copy()
    S = np.broadcast_to(np.asarray(S, dtype=float), (WL.shape[0],))
    WL[:, 1] -= S
    WR[:, 1] -= S
    r = rp(WL, WR, gamma)
    ws = r["ws"].copy()
    ws[:, 1] += S
    return ws


def _wave_pairs(gamma):
    WL, WR = workloads.random_states(600, seed=23, gamma=gamma)
    keep = no_vacuum(WL, WR, gamma)
    return WL[keep], WR[keep]


def _fan_error(rp, gamma):
    """Largest relative violation, over random pairs and points inside each
    rarefaction fan, of u -+ a = x/t, the Riemann invariant u +- 2a/(gamma-1) of
    the data side and its isentrope p/rho^gamma; and of the fan's edges: the
    data state just outside the head, the star state just inside the tail.
    The head and tail speeds come from the data and from p* (pinned above)."""
    WL, WR = _wave_pairs(gamma)
    r = oracle.riemann_prim(WL, WR, gamma)  # p*, u* of the pinned oracle
    pm, um = r["pm"], r["um"]
    worst = 0.0
    for sgn, W in ((-1.0, WL), (1.0, WR)):  # -1: left fan (u - a), +1: right fan (u + a)
        rho, u, p = W[:, 0], W[:, 1], W[:, 4]
        i = pm < p
        rho, u, p, pmi, umi = rho[i], u[i], p[i], pm[i], um[i]
        Wi = W[i]
        a = np.sqrt(gamma * p / rho)
        a_star = a * (pmi / p) ** ((gamma - 1.0) / (2.0 * gamma))
        head = u + sgn * a
        tail = umi + sgn * a_star
        inv = u - sgn * 2.0 * a / (gamma - 1.0)
        entropy = p / rho ** gamma
        WLi, WRi = WL[i], WR[i]
        scale = np.abs(u) + a
        for theta in (0.1, 0.37, 0.63, 0.9):
            S = head + theta * (tail - head)
            ws = _sample_with(rp, WLi, WRi, gamma, S)
            rs, us, ps = ws[:, 0], ws[:, 1], ws[:, 4]
            as_ = np.sqrt(gamma * np.maximum(ps, 0.0) / rs)
            worst = max(worst,
                        np.max(np.abs(us + sgn * as_ - S) / scale),
                        np.max(np.abs(us - sgn * 2.0 * as_ / (gamma - 1.0) - inv) / scale),
                        np.max(np.abs(ps / rs ** gamma / entropy - 1.0)))
        d = 1e-9 * scale
        outside = _sample_with(rp, WLi, WRi, gamma, head + sgn * d)
        worst = max(worst, np.max(np.abs(outside - Wi) / np.maximum(np.abs(Wi), 1.0)))
        inside = _sample_with(rp, WLi, WRi, gamma, tail - sgn * d)
        rho_star = rho * (pmi / p) ** (1.0 / gamma)
        worst = max(worst, np.max(np.abs(inside[:, 0] / rho_star - 1.0)),
                    np.max(np.abs(inside[:, 4] / pmi - 1.0)),
                    np.max(np.abs(inside[:, 1] - umi) / scale))
    return worst


def _shock_position_error(rp, gamma):
    """Largest relative violation of a shock's position: just outside the speed
    s = u_k -+ m/rho_k given by the Rankine-Hugoniot mass flux m = (p* -
    p_k)/|u_k - u*| the solution is the data state, just inside it is the
    post-shock state (density rho_k m / (m -+ rho_k (u* - u_k)), velocity u*,
    pressure p*)."""
    WL, WR = _wave_pairs(gamma)
    r = oracle.riemann_prim(WL, WR, gamma)
    pm, um = r["pm"], r["um"]
    worst = 0.0
    for sgn, W in ((-1.0, WL), (1.0, WR)):
        rho, u, p = W[:, 0], W[:, 1], W[:, 4]
        i = pm > p * (1.0 + 1e-6)
        rho, u, p, pmi, umi = rho[i], u[i], p[i], pm[i], um[i]
        Wi = W[i]
        m = (pmi - p) / np.abs(u - umi)
        s = u + sgn * m / rho
        rho_post = rho * (u - s) / (umi - s)
        a = np.sqrt(gamma * p / rho)
        scale = np.abs(u) + a
        d = 1e-9 * scale
        WLi, WRi = WL[i], WR[i]
        outside = _sample_with(rp, WLi, WRi, gamma, s + sgn * d)
        worst = max(worst, np.max(np.abs(outside - Wi) / np.maximum(np.abs(Wi), 1.0)))
        inside = _sample_with(rp, WLi, WRi, gamma, s - sgn * d)
        worst = max(worst, np.max(np.abs(inside[:, 0] / rho_post - 1.0)),
                    np.max(np.abs(inside[:, 4] / pmi - 1.0)),
                    np.max(np.abs(inside[:, 1] - umi) / scale))
    return worst


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_rarefaction_fans_are_centred_simple_waves(gamma):
    """Inside every rarefaction fan the sampled state lies on the characteristic
    through the origin (u - a = x/t on the left, u + a = x/t on the right), on the
    data side's Riemann invariant and on its isentrope; the fan's head leaves the
    data state and its tail the star state (to rounding)."""
    assert _fan_error(oracle.riemann_prim, gamma) < 1e-9


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_shocks_sit_where_the_mass_flux_puts_them(gamma):
    """Every shock separates the data state from the post-shock state exactly at
    the speed the Rankine-Hugoniot mass flux gives (to rounding)."""
    assert _shock_position_error(oracle.riemann_prim, gamma) < 1e-8


def _toro_violation(rp):
    """Largest error of p*, u* in Toro's tables 4.1-4.3 (tests 1-4, gamma 1.4),
    in units of half the last printed digit (1: agreement to the printed
    digits)."""
    worst = 0.0
    for row in read_golden(GOLDEN):
        if row[11] != "print":
            continue
        rl, ul, pl, rr, ur, pr = (float(x) for x in row[1:7])
        r = rp(np.array([[rl, ul, 0.0, 0.0, pl]]), np.array([[rr, ur, 0.0, 0.0, pr]]), 1.4)
        for got, printed in ((r["pm"][0], row[7]), (r["um"][0], row[8])):
            worst = max(worst, abs(got - float(printed)) / half_ulp_of_printed(printed))
    return worst


def _supersonic_violation(rp):
    rng = np.random.Generator(np.random.PCG64(5))
    n = 50
    rho = np.exp(rng.uniform(-1, 1, (n, 2)))
    p = np.exp(rng.uniform(-1, 1, (n, 2)))
    a = np.sqrt(1.4 * p / rho)
    u = a.max(axis=1, keepdims=True) * rng.uniform(3.0, 6.0, (n, 1)) * np.ones((1, 2))
    WL = np.column_stack([rho[:, 0], u[:, 0], rng.normal(size=n), rng.normal(size=n), p[:, 0]])
    WR = np.column_stack([rho[:, 1], u[:, 1], rng.normal(size=n), rng.normal(size=n), p[:, 1]])
    F = rp(WL, WR, 1.4)["F"]
    ref = physical_flux(WL, 1.4)
    return np.max(np.abs(F - ref) / np.maximum(np.abs(ref), 1.0))


_H_PF = "void pressure_function("
_H_RP = "void riemann_exact_prim("
_RIEMANN_MUTANTS = {
    # the shock branch of the pressure function with p - B_k for p + B_k
    "shock_B_sign": [(_H_PF, "sqrt(Ak / (p + Bk))", "sqrt(Ak / (p - Bk))")],
    # the rarefaction branch with exponent 1/gamma for (gamma-1)/(2 gamma)
    "raref_exponent": [(_H_PF, "pow(ratio, R(g.z))", "pow(ratio, R(g.inv_g))")],
    # u* with f_L - f_R for f_R - f_L
    "ustar_sign": [(_H_RP, "(uL + uR + fR - fL)", "(uL + uR + fL - fR)")],
    # A_k = 2/((gamma-1) rho_k) for 2/((gamma+1) rho_k)
    "A_gamma": [(_H_RP, "AL = R(2.0) / (R(g.gp1) * dL), AR = R(2.0) / (R(g.gp1) * dR)",
                 "AL = R(2.0) / (R(g.gm1) * dL), AR = R(2.0) / (R(g.gm1) * dR)")],
    # the left fan's sound speed with the sign of the velocity term flipped
    "fan_sign": [(_H_RP, "(aL + R(g.half_gm1) * uL)", "(aL - R(g.half_gm1) * uL)")],
    # the right fan's sound speed as printed, a_R + (gamma-1) u_R / 2 (reading R18)
    "right_fan_printed": [(_H_RP, "const R a = R(g.two_gp1) * (aR - R(g.half_gm1) * uR);",
                           "const R a = aR + R(g.half_gm1) * uR;")],
    # the left shock speed with the two coefficients of the square root swapped
    "shock_speed": [(_H_RP, "sqrt(R(g.sh_a) * pm / pL + R(g.sh_b))",
                     "sqrt(R(g.sh_b) * pm / pL + R(g.sh_a))")],
    # the star density of a left rarefaction with the exponent (gamma-1)/(2 gamma)
    "star_density": [(_H_RP, "d = dL * pow(pm / pL, R(g.inv_g))", "d = dL * pow(pm / pL, R(g.z))")],
    # the transverse velocities taken from the wrong side
    "transverse_side": [(_H_RP, "const R v = (u >= R(0.0)) ? WL[2] : WR[2];",
                         "const R v = (u >= R(0.0)) ? WR[2] : WL[2];")],
}


def test_riemann_pins_catch_planted_mistakes():
    """Each plausible slip in the exact solver, planted in a copy of the oracle
    source, fails at least one of its pins: Toro's star states, the jump
    relations at the contact, the fan and shock-position pins, the supersonic
    upwind flux.  The pins agree with the unchanged oracle (a few ulp)."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_RIEMANN_MUTANTS)) as ex:
        libs = dict(zip(_RIEMANN_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                   _RIEMANN_MUTANTS.items())))
    import oracle as oracle_mod
    def violations(rp):
        # each pin's error over its tolerance (1: at the tolerance)
        with np.errstate(all="ignore"):
            return {"toro": _toro_violation(rp) / 1.0001,
                    "fans": _fan_error(rp, 1.4) / 1e-9,
                    "shocks": _shock_position_error(rp, 1.4) / 1e-8,
                    "supersonic": _supersonic_violation(rp) / 1e-12}

    for tag, L in libs.items():
        v = violations(_riemann_lib(L))
        assert max(v.values()) > 10.0 or not np.all(np.isfinite(list(v.values()))), (
            "planted mistake %r passes the exact solver's pins: %s" % (tag, v))
        print("%s: %s" % (tag, {k: "%.3g" % x for k, x in v.items()}))
    base = violations(oracle_mod.riemann_prim)  # the oracle as it is passes them all
    assert max(base.values()) <= 1.0, base

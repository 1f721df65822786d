"""Pins of the oracle's exact Riemann solver (App. B.1, after Toro ch. 4).

Each test fixes the oracle against something other than itself:
  * Toro's tabulated exact star states (tests/golden), to the printed digits;
  * the Rankine-Hugoniot jump conditions across a shock and the Riemann
    invariant plus isentrope across a rarefaction, which the exact solution must
    satisfy for any data (these are physics, not the solver's formulas);
  * closed-form special cases: identical states give the physical flux,
    supersonic data give the upwind flux exactly, mirror data mirror the flux.
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

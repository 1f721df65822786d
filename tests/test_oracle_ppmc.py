"""Pins of the oracle's PPMC reconstruction (App. A.3; slopes from App. A.2).

Closed forms that fix it:
  * constant data are reproduced exactly for any dt;
  * for smooth monotone data (no limiter or monotonicity step active) the face
    values with dt = 0 equal the point values of the cubic whose cell averages
    are the data -- this holds only if the characteristic projection and
    back-projection compose to the identity and the parabola coefficients are
    the printed ones;
  * a quadratic density profile carried by a uniform subsonic flow: the state
    traced to the upwind face equals the exact average of that quadratic over
    the contact's domain of dependence (pins w6, the 2/3 factors and the
    contact correction);
  * mirror data give mirrored face states;
  * a small-amplitude acoustic simple wave carried by a supersonic flow: the
    state traced to the downwind face equals the background plus the wave's
    eigenvector times the exact average of its profile over that wave's domain
    of dependence (pins the acoustic corrections B and C: their signs, the
    factors 1/2, rho/a and a rho, and which wave speed bounds each integral).
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4


def cell_averages(coef, xc, h):
    """Exact averages of the polynomial sum coef[k] x^k over [xc-h/2, xc+h/2]."""
    a, b = xc - 0.5 * h, xc + 0.5 * h
    tot = 0.0
    for k, c in enumerate(coef):
        tot = tot + c * (b ** (k + 1) - a ** (k + 1)) / (k + 1)
    return tot / h


def poly(coef, x):
    return sum(c * x ** k for k, c in enumerate(coef))


def stencils_from_profiles(profiles, x0s, h):
    """Five-cell primitive stencils [n, 5, 5] from polynomial profiles per variable."""
    n = len(x0s)
    w = np.zeros((n, 5, 5))
    for i, x0 in enumerate(x0s):
        for s in range(5):
            xc = x0 + (s - 2) * h
            for q in range(5):
                w[i, s, q] = cell_averages(profiles[q], xc, h)
    return w


def test_constant_data_exact():
    rng = np.random.Generator(np.random.PCG64(1))
    n = 50
    base = np.column_stack([np.exp(rng.normal(size=n)), rng.normal(size=(n, 3)),
                            np.exp(rng.normal(size=n))])
    w = np.repeat(base[:, None, :], 5, axis=1)
    for dtdx in (0.0, 0.1, 0.37):
        WsL, WsR = oracle.ppmc(w, dtdx, GAMMA)
        assert np.array_equal(WsL, base)
        assert np.array_equal(WsR, base)


def test_cubic_face_values_dt0():
    """Smooth monotone cubics in all five primitives: W_L, W_R are exact point values."""
    profiles = [
        [1.0, 0.30, 0.05, 0.01],    # rho
        [0.20, 0.40, -0.03, 0.02],  # u (normal)
        [-0.1, 0.25, 0.02, -0.01],  # v
        [0.05, -0.2, 0.01, 0.005],  # w
        [1.0, 0.60, 0.04, 0.02],    # p
    ]
    h = 0.01
    x0s = np.linspace(-0.3, 0.3, 13)
    w = stencils_from_profiles(profiles, x0s, h)
    WsL, WsR = oracle.ppmc(w, 0.0, GAMMA)
    for i, x0 in enumerate(x0s):
        for q in range(5):
            exact_L = poly(profiles[q], x0 - 0.5 * h)
            exact_R = poly(profiles[q], x0 + 0.5 * h)
            assert abs(WsL[i, q] - exact_L) < 1e-12, (i, q)
            assert abs(WsR[i, q] - exact_R) < 1e-12, (i, q)


@pytest.mark.parametrize("U", [0.3, -0.3])
def test_advected_quadratic_traces_to_exact_upwind_average(U):
    """rho quadratic, u = U subsonic, p and v, w uniform.

    With |U| < a only the contact (speed U) carries rho.  For U > 0 the right
    face state is the average of rho(x) over [x_{i+1/2} - U dt, x_{i+1/2}]; for
    U < 0 the left face state is the average over [x_{i-1/2}, x_{i-1/2} - U dt].
    """
    h = 0.02
    rho = [2.0, 0.8, 0.9, 0.0]
    profiles = [rho, [U, 0, 0, 0], [0.1, 0, 0, 0], [-0.2, 0, 0, 0], [1.0, 0, 0, 0]]
    x0s = np.linspace(-0.2, 0.2, 9)
    w = stencils_from_profiles(profiles, x0s, h)
    for cfl in (0.1, 0.25, 0.4):
        dt = cfl * h / (abs(U) + np.sqrt(GAMMA * 1.0 / 2.5))
        WsL, WsR = oracle.ppmc(w, dt / h, GAMMA)
        for i, x0 in enumerate(x0s):
            if U > 0:
                b = x0 + 0.5 * h
                a = b - U * dt
                got = WsR[i, 0]
            else:
                a = x0 - 0.5 * h
                b = a - U * dt
                got = WsL[i, 0]
            F = lambda x: sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(rho))
            exact = (F(b) - F(a)) / (b - a)
            assert abs(got - exact) < 1e-12, (U, cfl, i, got, exact)
            # velocity, pressure and transverse velocities stay uniform
            for q, val in ((1, U), (2, 0.1), (3, -0.2), (4, 1.0)):
                assert abs(WsR[i, q] - val) < 1e-13 and abs(WsL[i, q] - val) < 1e-13


def test_mirror_symmetric_states():
    rng = np.random.Generator(np.random.PCG64(4))
    n = 200
    w = np.zeros((n, 5, 5))
    w[:, :, 0] = np.exp(rng.normal(scale=0.5, size=(n, 5)))
    w[:, :, 1:4] = rng.normal(size=(n, 5, 3))
    w[:, :, 4] = np.exp(rng.normal(scale=0.5, size=(n, 5)))
    m = w[:, ::-1, :].copy()
    m[:, :, 1] *= -1
    dtdx = 0.2
    WsL, WsR = oracle.ppmc(w, dtdx, GAMMA)
    mL, mR = oracle.ppmc(m, dtdx, GAMMA)
    flip = np.array([1, -1, 1, 1, 1])
    scale = np.abs(w).max(axis=(1, 2))[:, None]
    assert np.all(np.abs(mL * flip - WsR) <= 1e-12 * scale)
    assert np.all(np.abs(mR * flip - WsL) <= 1e-12 * scale)


def test_extremum_is_flattened_and_bounded():
    """A cell holding a local maximum gets flat faces; faces never leave the
    range of the neighbouring averages (Eqs. max_min and the bounding step)."""
    w = np.zeros((1, 5, 5))
    w[0, :, 0] = [1.0, 1.5, 2.0, 1.5, 1.0]   # density peak in the centre cell
    w[0, :, 4] = 1.0
    WsL, WsR = oracle.ppmc(w, 0.0, GAMMA)
    assert WsL[0, 0] == 2.0 and WsR[0, 0] == 2.0
    rng = np.random.Generator(np.random.PCG64(8))
    w = np.zeros((300, 5, 5))
    w[:, :, 0] = np.exp(rng.normal(size=(300, 5)))
    w[:, :, 4] = np.exp(rng.normal(size=(300, 5)))
    WsL, WsR = oracle.ppmc(w, 0.0, GAMMA)
    lo = np.minimum(w[:, 1:4, :].min(axis=1), w[:, 2, :])
    hi = np.maximum(w[:, 1:4, :].max(axis=1), w[:, 2, :])
    assert np.all(WsL >= lo - 1e-14) and np.all(WsL <= hi + 1e-14)
    assert np.all(WsR >= lo - 1e-14) and np.all(WsR <= hi + 1e-14)


def _ppmc_lib(L, w, dtdx, gamma):
    """oracle.ppmc through a given oracle library (a planted-mistake copy)."""
    import ctypes
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 5, 5)
    n = w.shape[0]
    WsL = np.zeros((n, 5)); WsR = np.zeros((n, 5))
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_ppmc.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp, dp]
    L.oracle_ppmc.restype = ctypes.c_int
    L.oracle_ppmc(n, w.ctypes.data_as(dp), float(dtdx), float(gamma), WsL.ctypes.data_as(dp),
                  WsR.ctypes.data_as(dp))
    return WsL, WsR


def _acoustic_wave_errors(family, ppmc_fn):
    """Largest deviation of the traced acoustic-wave perturbation from its exact
    first-order value, relative to the perturbation's size (see the test)."""
    rho0, p0 = 1.3, 0.9
    a0 = np.sqrt(GAMMA * p0 / rho0)
    eps = 1e-6
    h = 0.02
    qc = [0.4, 0.9, 1.3]  # q(x) = 0.4 + 0.9 x + 1.3 x^2, monotone on the stencils
    if family == "left":
        U, lam, r = 2.0 * a0, 2.0 * a0 - a0, np.array([1.0, -a0 / rho0, 0.0, 0.0, a0 * a0])
    else:
        U, lam, r = -2.0 * a0, -2.0 * a0 + a0, np.array([1.0, a0 / rho0, 0.0, 0.0, a0 * a0])
    w0 = np.array([rho0, U, 0.15, -0.05, p0])
    profiles = [[w0[q] + eps * r[q] * qc[0], eps * r[q] * qc[1], eps * r[q] * qc[2]]
                for q in range(5)]
    x0s = np.linspace(0.05, 0.25, 5)
    w = stencils_from_profiles(profiles, x0s, h)
    F = lambda x: sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(qc))
    worst = 0.0
    for cfl in (0.1, 0.3):
        dt = cfl * h / (abs(U) + a0)
        WsL, WsR = ppmc_fn(w, dt / h, GAMMA)
        for i, x0 in enumerate(x0s):
            if family == "left":
                b = x0 + 0.5 * h
                aa = b - lam * dt
                got = WsR[i]
            else:
                aa = x0 - 0.5 * h
                b = aa - lam * dt
                got = WsL[i]
            avg = (F(b) - F(aa)) / (b - aa)
            pert = (got - w0) / eps
            worst = max(worst, float(np.abs(pert - r * avg).max() / (np.abs(r).max() * abs(avg))))
    return worst


@pytest.mark.parametrize("family", ["left", "right"])
def test_supersonic_acoustic_wave_traces_to_exact_average(family):
    """A linear acoustic simple wave, w = w0 + eps r_k q(x) with q quadratic and
    r_k the wave's right eigenvector in primitive variables (left-going family:
    (1, -a/rho, 0, 0, a^2); right-going: (1, a/rho, 0, 0, a^2)), on a uniform
    flow moving supersonically so that the wave reaches the downwind face only
    through the correction terms: the left-going wave in a flow u = 2a to the
    right face (the C term, lambda^m = u - a > 0), the right-going wave in u =
    -2a to the left face (the B term, lambda^p = u + a < 0).  To first order in
    eps the traced state is w0 + eps r_k <q>, <q> the exact average of q over
    [x_f - lambda dt, x_f] (right face) or [x_f, x_f - lambda dt] (left face);
    the O(eps^2) remainder bounds the tolerance (1e-5 of the perturbation)."""
    assert _acoustic_wave_errors(family, lambda w, dtdx, g: oracle.ppmc(w, dtdx, g)) <= 1e-5


_PPMC = "void ppmc_cell(const R (*w)[5], R dtdx, const Gas& g, R WsL[5], R WsR[5]) {"
_ACOUSTIC_MUTANTS = {
    # the left-going wave's correction with the wrong sign of its velocity term
    "C_sign": [(_PPMC, "sR[0] = sR[0] + R(0.5) * (-(d * C[1]) / a + C[4] / a2);",
                "sR[0] = sR[0] + R(0.5) * ((d * C[1]) / a + C[4] / a2);")],
    # the right-going wave's velocity correction without its factor 1/2
    "B_half": [(_PPMC, "sL[1] = sL[1] + R(0.5) * (B[1] + B[4] / (a * d));",
                "sL[1] = sL[1] + (B[1] + B[4] / (a * d));")],
    # B bounded by the contact's speed instead of the right-going wave's
    "B_wave": [(_PPMC, "B[q] = TL_m[q] - TL_p[q];", "B[q] = TL_m[q] - TL_0[q];")],
    # C bounded by the contact's speed instead of the left-going wave's
    "C_wave": [(_PPMC, "C[q] = TR_p[q] - TR_m[q];", "C[q] = TR_p[q] - TR_0[q];")],
    # the pressure part of the C term's density correction dropped
    "C_pressure": [(_PPMC, "sR[0] = sR[0] + R(0.5) * (-(d * C[1]) / a + C[4] / a2);",
                    "sR[0] = sR[0] + R(0.5) * (-(d * C[1]) / a);")],
}


def test_acoustic_pin_catches_planted_mistakes():
    """Each plausible slip in the acoustic corrections, planted in a copy of the
    oracle source, fails the supersonic acoustic-wave pin (on the face its term
    reaches): a sign of the velocity term, a dropped factor 1/2, the wrong wave
    speed bounding the integral, a dropped pressure term."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_ACOUSTIC_MUTANTS)) as ex:
        libs = dict(zip(_ACOUSTIC_MUTANTS, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                    _ACOUSTIC_MUTANTS.items())))
    for tag, L in libs.items():
        errs = {fam: _acoustic_wave_errors(fam, lambda w, dtdx, g: _ppmc_lib(L, w, dtdx, g))
                for fam in ("left", "right")}
        assert max(errs.values()) > 1e-3, "planted mistake %r passes the acoustic pin: %s" % (
            tag, errs)
        print("%s: %s" % (tag, errs))


# ---------------------------------------------------------------------------
# Planted mistakes in the rest of PPMC (the slopes, the parabola, the traced
# integrals, the contact correction, monotonicity): each fails one of the pins
# above, re-run through a copy of the oracle with the mistake.

def _smooth_pin_violations(ppmc_fn):
    """Each pin's largest error over its tolerance (1: at the tolerance): the
    cubic face values, the advected quadratic, the flattened extremum and the
    neighbour bounds (test_cubic_face_values_dt0,
    test_advected_quadratic_traces_to_exact_upwind_average,
    test_extremum_is_flattened_and_bounded)."""
    out = {}
    profiles = [[1.0, 0.30, 0.05, 0.01], [0.20, 0.40, -0.03, 0.02], [-0.1, 0.25, 0.02, -0.01],
                [0.05, -0.2, 0.01, 0.005], [1.0, 0.60, 0.04, 0.02]]
    h = 0.01
    x0s = np.linspace(-0.3, 0.3, 13)
    WsL, WsR = ppmc_fn(stencils_from_profiles(profiles, x0s, h), 0.0, GAMMA)
    err = 0.0
    for i, x0 in enumerate(x0s):
        for q in range(5):
            err = max(err, abs(WsL[i, q] - poly(profiles[q], x0 - 0.5 * h)),
                      abs(WsR[i, q] - poly(profiles[q], x0 + 0.5 * h)))
    out["cubic"] = err / 1e-12
    err = 0.0
    h = 0.02
    rho = [2.0, 0.8, 0.9, 0.0]
    F = lambda x: sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(rho))
    for U in (0.3, -0.3):
        profiles = [rho, [U, 0, 0, 0], [0.1, 0, 0, 0], [-0.2, 0, 0, 0], [1.0, 0, 0, 0]]
        x0s = np.linspace(-0.2, 0.2, 9)
        w = stencils_from_profiles(profiles, x0s, h)
        for cfl in (0.1, 0.25, 0.4):
            dt = cfl * h / (abs(U) + np.sqrt(GAMMA * 1.0 / 2.5))
            WsL, WsR = ppmc_fn(w, dt / h, GAMMA)
            for i, x0 in enumerate(x0s):
                if U > 0:
                    b = x0 + 0.5 * h
                    a = b - U * dt
                    got = WsR[i, 0]
                else:
                    a = x0 - 0.5 * h
                    b = a - U * dt
                    got = WsL[i, 0]
                err = max(err, abs(got - (F(b) - F(a)) / (b - a)))
    out["quadratic"] = err / 1e-12
    w = np.zeros((1, 5, 5))
    w[0, :, 0] = [1.0, 1.5, 2.0, 1.5, 1.0]
    w[0, :, 4] = 1.0
    WsL, WsR = ppmc_fn(w, 0.0, GAMMA)
    out["extremum"] = max(abs(WsL[0, 0] - 2.0), abs(WsR[0, 0] - 2.0)) / 1e-15
    return out


_P = "void ppmc_cell("
_MUTANTS_SMOOTH = {
    # w6 as printed, 6 w_i - 3 (W_L - W_R): the parabola's mean is then not w_i
    "w6_printed": [(_P, "w6[q] = R(6.0) * wi[q] - R(3.0) * (L + Rr);",
                    "w6[q] = R(6.0) * wi[q] - R(3.0) * (L - Rr);")],
    # the parabolic interpolation with a third of the slope difference
    "face_third": [(_P, "R L = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(6.0);",
                    "R L = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(3.0);")],
    # the contact's traced integral with the sign of its 2/3 term flipped
    "two_thirds_sign": [(_P, "TL_0[q] = R(0.5) * a0 * (dw[q] + w6[q] * (R(1.0) + two3 * a0));",
                         "TL_0[q] = R(0.5) * a0 * (dw[q] + w6[q] * (R(1.0) - two3 * a0));")],
    # the contact correction of the density left out
    "contact_density": [(_P, "sL[0] = sL[0] + (E[0] - E[4] / a2);",
                         "sL[0] = sL[0] + (-E[4] / a2);")],
    # an extremum not flattened
    "no_flattening": [(_P, "{ L = wi[q]; Rr = wi[q]; }", "{ }")],
    # the left face bounded by the right neighbour
    "bound_side": [(_P, "L = mn(mx(wi[q], wim[q]), mx(mn(wi[q], wim[q]), L));",
                    "L = mn(mx(wi[q], wip[q]), mx(mn(wi[q], wip[q]), L));")],
    # the characteristic projection's first component as printed (R7 reading)
    "xi0_printed": [("void project(", "x[0] = R(0.5) * (-(d * dv[1]) / a + dv[4] / (a * a));",
                     "x[0] = R(-0.5) * (d * dv[1] / a + dv[4] / (a * a));")],
    # the MC limiter without its factor 2 (a minmod of three differences)
    "mc_factor": [("void plmc_slope(",
                   "const R lim = mn(mn(fabs(xC[q]), R(2.0) * fabs(xL[q])), R(2.0) * fabs(xR[q]));",
                   "const R lim = mn(mn(fabs(xC[q]), fabs(xL[q])), fabs(xR[q]));")],
}


def test_ppmc_pins_catch_planted_mistakes():
    """Each plausible slip in the slopes, the parabola, the traced integrals,
    the contact correction or the monotonicity step, planted in a copy of the
    oracle source, fails at least one PPMC pin by far more than its tolerance;
    the oracle as it is passes them all."""
    from concurrent.futures import ThreadPoolExecutor

    from tests.helpers import build_oracle_mutant
    with ThreadPoolExecutor(max_workers=len(_MUTANTS_SMOOTH)) as ex:
        libs = dict(zip(_MUTANTS_SMOOTH, ex.map(lambda kv: build_oracle_mutant(*kv),
                                                  _MUTANTS_SMOOTH.items())))
    for tag, L in libs.items():
        with np.errstate(all="ignore"):
            v = _smooth_pin_violations(lambda w, dtdx, g: _ppmc_lib(L, w, dtdx, g))
        assert max(v.values()) > 10.0 or not np.all(np.isfinite(list(v.values()))), (
            "planted mistake %r passes the PPMC pins: %s" % (tag, v))
        print("%s: %s" % (tag, {k: "%.3g" % x for k, x in v.items()}))
    base = _smooth_pin_violations(oracle.ppmc)
    assert max(base.values()) <= 1.0, base

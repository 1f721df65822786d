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
  * mirror data give mirrored face states.
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

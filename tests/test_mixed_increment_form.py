"""The transverse half-step of the mixed-precision path in increment form
(Eq. transverse_evolution, primitive recovery of U* + dU).

With v the velocity of the face state, rho' = rho + d rho and q = d m - v d rho,
  v' = v + q / rho'
  p' = p + (gamma - 1) (dE - v.q - |v|^2 d rho / 2 - |q|^2 / (2 rho'))
is the primitive recovery of U* + dU rearranged exactly.  These checks, in plain
numpy: the identity holds in float64 against the direct recovery; evaluated in
float32 it keeps the accuracy of the float increments where the direct float32
recovery loses digits to the total-minus-kinetic-energy cancellation (smooth
flow at Mach 30).  The GPU kernel's results are checked against the oracle by
the -m gpu tests.
"""
import numpy as np


def cons(rho, v, p, g):
    m = rho[:, None] * v
    E = p / (g - 1) + 0.5 * rho * (v * v).sum(axis=1)
    return rho, m, E


def direct(rho, m, E, g):
    r = rho
    v = m / r[:, None]
    p = (g - 1) * (E - 0.5 * (m * v).sum(axis=1))
    return r, v, p


def increment(rho, v, p, drho, dm, dE, g):
    one = rho.dtype.type(1)
    half = rho.dtype.type(0.5)
    gm1 = rho.dtype.type(g - 1)
    rn = rho + drho
    inv = one / rn
    q = dm - v * drho[:, None]
    vq = (v * q).sum(axis=1)
    v2 = (v * v).sum(axis=1)
    q2 = (q * q).sum(axis=1)
    de = dE - vq - half * (v2 * drho + q2 * inv)
    return rn, v + q * inv[:, None], p + gm1 * de


def samples(n, mach, delta, g=5.0 / 3.0, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = np.exp(rng.uniform(-1, 1, n))
    p = np.exp(rng.uniform(-1, 1, n))
    a = np.sqrt(g * p / rho)
    dirs = rng.standard_normal((n, 3))
    v = dirs / np.linalg.norm(dirs, axis=1)[:, None] * (mach * a)[:, None]
    # a nearby state W' = W (1 + delta z): dU = U(W') - U(W)
    rho2 = rho * (1 + delta * rng.standard_normal(n))
    v2 = v * (1 + delta * rng.standard_normal((n, 3)))
    p2 = p * (1 + delta * rng.standard_normal(n))
    U = cons(rho, v, p, g)
    U2 = cons(rho2, v2, p2, g)
    dU = tuple(b - a_ for a_, b in zip(U, U2))
    return (rho, v, p), dU, (rho2, v2, p2), g


def test_identity_in_float64():
    (rho, v, p), (drho, dm, dE), (rho2, v2, p2), g = samples(2000, 3.0, 0.05)
    rn, vn, pn = increment(rho, v, p, drho, dm, dE, g)
    rd, vd, pd = direct(rho + drho, cons(rho, v, p, g)[1] + dm, cons(rho, v, p, g)[2] + dE, g)
    np.testing.assert_allclose(rn, rho2, rtol=1e-14)
    np.testing.assert_allclose(vn, vd, rtol=1e-11, atol=1e-11 * np.abs(vd).max())
    np.testing.assert_allclose(pn, pd, rtol=1e-10)
    np.testing.assert_allclose(pn, p2, rtol=1e-10)


def test_float32_keeps_the_increments_accuracy_at_high_mach():
    (rho, v, p), (drho, dm, dE), (rho2, v2, p2), g = samples(4000, 30.0, 1e-3)
    f = np.float32
    # float32 inputs as the kernel has them: the face state and the increments
    rho32, v32, p32 = rho.astype(f), v.astype(f), p.astype(f)
    drho32, dm32, dE32 = drho.astype(f), dm.astype(f), dE.astype(f)
    _, _, p_inc = increment(rho32, v32, p32, drho32, dm32, dE32, g)
    # direct float32 recovery of U* + dU from the same float inputs
    U = cons(rho32, v32, p32, f(g))
    _, _, p_dir = direct(U[0] + drho32, U[1] + dm32, U[2] + dE32, f(g))
    # reference: the increment form in float64 on the same float32 inputs
    _, _, p_ref = increment(rho32.astype(np.float64), v32.astype(np.float64),
                            p32.astype(np.float64), drho32.astype(np.float64),
                            dm32.astype(np.float64), dE32.astype(np.float64), g)
    err_inc = np.abs(p_inc / p_ref - 1)
    err_dir = np.abs(p_dir / p_ref - 1)
    # kinetic over internal energy is ~g M^2 / 2 ~ 750: the direct form loses
    # about three digits of float32, the increment form keeps its float ulps
    assert np.median(err_inc) < 1e-7 and err_inc.max() < 2e-6, (np.median(err_inc), err_inc.max())
    assert np.median(err_dir) > 1e-5, np.median(err_dir)

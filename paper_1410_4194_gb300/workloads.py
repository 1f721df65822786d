"""Seeded synthetic initial conditions for the five benchmark workloads.

This module builds inputs only.  It contains none of the solver's arithmetic
(no reconstruction, Riemann solve or update); it turns primitive initial
conditions into conserved variables with the ideal-gas relation
E = p/(gamma-1) + rho |v|^2 / 2 and nothing else.  Both the CUDA path and the
CPU oracle consume its arrays, so it imports neither of them.

Every generator returns a dict with the conserved state ``u`` of shape
``[5, nz, ny, nx]`` (rho, rho u, rho v, rho w, E; float64), the cell width
``dx``, ``gamma``, the boundary codes ``bc`` (x-, x+, y-, y+, z-, z+; 0 periodic,
1 reflective, 2 outflow, 3 inflow) and, where needed, ``inflow`` primitive
states keyed by face.

Workloads (the paper's own data -- turbulence snapshots and cloud
distributions -- are not available, so seeded stand-ins of the same shape and
statistics are used):
  * ``sod``: 1D shock tube, gamma 1.4, (1,0,1) | (0.125,0,0.1) at x = 0.5.
  * ``sedov``: 3D blast, unit energy in the cells within 3.5 cells of the centre.
  * ``shock_cloud``: Mach-10 planar shock on a cloud with a lognormal density
    field (k^-11/3, wavelengths 4-64 cells), mean contrast 10.
  * ``turbulence``: Gaussian solenoidal velocity field, E(k) ~ k^-2, k = 1..16,
    rms Mach 5.
  * ``batched``: 96 grids of edges drawn from {32, 48, 64, 96, 128}, each a
    Sedov blast or an x shock tube.
"""
import numpy as np

PERIODIC, REFLECT, OUTFLOW, INFLOW = 0, 1, 2, 3


def prim_to_cons(rho, vx, vy, vz, p, gamma):
    """Stack primitive fields into the conserved layout [5, nz, ny, nx]."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    vx = np.broadcast_to(np.asarray(vx, dtype=np.float64), shape)
    vy = np.broadcast_to(np.asarray(vy, dtype=np.float64), shape)
    vz = np.broadcast_to(np.asarray(vz, dtype=np.float64), shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    u = np.empty((5,) + shape, dtype=np.float64)
    u[0] = rho
    u[1] = rho * vx
    u[2] = rho * vy
    u[3] = rho * vz
    u[4] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return u


def _centres(n, dx):
    return (np.arange(n, dtype=np.float64) + 0.5) * dx


def sod(nx=512, gamma=1.4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5):
    """1D Sod shock tube on [0, 1] with outflow ends; cells centred at (i+1/2)dx."""
    dx = 1.0 / nx
    x = _centres(nx, dx)
    L = x < x0
    rho = np.where(L, left[0], right[0]).reshape(1, 1, nx)
    vx = np.where(L, left[1], right[1]).reshape(1, 1, nx)
    p = np.where(L, left[2], right[2]).reshape(1, 1, nx)
    u = prim_to_cons(rho, vx, 0.0, 0.0, p, gamma)
    return dict(name="sod", u=u, dx=dx, gamma=gamma,
                bc=[OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC])


def sedov_blast_cells(shape, r_cells=3.5):
    """Mask of the cells whose centres lie within ``r_cells`` of the box centre."""
    nz, ny, nx = shape
    ci = [np.arange(n, dtype=np.float64) + 0.5 - n / 2.0 for n in (nz, ny, nx)]
    z, y, x = np.meshgrid(*ci, indexing="ij")
    return (x * x + y * y + z * z) < r_cells * r_cells


def sedov(n=256, shape=None, dx=None, gamma=5.0 / 3.0, rho0=1.0, p0=1e-5, energy=1.0,
          r_cells=3.5):
    """3D Sedov-Taylor blast in a periodic box.

    ``energy`` is spread as thermal energy uniformly over the cells within
    ``r_cells`` cell widths of the box centre (a cell corner for even edges).
    """
    if shape is None:
        shape = (n, n, n)
    nz, ny, nx = shape
    if dx is None:
        dx = 1.0 / nx
    mask = sedov_blast_cells(shape, r_cells)
    ncell = int(mask.sum())
    p_in = (gamma - 1.0) * energy / (ncell * dx ** 3)
    p = np.where(mask, p_in, p0)
    rho = np.full(shape, rho0)
    u = prim_to_cons(rho, 0.0, 0.0, 0.0, p, gamma)
    return dict(name="sedov", u=u, dx=dx, gamma=gamma, bc=[PERIODIC] * 6,
                blast_cells=ncell, p_blast=p_in, energy=energy)


def rankine_hugoniot(mach, rho1=1.0, p1=1.0, gamma=5.0 / 3.0):
    """Post-shock (rho, u, p) behind a shock of Mach ``mach`` moving into gas at rest."""
    a1 = np.sqrt(gamma * p1 / rho1)
    vs = mach * a1
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    u2 = vs * (1.0 - rho1 / rho2)
    return rho2, u2, p2, vs


def gaussian_random_field(shape, seed, slope, kmin, kmax):
    """Periodic Gaussian random field with power P(k) ~ k^slope for kmin <= |k| <= kmax.

    ``k`` is in cycles per box; the field is normalised to zero mean, unit variance.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    band = (k >= kmin) & (k <= kmax)
    amp = np.zeros_like(k)
    amp[band] = k[band] ** (slope / 2.0)
    noise = rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)
    f = np.fft.irfftn(noise * amp, s=shape, axes=(0, 1, 2))
    f -= f.mean()
    f /= f.std()
    return f


def shock_cloud(nx=512, ny=256, nz=256, mach=10.0, gamma=5.0 / 3.0, chi=10.0,
                radius=32, centre=(176, 128, 128), shock_x=128, seed=4194):
    """Mach-10 planar shock moving in +x onto a lognormal cloud (mean contrast ``chi``).

    Cloud density is max(1, s exp(g)) with g a unit-variance Gaussian field of
    spectrum k^-11/3 between wavelengths 4 and 64 cells; s is found by
    bisection so that the mean density over the cloud cells is ``chi``.  The
    cloud sits in pressure equilibrium (p = 1) with the ambient gas.
    """
    dx = 1.0 / ny
    rho2, u2, p2, vs = rankine_hugoniot(mach, 1.0, 1.0, gamma)
    box = 128
    g = gaussian_random_field((box, box, box), seed, -11.0 / 3.0, box / 64.0, box / 4.0)
    rho = np.ones((nz, ny, nx))
    vx = np.zeros((nz, ny, nx))
    p = np.ones((nz, ny, nx))
    cx, cy, cz = centre
    zi = np.arange(nz) + 0.5 - (cz + 0.0)
    yi = np.arange(ny) + 0.5 - (cy + 0.0)
    xi = np.arange(nx) + 0.5 - (cx + 0.0)
    # cloud region: a (2r)^3 box around the centre; the field is sampled from the
    # periodic box by cell offset
    z0, z1 = cz - radius, cz + radius
    y0, y1 = cy - radius, cy + radius
    x0, x1 = cx - radius, cx + radius
    Z, Y, X = np.meshgrid(zi[z0:z1], yi[y0:y1], xi[x0:x1], indexing="ij")
    inside = (X * X + Y * Y + Z * Z) < radius * radius
    gsub = g[:z1 - z0, :y1 - y0, :x1 - x0]
    eg = np.exp(gsub[inside])
    lo, hi = 0.0, 1e3
    for _ in range(200):
        s = 0.5 * (lo + hi)
        if np.maximum(1.0, s * eg).mean() < chi:
            lo = s
        else:
            hi = s
    s = 0.5 * (lo + hi)
    sub = rho[z0:z1, y0:y1, x0:x1]
    sub[inside] = np.maximum(1.0, s * eg)
    rho[:, :, :shock_x] = rho2
    vx[:, :, :shock_x] = u2
    p[:, :, :shock_x] = p2
    u = prim_to_cons(rho, vx, 0.0, 0.0, p, gamma)
    return dict(name="shock_cloud", u=u, dx=dx, gamma=gamma,
                bc=[INFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                inflow={0: (rho2, u2, 0.0, 0.0, p2)}, shock_speed=vs, cloud_scale=s)


def turbulence(n=512, gamma=5.0 / 3.0, mach=5.0, kmin=1, kmax=16, seed=1410):
    """Periodic box at rho = 1, p = 1 with a Gaussian solenoidal velocity field.

    Complex normal modes with shell spectrum E(k) ~ k^-2 (mode amplitude ~ k^-2)
    for integer shells kmin <= |k| <= kmax, projected onto the plane normal to
    k, scaled to rms |v| = mach * sqrt(gamma).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    kz = np.fft.fftfreq(n) * n
    ky = np.fft.fftfreq(n) * n
    kx = np.fft.rfftfreq(n) * n
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k = np.sqrt(k2)
    shell = np.rint(k)
    band = (shell >= kmin) & (shell <= kmax)
    amp = np.zeros_like(k)
    amp[band] = k[band] ** -2.0
    comps = []
    for _ in range(3):
        comps.append((rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)) * amp)
    k2s = np.where(k2 > 0, k2, 1.0)
    div = (KX * comps[0] + KY * comps[1] + KZ * comps[2]) / k2s
    comps[0] = comps[0] - KX * div
    comps[1] = comps[1] - KY * div
    comps[2] = comps[2] - KZ * div
    v = [np.fft.irfftn(c, s=(n, n, n), axes=(0, 1, 2)) for c in comps]
    rms = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    scale = mach * np.sqrt(gamma) / rms
    rho = np.ones((n, n, n))
    u = prim_to_cons(rho, v[0] * scale, v[1] * scale, v[2] * scale, 1.0, gamma)
    return dict(name="turbulence", u=u, dx=1.0 / n, gamma=gamma, bc=[PERIODIC] * 6)


def batched(ngrids=96, seed=14104194, edges=(32, 48, 64, 96, 128), gamma=5.0 / 3.0,
            dx=1.0 / 64.0):
    """Independent grids of uneven sizes: Sedov blasts and x shock tubes.

    Each axis edge is drawn uniformly from ``edges``; a fair coin picks the
    problem.  Shock tubes have (rho, p) on each side log-uniform in [0.1, 10],
    v = 0, the diaphragm at x = nx/2, outflow in x and periodic y, z.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(ngrids):
        nx, ny, nz = (int(e) for e in rng.choice(edges, size=3))
        kind = "sedov" if rng.random() < 0.5 else "tube"
        if kind == "sedov":
            w = sedov(shape=(nz, ny, nx), dx=dx, gamma=gamma)
            w["name"] = "sedov"
        else:
            rl, pl, rr, pr = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=4))
            x = np.arange(nx)
            L = (x < nx // 2).reshape(1, 1, nx)
            rho = np.broadcast_to(np.where(L, rl, rr), (nz, ny, nx)).copy()
            p = np.broadcast_to(np.where(L, pl, pr), (nz, ny, nx)).copy()
            u = prim_to_cons(rho, 0.0, 0.0, 0.0, p, gamma)
            w = dict(name="tube", u=u, dx=dx, gamma=gamma,
                     bc=[OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                     tube=(rl, pl, rr, pr))
        out.append(w)
    return out


def noh(n=200, nd=3, gamma=5.0 / 3.0, rho0=1.0, speed=1.0, p0=1e-6):
    """Noh's strong shock (Sec. 4.3.1) on the octant [0, 1]^nd: uniform density
    rho0 and pressure p0 streaming at `speed` toward the origin; reflecting
    inner faces, analytic (HYDRO_BC_NOH) outer faces whose prescribed state is
    (rho0, speed, 0, 0, p0).  Also returns the cells' radius r."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    if nd == 3:
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
        u = prim_to_cons(np.full_like(r, rho0), -speed * X / r, -speed * Y / r,
                         -speed * Z / r, np.full_like(r, p0), gamma)
        bc, faces = [1, 4, 1, 4, 1, 4], (1, 3, 5)
    elif nd == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        r = np.sqrt(X ** 2 + Y ** 2)[None]
        u = prim_to_cons(np.full_like(r, rho0), (-speed * X / r[0])[None],
                         (-speed * Y / r[0])[None], 0.0, np.full_like(r, p0), gamma)
        bc, faces = [1, 4, 1, 4, 0, 0], (1, 3)
    else:
        raise ValueError("nd must be 2 or 3")
    return dict(u=u, dx=dx, gamma=gamma, bc=bc, r=r,
                inflow={f: (rho0, speed, 0.0, 0.0, p0) for f in faces})


def smooth_periodic(shape, gamma=1.4, seed=7, amp=0.2, vamp=0.5):
    """Smooth random periodic state (a few low Fourier modes per field), for tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                             indexing="ij")

    def field():
        f = np.zeros(shape)
        for _ in range(3):
            kx, ky, kz = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * xx + ky * yy + kz * zz) + ph)
        return f / 3.0

    rho = 1.0 + amp * field()
    p = 1.0 + amp * field()
    vx = vamp * field() if nx > 1 else np.zeros(shape)
    vy = vamp * field() if ny > 1 else np.zeros(shape)
    vz = vamp * field() if nz > 1 else np.zeros(shape)
    return prim_to_cons(rho, vx, vy, vz, p, gamma)


def random_states(n, seed, gamma=1.4, rho_range=(0.1, 10.0), p_range=(0.01, 100.0), vmax=3.0):
    """Random primitive state pairs [n, 5] (rho, u, v, w, p) for Riemann tests."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def one():
        rho = np.exp(rng.uniform(np.log(rho_range[0]), np.log(rho_range[1]), n))
        p = np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1]), n))
        v = rng.uniform(-vmax, vmax, (n, 3))
        return np.column_stack([rho, v, p])

    return one(), one()

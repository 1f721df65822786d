"""CPU oracle for one CTU + PPMC + exact-Riemann step -- TEST INFRASTRUCTURE.

A ctypes front end to ``hydro_oracle.cpp`` (plain FP64 C++, no fused
multiply-add).  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path
(``paper_1410_4194_gb300``) never does, and the oracle imports nothing from it.

Functions follow Schneider & Robertson, "Cholla": the CTU step of Sec. 2.3,
PPMC of App. A.3 and the exact solver of App. B.1.  Pins (the values and
properties that fix the oracle independently of itself) live in
``tests/test_oracle_*.py``.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None

FLAG_NEWTON = 1
FLAG_NONPHYS = 2

BC_PERIODIC, BC_REFLECT, BC_OUTFLOW, BC_INFLOW, BC_NOH = 0, 1, 2, 3, 4
RECON_PPMC, RECON_PPMP, RECON_PLMC, RECON_PLMP, RECON_PCM = 0, 1, 2, 3, 4
SOLVER_EXACT, SOLVER_ROE = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.oracle_init.restype = ctypes.c_void_p
        L.oracle_init.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_ip]
        L.oracle_free.argtypes = [ctypes.c_void_p]
        L.oracle_set_inflow.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.oracle_set_recon.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_set_solver.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_riemann_roe.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp]
        L.oracle_reconstruct.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.oracle_set_state.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_get_state.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_compute_dt.restype = ctypes.c_double
        L.oracle_compute_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.oracle_step_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.oracle_set_time.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.oracle_get_time.argtypes = [ctypes.c_void_p]
        L.oracle_get_time.restype = ctypes.c_double
        L.oracle_fill_ghosts.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_riemann_prim.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double,
                                          _dp, _dp, _dp, _dp, _ip]
        L.oracle_riemann_cons.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp]
        L.oracle_ppmc.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.oracle_count_step.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp]
        L.oracle_count_step_stages.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp]
        _lib = L
    return _lib


def set_threads(n):
    """Set the OpenMP thread count of the oracle (0: every processor); returns
    the count in effect."""
    return lib().oracle_set_threads(int(n))


def riemann_prim(WL, WR, gamma):
    """Exact Riemann solver on primitive pairs ``[n, 5]`` (rho, u_n, u_t1, u_t2, p).

    Returns a dict with the flux ``F [n,5]``, star pressure ``pm``, star
    velocity ``um``, the sampled interface state ``ws [n,5]``, Newton
    iteration counts and the OR of the status flags.
    """
    WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(-1, 5)
    WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(-1, 5)
    n = WL.shape[0]
    F = np.zeros((n, 5)); ws = np.zeros((n, 5))
    pm = np.zeros(n); um = np.zeros(n); it = np.zeros(n, dtype=np.int32)
    fl = lib().oracle_riemann_prim(n, _ptr(WL), _ptr(WR), float(gamma), _ptr(F), _ptr(pm),
                                   _ptr(um), _ptr(ws), _ptr(it, _ip))
    return dict(F=F, pm=pm, um=um, ws=ws, iters=it, flags=fl)


def riemann_cons(UL, UR, gamma):
    """Exact Riemann flux on conserved pairs ``[n, 5]`` in sweep order."""
    UL = np.ascontiguousarray(UL, dtype=np.float64).reshape(-1, 5)
    UR = np.ascontiguousarray(UR, dtype=np.float64).reshape(-1, 5)
    F = np.zeros_like(UL)
    fl = lib().oracle_riemann_cons(UL.shape[0], _ptr(UL), _ptr(UR), float(gamma), _ptr(F))
    return F, fl


def ppmc(w, dtdx, gamma):
    """PPMC on five-cell primitive stencils ``w [n, 5 cells, 5]``.

    Returns ``(WsL, WsR)``: the time-evolved states at the left and right face
    of the centre cell, each ``[n, 5]``.
    """
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 5, 5)
    n = w.shape[0]
    WsL = np.zeros((n, 5)); WsR = np.zeros((n, 5))
    lib().oracle_ppmc(n, _ptr(w), float(dtdx), float(gamma), _ptr(WsL), _ptr(WsR))
    return WsL, WsR


def riemann_roe(UL, UR, gamma, etaH=None):
    """Roe solver with the HLLE fallback on conserved pairs ``[n, 5]`` (rho,
    normal momentum, two transverse momenta, E); ``etaH [n]`` the H correction
    (None: none).  Returns the fluxes ``[n, 5]``."""
    UL = np.ascontiguousarray(UL, dtype=np.float64).reshape(-1, 5)
    UR = np.ascontiguousarray(UR, dtype=np.float64).reshape(-1, 5)
    n = UL.shape[0]
    F = np.zeros((n, 5))
    e = None if etaH is None else np.ascontiguousarray(etaH, dtype=np.float64).reshape(-1)
    lib().oracle_riemann_roe(n, _ptr(UL), _ptr(UR), None if e is None else _ptr(e), float(gamma),
                             _ptr(F))
    return F


def reconstruct(recon, w, dtdx, dx, gamma):
    """Reconstruction ``recon`` (RECON_*) on seven-cell primitive stencils
    ``w [n, 7 cells, 5]`` (cells i-3..i+3; rho, normal velocity, two transverse
    velocities, p).  Returns ``(UsL, UsR)``: the conserved time-evolved states at
    the left and right face of the centre cell, each ``[n, 5]``."""
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 7, 5)
    n = w.shape[0]
    UsL = np.zeros((n, 5)); UsR = np.zeros((n, 5))
    rc = lib().oracle_reconstruct(n, int(recon), _ptr(w), float(dtdx), float(dx), float(gamma),
                                  _ptr(UsL), _ptr(UsR))
    if rc != 0:
        raise ValueError("unknown reconstruction %r" % (recon,))
    return UsL, UsR


class Grid:
    """One grid advanced by the oracle's CTU step.

    ``u`` arrays are conserved variables ``[5, nz, ny, nx]`` (rho, rho u,
    rho v, rho w, E) of the real cells.  ``bc`` lists x-, x+, y-, y+, z-, z+.
    """

    def __init__(self, nx, ny, nz, dx, gamma, bc):
        bca = np.ascontiguousarray(bc, dtype=np.int32)
        self.shape = (nz, ny, nx)
        self.h = lib().oracle_init(nx, ny, nz, float(dx), float(gamma), _ptr(bca, _ip))
        if not self.h:
            raise ValueError("oracle_init rejected the grid")
        self.n = (nx, ny, nz)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.oracle_free(h)
            self.h = None

    def set_inflow(self, face, prim):
        """Prescribed state of an inflow face (rho, u, v, w, p), or of a Noh face
        (rho0, V, -, -, p0)."""
        p = np.ascontiguousarray(prim, dtype=np.float64)
        lib().oracle_set_inflow(self.h, int(face), _ptr(p))

    def set_time(self, t):
        """Time at the start of the next step (the Noh boundary's t)."""
        lib().oracle_set_time(self.h, float(t))

    def get_time(self):
        return lib().oracle_get_time(self.h)

    def set_recon(self, recon):
        """Reconstruction (Sec. 2.2.1): RECON_PPMC (default), RECON_PPMP, RECON_PLMC,
        RECON_PLMP or RECON_PCM."""
        if lib().oracle_set_recon(self.h, int(recon)) != 0:
            raise ValueError("unknown reconstruction %r" % (recon,))

    def set_solver(self, solver):
        """Riemann solver (Sec. 2.2.2): SOLVER_EXACT (default) or SOLVER_ROE (Roe with
        the HLLE fallback; H correction in the second set of solves)."""
        if lib().oracle_set_solver(self.h, int(solver)) != 0:
            raise ValueError("unknown Riemann solver %r" % (solver,))

    def set_state(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (5,) + self.shape
        lib().oracle_set_state(self.h, _ptr(u))

    def get_state(self):
        u = np.zeros((5,) + self.shape)
        lib().oracle_get_state(self.h, _ptr(u))
        return u

    def compute_dt(self, cfl):
        return lib().oracle_compute_dt(self.h, float(cfl))

    def step_dt(self, dt):
        """Advance one CTU step with the given dt; returns the status flags."""
        return lib().oracle_step_dt(self.h, float(dt))

    def step(self, cfl):
        """Advance one step with dt from the CFL condition; returns (dt, flags)."""
        dt = self.compute_dt(cfl)
        return dt, self.step_dt(dt)

    def padded_after_ghost_fill(self):
        nx, ny, nz = self.n
        N = [n + 8 if n > 1 else 1 for n in (nx, ny, nz)]
        out = np.zeros((5, N[2], N[1], N[0]))
        lib().oracle_fill_ghosts(self.h, _ptr(out))
        return out

    def count_step(self, dt):
        """Algorithmic operation counts of one step (state unchanged).

        Returns a dict with add (incl. subtract), mul, div, sqrt, pow and cmp
        (compare/min/max/abs) counts, plus the status flags.
        """
        c = np.zeros(6)
        fl = lib().oracle_count_step(self.h, float(dt), _ptr(c))
        keys = ("add", "mul", "div", "sqrt", "pow", "cmp")
        out = {k: int(v) for k, v in zip(keys, c)}
        out["flags"] = fl
        return out

    STAGES = ("prims", "ppmc", "riemann1", "riemann2", "update", "slopes")

    def count_step_stages(self, dt):
        """Per-stage algorithmic operation counts of one step (state unchanged).

        Returns {stage: {"ops": {kind: count}, "units": n}} for the stages
        prims (incl. the dt minimum), ppmc (without slopes), riemann1,
        riemann2 (incl. the transverse half-step), update and slopes.
        """
        c = np.zeros(36)
        u = np.zeros(6)
        lib().oracle_count_step_stages(self.h, float(dt), _ptr(c), _ptr(u))
        keys = ("add", "mul", "div", "sqrt", "pow", "cmp")
        out = {}
        for k, name in enumerate(self.STAGES):
            out[name] = {"ops": {kk: int(c[6 * k + q]) for q, kk in enumerate(keys)},
                         "units": int(u[k])}
        return out


def run(u0, dx, gamma, bc, nsteps=None, cfl=0.3, t_end=None, inflow=None, max_steps=100000,
        recon=RECON_PPMC, solver=SOLVER_EXACT):
    """Advance ``u0`` with the oracle; returns ``(u, t, nsteps, flags)``.

    Either ``nsteps`` CFL steps, or steps until ``t_end`` with the last step
    clamped so that the final time is exactly ``t_end``.
    """
    _, nz, ny, nx = u0.shape
    g = Grid(nx, ny, nz, dx, gamma, bc)
    g.set_recon(recon)
    g.set_solver(solver)
    if inflow:
        for face, prim in inflow.items():
            g.set_inflow(face, prim)
    g.set_state(u0)
    t = 0.0
    steps = 0
    flags = 0
    while steps < max_steps:
        if nsteps is not None and steps >= nsteps:
            break
        if t_end is not None and t >= t_end:
            break
        dt = g.compute_dt(cfl)
        last = t_end is not None and t + dt >= t_end
        if last:
            dt = t_end - t
        flags |= g.step_dt(dt)
        t = t_end if last else t + dt
        steps += 1
    return g.get_state(), t, steps, flags

"""Python binding of the C-ABI in ``include/hydro.h`` (ctypes, marshalling only).

Every step of the method runs in the CUDA library ``_build/libhydro.so``; this
module only converts arguments.  There is no CPU fallback: if the library has
not been built, or no GPU is present, the calls raise.

Arrays are conserved states ``[5, nz, ny, nx]`` float64 (rho, rho u, rho v,
rho w, E).  A ``torch`` CUDA tensor is passed by device pointer on the current
torch stream; a numpy array or CPU tensor by host pointer.
"""
import ctypes
import math
import os

import numpy as np

HYDRO_BC_PERIODIC, HYDRO_BC_REFLECT, HYDRO_BC_OUTFLOW, HYDRO_BC_INFLOW, HYDRO_BC_NOH = 0, 1, 2, 3, 4
HYDRO_FP64, HYDRO_MIXED, HYDRO_FP64_STRICT = 0, 1, 2
HYDRO_RECON_PPMC, HYDRO_RECON_PPMP, HYDRO_RECON_PLMC, HYDRO_RECON_PLMP, HYDRO_RECON_PCM = range(5)
HYDRO_RIEMANN_EXACT, HYDRO_RIEMANN_ROE = 0, 1
ERRORS = {0: "HYDRO_OK", -1: "HYDRO_EINVAL", -2: "HYDRO_ENOMEM", -3: "HYDRO_ECUDA",
          -4: "HYDRO_ENONPHYS", -5: "HYDRO_ENEWTON", -6: "HYDRO_ENOSTATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhydro.so")

# every entry point that include/hydro.h declares
EXPORTS = ("hydro_init", "hydro_set_inflow", "hydro_set_time", "hydro_get_time",
           "hydro_set_precision", "hydro_set_stream", "hydro_set_block_size", "hydro_block_size",
           "hydro_set_state", "hydro_get_state", "hydro_step", "hydro_step_dt",
           "hydro_compute_dt", "hydro_advance",
           "hydro_set_state_async", "hydro_get_state_async", "hydro_step_async", "hydro_sync", "hydro_last_error", "hydro_error_string",
           "hydro_cuda_error_string", "hydro_profile", "hydro_profile_read", "hydro_free",
           "hydro_riemann_exact", "hydro_ppmc", "hydro_compute_dt_noalloc",
           "hydro_batch_init", "hydro_batch_set_inflow", "hydro_batch_set_precision",
           "hydro_batch_set_stream", "hydro_batch_set_state", "hydro_batch_get_state",
           "hydro_batch_step", "hydro_batch_step_async", "hydro_batch_sync",
           "hydro_batch_set_state_async", "hydro_batch_get_state_async", "hydro_batch_autotune", "hydro_batch_last_error",
           "hydro_batch_cuda_error_string", "hydro_batch_free", "hydro_check_conversions",
           "hydro_check_fastdiv", "hydro_check_newton", "hydro_check_scaling",
           "hydro_probe_fp64_rate",
           "hydro_set_reconstruction", "hydro_batch_set_reconstruction",
           "hydro_set_riemann_solver", "hydro_batch_set_riemann_solver")
STAGES = ("prims", "set_dt", "slopes", "ppmc", "riemann1", "riemann2", "update")

_lib = None


class HydroError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERRORS.get(code, "?"), code, (": " + msg) if msg else ""))


def load():
    """Load libhydro.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhydro.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.hydro_init.argtypes = [ctypes.POINTER(vp)] + [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ip]
    L.hydro_set_inflow.argtypes = [vp, ctypes.c_int, dp]
    L.hydro_set_time.argtypes = [vp, ctypes.c_double]
    L.hydro_get_time.argtypes = [vp]
    L.hydro_get_time.restype = ctypes.c_double
    L.hydro_set_precision.argtypes = [vp, ctypes.c_int]
    L.hydro_set_stream.argtypes = [vp, vp]
    L.hydro_set_block_size.argtypes = [vp, ctypes.c_int]
    L.hydro_block_size.argtypes = [vp]
    L.hydro_set_state.argtypes = [vp, vp, ctypes.c_int]
    L.hydro_get_state.argtypes = [vp, vp, ctypes.c_int]
    for f in (L.hydro_step, L.hydro_step_dt, L.hydro_compute_dt):
        f.argtypes = [vp, ctypes.c_double]
        f.restype = ctypes.c_double
    L.hydro_last_error.argtypes = [vp]
    L.hydro_error_string.argtypes = [ctypes.c_int]
    L.hydro_error_string.restype = ctypes.c_char_p
    L.hydro_cuda_error_string.argtypes = [vp]
    L.hydro_cuda_error_string.restype = ctypes.c_char_p
    L.hydro_free.argtypes = [vp]
    L.hydro_profile.argtypes = [vp, ctypes.c_int]
    llp = ctypes.POINTER(ctypes.c_longlong)
    L.hydro_profile_read.argtypes = [vp, ctypes.c_int, dp, llp, llp, llp]
    L.hydro_advance.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, llp]
    L.hydro_set_state_async.argtypes = [vp, vp, ctypes.c_int]
    L.hydro_get_state_async.argtypes = [vp, vp, ctypes.c_int]
    L.hydro_step_async.argtypes = [vp, ctypes.c_double]
    L.hydro_sync.argtypes = [vp, dp]
    L.hydro_riemann_exact.argtypes = [ctypes.c_int, vp, vp, ctypes.c_double, vp, vp, vp]
    L.hydro_ppmc.argtypes = [ctypes.c_int, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    L.hydro_compute_dt_noalloc.argtypes = [vp] + [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [vp, vp]
    L.hydro_batch_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ip, dp, dp, ip]
    L.hydro_batch_set_inflow.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    L.hydro_batch_set_precision.argtypes = [vp, ctypes.c_int]
    L.hydro_batch_set_stream.argtypes = [vp, vp]
    L.hydro_batch_set_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_batch_get_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_batch_step.argtypes = [vp, ctypes.c_double, ctypes.c_int, dp]
    L.hydro_batch_step_async.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.hydro_batch_sync.argtypes = [vp]
    L.hydro_batch_set_state_async.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_batch_get_state_async.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_batch_autotune.argtypes = [vp, ctypes.c_int, ip, ip, ctypes.POINTER(ctypes.c_float)]
    L.hydro_batch_last_error.argtypes = [vp]
    L.hydro_batch_cuda_error_string.argtypes = [vp]
    L.hydro_batch_cuda_error_string.restype = ctypes.c_char_p
    L.hydro_batch_free.argtypes = [vp]
    L.hydro_check_conversions.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), vp]
    L.hydro_check_scaling.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), vp]
    L.hydro_check_newton.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), vp]
    L.hydro_probe_fp64_rate.argtypes = [dp, vp]
    L.hydro_check_fastdiv.argtypes = []
    L.hydro_check_fastdiv.restype = ctypes.c_longlong
    L.hydro_set_reconstruction.argtypes = [vp, ctypes.c_int]
    L.hydro_batch_set_reconstruction.argtypes = [vp, ctypes.c_int]
    L.hydro_set_riemann_solver.argtypes = [vp, ctypes.c_int]
    L.hydro_batch_set_riemann_solver.argtypes = [vp, ctypes.c_int]
    _lib = L
    return L


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _torch_stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _buffer(u, shape, writable):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if _is_torch(u):
        if tuple(u.shape) != shape or str(u.dtype) != "torch.float64" or not u.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor of shape %s" % (shape,))
        return ctypes.c_void_p(u.data_ptr()), int(u.is_cuda), u
    a = u if writable else np.ascontiguousarray(u, dtype=np.float64)
    if a.shape != shape or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float64 array of shape %s" % (shape,))
    return ctypes.c_void_p(a.ctypes.data), 0, a


class Grid:
    """One grid advanced by the CUDA CTU step (see include/hydro.h)."""

    def __init__(self, nx, ny, nz, dx, gamma, bc, precision=HYDRO_FP64, stream=None,
                 recon=HYDRO_RECON_PPMC, solver=HYDRO_RIEMANN_EXACT):
        L = load()
        self._L = L
        h = ctypes.c_void_p()
        bca = (ctypes.c_int * 6)(*[int(b) for b in bc])
        rc = L.hydro_init(ctypes.byref(h), int(nx), int(ny), int(nz), float(dx), float(gamma), bca)
        if rc != 0:
            raise HydroError(rc, "hydro_init")
        self.h = h
        self.shape = (5, nz, ny, nx)
        self.n = (nx, ny, nz)
        self._pending = []
        if stream is not None:
            self.set_stream(stream)
        if recon != HYDRO_RECON_PPMC:
            self.set_reconstruction(recon)
        if solver != HYDRO_RIEMANN_EXACT:
            self.set_riemann_solver(solver)
        if precision != HYDRO_FP64:
            self.set_precision(precision)

    def _check(self, rc, what):
        if rc != 0:
            msg = what
            if rc == -3:
                msg += ": " + self._L.hydro_cuda_error_string(self.h).decode()
            raise HydroError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self._L.hydro_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_inflow(self, face, prim):
        """Prescribed state of an inflow face (rho, u, v, w, p), or of a Noh face
        (rho0, V, -, -, p0)."""
        p = (ctypes.c_double * 5)(*[float(x) for x in prim])
        self._check(self._L.hydro_set_inflow(self.h, int(face), p), "set_inflow")

    def set_time(self, t):
        """Time at the start of the next step (the Noh boundary's t)."""
        self._check(self._L.hydro_set_time(self.h, float(t)), "set_time")

    def get_time(self):
        t = self._L.hydro_get_time(self.h)
        if t < 0:
            raise HydroError(int(t), "get_time")
        return t

    def set_precision(self, mode):
        self._check(self._L.hydro_set_precision(self.h, int(mode)), "set_precision")

    def set_reconstruction(self, recon):
        self._check(self._L.hydro_set_reconstruction(self.h, int(recon)), "set_reconstruction")

    def set_riemann_solver(self, solver):
        self._check(self._L.hydro_set_riemann_solver(self.h, int(solver)), "set_riemann_solver")

    def set_block_size(self, bs):
        """Threads a block of the fast FP64 / mixed launches: 128, 256 or 0 (auto)."""
        self._check(self._L.hydro_set_block_size(self.h, int(bs)), "set_block_size")

    def block_size(self):
        return self._L.hydro_block_size(self.h)

    def set_stream(self, stream):
        """Order this grid's work on a stream: a torch.cuda.Stream, a raw
        cudaStream_t integer, or "torch" for torch's current stream."""
        if stream == "torch":
            ptr = _torch_stream_ptr()
        elif hasattr(stream, "cuda_stream"):
            ptr = ctypes.c_void_p(stream.cuda_stream)
        else:
            ptr = ctypes.c_void_p(int(stream) if stream else 0)
        self._check(self._L.hydro_set_stream(self.h, ptr), "set_stream")

    def set_state(self, u):
        ptr, dev, keep = _buffer(u, self.shape, False)
        self._check(self._L.hydro_set_state(self.h, ptr, dev), "set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, dev, keep = _buffer(out, self.shape, True)
        self._check(self._L.hydro_get_state(self.h, ptr, dev), "get_state")
        return out

    # asynchronous forms: the buffers are held until sync(); a host buffer should
    # be page-locked (a pinned torch tensor) for the copy to overlap other work
    def _async_buffer(self, u, writable):
        ptr, dev, keep = _buffer(u, self.shape, writable)
        if keep is not u:
            raise ValueError("asynchronous copies need a C-contiguous float64 buffer (no temporary)")
        self._pending.append(u)
        return ptr, dev

    def set_state_async(self, u):
        ptr, dev = self._async_buffer(u, False)
        self._check(self._L.hydro_set_state_async(self.h, ptr, dev), "set_state_async")

    def get_state_async(self, out):
        ptr, dev = self._async_buffer(out, True)
        self._check(self._L.hydro_get_state_async(self.h, ptr, dev), "get_state_async")
        return out

    def step_async(self, cfl):
        """Enqueue one CFL step; dt and the status stay on the device until sync()."""
        self._check(self._L.hydro_step_async(self.h, float(cfl)), "step_async")

    def sync(self, check=True):
        """Wait for this grid's stream; returns the last step's dt (raises on a
        step's error status when check)."""
        dt = ctypes.c_double(0.0)
        rc = self._L.hydro_sync(self.h, ctypes.byref(dt))
        self._pending = []
        if check:
            self._check(rc, "sync")
        return dt.value

    def _dt_result(self, dt, what, check):
        if dt < 0:
            rc = self._L.hydro_last_error(self.h)
            if check:
                self._check(rc, what)
            return dt
        return dt

    def step(self, cfl, check=True):
        """One CTU step with the CFL time step; returns dt (raises on error)."""
        return self._dt_result(self._L.hydro_step(self.h, float(cfl)), "step", check)

    def step_dt(self, dt, check=True):
        """One CTU step with a given dt; returns dt (raises on error)."""
        return self._dt_result(self._L.hydro_step_dt(self.h, float(dt)), "step_dt", check)

    def compute_dt(self, cfl):
        return self._dt_result(self._L.hydro_compute_dt(self.h, float(cfl)), "compute_dt", True)

    def advance(self, cfl, t_end=math.inf, max_steps=None, check=True):
        """CFL steps until the time reaches t_end (the last step shortened to land
        on it) or max_steps steps were taken, looped on the device inside one CUDA
        graph; returns the number of steps taken (raises on error when check).
        One of t_end and max_steps must bound the run."""
        if max_steps is None:
            if math.isinf(t_end):
                raise ValueError("advance needs a finite t_end or max_steps")
            max_steps = 1 << 52
        n = ctypes.c_longlong(0)
        rc = self._L.hydro_advance(self.h, float(cfl), float(t_end), int(max_steps),
                                   ctypes.byref(n))
        if check:
            self._check(rc, "advance")
        return n.value

    def last_error(self):
        return self._L.hydro_last_error(self.h)

    def profile(self, enable=True):
        """Enable/disable per-stage CUDA-event timing; resets the totals."""
        self._check(self._L.hydro_profile(self.h, int(bool(enable))), "profile")

    def profile_read(self):
        """Per-stage totals: {stage: (ms, launches, units)} and total launches."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_longlong * n)()
        un = (ctypes.c_longlong * n)()
        tot = ctypes.c_longlong()
        self._check(self._L.hydro_profile_read(self.h, n, ms, la, un, ctypes.byref(tot)),
                    "profile_read")
        return {STAGES[k]: (ms[k], la[k], un[k]) for k in range(n)}, tot.value


def run(u0, dx, gamma, bc, nsteps=None, cfl=0.3, t_end=None, inflow=None, precision=HYDRO_FP64,
        max_steps=100000, recon=HYDRO_RECON_PPMC, solver=HYDRO_RIEMANN_EXACT, loop="device"):
    """Advance ``u0`` on the GPU; returns ``(u, t, nsteps)`` (host numpy state).
    loop="device" runs the steps inside a CUDA graph (Grid.advance); loop="host"
    takes them one call at a time; both give the same dt sequence and state."""
    _, nz, ny, nx = u0.shape
    g = Grid(nx, ny, nz, dx, gamma, bc, precision=precision, recon=recon, solver=solver)
    try:
        if inflow:
            for face, prim in inflow.items():
                g.set_inflow(face, prim)
        g.set_state(np.ascontiguousarray(u0, dtype=np.float64))
        if loop == "device":
            limit = max_steps if nsteps is None else min(nsteps, max_steps)
            steps = g.advance(cfl, math.inf if t_end is None else t_end, limit)
            return g.get_state(), g.get_time(), steps
        if loop != "host":
            raise ValueError("loop must be 'device' or 'host'")
        t, steps = 0.0, 0
        while steps < max_steps:
            if nsteps is not None and steps >= nsteps:
                break
            if t_end is not None and t >= t_end:
                break
            if t_end is None:
                dt = g.step(cfl)
                t += dt
            else:
                dt = g.compute_dt(cfl)
                last = t + dt >= t_end
                if last:
                    dt = t_end - t
                g.step_dt(dt)
                t = t_end if last else t + dt
            steps += 1
        return g.get_state(), t, steps
    finally:
        g.close()


def riemann_exact(UL, UR, gamma, F, flags=None):
    """Exact Riemann fluxes of device SoA arrays [5, n] (torch CUDA tensors)."""
    L = load()
    n = UL.shape[1]
    fp = ctypes.c_void_p(flags.data_ptr()) if flags is not None else None
    rc = L.hydro_riemann_exact(n, ctypes.c_void_p(UL.data_ptr()), ctypes.c_void_p(UR.data_ptr()),
                               float(gamma), ctypes.c_void_p(F.data_ptr()), fp, _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "riemann_exact")


def ppmc(w, dtdx, gamma, WsL, WsR):
    """PPMC of device stencils w [5 cells, 5, n] into WsL, WsR [5, n] (torch CUDA tensors)."""
    L = load()
    n = w.shape[2]
    rc = L.hydro_ppmc(n, ctypes.c_void_p(w.data_ptr()), float(dtdx), float(gamma),
                      ctypes.c_void_p(WsL.data_ptr()), ctypes.c_void_p(WsR.data_ptr()),
                      _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "ppmc")


def _check_device_f64(name, t, ndim=None, lead=None):
    """Raise ValueError unless t is a contiguous float64 CUDA tensor on the
    current device (checked before any pointer reaches a kernel)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise ValueError("%s must be float64, got %s" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if ndim is not None and (t.dim() != ndim or (lead is not None and t.shape[0] != lead)):
        raise ValueError("%s must have shape [%s, ...] with %d dimensions, got %s"
                         % (name, lead, ndim, tuple(t.shape)))
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on %s, not on the current device cuda:%d"
                         % (name, t.device, torch.cuda.current_device()))


def compute_dt_noalloc(u, dx, gamma, cfl, dt_out):
    """CFL dt of a device state u [5, nz, ny, nx] (torch CUDA float64) into the
    one-element CUDA tensor dt_out, without any device allocation; returns the
    C-ABI status code (0 on success).  A cell with rho <= 0 or a NaN gives a
    NaN dt.  Raises ValueError, before anything is launched, unless both are
    contiguous float64 tensors on the current CUDA device and u has 5 planes."""
    _check_device_f64("u", u, ndim=4, lead=5)
    _check_device_f64("dt_out", dt_out)
    if dt_out.numel() < 1:
        raise ValueError("dt_out must hold at least one element")
    L = load()
    _, nz, ny, nx = u.shape
    return L.hydro_compute_dt_noalloc(ctypes.c_void_p(u.data_ptr()), int(nx), int(ny), int(nz),
                                      float(dx), float(gamma), float(cfl),
                                      ctypes.c_void_p(dt_out.data_ptr()), _torch_stream_ptr())


def check_conversions():
    """Mismatch counts (widening, narrowing) of the library's integer-arithmetic
    float <-> double conversions against the hardware conversions."""
    L = load()
    out = (ctypes.c_ulonglong * 2)()
    rc = L.hydro_check_conversions(out, _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "check_conversions")
    return int(out[0]), int(out[1])


def probe_fp64_rate():
    """Measured FP64 throughput of the current device in flop/s (2 per fused
    multiply-add), from a kernel of independent FMA chains on every SM."""
    L = load()
    out = ctypes.c_double(0.0)
    rc = L.hydro_probe_fp64_rate(ctypes.byref(out), _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "probe_fp64_rate")
    return float(out.value)


def check_scaling():
    """Mismatch counts (halving, doubling, sign tests, float-float sums) of the
    kernels' integer-pipe helpers against the FP64 arithmetic."""
    L = load()
    out = (ctypes.c_ulonglong * 4)()
    rc = L.hydro_check_scaling(out, _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "check_scaling")
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def check_newton():
    """Largest ulp distances (reciprocal, quotient, square root, reciprocal
    square root, fifth root, square-root form) of the kernels' Newton-refined
    FP64 operations from correctly rounded references."""
    L = load()
    out = (ctypes.c_ulonglong * 6)()
    rc = L.hydro_check_newton(out, _torch_stream_ptr())
    if rc != 0:
        raise HydroError(rc, "check_newton")
    return tuple(int(v) for v in out)


def check_fastdiv():
    """Mismatches of the kernels' multiply-high index division against plain
    integer division (host-only; 0 expected)."""
    return int(load().hydro_check_fastdiv())


class Batch:
    """Independent grids of uneven sizes advanced together (see include/hydro.h)."""

    def __init__(self, grids, precision=HYDRO_FP64, recon=HYDRO_RECON_PPMC,
                 solver=HYDRO_RIEMANN_EXACT):
        """grids: list of dicts with "u" [5, nz, ny, nx], "dx", "gamma", "bc" and
        optionally "inflow" {face: prim}."""
        L = load()
        self._L = L
        n = len(grids)
        dims = (ctypes.c_int * (3 * n))()
        dx = (ctypes.c_double * n)()
        gam = (ctypes.c_double * n)()
        bc = (ctypes.c_int * (6 * n))()
        self.shapes = []
        for i, w in enumerate(grids):
            _, nz, ny, nx = w["u"].shape
            dims[3 * i:3 * i + 3] = [nx, ny, nz]
            dx[i] = float(w["dx"])
            gam[i] = float(w["gamma"])
            bc[6 * i:6 * i + 6] = [int(b) for b in w["bc"]]
            self.shapes.append((5, nz, ny, nx))
        h = ctypes.c_void_p()
        rc = L.hydro_batch_init(ctypes.byref(h), n, dims, dx, gam, bc)
        if rc != 0:
            raise HydroError(rc, "hydro_batch_init")
        self.h = h
        self.n = n
        self._pending = []
        if recon != HYDRO_RECON_PPMC:
            self._check(L.hydro_batch_set_reconstruction(h, int(recon)), "set_reconstruction")
        if solver != HYDRO_RIEMANN_EXACT:
            self._check(L.hydro_batch_set_riemann_solver(h, int(solver)), "set_riemann_solver")
        if precision != HYDRO_FP64:
            self._check(L.hydro_batch_set_precision(h, int(precision)), "set_precision")
        for i, w in enumerate(grids):
            for face, prim in (w.get("inflow") or {}).items():
                p = (ctypes.c_double * 5)(*[float(x) for x in prim])
                self._check(L.hydro_batch_set_inflow(h, i, int(face), p), "set_inflow")
            self.set_state(i, w["u"])

    def _check(self, rc, what):
        if rc != 0:
            msg = what
            if rc == -3:
                msg += ": " + self._L.hydro_batch_cuda_error_string(self.h).decode()
            raise HydroError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self._L.hydro_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, i, u):
        ptr, dev, keep = _buffer(u, self.shapes[i], False)
        self._check(self._L.hydro_batch_set_state(self.h, int(i), ptr, dev), "set_state")

    def get_state(self, i, out=None):
        if out is None:
            out = np.empty(self.shapes[i], dtype=np.float64)
        ptr, dev, keep = _buffer(out, self.shapes[i], True)
        self._check(self._L.hydro_batch_get_state(self.h, int(i), ptr, dev), "get_state")
        return out

    def set_state_async(self, i, u):
        ptr, dev, keep = _buffer(u, self.shapes[i], False)
        if keep is not u:
            raise ValueError("asynchronous copies need a C-contiguous float64 buffer (no temporary)")
        self._pending.append(u)
        self._check(self._L.hydro_batch_set_state_async(self.h, int(i), ptr, dev), "set_state_async")

    def get_state_async(self, i, out):
        ptr, dev, keep = _buffer(out, self.shapes[i], True)
        if keep is not out:
            raise ValueError("asynchronous copies need a C-contiguous float64 buffer (no temporary)")
        self._pending.append(out)
        self._check(self._L.hydro_batch_get_state_async(self.h, int(i), ptr, dev), "get_state_async")
        return out

    def step_async(self, cfl, nsteps=1):
        self._check(self._L.hydro_batch_step_async(self.h, float(cfl), int(nsteps)), "step_async")

    def sync(self):
        """Wait for the batch's stream; raises on the last step call's error status."""
        rc = self._L.hydro_batch_sync(self.h)
        self._pending = []
        self._check(rc, "sync")

    def set_stream(self, stream):
        """Order the batch's work on a torch CUDA stream (or a raw cudaStream_t)."""
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._check(self._L.hydro_batch_set_stream(self.h, ctypes.c_void_p(ptr)), "set_stream")

    def step(self, cfl, nsteps=1):
        """Advance every grid nsteps steps; returns dt [nsteps, ngrids]."""
        dt = np.zeros((nsteps, self.n))
        rc = self._L.hydro_batch_step(self.h, float(cfl), int(nsteps),
                                      dt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self._check(rc, "batch_step")
        return dt

    def autotune(self, use_cache=True):
        """Pick the launch schedule; returns (block_size, order, ms_per_step)."""
        bs, order, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._check(self._L.hydro_batch_autotune(self.h, int(bool(use_cache)), ctypes.byref(bs),
                                                 ctypes.byref(order), ctypes.byref(ms)), "autotune")
        return bs.value, order.value, ms.value

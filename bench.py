#!/usr/bin/env python
"""Throughput of the CTU + PPMC + exact-Riemann step on GB300, in cell-updates/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload sedov256]
                    [--precision fp64|mixed|strict] [--impl ours|reference] [--no-extra]

One step = one full CTU step (ghost remap, dt minimum, three PPMC sweeps, six
sets of exact Riemann solves, transverse half-step, conserved update) of every
real cell.  ``value`` = real cells x steps x ranks / max-over-ranks wall time of
the K timed steps (CUDA events on the grid's stream, barrier + synchronize on
both sides), state resident in HBM.  ``e2e`` = the same through the public API
with the state copied host->device before and device->host after every step.

The default run (Sedov 256^3, FP64, one GPU) adds to the same JSON line one
record per other form the metric names, each timed the same way with its own
clock samples: ``mixed`` and ``fp64_strict`` (Sedov 256^3), ``batched96_fp64``
and ``batched96_mixed`` (96 uneven grids), ``turbulence512_fp64/_mixed`` and
``shock_cloud_fp64/_mixed``; every mixed record carries its L1 difference to
the FP64 path from the same initial state after the same steps.

Under torchrun each rank advances its own independent replica of the workload
(the method's grids share nothing, so there is no collective on the data path:
"scaling": "weak").

``--impl reference`` times the CPU oracle (test infrastructure, plain FP64 C++)
on the host cores on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s on 1 GB300 (CTU+PPM+exact RS), FP64 vs mixed/batched at matched L1"
UNIT = "cell-updates/s"
# independent grids (or batches) the end-to-end measurement rotates over: one
# is uploaded, one steps and one is downloaded at a time
E2E_PIPELINE = 3

# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2070 MHz x 2 FP64 FMA
# per clock per SM x 2 flops per FMA (NVIDIA's nominal 1.25 TFLOP/s).
FP64_FLOPS_PEAK = 152 * 2070e6 * 2 * 2
PEAK_SOURCE = "152 SMs x 2070 MHz x 2 FP64 FMA/clk/SM x 2 flop/FMA (unit counts and clock)"

# Algorithmic FP64 flops per unit of each stage (add, multiply, divide, square
# root and pow one flop each; compares not counted): printed by
# `python oracle/count_ops.py`, the operation-counting build of the CPU reference
# run on one step of a 32^3 sample of each workload's initial-condition recipe.
# Units: padded cells (prims), real cells (slopes, ppmc, update), faces (riemann1,
# riemann2).  The benchmark never runs the oracle for these.
ALGORITHMIC_FLOPS = {
    "batched": {"ppmc": 406.0, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 81.0, "update": 45.0},
    "sedov": {"ppmc": 406.0, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 81.0, "update": 45.0},
    "sedov/pcm": {"ppmc": 0.0, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 0.0, "update": 45.0},
    "sedov/pcm+roe": {"ppmc": 0.0, "prims": 22.752, "riemann1": 305.0, "riemann2": 328.0, "slopes": 0.0, "update": 45.0},
    "sedov/plmc": {"ppmc": 108.0, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 81.0, "update": 45.0},
    "sedov/plmc+roe": {"ppmc": 108.0, "prims": 22.752, "riemann1": 305.0, "riemann2": 328.0, "slopes": 81.0, "update": 45.0},
    "sedov/plmp": {"ppmc": 107.0, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 25.0, "update": 45.0},
    "sedov/plmp+roe": {"ppmc": 107.0, "prims": 22.752, "riemann1": 305.0, "riemann2": 328.0, "slopes": 25.0, "update": 45.0},
    "sedov/ppmc+roe": {"ppmc": 406.0, "prims": 22.752, "riemann1": 305.0, "riemann2": 328.0, "slopes": 81.0, "update": 45.0},
    "sedov/ppmp": {"ppmc": 511.042, "prims": 22.752, "riemann1": 136.078, "riemann2": 196.262, "slopes": 25.0, "update": 45.0},
    "sedov/ppmp+roe": {"ppmc": 511.042, "prims": 22.752, "riemann1": 305.0, "riemann2": 328.0, "slopes": 25.0, "update": 45.0},
    "shock_cloud": {"ppmc": 413.0, "prims": 22.752, "riemann1": 135.667, "riemann2": 195.667, "slopes": 81.0, "update": 45.0},
    "sod512": {"ppmc": 406.0, "prims": 28.742, "riemann1": 136.125, "riemann2": 136.125, "slopes": 81.0, "update": 15.0},
    "turbulence": {"ppmc": 423.374, "prims": 22.752, "riemann1": 140.154, "riemann2": 200.574, "slopes": 91.922, "update": 45.0},
    "noh": {"ppmc": 428.076, "prims": 22.752, "riemann1": 207.456, "riemann2": 253.292, "slopes": 92.761, "update": 45.0},
    "noh/ppmc+roe": {"ppmc": 428.076, "prims": 22.752, "riemann1": 135.303, "riemann2": 158.299, "slopes": 92.761, "update": 45.0},
}

# The FP64 part of the mixed-precision stages, flops per unit, from the kernels'
# own FP64 arithmetic (everything else in them is float; a fused multiply-add
# counts 2): the primitive stage forms |m|^2 (1 multiply + 2 FMA), rho E -
# |m|^2/2 (1 FMA; the halving is integer arithmetic) and its product with
# (gamma-1)/rho taken in float (1 multiply), 8 flops a padded cell; the update
# converts the float-float flux sum to a double in integer arithmetic and
# applies it with 1 FMA a variable, 10 flops a cell; the Riemann stages, the
# reconstruction and the transverse half-step are float.
def mixed_fp64_flops(active_axes):
    return {"riemann2": 0, "riemann1": 0, "ppmc": 0, "update": 10, "prims": 8}

# Algorithmic HBM bytes per unit of each stage's kernel (every plane read and
# written once; stencil neighbours come from cache): FP64 intermediates are
# 8-byte planes, the mixed path's 4-byte ones.  prims: 5 conserved in, 8
# primitive planes out; slopes: 8 in, 5 out; ppmc: 8 + 5 in, 10 face states out;
# riemann1: 10 in, 5 out; riemann2: 10 face states + 2 x 5 transverse fluxes in,
# 5 out; update: 5 conserved + 3 x 5 fluxes in, 5 out.  The mixed PPMC kernel
# forms its slopes itself: 8 in, 10 out (the mixed path launches no slope pass).
ALGORITHMIC_BYTES = {
    "fp64": {"prims": 104, "slopes": 104, "ppmc": 184, "riemann1": 120, "riemann2": 200,
             "update": 200},
    "mixed": {"prims": 72, "slopes": 52, "ppmc": 72, "riemann1": 60, "riemann2": 100,
              "update": 140},
}


def mixed_bytes_per_cell_update(active_axes=3):
    """Algorithmic HBM bytes of one mixed-precision cell update: primitives and
    update once, reconstruction and both Riemann sets once per active axis
    (the PPMC kernel forms its own slopes)."""
    b = ALGORITHMIC_BYTES["mixed"]
    return b["prims"] + b["update"] + active_axes * (b["ppmc"] + b["riemann1"] + b["riemann2"])

# dram bytes (read + write) per unit of the stage's kernel from an ncu capture,
# with the digest of the sources that kernel is built from and the threads a
# block of the captured launches; a digest or block-size mismatch (the kernel
# changed since the capture) reports null.  Captured on Sedov 160^3
# (the 256^3 launches exceed the capture size rule) and scaled by the units of
# a launch: these kernels stream each plane once, so traffic grows in
# proportion to the units.  Units at 160^3: riemann2 161 x 160 x 160 faces,
# riemann1 161 x 162 x 162 faces, ppmc 162^3 cells, slopes 164 x 162 x 162
# cells, prims 168^3 padded cells, update 160^3 cells.
_FP64_SRC = ["hydro_fp64_fast.cu", "hydro_internal.h", "hydro_kernels.cuh", "hydro_math.cuh"]
_MIXED_SRC = ["hydro_ffsum.cuh", "hydro_internal.h", "hydro_kernels.cuh", "hydro_math.cuh",
              "hydro_mixed.cu"]
NCU_TRAFFIC = {
    # the x sweep (one face a thread, 207.7 B) and the y, z sweeps (segments of
    # four faces, 213.3 B)
    ("fp64", "riemann2"): {"bytes_per_unit": 211.4, "digest": "d32566f3c692a888", "bs": 128,
                           "sources": _FP64_SRC},
    # the x sweep (face values shared through the warp, 184.0 B) and the y, z
    # sweeps (segments, 200.7 B)
    ("fp64", "ppmc"): {"bytes_per_unit": 195.1, "digest": "d32566f3c692a888", "bs": 128,
                       "sources": _FP64_SRC},
    ("fp64", "riemann1"): {"bytes_per_unit": 120.4, "digest": "d32566f3c692a888", "bs": 128,
                           "sources": _FP64_SRC},
    ("fp64", "slopes"): {"bytes_per_unit": 99.5, "digest": "d32566f3c692a888", "bs": 128,
                         "sources": _FP64_SRC},
    ("mixed", "riemann2"): {"bytes_per_unit": 99.7, "digest": "ee5a686edf4a7f81", "bs": 128,
                            "sources": _MIXED_SRC},
    ("mixed", "update"): {"bytes_per_unit": 137.9, "digest": "ee5a686edf4a7f81", "bs": 128,
                          "sources": _MIXED_SRC},
    # the x sweep (one thread a cell, 62.6 B) and the y, z sweeps (segments, 64.4 B)
    ("mixed", "ppmc"): {"bytes_per_unit": 63.8, "digest": "ee5a686edf4a7f81", "bs": 128,
                        "sources": _MIXED_SRC},
    ("mixed", "riemann1"): {"bytes_per_unit": 55.1, "digest": "ee5a686edf4a7f81", "bs": 128,
                            "sources": _MIXED_SRC},
    ("mixed", "prims"): {"bytes_per_unit": 59.3, "digest": "ee5a686edf4a7f81", "bs": 128,
                         "sources": _MIXED_SRC},
}

# FP64 pipe lane-slots (warp FP64 instructions x 32) per unit of the FP64
# kernels from one-launch ncu captures with the FP64 instruction counters
# (Sedov 160^3 and Mach-5 turbulence 128^3, the same recipes as the benchmark
# workloads at a capturable size; the counts are per unit of work and depend on
# the data, not the size).  With the live launch time they give the fraction of
# the FP64 pipe's issue capacity (2 lanes a clock an SM) a kernel uses: what
# bounds the FP64 path, beside the algorithmic-flop fraction (an FMA counts 2
# flops; divisions and roots take several slots a flop).  Null once the sources
# change.
NCU_FP64_SLOTS = {
    ("sedov", "riemann2"): 177.8, ("sedov", "riemann1"): 105.1, ("sedov", "ppmc"): 75.4,
    ("sedov", "slopes"): 23.0,
    ("turbulence", "riemann2"): 250.9, ("turbulence", "riemann1"): 176.1,
    ("turbulence", "ppmc"): 113.4, ("turbulence", "slopes"): 42.0,
}
NCU_FP64_SLOTS_DIGEST = "d32566f3c692a888"


def workload(name):
    from paper_1410_4194_gb300 import workloads as W
    if name == "sedov256":
        w = W.sedov(256)
        w["desc"] = "3D Sedov-Taylor blast, 256^3 periodic, gamma 5/3, CFL 0.3"
    elif name.startswith("sedov"):
        n = int(name[5:])
        w = W.sedov(n)
        w["desc"] = "3D Sedov-Taylor blast, %d^3 periodic, gamma 5/3, CFL 0.3" % n
    elif name == "sod512":
        w = W.sod(512)
        w["desc"] = "1D Sod shock tube, 512 cells, gamma 1.4, CFL 0.3"
    elif name == "shock_cloud":
        w = W.shock_cloud()
        w["desc"] = "3D Mach-10 shock-cloud, 512x256x256, gamma 5/3, CFL 0.3"
    elif name == "turbulence":
        w = W.turbulence(512)
        w["desc"] = "3D supersonic turbulence, 512^3 periodic, rms Mach 5, CFL 0.3"
    elif name.startswith("turbulence"):
        # the same recipe on a smaller box, shells scaled with the box so that
        # the shortest wavelength keeps its 32 cells
        n = int(name[10:])
        w = W.turbulence(n, kmax=max(1, 16 * n // 512))
        w["desc"] = ("3D supersonic turbulence, %d^3 periodic, rms Mach 5, shells 1..%d, CFL 0.3"
                     % (n, max(1, 16 * n // 512)))
    elif name.startswith("noh"):
        n = int(name[3:] or 200)
        w = W.noh(n)
        w["desc"] = ("3D Noh strong shock, %d^3 octant, reflecting inner and analytic outer "
                     "faces, gamma 5/3, p0 1e-6, CFL 0.3" % n)
    elif name.startswith("batched"):
        n = int(name[7:] or 96)
        grids = W.batched(ngrids=n)
        w = dict(grids=grids, desc="%d independent 3D grids, edges from {32,48,64,96,128}, "
                                   "Sedov or x shock tube, gamma 5/3, CFL 0.3, per-grid dt" % n)
    else:
        raise SystemExit("unknown workload %s" % name)
    w["key"] = name
    return w


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x, ws, device="cuda"):
    """Maximum of a per-rank number over all ranks (identity for one rank)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(units_per_rank, steps, ws, ms_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (each rank advances its own replica)."""
    return ws * units_per_rank * steps / (ms_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


RECON_CODES = {"ppmc": 0, "ppmp": 1, "plmc": 2, "plmp": 3, "pcm": 4}
SOLVER_CODES = {"exact": 0, "roe": 1}


def flops_table(key, recon="ppmc", solver="exact"):
    """Algorithmic FP64 flops per unit for a workload key, reconstruction and
    Riemann solver (the other methods are counted on the Sedov sample)."""
    if key.startswith("sedov"):
        key = "sedov"
    elif key.startswith("turbulence"):
        key = "turbulence"
    elif key.startswith("batched"):
        key = "batched"
    elif key.startswith("noh"):
        key = "noh" if solver == "exact" else "noh/ppmc+roe"
        if recon == "ppmc":
            return ALGORITHMIC_FLOPS[key], key
    if recon != "ppmc" or solver != "exact":
        key = "sedov/%s" % recon + ("+roe" if solver == "roe" else "")
    return ALGORITHMIC_FLOPS[key], key


def run_cpu_baseline(wname, max_steps, cfl=0.3, min_seconds=10.0):
    """Oracle on the host cores, bounded sample: steps of the same IC recipe at a
    size the host finishes quickly, repeated until ``min_seconds`` have passed
    (at most ``max_steps``), so that the sample is ~10-30 s of CPU work."""
    import oracle
    from paper_1410_4194_gb300 import workloads as W
    if wname.startswith("sedov"):
        s = W.sedov(128)
        sample = "Sedov blast at 128^3 (same IC recipe as 256^3), %d oracle steps"
    elif wname == "sod512":
        s = W.sod(512)
        sample = "Sod 512 cells, %d oracle steps"
    elif wname.startswith("noh"):
        s = W.noh(64)
        sample = "Noh octant at 64^3 (same recipe), %d oracle steps"
    else:
        full = workload(wname)
        s = dict(u=np.ascontiguousarray(full["u"][:, :64, :64, :128]), dx=full["dx"],
                 gamma=full["gamma"], bc=[2, 2, 0, 0, 0, 0])
        sample = wname + " sub-block 128x64x64, %d oracle steps"
    cores = oracle.set_threads(0)
    _, nz, ny, nx = s["u"].shape
    g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
    for face, prim in (s.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    g.set_state(s["u"])
    g.step(cfl)  # untimed: first touch of the oracle's arrays
    steps = 0
    t0 = time.perf_counter()
    while steps < max(1, max_steps):
        g.step(cfl)
        steps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    el = time.perf_counter() - t0
    return {"value": nx * ny * nz * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample % steps, "seconds": el}


PRECISIONS = {"fp64": 0, "mixed": 1, "strict": 2}  # HYDRO_FP64, HYDRO_MIXED, HYDRO_FP64_STRICT
DTYPES = {"fp64": "f64", "mixed": "f32+f64", "strict": "f64"}


def timed(stream, fn, ws, local):
    """Run fn() between CUDA events on `stream` with a barrier and a
    synchronize on both sides, nvidia-smi sampling the clocks meanwhile;
    returns (max-over-ranks ms, clocks)."""
    import torch
    import torch.distributed as dist
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    return max_over_ranks(ev0.elapsed_time(ev1), ws), clocks


def fp64_peak_live(hydro):
    """Measured FP64 throughput of this device (flop/s), or None."""
    try:
        return hydro.probe_fp64_rate()
    except Exception:  # reported as unavailable, the nominal peak stands
        return None


def single_roofline(stages, precision, wkey, recon, solver, active, block_size, fp64_live,
                    sm_mhz):
    """Roofline of the dominant kernel of a single-grid run from the per-stage
    CUDA-event split: FP64 flops (FP64 and strict modes) or HBM bytes (mixed)."""
    dom = max((k for k in stages if stages[k][1] > 0), key=lambda k: stages[k][0])
    dms, dl, dunits = stages[dom]
    units_per_launch = dunits / dl
    avg_ms = dms / dl
    # the dominant stage's kernel: the reconstruction stage runs the selected
    # reconstruction's kernel, the Riemann stages the Roe kernels with roe
    if precision == "mixed":
        kname = "kb_%s_mixed" % dom
    elif precision == "strict":
        kname = "k_%s (strict)" % dom
    elif dom == "ppmc":
        # fast FP64 PPMC: face values shared through the warp along x, by
        # segments along y and z
        kname = "kb_ppmc_xs (x) / kb_ppmc_seg (y, z)" if recon == "ppmc" else "kb_" + recon
    elif dom in ("riemann1", "riemann2") and solver == "roe":
        kname = "kb_%s_roe" % dom
    elif dom == "riemann2" and active > 1:
        # the fast FP64 exact second set: one face a thread along x, by
        # segments along y and z
        kname = "kb_riemann2 (x) / kb_riemann2_seg (y, z)"
    else:
        kname = "kb_" + dom
    # captured traffic applies to the kernels captured (PPMC + exact solver, 3D
    # grids: a 1D or 2D face carries no or fewer transverse terms)
    traffic = None
    tinfo = NCU_TRAFFIC.get((precision, dom))
    if (tinfo and active == 3 and recon == "ppmc" and solver == "exact"
            and tinfo["digest"] == source_digest(tinfo["sources"])
            and tinfo["bs"] == block_size):
        traffic = tinfo["bytes_per_unit"] * units_per_launch
    bytes_per_unit = ALGORITHMIC_BYTES["mixed" if precision == "mixed" else "fp64"][dom]
    if precision != "mixed":
        # FP64 kernels: bound by the FP64 pipe (DRAM a few % busy)
        table, tkey = flops_table(wkey, recon, solver)
        per_unit = table[dom]
        achieved = per_unit * units_per_launch / (avg_ms / 1e3)
        r = {"bound": "alu", "achieved": achieved, "peak": FP64_FLOPS_PEAK,
             "unit": "FP64 FLOP/s", "frac": achieved / FP64_FLOPS_PEAK,
             "traffic": traffic, "kernel": kname, "flops_per_unit": per_unit,
             "units_per_launch": units_per_launch, "avg_launch_ms": avg_ms,
             "flops_source": "algorithmic FP64 flops per unit (oracle/count_ops.py, %s)" % tkey,
             "peak_source": PEAK_SOURCE, "bytes_per_unit_algorithmic": bytes_per_unit}
        wbase = tkey.split("/")[0]
        slots = NCU_FP64_SLOTS.get((wbase, dom))
        if (precision == "fp64" and slots and active == 3 and recon == "ppmc"
                and solver == "exact" and block_size == 128
                and NCU_FP64_SLOTS_DIGEST == source_digest(_FP64_SRC)):
            clk = (sm_mhz or 2070.0) * 1e6
            r["fp64_lane_slots_per_unit"] = slots
            r["fp64_issue_frac"] = slots * units_per_launch / (avg_ms / 1e3) / (2 * 152 * clk)
            r["fp64_issue_source"] = (
                "ncu FP64-pipe lane-slots per unit (smsp__inst_executed_pipe_fp64 x 32, "
                "%s recipe at 160^3 / 128^3) x units / live launch time, against "
                "2 lanes a clock x 152 SMs at the %s SM clock"
                % (wbase, "median sampled" if sm_mhz else "maximum"))
        if fp64_live:
            r["peak_measured"] = fp64_live
            r["frac_of_measured"] = achieved / fp64_live
            r["peak_measured_source"] = (
                "FP64 FMA throughput measured live on this GPU (hydro_probe_fp64_rate: "
                "independent FMA chains on every SM, 2 flop/FMA)"
                + (", %.2f FMA/clk/SM at the %.0f MHz median SM clock of the timed region"
                   % (fp64_live / 2 / 152 / (sm_mhz * 1e6), sm_mhz) if sm_mhz else ""))
        return r
    # mixed kernels: float arithmetic on a pipe 64x the FP64 rate, streaming
    # float planes: the roofline that bounds them is HBM bandwidth
    peak, psrc = hbm_peak_gbs()
    achieved = bytes_per_unit * units_per_launch / (avg_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kname,
            "bytes_per_unit_algorithmic": bytes_per_unit,
            "units_per_launch": units_per_launch, "avg_launch_ms": avg_ms,
            "bytes_source": "every plane the kernel reads or writes, once per unit",
            "peak_source": "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % psrc
                           if psrc == "measured" else "fallback HBM bandwidth",
            "fp64_flops_per_unit": mixed_fp64_flops(active).get(dom, 0)}


def measure_single(w, precision, steps, warmup, cfl, ws, local, recon="ppmc", solver="exact",
                   e2e=True, device_loop=True, keep_state=False, fp64_live=None):
    """Time `steps` device-resident CTU steps of one grid after `warmup` steps;
    returns the record (value, ms_per_step, clocks, roofline, stages, e2e,
    device_loop, gpu_launches) and, with keep_state, the device state right
    after the timed steps (warmup + steps steps from the initial state)."""
    import torch
    from paper_1410_4194_gb300 import hydro
    _, nz, ny, nx = w["u"].shape
    nreal = nx * ny * nz
    prec = PRECISIONS[precision]
    stream = torch.cuda.current_stream()
    g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=prec, stream=stream,
                   recon=RECON_CODES[recon], solver=SOLVER_CODES[solver])
    for face, prim in (w.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    u_host = torch.from_numpy(w["u"]).pin_memory() if e2e else None
    g.set_state(w["u"])
    for _ in range(warmup):
        g.step(cfl)
    torch.cuda.synchronize()

    # ---- timed region: K device-resident steps ------------------------------
    g.profile(True)

    def run_steps():
        for _ in range(steps):
            g.step(cfl)
    ms, clocks = timed(stream, run_steps, ws, local)
    stages, launches_total = g.profile_read()
    g.profile(False)
    rec = {"value": replicas_value(nreal, steps, ws, ms), "unit": UNIT, "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps, "precision": precision,
           "dtype": DTYPES[precision], "gpu_launches": launches_total, "clocks": clocks}
    state = None
    if keep_state:
        state = torch.empty((5, nz, ny, nx), dtype=torch.float64, device="cuda")
        g.get_state(state)

    # ---- the same K steps looped on the device (hydro_advance: one CUDA graph
    # with a WHILE node, no host round trip and no tracing events per step) ----
    if device_loop:
        g.advance(cfl, math.inf, 0)  # captures the loop graph outside the timed region
        box = {}

        def run_loop():
            box["taken"] = g.advance(cfl, math.inf, steps)
        ms_dev, _ = timed(stream, run_loop, ws, local)
        rec["device_loop"] = {"value": replicas_value(nreal, box["taken"], ws, ms_dev),
                              "unit": UNIT, "ms_per_step": ms_dev / max(box["taken"], 1),
                              "steps": box["taken"]}

    # ---- end to end through the public API with host buffers ----------------
    # Every step uploads its input state from pinned host memory, steps, and
    # downloads the resulting state.  Steps rotate over E2E_PIPELINE grids on as
    # many streams (the asynchronous API), so that the host-to-device copy of
    # one grid, the step of another and the device-to-host copy of a third run
    # at once, as a pipeline of independent problems would run.
    rec["e2e"] = None
    if e2e:
        import torch.distributed as dist
        npipe = E2E_PIPELINE
        out_host = [torch.empty_like(u_host).pin_memory() for _ in range(npipe)]
        pipe, streams = [g], [stream]
        for _ in range(npipe - 1):
            sk = torch.cuda.Stream()
            gk = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=prec,
                            stream=sk, recon=RECON_CODES[recon], solver=SOLVER_CODES[solver])
            for face, prim in (w.get("inflow") or {}).items():
                gk.set_inflow(face, prim)
            pipe.append(gk)
            streams.append(sk)

        def e2e_step(k):
            gk = pipe[k % npipe]
            gk.set_state_async(u_host)
            gk.step_async(cfl)
            gk.get_state_async(out_host[k % npipe])

        for k in range(npipe):
            e2e_step(k)
        for gk in pipe:
            gk.sync()
        ke = max(npipe, min(steps, 12))
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sk in streams[1:]:
            sk.wait_event(e0)
        for k in range(ke):
            e2e_step(k)
        for sk in streams[1:]:
            eb = torch.cuda.Event()
            eb.record(sk)
            stream.wait_event(eb)
        e1.record(stream)
        for gk in pipe:
            gk.sync()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        te = max_over_ranks(e0.elapsed_time(e1), ws)
        rec["e2e"] = {"value": replicas_value(nreal, ke, ws, te), "unit": UNIT,
                      "h2d_bytes_per_step": int(u_host.numel() * 8),
                      "d2h_bytes_per_step": int(out_host[0].numel() * 8), "steps": ke,
                      "host_wall_s": wall,
                      "pipeline": "%d grids on %d streams: one grid's upload, another's step "
                                  "and a third's download overlap" % (npipe, npipe)}
        for gk in pipe[1:]:
            gk.close()
    active = sum(1 for n in (nx, ny, nz) if n > 1)
    rec["roofline"] = single_roofline(stages, precision, w["key"], recon, solver, active,
                                      g.block_size(), fp64_live, clocks.get("sm_mhz"))
    rec["stages"] = {k: {"ms": v[0], "launches": v[1], "share": v[0] / max(ms, 1e-9)}
                     for k, v in stages.items()}
    rec["hbm"] = hbm_report(rec["value"] / ws, rec["roofline"]["traffic"],
                            rec["roofline"]["avg_launch_ms"])
    if precision == "mixed":
        rec["bytes_per_cell_update_algorithmic"] = mixed_bytes_per_cell_update(active)
    g.close()
    return rec, state


def l1_rel(a, ref):
    """Relative L1 difference per field (rho, three momenta against their
    group's scale, E) of two states [5, ...] (torch or numpy)."""
    d = [float(abs(a[q] - ref[q]).sum()) for q in range(5)]
    s = [float(abs(ref[q]).sum()) for q in range(5)]
    mom = max(s[1:4])
    den = [s[0], mom, mom, mom, s[4]]
    return [x / y if y > 0 else 0.0 for x, y in zip(d, den)]


def measure_batch(grids, desc, precision, steps, warmup, cfl, ws, local, e2e=True,
                  keep_states=False):
    """Config 5: a batch of independent grids advanced by hydro_batch_step (one
    CUDA-graph launch a call; here one step a call so that the timed region is
    exactly K steps).  Returns the record and, with keep_states, the host states
    after warmup + steps steps."""
    import torch
    import torch.distributed as dist
    from paper_1410_4194_gb300 import hydro
    ncells = sum(int(np.prod(g["u"].shape[1:])) for g in grids)
    prec = PRECISIONS[precision]
    stream = torch.cuda.Stream()
    b = hydro.Batch(grids, precision=prec)
    b.set_stream(stream)
    bs, order, tune_ms = b.autotune(use_cache=True)
    for _ in range(warmup):
        b.step(cfl, nsteps=1)
    torch.cuda.synchronize()

    def run_steps():
        for _ in range(steps):
            b.step(cfl, nsteps=1)
    ms, clocks = timed(stream, run_steps, ws, local)
    value = replicas_value(ncells, steps, ws, ms)
    states = [b.get_state(i) for i in range(len(grids))] if keep_states else None
    # end to end: every step uploads every grid's state from pinned host memory,
    # steps and downloads the states; steps rotate over E2E_PIPELINE batches on
    # as many streams (the asynchronous API), each synced once the next two
    # batches' work is queued, so that one batch's upload, another's step and a
    # third's download overlap
    e2e_rec = None
    if e2e:
        npipe = E2E_PIPELINE
        hosts = [torch.from_numpy(g["u"]).pin_memory() for g in grids]
        outs = [[torch.empty_like(x).pin_memory() for x in hosts] for _ in range(npipe)]
        pipe, streams = [b], [stream]
        for _ in range(npipe - 1):
            sk = torch.cuda.Stream()
            bk = hydro.Batch(grids, precision=prec)
            bk.set_stream(sk)
            bk.autotune(use_cache=True)
            pipe.append(bk)
            streams.append(sk)

        def e2e_step(k):
            bk = pipe[k % npipe]
            for i, x in enumerate(hosts):
                bk.set_state_async(i, x)
            bk.step_async(cfl, nsteps=1)
            for i, x in enumerate(outs[k % npipe]):
                bk.get_state_async(i, x)

        for k in range(npipe):
            e2e_step(k)
        for bk in pipe:
            bk.sync()
        ke = max(npipe, min(steps, 6))
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sk in streams[1:]:
            sk.wait_event(e0)
        for k in range(ke):
            e2e_step(k)
            if k >= npipe - 1:
                pipe[(k - npipe + 1) % npipe].sync()
        for sk in streams[1:]:
            eb = torch.cuda.Event()
            eb.record(sk)
            stream.wait_event(eb)
        e1.record(stream)
        for j in range(max(0, ke - npipe + 1), ke):
            pipe[j % npipe].sync()
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1), ws)
        e2e_rec = {"value": replicas_value(ncells, ke, ws, te), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(x.numel() * 8 for x in hosts)),
                   "d2h_bytes_per_step": int(sum(x.numel() * 8 for x in outs[0])), "steps": ke,
                   "pipeline": "%d batches on %d streams: one batch's upload, another's step "
                               "and a third's download overlap" % (npipe, npipe)}
        for bk in pipe[1:]:
            bk.close()
    b.close()
    # kernels of one step of the graph (3D grids): primitives + dt, update, and
    # per axis the slope pass (none in mixed precision, whose PPMC kernel forms
    # its own slopes), reconstruction and the two Riemann sets
    slope_pass = 0 if precision == "mixed" else 1
    launches_per_step = 3 + 3 * (3 + slope_pass)
    # step-level roofline (the graph's kernels are not timed one by one):
    # FP64 flops of a cell update times the cell-update rate
    if precision == "fp64":
        pu = ALGORITHMIC_FLOPS["batched"]
        per_cell = (pu["prims"] + 3 * (pu["slopes"] + pu["ppmc"] + pu["riemann1"]
                                       + pu["riemann2"]) + pu["update"])
        achieved = per_cell * value / ws
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_FLOPS_PEAK,
                    "unit": "FP64 FLOP/s", "frac": achieved / FP64_FLOPS_PEAK, "traffic": None,
                    "kernel": "whole step (graph)", "flops_per_cell_update": per_cell,
                    "flops_source": "algorithmic FP64 flops per cell update "
                                    "(oracle/count_ops.py, Sedov sample)",
                    "peak_source": PEAK_SOURCE}
    else:
        per_cell = mixed_bytes_per_cell_update(3)
        achieved = per_cell * value / ws / 1e9
        peak, psrc = hbm_peak_gbs()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None, "kernel": "whole step (graph)",
                    "bytes_per_cell_update": per_cell,
                    "bytes_source": "algorithmic HBM bytes of the mixed-precision kernels per "
                                    "cell update",
                    "peak_source": "%s HBM copy bandwidth" % psrc}
    rec = {"value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps, "precision": precision, "dtype": DTYPES[precision],
           "config": {"workload": desc, "cells": ncells, "grids": len(grids),
                      "precision": precision, "schedule": {"block": bs, "order": order},
                      "l2": "inputs larger than L2 (states %.2f GB)" % (ncells * 40 / 1e9)},
           "e2e": e2e_rec, "gpu_launches": launches_per_step * steps, "clocks": clocks,
           "hbm": hbm_report(value / ws), "roofline": roofline}
    return rec, states


def extra_records(args, ws, local, main_state, fp64_live):
    """The other forms the metric names, each measured on this GPU right after
    the headline line and carried in the same JSON line: mixed precision and
    the strict FP64 mode on the same Sedov 256^3 workload, the 96-grid batch in
    FP64 and mixed precision, and the FP64 and mixed paths on the two harder
    workloads (Mach-5 turbulence 512^3, Mach-10 shock-cloud 512x256x256), each
    with the L1 difference of mixed to FP64 from the same initial state after
    the same steps.  Fewer steps on the large workloads (stated per record)."""
    import torch
    out = {}
    wu = 3 if args.warmup >= 3 else args.warmup
    sed = workload("sedov256")
    # mixed, same steps as the headline: L1 against the headline's FP64 state
    rec, st = measure_single(sed, "mixed", args.steps, args.warmup, args.cfl, ws, local,
                             keep_state=True)
    rec["config"] = single_config("sedov256", "mixed", ws)
    rec["l1_vs_fp64"] = {"steps": args.warmup + args.steps,
                         "fields": ["rho", "mx", "my", "mz", "E"],
                         "l1_rel": l1_rel(st, main_state),
                         "reference": "HYDRO_FP64 GPU path (the headline run) from the same "
                                      "initial state after the same steps"}
    out["mixed"] = rec
    del st
    # strict FP64: the printed formulas in the oracle's operation order
    ks = min(args.steps, 5)
    rec, _ = measure_single(sed, "strict", ks, wu, args.cfl, ws, local, e2e=False,
                            device_loop=False, fp64_live=fp64_live)
    rec["config"] = single_config("sedov256", "strict", ws)
    out["fp64_strict"] = rec
    del sed
    torch.cuda.empty_cache()
    # the 96-grid batch (config 5)
    bw = workload("batched96")
    kb = min(args.steps, 10)
    rec64, s64 = measure_batch(bw["grids"], bw["desc"], "fp64", kb, wu, args.cfl, ws, local,
                               keep_states=True)
    out["batched96_fp64"] = rec64
    recm, sm = measure_batch(bw["grids"], bw["desc"], "mixed", kb, wu, args.cfl, ws, local,
                             keep_states=True)
    per_grid = np.array([l1_rel(a, c) for a, c in zip(sm, s64)])
    worst = int(np.argmax(per_grid[:, 0]))
    recm["l1_vs_fp64"] = {"steps": wu + kb, "fields": ["rho", "mx", "my", "mz", "E"],
                          "per_grid_max": per_grid.max(axis=0).tolist(),
                          "per_grid_median": np.median(per_grid, axis=0).tolist(),
                          "worst_grid_rho": worst,
                          "reference": "HYDRO_FP64 batch from the same initial states after "
                                       "the same steps"}
    out["batched96_mixed"] = recm
    del bw, s64, sm
    # the two large workloads, FP64 and mixed from the same initial state
    for name in ("turbulence", "shock_cloud"):
        wl = workload(name)
        kl = min(args.steps, 5)
        r64, s64 = measure_single(wl, "fp64", kl, wu, args.cfl, ws, local, e2e=False,
                                  device_loop=False, keep_state=True, fp64_live=fp64_live)
        r64["config"] = single_config(name, "fp64", ws)
        rmx, smx = measure_single(wl, "mixed", kl, wu, args.cfl, ws, local, e2e=False,
                                  device_loop=False, keep_state=True)
        rmx["config"] = single_config(name, "mixed", ws)
        rmx["l1_vs_fp64"] = {"steps": wu + kl, "fields": ["rho", "mx", "my", "mz", "E"],
                             "l1_rel": l1_rel(smx, s64),
                             "reference": "HYDRO_FP64 GPU path from the same initial state "
                                          "after the same steps"}
        key = "turbulence512" if name == "turbulence" else "shock_cloud"
        out[key + "_fp64"] = r64
        out[key + "_mixed"] = rmx
        del wl, s64, smx
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sedov256")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "strict"])
    ap.add_argument("--recon", default="ppmc", choices=list(RECON_CODES),
                    help="reconstruction (Sec. 2.2.1): ppmc (default), ppmp, plmc, plmp, pcm")
    ap.add_argument("--solver", default="exact", choices=["exact", "roe"],
                    help="Riemann solver (Sec. 2.2.2): exact (default) or roe (HLLE fallback, "
                         "H correction)")
    ap.add_argument("--cfl", type=float, default=0.3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="the headline line only (no mixed, strict, batched, turbulence and "
                         "shock-cloud records)")
    ap.add_argument("--cpu-steps", type=int, default=1000,
                    help="cap on the oracle steps of the CPU baseline (it stops after 10 s)")
    ap.add_argument("--compare-l1", action="store_true",
                    help="mixed precision: also run the FP64 path from the same state for the "
                         "same steps and report the L1 difference per field")
    args = ap.parse_args()
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist
    from paper_1410_4194_gb300 import hydro

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    w = workload(args.workload)
    if "grids" in w:
        return run_batch(args, w, ws, rank)
    fp64_live = fp64_peak_live(hydro) if args.precision != "mixed" else None
    # the sub-records run after the headline default (Sedov 256^3, FP64, PPMC +
    # exact) on one GPU; under torchrun every rank times the headline only
    extras = (not args.no_extra and ws == 1 and args.workload == "sedov256"
              and args.precision == "fp64" and args.recon == "ppmc" and args.solver == "exact")
    rec, state = measure_single(w, args.precision, args.steps, args.warmup, args.cfl, ws, local,
                                recon=args.recon, solver=args.solver, e2e=not args.no_e2e,
                                keep_state=extras, fp64_live=fp64_live)
    l1 = None
    if args.compare_l1 and args.precision == "mixed":
        l1 = compare_l1(w, args, hydro)
    extra = extra_records(args, ws, local, state, fp64_live) if extras else {}
    del state
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args.workload, args.cpu_steps, args.cfl)
    line = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
        "config": single_config(args.workload, args.precision, ws, args.recon, args.solver),
        "e2e": rec["e2e"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
        "roofline": rec["roofline"], "device_loop": rec.get("device_loop"),
        "stages": rec["stages"], "cpu_baseline": cpu, "hbm": rec["hbm"],
    }
    if l1 is not None:
        line["l1_vs_fp64"] = l1
    line.update(extra)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_batch(args, w, ws, rank):
    """The batched workload as the headline line (--workload batchedN)."""
    import torch.distributed as dist
    _, _, local = dist_env()
    rec, _ = measure_batch(w["grids"], w["desc"], args.precision, args.steps, args.warmup,
                           args.cfl, ws, local, e2e=not args.no_e2e,
                           keep_states=args.compare_l1 and args.precision == "mixed")
    l1 = None
    if args.compare_l1 and args.precision == "mixed":
        from paper_1410_4194_gb300 import hydro
        res = {}
        for name, pr in (("mixed", hydro.HYDRO_MIXED), ("fp64", hydro.HYDRO_FP64)):
            bb = hydro.Batch(w["grids"], precision=pr)
            bb.step(args.cfl, nsteps=args.warmup + args.steps)
            res[name] = [bb.get_state(i) for i in range(len(w["grids"]))]
            bb.close()
        d = sum(np.abs(a - c).reshape(5, -1).sum(axis=1) for a, c in zip(res["mixed"], res["fp64"]))
        s_ = sum(np.abs(c).reshape(5, -1).sum(axis=1) for c in res["fp64"])
        mom = s_[1:4].max()
        l1 = {"steps": args.warmup + args.steps, "fields": ["rho", "mx", "my", "mz", "E"],
              "l1_rel": list(d / np.array([s_[0], mom, mom, mom, s_[4]])),
              "reference": "HYDRO_FP64 batch from the same initial states"}
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cfg = dict(rec["config"])
    cfg["parallelism"] = "replicas" if ws > 1 else "single"
    line = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
        "config": cfg, "e2e": rec["e2e"], "gpu_launches": rec["gpu_launches"],
        "clocks": rec["clocks"], "hbm": rec["hbm"], "roofline": rec["roofline"],
        "cpu_baseline": None,
    }
    if l1 is not None:
        line["l1_vs_fp64"] = l1
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline("sedov", args.cpu_steps, args.cfl)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def compare_l1(w, args, hydro):
    """Run the mixed and the FP64 path from the workload's initial state for
    warmup + steps steps and report the relative L1 difference per field (the
    momenta against their group's scale)."""
    import torch
    _, nz, ny, nx = w["u"].shape
    n = args.warmup + args.steps
    stream = torch.cuda.current_stream()
    res = {}
    for name, prec in (("mixed", hydro.HYDRO_MIXED), ("fp64", hydro.HYDRO_FP64)):
        h = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=prec, stream=stream)
        for face, prim in (w.get("inflow") or {}).items():
            h.set_inflow(face, prim)
        h.set_state(w["u"])
        for _ in range(n):
            h.step(args.cfl)
        out = torch.empty((5, nz, ny, nx), dtype=torch.float64, device="cuda")
        h.get_state(out)
        h.close()
        res[name] = out
    return {"steps": n, "fields": ["rho", "mx", "my", "mz", "E"],
            "l1_rel": l1_rel(res["mixed"], res["fp64"]),
            "reference": "HYDRO_FP64 GPU path from the same initial state"}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine's GB300 (MEASURED_PEAKS.json), else
    the fallback measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def hbm_report(cells_per_s, kernel_traffic=None, kernel_ms=None):
    """HBM roofline of the step (80 B per cell update: the FP64 conserved state
    read once and written once) and, when known, the dominant kernel's DRAM rate."""
    peak, src = hbm_peak_gbs()
    out = {"bytes_per_cell_update": 80, "achieved_gbs": cells_per_s * 80 / 1e9,
           "peak_gbs": peak, "peak_source": src, "frac": cells_per_s * 80 / 1e9 / peak}
    if kernel_traffic is not None and kernel_ms:
        gbs = kernel_traffic / (kernel_ms / 1e3) / 1e9
        out["dominant_kernel_dram_gbs"] = gbs
        out["dominant_kernel_dram_frac"] = gbs / peak
    return out


def source_digest(files):
    """Digest of the kernel sources (paths under the package's csrc/)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_4194_gb300", "csrc")
    for f in sorted(files):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def run_reference(args, ws, rank):
    """The oracle timed on the host cores (rank 0 only), each step a bounded
    sample of the workload: Sedov at 128^3 (same recipe), Sod in full, a
    128x64x64 block of the large fields, the first grids of a batch."""
    if rank != 0:
        return
    import oracle
    from paper_1410_4194_gb300 import workloads as W
    if args.workload.startswith("batched"):
        grids, cells = [], 0
        for gw in workload(args.workload)["grids"]:
            grids.append(gw)
            cells += int(np.prod(gw["u"].shape[1:]))
            if cells >= 1 << 20:
                break
        samples = grids
        sample = "the first %d grids of the batch (%d cells), one oracle step each per step" % (
            len(grids), cells)
        config = {"workload": workload(args.workload)["desc"], "precision": args.precision,
                  "parallelism": "replicas" if ws > 1 else "single"}
    else:
        if args.workload.startswith("sedov"):
            s = W.sedov(128)
            sample = ("Sedov blast at 128^3 (same IC recipe as the %s workload), one oracle step "
                      "per step" % args.workload)
        elif args.workload == "sod512":
            s = W.sod(512)
            sample = "Sod 512 cells, one oracle step per step"
        elif args.workload.startswith("noh"):
            s = W.noh(64)
            sample = ("Noh octant at 64^3 (same recipe as the %s workload), one oracle step per "
                      "step" % args.workload)
        else:
            full = workload(args.workload)
            s = dict(u=np.ascontiguousarray(full["u"][:, :64, :64, :128]), dx=full["dx"],
                     gamma=full["gamma"], bc=[2, 2, 0, 0, 0, 0])
            sample = "%s sub-block 128x64x64, one oracle step per step" % args.workload
        samples = [s]
        config = single_config(args.workload, args.precision, ws)
    cores = oracle.set_threads(0)
    gs, cells = [], 0
    for s in samples:
        _, nz, ny, nx = s["u"].shape
        g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
        for face, prim in (s.get("inflow") or {}).items():
            g.set_inflow(face, prim)
        g.set_state(s["u"])
        gs.append(g)
        cells += nx * ny * nz
    for _ in range(args.warmup):
        for g in gs:
            g.step(args.cfl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for g in gs:
            g.step(args.cfl)
    el = time.perf_counter() - t0
    value = cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOAD_DESC = {
    "sod512": "1D Sod shock tube, 512 cells, gamma 1.4, CFL 0.3",
    "shock_cloud": "3D Mach-10 shock-cloud, 512x256x256, gamma 5/3, CFL 0.3",
    "turbulence": "3D supersonic turbulence, 512^3 periodic, rms Mach 5, CFL 0.3",
}


def workload_shape(name):
    """(nx, ny, nz) of a single-grid workload without building it."""
    if name.startswith("sedov"):
        n = int(name[5:])
        return n, n, n
    if name.startswith("noh"):
        n = int(name[3:] or 200)
        return n, n, n
    if name.startswith("turbulence") and name != "turbulence":
        n = int(name[10:])
        return n, n, n
    return {"sod512": (512, 1, 1), "shock_cloud": (512, 256, 256),
            "turbulence": (512, 512, 512)}[name]


def workload_desc(name):
    if name.startswith("sedov"):
        n = int(name[5:])
        return "3D Sedov-Taylor blast, %d^3 periodic, gamma 5/3, CFL 0.3" % n
    if name.startswith("noh"):
        n = int(name[3:] or 200)
        return ("3D Noh strong shock, %d^3 octant, reflecting inner and analytic outer faces, "
                "gamma 5/3, p0 1e-6, CFL 0.3" % n)
    if name.startswith("turbulence") and name != "turbulence":
        n = int(name[10:])
        return ("3D supersonic turbulence, %d^3 periodic, rms Mach 5, shells 1..%d, CFL 0.3"
                % (n, max(1, 16 * n // 512)))
    return WORKLOAD_DESC.get(name, name)


def single_config(name, precision, ws, recon="ppmc", solver="exact"):
    nx, ny, nz = workload_shape(name)
    return {"workload": workload_desc(name), "cells": nx * ny * nz, "precision": precision,
            "reconstruction": recon, "riemann_solver": solver,
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (state %.2f GB, step working set %.1f GB)" % (
                nx * ny * nz * 40 / 1e9,
                (nx + 8) * (ny + 8 if ny > 1 else 1) * (nz + 8 if nz > 1 else 1) * 8 * 56 / 1e9)}


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Throughput of the CTU + PPMC + exact-Riemann step on GB300, in cell-updates/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload sedov256]
                    [--precision fp64|mixed] [--impl ours|reference]

One step = one full CTU step (ghost remap, dt minimum, three PPMC sweeps, six
sets of exact Riemann solves, transverse half-step, conserved update) of every
real cell.  ``value`` = real cells x steps x ranks / max-over-ranks wall time of
the K timed steps (CUDA events on the grid's stream, barrier + synchronize on
both sides), state resident in HBM.  ``e2e`` = the same through the public API
with the state copied host->device before and device->host after every step.

Under torchrun each rank advances its own independent replica of the workload
(the method's grids share nothing, so there is no collective on the data path:
"scaling": "weak").

``--impl reference`` times the CPU oracle (test infrastructure, plain FP64 C++)
on the host cores on a bounded sample of the same workload.
"""
import argparse
import json
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

# FP64 issue rate of GB300 derived from unit counts and clock: 152 SMs x 2070 MHz x
# 2 FP64 FMA instructions per clock per SM (NVIDIA's nominal 1.25 TFLOP/s counts an
# FMA as two flops).  The algorithmic count below counts every add, multiply,
# divide, square root, pow and compare as one operation.
FP64_OPS_PEAK = 152 * 2070e6 * 2
FP32_OPS_PEAK = 152 * 2070e6 * 128

# dram bytes (read + write) per launch from an ncu capture, per stage, with the
# kernel source digest they were taken on; a digest mismatch reports null.
NCU_TRAFFIC = {}

ORACLE_STAGE = {"prims": "prims", "slopes": "slopes", "ppmc": "ppmc", "riemann1": "riemann1",
                "riemann2": "riemann2", "update": "update"}


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


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_ops(w, cfl):
    """Per-unit algorithmic FP64 operation counts of each stage, measured by the
    op-counting oracle on a 32^3 sample of the same problem (same IC recipe)."""
    import oracle
    from paper_1410_4194_gb300 import workloads as W
    key = w["key"]
    if key.startswith("sedov") or key.startswith("batched"):
        s = W.sedov(32)
    elif key == "sod512":
        s = W.sod(512)
    else:
        s = dict(u=w["u"][:, :32, :32, :32].copy(), dx=w["dx"], gamma=w["gamma"], bc=[0] * 6)
    _, nz, ny, nx = s["u"].shape
    g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
    for face, prim in (s.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    g.set_state(s["u"])
    dt = g.compute_dt(cfl)
    st = g.count_step_stages(dt)
    out = {}
    for k, v in st.items():
        tot = sum(v["ops"].values())
        out[k] = tot / max(v["units"], 1)
    return out, "op-counting oracle on %dx%dx%d %s, one step" % (nx, ny, nz, key)


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
    else:
        full = workload(wname)
        s = dict(u=np.ascontiguousarray(full["u"][:, :64, :64, :128]), dx=full["dx"],
                 gamma=full["gamma"], bc=[2, 2, 0, 0, 0, 0])
        sample = wname + " sub-block 128x64x64, %d oracle steps"
    cores = oracle.set_threads(0)
    _, nz, ny, nx = s["u"].shape
    g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sedov256")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cfl", type=float, default=0.3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
        return run_batch(args, w, ws, rank, local)
    _, nz, ny, nx = w["u"].shape
    nreal = nx * ny * nz
    prec = hydro.HYDRO_FP64 if args.precision == "fp64" else hydro.HYDRO_MIXED
    stream = torch.cuda.current_stream()
    g = hydro.Grid(nx, ny, nz, w["dx"], w["gamma"], w["bc"], precision=prec, stream=stream)
    for face, prim in (w.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    u_host = torch.from_numpy(w["u"]).pin_memory()
    g.set_state(u_host.numpy())
    for _ in range(args.warmup):
        g.step(args.cfl)
    torch.cuda.synchronize()

    # ---- timed region: K device-resident steps ------------------------------
    g.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.step(args.cfl)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    stages, launches_total = g.profile_read()
    g.profile(False)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * nreal * args.steps / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty_like(u_host).pin_memory()
        ke = max(1, min(args.steps, 5))
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            g.set_state(u_host.numpy())
            g.step(args.cfl)
            g.get_state(out_host.numpy())
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        te = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * nreal * ke / (float(te.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(u_host.numel() * 8),
               "d2h_bytes_per_step": int(out_host.numel() * 8), "steps": ke,
               "host_wall_s": wall}

    l1 = None
    if args.compare_l1 and args.precision == "mixed":
        l1 = compare_l1(w, args, g, hydro, stream)
    if rank != 0:
        g.close()
        if ws > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel -------------------------------------
    dom = max((k for k in stages if stages[k][1] > 0), key=lambda k: stages[k][0])
    dms, dl, dunits = stages[dom]
    per_unit, count_src = algorithmic_ops(w, args.cfl)
    ops_per_launch = per_unit[ORACLE_STAGE[dom]] * dunits / dl
    avg_ms = dms / dl
    achieved = ops_per_launch / (avg_ms / 1e3)
    peak = FP64_OPS_PEAK if args.precision == "fp64" else FP32_OPS_PEAK
    traffic = None
    tinfo = NCU_TRAFFIC.get(dom)
    if tinfo and tinfo.get("digest") == kernel_digest():
        traffic = tinfo["bytes_per_launch"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP64 op/s"
                if args.precision == "fp64" else "FP32 op/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_" + dom,
                "ops_per_launch": ops_per_launch, "avg_launch_ms": avg_ms,
                "ops_source": count_src,
                "peak_source": "152 SMs x 2070 MHz x 2 FP64 FMA/clk/SM (unit counts and clock)"}
    stage_report = {k: {"ms": v[0], "launches": v[1], "share": v[0] / max(ms, 1e-9)}
                    for k, v in stages.items()}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args.workload, args.cpu_steps, args.cfl)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": w["desc"], "cells": nreal, "precision": args.precision,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (state %.2f GB, step working set %.1f GB)" % (
                       nreal * 40 / 1e9, (nx + 8) * (ny + 8) * (nz + 8) * 8 * 56 / 1e9)},
        "e2e": e2e, "gpu_launches": launches_total, "clocks": clocks, "roofline": roofline,
        "stages": stage_report, "cpu_baseline": cpu,
    }
    if l1 is not None:
        line["l1_vs_fp64"] = l1
    print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        dist.destroy_process_group()


def run_batch(args, w, ws, rank, local):
    """Config 5: a batch of independent grids advanced by hydro_batch_step (one
    CUDA-graph launch a call; here one step a call so that the timed region is
    exactly K steps)."""
    import torch
    import torch.distributed as dist
    from paper_1410_4194_gb300 import hydro
    grids = w["grids"]
    ncells = sum(int(np.prod(g["u"].shape[1:])) for g in grids)
    prec = hydro.HYDRO_FP64 if args.precision == "fp64" else hydro.HYDRO_MIXED
    stream = torch.cuda.Stream()
    b = hydro.Batch(grids, precision=prec)
    b._check(b._L.hydro_batch_set_stream(b.h, hydro.ctypes.c_void_p(stream.cuda_stream)),
             "set_stream")
    bs, order, tune_ms = b.autotune(use_cache=True)
    for _ in range(args.warmup):
        b.step(args.cfl, nsteps=1)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.step(args.cfl, nsteps=1)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * ncells * args.steps / (ms_max / 1e3)
    e2e = None
    if not args.no_e2e:
        hosts = [torch.from_numpy(g["u"]).pin_memory() for g in grids]
        outs = [torch.empty_like(x).pin_memory() for x in hosts]
        ke = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            for i, x in enumerate(hosts):
                b.set_state(i, x.numpy())
            b.step(args.cfl, nsteps=1)
            for i, x in enumerate(outs):
                b.get_state(i, x.numpy())
        e1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": ws * ncells * ke / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(x.numel() * 8 for x in hosts)),
               "d2h_bytes_per_step": int(sum(x.numel() * 8 for x in outs)), "steps": ke}
    l1 = None
    if args.compare_l1 and args.precision == "mixed":
        res = {}
        for name, pr in (("mixed", hydro.HYDRO_MIXED), ("fp64", hydro.HYDRO_FP64)):
            bb = hydro.Batch(grids, precision=pr)
            bb.step(args.cfl, nsteps=args.warmup + args.steps)
            res[name] = [bb.get_state(i) for i in range(len(grids))]
            bb.close()
        d = sum(np.abs(a - c).reshape(5, -1).sum(axis=1) for a, c in zip(res["mixed"], res["fp64"]))
        s_ = sum(np.abs(c).reshape(5, -1).sum(axis=1) for c in res["fp64"])
        mom = s_[1:4].max()
        l1 = {"steps": args.warmup + args.steps, "fields": ["rho", "mx", "my", "mz", "E"],
              "l1_rel": list(d / np.array([s_[0], mom, mom, mom, s_[4]])),
              "reference": "HYDRO_FP64 batch from the same initial states"}
    b.close()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    # step-level roofline: algorithmic FP64 operations of a cell update
    # (op-counting oracle, Sedov sample) times the cell-update rate
    per_unit, count_src = algorithmic_ops(dict(key="sedov32"), args.cfl)
    per_cell = (per_unit["prims"] + 3 * (per_unit["slopes"] + per_unit["ppmc"] + per_unit["riemann1"]
                                        + per_unit["riemann2"]) + per_unit["update"])
    achieved = per_cell * value / ws
    peak = FP64_OPS_PEAK if args.precision == "fp64" else FP32_OPS_PEAK
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": w["desc"], "cells": ncells, "grids": len(grids),
                   "precision": args.precision, "schedule": {"block": bs, "order": order},
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (states %.2f GB)" % (ncells * 40 / 1e9)},
        "e2e": e2e, "gpu_launches": 15 * args.steps, "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "FP64 op/s" if args.precision == "fp64" else "FP32 op/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "whole step (graph)",
                     "ops_per_cell_update": per_cell, "ops_source": count_src},
        "cpu_baseline": None,
    }
    if l1 is not None:
        line["l1_vs_fp64"] = l1
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline("sedov", args.cpu_steps, args.cfl)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def compare_l1(w, args, g, hydro, stream):
    """Run the mixed and the FP64 path from the workload's initial state for
    warmup + steps steps and report the relative L1 difference per field (the
    momenta against their group's scale)."""
    import torch
    _, nz, ny, nx = w["u"].shape
    n = args.warmup + args.steps
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
    d = (res["mixed"] - res["fp64"]).abs().reshape(5, -1).sum(dim=1)
    s = res["fp64"].abs().reshape(5, -1).sum(dim=1)
    mom = s[1:4].max()
    den = torch.stack([s[0], mom, mom, mom, s[4]])
    l1 = (d / den).tolist()
    return {"steps": n, "fields": ["rho", "mx", "my", "mz", "E"], "l1_rel": l1,
            "reference": "HYDRO_FP64 GPU path from the same initial state"}


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_4194_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def run_reference(args, ws, rank):
    """The oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    from paper_1410_4194_gb300 import workloads as W
    if args.workload.startswith("sedov"):
        s = W.sedov(128)
        sample = "Sedov blast at 128^3 (same IC recipe as the 256^3 workload), one oracle step per step"
    elif args.workload == "sod512":
        s = W.sod(512)
        sample = "Sod 512 cells"
    else:
        full = workload(args.workload)
        s = dict(u=np.ascontiguousarray(full["u"][:, :64, :64, :128]), dx=full["dx"],
                 gamma=full["gamma"], bc=[2, 2, 0, 0, 0, 0])
        sample = "%s sub-block 128x64x64" % args.workload
    cores = oracle.set_threads(0)
    _, nz, ny, nx = s["u"].shape
    g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
    g.set_state(s["u"])
    for _ in range(args.warmup):
        g.step(args.cfl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.step(args.cfl)
    el = time.perf_counter() - t0
    value = nx * ny * nz * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload), "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_desc(name):
    return {"sedov256": "3D Sedov-Taylor blast, 256^3 periodic, gamma 5/3, CFL 0.3",
            "sod512": "1D Sod shock tube, 512 cells, gamma 1.4, CFL 0.3"}.get(name, name)


if __name__ == "__main__":
    main()

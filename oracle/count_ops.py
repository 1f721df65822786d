"""Algorithmic operation counts per unit of work of each stage of the CTU step
-- TEST INFRASTRUCTURE.  Prints the table that bench.py holds as
ALGORITHMIC_FLOPS (the benchmark itself never runs the oracle for it):

    python oracle/count_ops.py

For each benchmark workload (and, on the Sedov sample, each other
reconstruction and the Roe solver) the op-counting build of the CPU oracle runs one
step of a 32^3 sample of the same initial-condition recipe (Sedov: a 32^3 blast
made the same way; shock-cloud and turbulence: the 32^3 corner block of the
full field; Sod: the full 512 cells) and counts every add, multiply, divide,
square root and pow as one floating-point operation (flop) and every compare
separately.  Units: padded cells for the
primitive stage (incl. the dt minimum), real cells for the slope and PPMC
stages and the update, faces for the two Riemann stages.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1410_4194_gb300 import workloads as W  # noqa: E402


def sample(name):
    if name in ("sedov", "batched"):
        return W.sedov(32), "Sedov blast 32^3, same recipe"
    if name == "noh":
        return W.noh(32), "Noh octant 32^3, same recipe"
    if name == "sod512":
        return W.sod(512), "Sod 512 cells"
    full = W.shock_cloud() if name == "shock_cloud" else W.turbulence(512)
    s = dict(u=np.ascontiguousarray(full["u"][:, :32, :32, :32]), dx=full["dx"],
             gamma=full["gamma"], bc=[0] * 6)
    return s, "32^3 corner block of the full field, periodic"


def counts(name, cfl=0.3, recon=oracle.RECON_PPMC, solver=oracle.SOLVER_EXACT):
    s, desc = sample(name)
    _, nz, ny, nx = s["u"].shape
    g = oracle.Grid(nx, ny, nz, s["dx"], s["gamma"], s["bc"])
    g.set_recon(recon)
    g.set_solver(solver)
    for face, prim in (s.get("inflow") or {}).items():
        g.set_inflow(face, prim)
    g.set_state(s["u"])
    st = g.count_step_stages(g.compute_dt(cfl))
    flops = {k: (sum(v["ops"].values()) - v["ops"]["cmp"]) / max(v["units"], 1)
             for k, v in st.items()}
    cmps = {k: v["ops"]["cmp"] / max(v["units"], 1) for k, v in st.items()}
    return {"flops_per_unit": flops, "compares_per_unit": cmps, "sample": desc}


def main():
    out = {name: counts(name) for name in ("sedov", "sod512", "shock_cloud", "turbulence", "noh")}
    out["batched"] = out["sedov"]
    out["noh/ppmc+roe"] = counts("noh", solver=oracle.SOLVER_ROE)
    recons = {"ppmp": oracle.RECON_PPMP, "plmc": oracle.RECON_PLMC, "plmp": oracle.RECON_PLMP,
              "pcm": oracle.RECON_PCM}
    for rname, r in recons.items():
        out["sedov/" + rname] = counts("sedov", recon=r)
    recons["ppmc"] = oracle.RECON_PPMC
    for rname, r in recons.items():
        out["sedov/%s+roe" % rname] = counts("sedov", recon=r, solver=oracle.SOLVER_ROE)
    json.dump(out, sys.stdout, indent=1, sort_keys=True)
    sys.stdout.write("\n")


if __name__ == "__main__":
    main()

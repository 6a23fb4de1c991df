"""Run one of the synthetic workloads through the C ABI and print its throughput.

    python -m paper_2605_22214_gb300.run WORKLOAD [--precision fp32] [--steps 50] [--size N]

WORKLOAD is one of: spinodal (D2Q9, N = 4, size^2), janus3d (D3Q19, N = 4, size^3),
lens (D2Q9, N = 3, size^2, walls in y), poiseuille3d (D3Q19, N = 7, 32 x 32 x 192),
porous (D2Q9, N = 4, (4 size) x size channel through solid posts, inlet and outflow),
porous3d (D3Q19, N = 4, size^3 block of solid cubes and a slab with a window, walls in z),
emulsion (D2Q9, N = 4, the 600 x 140 emulsion generator),
pals (D2Q9, N = 4, the 400 x 140 patterned liquid surface),
batch (--sims D2Q9 lens/Janus simulations of mixed size and N in one batch, FP32;
--mode persistent | per_step | auto).
The time is taken with CUDA events around the steps, after three warm-up steps.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make(name, size):
    import nfe_workloads as W
    if name == "spinodal":
        return W.spinodal_2d(nx=size, ny=size)
    if name == "janus3d":
        return W.janus_3d(n=size)
    if name == "lens":
        return W.lens_2d(nx=size, ny=size, radius=12.0 * size / 64.0)
    if name == "poiseuille3d":
        return W.layered_poiseuille()
    if name == "porous":
        return W.porous_channel_2d(nx=4 * size, ny=size)
    if name == "porous3d":
        return W.porous_3d(size, size, size, 4, walls=(False, False, True))
    if name == "emulsion":
        return W.emulsion_2d()
    if name == "pals":
        return W.pals_2d()
    raise SystemExit(f"unknown workload {name}")


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("workload")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "f16", "bf16"])
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--variant", type=int, default=-1, help="tile shape (-1: autotune)")
    ap.add_argument("--tau-g", type=float, default=1.0, help="relaxation time of the component populations")
    ap.add_argument("--sims", type=int, default=512, help="batch: number of simulations")
    ap.add_argument("--mode", default="auto", choices=["persistent", "per_step", "auto"], help="batch: launch form")
    args = ap.parse_args()
    import torch

    import paper_2605_22214_gb300 as nfe
    from paper_2605_22214_gb300 import build
    build.build()
    if args.workload == "batch":
        return run_batch(nfe, torch, args)
    p = make(args.workload, args.size)
    p["tau_g"] = args.tau_g
    stream = torch.cuda.Stream()
    with nfe.Sim(p, args.precision, stream=stream.cuda_stream, scale_exp=10) as s:
        s.set_fields(p["C0"])
        if "geometry" in p:
            geo = p["geometry"]
            s.set_geometry(geo["node"], geo["inlets"], geo["outflow"])
        s.set_variant(args.variant)
        with torch.cuda.stream(stream):
            s.step(3)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(args.steps)
            b.record(stream)
        b.synchronize()
        s.sync()
        ms = a.elapsed_time(b) / args.steps
        info = s.info()
    n = info["sites"]
    print(json.dumps({"workload": p["name"], "precision": args.precision, "sites": n, "ms_per_step": round(ms, 5),
                      "mlups": round(n / ms / 1e3, 1), "variant": info["variant"],
                      "effective_gbs": round(info["min_bytes_per_site"] * n / ms / 1e6, 1)}))


def run_batch(nfe, torch, args):
    import nfe_workloads as W
    sims = W.batch_sweep(args.sims, seed=1005)
    sites = sum(p["nx"] * p["ny"] for p in sims)
    mode = {"persistent": nfe.NFE_BATCH_PERSISTENT, "per_step": nfe.NFE_BATCH_PER_STEP, "auto": nfe.NFE_BATCH_AUTO}[args.mode]
    stream = torch.cuda.Stream()
    with nfe.Batch(sims, "fp32", stream=stream.cuda_stream) as bt:
        for i, p in enumerate(sims):
            bt.set_fields(i, p["C0"])
        bt.set_mode(mode)
        with torch.cuda.stream(stream):
            bt.step(3)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bt.step(args.steps)
            b.record(stream)
        b.synchronize()
        bt.sync()
        ms = a.elapsed_time(b) / args.steps
        info = bt.info()
    print(json.dumps({"workload": f"batch of {args.sims} D2Q9 simulations", "mode": args.mode, "sites": sites,
                      "ms_per_step": round(ms, 5), "mlups": round(sites / ms / 1e3, 1), "form": info["form"],
                      "tile_y": info["tile_y"]}))


if __name__ == "__main__":
    main()

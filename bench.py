#!/usr/bin/env python3
"""Throughput of the N-component free-energy LBM time step on GB300.

Workload: the quaternary spinodal mixture, 512 x 512 D2Q9, N = 4, all
sigma_ij = 0.005, tau = 0.8, m = 0.1, C_i = 1/4 + U(-0.02, 0.02) renormalised
(seed 1002).  One bench step = one time step of the whole lattice (stencils,
flux potential, conservative force, collide+stream of f, Cahn-Hilliard update
of C).  The whole working set (~30 MB in FP32) fits in the 129 MB L2, so a
256 MiB buffer is written between timed steps and every timed step starts
with a cold L2; CUDA events on the library's stream bracket each step.

Metric: MLUPS x N (million lattice-site updates per second times the number
of components), for the FP32 path (headline `value`) with the FP64 path
reported beside it (`fp64_path`).  `roofline` is for the dominant kernel,
against the measured HBM copy bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nfe|reference]

Under torchrun (N > 1) every rank runs an independent replica (the path has
no data exchange between simulations); the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import nfe_workloads as W  # noqa: E402

WORKLOAD = "spinodal 512x512 D2Q9 N=4 (sigma=0.005, tau=0.8, m=0.1, seed 1002)"
METRIC = "MLUPS x N (FP32 path; FP64 path beside), cold-L2 time per step"
UNIT = "MLUPS*N"
FLUSH_BYTES = 256 << 20


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def max_over_ranks_of(x, world_size, device):
    """Largest value of x over all ranks (the slowest replica sets the time)."""
    if world_size == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(sites_per_rank, steps, n_components, world_size, ms_total_max):
    """Whole-job MLUPS x N of independent replicas: all ranks' site updates / slowest rank's time."""
    return world_size * sites_per_rank * steps * n_components / (ms_total_max * 1e-3) / 1e6


def _captured_traffic(variant):
    """DRAM bytes per launch of the fused D2Q9 kernel with tile shape `variant`, from the
    committed ncu capture (one value per tile shape), or None when the kernel sources changed
    since that capture or that shape was not captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_fused2d_spinodal512_N4.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2605_22214_gb300", "csrc")
    for f in ("nfe_fused2d.cuh", "nfe_kernels.cuh", "nfe_internal.h"):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["source_sha256"]:
        return None
    return rec["dram_bytes_per_launch"].get(str(variant))


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def run_nfe(args):
    import torch
    import torch.distributed as dist

    import paper_2605_22214_gb300 as nfe
    from paper_2605_22214_gb300 import build as nfe_build

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    nfe_build.build()
    hbm, peak_kind = _peaks()
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    p = W.spinodal_2d(seed=1002 + 1000 * rank)
    n = p["nx"] * p["ny"] * p["nz"]
    N = p["N"]

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, ws, "cuda")

    def timed_steps(sim, K, W_, clocks=None):
        """Sum of per-step event times with an L2 flush before every step (ms)."""
        with torch.cuda.stream(stream):
            for _ in range(W_):
                flush.zero_()
                sim.step(1)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        total = 0.0
        pending = []
        t0 = time.perf_counter()
        ctx = clocks if clocks is not None else _Null()
        with ctx:
            with torch.cuda.stream(stream):
                for i in range(K):
                    flush.zero_()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    sim.step(1)
                    b.record(stream)
                    pending.append((a, b))
                    if len(pending) >= 256:
                        b.synchronize()
                        total += sum(x.elapsed_time(y) for x, y in pending)
                        pending.clear()
            torch.cuda.synchronize()
        total += sum(x.elapsed_time(y) for x, y in pending)
        wall = time.perf_counter() - t0
        barrier()
        return total, wall

    def kernel_times(sim, K):
        """Per-kernel average duration (ms) from the library's own events, flushed L2."""
        sim.profile_enable(True)
        with torch.cuda.stream(stream):
            for _ in range(K):
                flush.zero_()
                sim.step(1)
        prof = sim.profile_read()
        sim.profile_enable(False)
        return {k: (cnt, ms / cnt) for k, (cnt, ms) in prof.items()}

    results = {}
    for prec in ("fp32", "fp64"):
        K = args.steps if prec == "fp32" else max(1, args.steps // 4)
        sim = nfe.Sim(p, prec, stream=stream.cuda_stream)
        sim.set_fields(p["C0"])
        clocks = Clocks(local) if prec == "fp32" else None
        ms_total, wall = timed_steps(sim, K, args.warmup, clocks)
        info = sim.info()
        ms_total = max_over_ranks(ms_total)
        ms_step = ms_total / K
        kt = kernel_times(sim, min(K, 500))
        d = sim.diagnostics()
        results[prec] = dict(sim=sim, info=info, ms_step=ms_step, K=K, kt=kt, diag=d, clocks=clocks, wall=wall)

    # end-to-end through the C ABI with host buffers: H2D of the full state from pinned
    # memory, one step, D2H of the full state, every step (wall clock, synchronised)
    r32 = results["fp32"]
    sim = r32["sim"]
    nbytes = r32["info"]["state_bytes"]
    hbuf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    nfe.nfe_get_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
    Ke = max(1, min(args.steps, 200))
    for _ in range(3):
        nfe.nfe_set_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
        sim.step(1)
        nfe.nfe_get_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
    barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        nfe.nfe_set_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
        sim.step(1)
        nfe.nfe_get_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_val = ws * n * Ke * N / e2e_s / 1e6

    def roofline(r):
        kt = r["kt"]
        prec_bytes = 4 if r is r32 else 8
        # dominant kernel and its compulsory bytes per site (each array it touches once)
        dom = max(kt, key=lambda k: kt[k][1])
        Q, D = 9, 2
        if dom == "fused_step":
            bps = r["info"]["min_bytes_per_site"]
        elif dom == "collide_stream":
            bps = prec_bytes * ((Q - 1) + (N - 1) + (Q - 1) + D + (N - 1))
        else:
            bps = prec_bytes * ((N - 1) + D + (N - 1) + (N - 1))
        ach = bps * n / (kt[dom][1] * 1e-3) / 1e9
        traffic = _captured_traffic(r["info"]["variant"]) if r is r32 else None
        return dict(bound="hbm", kernel=dom, variant=r["info"]["variant"], bytes_per_site=bps, achieved=round(ach, 1), peak=hbm,
                    unit="GB/s", frac=round(ach / hbm, 4), peak_source=peak_kind, traffic=traffic,
                    kernel_ms=round(kt[dom][1], 5), algorithmic_bytes=bps * n)

    def path_summary(r):
        mlups = ws * n / (r["ms_step"] * 1e-3) / 1e6
        eff = r["info"]["min_bytes_per_site"] * n / (r["ms_step"] * 1e-3) / 1e9
        return dict(value=round(mlups * N, 1), mlups=round(mlups, 1), ms_per_step=round(r["ms_step"], 5),
                    effective_gbs=round(eff, 1), effective_frac=round(eff / hbm, 4),
                    min_bytes_per_site=r["info"]["min_bytes_per_site"],
                    kernels={k: dict(launches=c, avg_ms=round(t, 5)) for k, (c, t) in r["kt"].items()},
                    )

    # the same time step on other sizes and storage formats (context for the roofline)
    extras = []
    if not args.no_extras:
        cases = [("spinodal 512x512 N=4", W.spinodal_2d(seed=1002), "f16", args.steps // 4, True),
                 ("spinodal 512x512 N=4", W.spinodal_2d(seed=1002), "bf16", args.steps // 4, True),
                 ("spinodal 4096x4096 N=4", W.spinodal_2d(nx=4096, ny=4096, seed=1012), "fp32", 60, False),
                 ("spinodal 4096x4096 N=4", W.spinodal_2d(nx=4096, ny=4096, seed=1012), "f16", 60, False),
                 ("spinodal 4096x4096 N=4", W.spinodal_2d(nx=4096, ny=4096, seed=1012), "fp64", 10, False),
                 ("spinodal 4096x4096 N=4, tau_g = 1.3 (stored g)", dict(W.spinodal_2d(nx=4096, ny=4096, seed=1012), tau_g=1.3),
                  "fp32", 30, False),
                 ("janus 256^3 D3Q19 N=4", W.janus_3d(seed=1004), "fp32", 20, False),
                 ("janus 256^3 D3Q19 N=4", W.janus_3d(seed=1004), "bf16", 20, False),
                 ("emulsion generator 600x140 D2Q9 N=4 (solid walls, 6 inlets, convective outflow)",
                  W.emulsion_2d(), "fp32", args.steps // 4, True),
                 ("porous channel 4096x1024 D2Q9 N=4 (4x4 posts every 16 sites, inlet, outflow)",
                  W.porous_channel_2d(), "fp32", 60, False),
                 ("patterned liquid surface 400x140 D2Q9 N=4 (walls, posts, force on fluid 2)",
                  W.pals_2d(), "fp32", args.steps // 4, True)]
        for name, q, prec, K, fl in cases:
            nq = q["nx"] * q["ny"] * q["nz"]
            with nfe.Sim(q, prec, stream=stream.cuda_stream, scale_exp=10) as sx:
                sx.set_fields(q["C0"])
                if "geometry" in q:
                    geo = q["geometry"]
                    sx.set_geometry(geo["node"], geo["inlets"], geo["outflow"])
                if fl:
                    ms_total, _ = timed_steps(sx, K, 5)
                    ms = ms_total / K
                else:
                    with torch.cuda.stream(stream):
                        sx.step(3)
                        a = torch.cuda.Event(enable_timing=True)
                        bb = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        sx.step(K)
                        bb.record(stream)
                    bb.synchronize()
                    ms = a.elapsed_time(bb) / K
                inf = sx.info()
            mlups = nq / (ms * 1e-3) / 1e6
            eff = inf["min_bytes_per_site"] * nq / (ms * 1e-3) / 1e9
            extras.append(dict(workload=name, precision=prec, sites=nq, ms_per_step=round(ms, 4),
                               mlups=round(mlups, 1), mlups_x_n=round(mlups * q["N"], 1),
                               min_bytes_per_site=inf["min_bytes_per_site"], effective_gbs=round(eff, 1),
                               effective_frac=round(eff / hbm, 4), kernels_per_step=inf["kernels_per_step"],
                               l2="flushed before every step" if fl else "working set > L2, steps back to back"))
            del q

    batched = None
    precision = None
    coarsening = None
    if not args.no_extras:
        batched = batch_sweep_measure(nfe, torch, stream, args.batch_steps)
        precision = precision_study(nfe, stream)
        coarsening = coarsening_measure(nfe, stream)

    s32 = path_summary(r32)
    s64 = path_summary(results["fp64"])
    s64["roofline"] = roofline(results["fp64"])
    line = {
        "metric": METRIC,
        "value": s32["value"],
        "unit": UNIT,
        "n_gpus": ws,
        "steps": r32["K"],
        "warmup": args.warmup,
        "ms_per_step": s32["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded spinodal mixture, numpy PCG64)",
        "config": {"workload": WORKLOAD, "sites": n, "N": N, "lattice": "D2Q9", "precision": "fp32",
                   "l2": "256 MiB buffer written before every timed step (cold L2)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "mlups": s32["mlups"],
        "effective_gbs": s32["effective_gbs"],
        "effective_frac": s32["effective_frac"],
        "roofline": roofline(r32),
        "kernels": s32["kernels"],
        "fp64_path": s64,
        "e2e": {"value": round(e2e_val, 1), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": Ke,
                "how": "nfe_set_state (pinned host -> device), nfe_step(1), nfe_get_state (device -> pinned host)"},
        "gpu_launches": r32["info"]["kernels_per_step"] * r32["K"],
        "extras": extras,
        "batched": batched,
        "precision_study": precision,
        "coarsening": coarsening,
        "clocks": r32["clocks"].summary() if r32["clocks"] is not None else None,
    }
    for r in results.values():
        r["sim"].close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def coarsening_measure(nfe, stream, n=1600, t_end=40000):
    """Domain growth of the paper's binary phase-separation run (Sec. IV): n^2, C_i ~ U(0, 1)
    renormalised, sigma = 0.005, eta = 1/6, FP32.  L (mean over the two components, the
    equation for L_i of Sec. IV, via nfe_domain_size) at geometric times; the late-time exponent
    is the least-squares slope of log L on log t over the last half of the samples."""
    p = W.phase_separation_2d(nx=n, ny=n, N=2, seed=1013)
    times = [int(round(500 * (t_end / 500) ** (i / 10))) for i in range(11)]
    Ls = []
    with nfe.Sim(p, "fp32", stream=stream.cuda_stream) as s:
        s.set_fields(p["C0"])
        t = 0
        for target in times:
            s.step(target - t)
            t = target
            Ls.append(s.domain_size()[1])
    half = len(times) // 2
    a = float(np.polyfit(np.log(times[half:]), np.log(Ls[half:]), 1)[0])
    return {"workload": f"binary phase separation {n}x{n} (C_i ~ U(0, 1) renormalised, sigma = 0.005, tau = 1, m = 0.1, "
                        "seed 1013), FP32", "t": times, "L": [round(x, 3) for x in Ls], "late_exponent": round(a, 3),
            "expected": "2/3 (inertial hydrodynamic coarsening, Sec. IV)"}


def precision_study(nfe, stream, n=128, steps=300):
    """Four Janus drops (the 256^3 layout scaled to n^3), FP32 compute with FP32 / FP16 / BF16
    storage of f against the FP64 path: volume-fraction error, Laplace-pressure error of each
    drop (mean P inside minus mean P in the matrix) and momentum drift per site."""
    p = W.janus_3d(n=n, radius=8.0, seed=1004)
    R = p["radius"]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    dists = [np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) for cx, cy, cz in p["centres"]]
    matrix = np.all([d > R + 6 for d in dists], axis=0)

    def run(prec):
        with nfe.Sim(p, prec, stream=stream.cuda_stream, scale_exp=10) as s:
            s.set_fields(p["C0"])
            s.step(steps)
            C, v, P = s.fields()
            d = s.diagnostics()
        dP = np.array([P[dd < R - 4].mean() - P[matrix].mean() for dd in dists])
        return C, P, dP, np.abs(d["momentum"]).max() / n ** 3

    C64, P64, dP64, m64 = run("fp64")
    out = {"workload": f"4 Janus drops {n}^3 (radius {R:g}), {steps} steps, FP32 compute vs the FP64 path",
           "fp64": {"momentum_per_site": m64, "laplace_dP": [float(v) for v in dP64]}}
    for prec in ("fp32", "f16", "bf16"):
        C, P, dP, m = run(prec)
        out[prec] = {"max_abs_C_err": float(np.abs(C - C64).max()),
                     "max_rel_P_err": float(np.abs(P - P64).max() / np.abs(P64).max()),
                     "laplace_rel_err": float(np.abs(dP - dP64).max() / np.abs(dP64).max()),
                     "momentum_per_site": m}
    return out


def batch_sweep_measure(nfe, torch, stream, steps):
    """The 512-simulation lens/Janus sweep (D2Q9, N in {3,4,5}, FP32): one persistent launch
    for all steps, one batched launch per step, and one launch per simulation per step."""
    sims = W.batch_sweep(512, seed=1005)
    sites = sum(p["nx"] * p["ny"] for p in sims)
    site_n = sum(p["nx"] * p["ny"] * p["N"] for p in sims)
    out = {"workload": "512 D2Q9 lens/Janus simulations, edge in {64,96,128,192,256}, N in {3,4,5}, "
                       "sigma ~ U(0.004, 0.012), seed 1005+i, FP32", "sites": sites, "steps": steps}
    with nfe.Batch(sims, "fp32", stream=stream.cuda_stream) as bt:
        for i, p in enumerate(sims):
            bt.set_fields(i, p["C0"])
        for mode, name in ((nfe.NFE_BATCH_PERSISTENT, "persistent"), (nfe.NFE_BATCH_PER_STEP, "per_step"),
                           (nfe.NFE_BATCH_AUTO, "autotuned")):
            bt.set_mode(mode)
            with torch.cuda.stream(stream):
                bt.step(4)
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                bt.step(steps)
                e.record(stream)
            e.synchronize()
            bt.sync()
            ms = a.elapsed_time(e) / steps
            inf = bt.info()
            out[name] = {"ms_per_step": round(ms, 4), "mlups": round(sites / (ms * 1e-3) / 1e6, 1),
                         "mlups_x_n": round(site_n / (ms * 1e-3) / 1e6, 1), "tile_y": inf["tile_y"],
                         "form": inf["form"], "grid": inf["grid"]}
        out["info"] = bt.info()
    # the same jobs, one launch per simulation per step
    singles = []
    for p in sims:
        s = nfe.Sim(p, "fp32", stream=stream.cuda_stream)
        s.set_fields(p["C0"])
        s.set_variant(1)
        singles.append(s)
    k = max(2, steps // 10)
    with torch.cuda.stream(stream):
        for s in singles:
            s.step(1)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            for s in singles:
                s.step(1)
        e.record(stream)
    e.synchronize()
    ms = a.elapsed_time(e) / k
    out["one_launch_per_simulation"] = {"ms_per_step": round(ms, 4), "mlups": round(sites / (ms * 1e-3) / 1e6, 1),
                                        "mlups_x_n": round(site_n / (ms * 1e-3) / 1e6, 1), "steps": k}
    for s in singles:
        s.close()
    return out


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def _oracle_rate(p, budget_s, min_steps=2):
    """Time the FP64 oracle, as it stands, on p for about budget_s seconds."""
    from oracle import lbm
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    st = lbm.step(prm, st)                      # warm-up
    steps = 0
    t0 = time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < budget_s:
        st = lbm.step(prm, st)
        steps += 1
    dt = time.perf_counter() - t0
    n = p["nx"] * p["ny"] * p["nz"]
    return n * steps / dt / 1e6, steps, dt


def cpu_baseline(p, budget_s=15.0):
    mlups, steps, dt = _oracle_rate(p, budget_s)
    return {"value": round(mlups * p["N"], 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} time steps of the full 512x512 N=4 workload in {dt:.1f} s "
                      "(numpy FP64 oracle, literal f and g populations, single thread)"}


def run_reference(args):
    """The oracle as it stands on the host cores, same config, metric and unit."""
    ws, rank = _dist()
    if rank != 0:
        return
    full = W.spinodal_2d(seed=1002)
    # each bench step: one time step of a periodic square sample of the workload's initial
    # field, sized so the whole --steps/--warmup run ends within about two minutes
    rate, _, _ = _oracle_rate(W.spinodal_2d(nx=64, ny=64, seed=1002), 2.0)
    per_step = 120.0 / max(1, args.steps + args.warmup)
    side = int(max(8, min(512, math.sqrt(rate * 1e6 * per_step))))
    p = dict(full)
    p["nx"] = p["ny"] = side
    p["C0"] = full["C0"][:, :, :side, :side] / full["C0"][:, :, :side, :side].sum(axis=0, keepdims=True)
    from oracle import lbm
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    for _ in range(args.warmup):
        st = lbm.step(prm, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = lbm.step(prm, st)
    dt = time.perf_counter() - t0
    val = side * side * args.steps * p["N"] / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded spinodal mixture, numpy PCG64)",
            "config": {"workload": WORKLOAD, "sample": f"{side}x{side} periodic corner of the 512x512 input"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(val, 4), "unit": UNIT,
                             "sample": f"{args.steps} steps of a {side}x{side} sample"},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["nfe", "reference"], default="nfe")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other sizes and storage formats")
    ap.add_argument("--batch-steps", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nfe(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Throughput of the N-component free-energy LBM time step on GB300.

Headline workload: four Janus droplets in a 256^3 periodic box, D3Q19, N = 4
(drops of radius 32 split by the plane x = x_c, sigma_ij ~ U(0.004, 0.012)
from seed 1004, tau = 1, m = 1/50), FP32 path.  One bench step = one time step
of the whole lattice (stencils, flux potential, conservative force,
collide+stream of f, Cahn-Hilliard update of C): the form of the D3Q19 step
the library's autotuner picked (the fused kernel, or the split physics and
gather kernels).  The working set (two 1.4 GB state buffers) is far larger
than the 129 MB L2, so steps run back to back; CUDA events on the library's
stream bracket the timed steps.

Metric: MLUPS x N (million lattice-site updates per second times the number
of components) of the FP32 path (headline `value`), the FP64 path on the same
lattice beside it (`fp64_path`).  `roofline`: the step's algorithmic bytes
(each population and volume fraction read once and written once) over the
step's time, against the measured HBM copy bandwidth, with every kernel of
the step beside it (`per_kernel`, each with its own algorithmic bytes).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nfe|reference]

Under torchrun (N > 1) every rank runs an independent replica (the path has
no data exchange between simulations); the slowest rank's time is used.
`--impl reference` times the FP64 oracle (the plain CPU restatement of the
method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import nfe_workloads as W  # noqa: E402

WORKLOAD = ("four Janus drops 256^3 D3Q19 N=4 (radius 32, sigma ~ U(0.004, 0.012) seed 1004, "
            "tau=1, m=1/50)")
METRIC = "MLUPS x N (FP32 path; FP64 path beside)"
UNIT = "MLUPS*N"
FLUSH_BYTES = 256 << 20
SAMPLE_EDGE = 32          # edge of the cubes the oracle is timed on


def _config(ws):
    return {"workload": WORKLOAD, "sites": 256 ** 3, "N": 4, "lattice": "D3Q19", "precision": "fp32",
            "l2": "inputs larger than L2 (2 x 1.4 GB state), steps back to back",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


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


def _sources_sha(files):
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2605_22214_gb300", "csrc")
    for f in files:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(name, variant):
    """DRAM bytes of one time step (summed over its launches) from a committed ncu capture
    (profiles/<name>.json, per tile-shape variant), or None when the kernel sources changed since
    that capture or the variant was not captured."""
    path = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    if _sources_sha(rec["sources"]) != rec["source_sha256"]:
        return None
    v = rec["dram_bytes_per_step"].get(str(variant))
    return None if v is None else float(sum(v.values()))


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class Clocks:
    """SM clock and throttle reasons sampled while the timed region runs.

    NVML (libnvidia-ml, loaded with ctypes) is polled every millisecond from a thread, so even
    a timed region of a few tens of milliseconds gets samples; nvidia-smi every 100 ms is the
    fallback.  The GPU is found by its UUID (the NVML index can differ from the CUDA index)."""

    # clock-event reason bits of the NVML API
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.samples = []
        self.max_mhz = None
        self.source = None
        self._stop = threading.Event()
        self._thread = None
        self._proc = None

    def _nvml_handle(self):
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.cuda_index).uuid)
        except Exception:
            uuid = None
        ok = False
        if uuid:
            u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        return lib, h

    def _poll_nvml(self, lib, h):
        mhz = ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0:
                r = reasons.value if get_reasons(h, ctypes.byref(reasons)) == 0 else 0
                self.samples.append((float(mhz.value), int(r)))
            time.sleep(0.001)

    def __enter__(self):
        try:
            lib, h = self._nvml_handle()
            self.source = "nvml, 1 ms polling"
            self._thread = threading.Thread(target=self._poll_nvml, args=(lib, h), daemon=True)
            self._thread.start()
        except (OSError, AttributeError):
            self.source = "nvidia-smi, 100 ms polling"
            q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            try:
                self._proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                               "-i", str(self.cuda_index), "-lms", "100"],
                                              stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self._proc = None
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._thread is not None:
            self._thread.join(timeout=2)
        if self._proc is not None:
            self._proc.terminate()
            try:
                out, _ = self._proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
                out, _ = self._proc.communicate()
            bits = [0x8, 0x40, 0x20, 0x4]
            for ln in out.splitlines():
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 6:
                    continue
                try:
                    mhz, mx = float(parts[0]), float(parts[1])
                except ValueError:
                    continue
                self.max_mhz = mx
                r = sum(b for b, v in zip(bits, parts[2:6]) if v.lower().startswith("active"))
                self.samples.append((mhz, r))
        return False

    def summary(self):
        mhz = [m for m, _ in self.samples]
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(mhz), "source": self.source}


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

def _oracle_worker(conn, p):
    """One host process: the FP64 oracle, as it stands, on one sample cube (periodic)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import lbm
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    conn.send("ready")
    while True:
        k = conn.recv()
        if k is None:
            break
        t0 = time.perf_counter()
        for _ in range(k):
            st = lbm.step(prm, st)
        conn.send(time.perf_counter() - t0)
    conn.close()


def sample_cubes(full, count, edge=SAMPLE_EDGE):
    """`count` periodic edge^3 cubes cut from the 256^3 input at seeded corners (drops and matrix)."""
    rng = np.random.default_rng(7)
    n = full["nx"]
    out = []
    for _ in range(count):
        z0, y0, x0 = (int(v) for v in rng.integers(0, n - edge, size=3))
        q = {k: v for k, v in full.items() if k not in ("C0", "centres")}
        C = np.ascontiguousarray(full["C0"][:, z0:z0 + edge, y0:y0 + edge, x0:x0 + edge])
        q["C0"] = C / C.sum(axis=0, keepdims=True)
        q["nx"] = q["ny"] = q["nz"] = edge
        out.append(q)
    return out


class OraclePool:
    """One spawned process per host core, each stepping the oracle on its own sample cube.
    Spawned (not forked), so a CUDA context in the parent is never copied."""

    def __init__(self, cubes):
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for q in cubes:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, q), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            c.recv()
        self.sites = sum(q["nx"] * q["ny"] * q["nz"] for q in cubes)
        self.N = cubes[0]["N"]

    def step(self, k):
        """Advance every cube by k steps in parallel; returns the wall time (s)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(k)
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except (BrokenPipeError, OSError):
                pass
        for pr in self.procs:
            pr.join(timeout=10)


def cpu_baseline(full, budget_s=15.0):
    """The oracle timed on all host cores: one process per core, each on its own 32^3 cube of the
    workload, for about budget_s seconds."""
    cores = os.cpu_count() or 1
    pool = OraclePool(sample_cubes(full, cores))
    try:
        pool.step(1)                                # warm-up
        steps, wall = 0, 0.0
        while steps < 2 or wall < budget_s:
            wall += pool.step(1)
            steps += 1
    finally:
        pool.close()
    val = pool.sites * steps * pool.N / wall / 1e6
    return {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each {steps} time steps of its own periodic {SAMPLE_EDGE}^3 cube of the "
                      f"256^3 input, {wall:.1f} s wall (numpy FP64 oracle, literal f and g populations, "
                      f"one thread per process)"}


# ----------------------------------------------------------------------------
# the library arm
# ----------------------------------------------------------------------------

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
    p = W.janus_3d(seed=1004 + 1000 * rank)
    n = p["nx"] * p["ny"] * p["nz"]
    N = p["N"]

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, ws, "cuda")

    def timed(sim, K, W_, clocks=None):
        """Device time (ms) of K steps back to back, after W_ warm-up steps."""
        with torch.cuda.stream(stream):
            sim.step(W_)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        ctx = clocks if clocks is not None else _Null()
        with ctx:
            with torch.cuda.stream(stream):
                a.record(stream)
                sim.step(K)
                b.record(stream)
            b.synchronize()
        torch.cuda.synchronize()
        barrier()
        return a.elapsed_time(b)

    def kernel_times(sim, K):
        """Per-kernel average duration (ms) from the library's own events on its stream."""
        sim.profile_enable(True)
        with torch.cuda.stream(stream):
            sim.step(K)
        prof = sim.profile_read()
        sim.profile_enable(False)
        return {k: (cnt, ms / cnt) for k, (cnt, ms) in prof.items()}

    results = {}
    for prec in ("fp32", "fp64"):
        K = args.steps if prec == "fp32" else max(1, args.steps // 4)
        sim = nfe.Sim(p, prec, stream=stream.cuda_stream)
        sim.set_fields(p["C0"])
        if prec == "fp32" and args.variant >= 0:
            sim.set_variant(args.variant)       # a fixed form instead of the autotuner's pick
        clocks = Clocks(local) if prec == "fp32" else None
        ms_total = max_over_ranks(timed(sim, K, args.warmup, clocks))
        info = sim.info()
        kt = kernel_times(sim, min(K, 20))
        results[prec] = dict(sim=sim, info=info, ms_step=ms_total / K, K=K, kt=kt, clocks=clocks)

    # end to end through the C ABI with host buffers: H2D of the full state from pinned memory,
    # one step, D2H of the full state, every step (wall clock, synchronised)
    r32 = results["fp32"]
    sim = r32["sim"]
    nbytes = r32["info"]["state_bytes"]
    hbuf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    nfe.nfe_get_state_ptr(sim.h, hbuf.data_ptr(), nbytes)
    Ke = max(1, min(args.steps, 50))
    for _ in range(2):
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
    del hbuf

    def kernel_bytes(kind, info, prec):
        """Algorithmic bytes per site of one kernel of the step: every array it must read or write,
        once (the split D3Q19 step moves its gather records through HBM)."""
        fb = {"fp64": 8, "fp32": 4, "f16": 2, "bf16": 2}[prec]
        cb = 8 if prec == "fp64" else 4
        Q = 19
        rec = 2 * N + 1           # the gather record: C, v and S of the site
        if kind == "step_physics":
            return 2 * (Q - 1) * fb + (N - 1) * cb + rec * cb
        if kind == "step_gather":
            return rec * cb + (N - 1) * cb
        return info["min_bytes_per_site"]

    def roofline(r, prec, traffic_name=None):
        """The step against the HBM roofline: its algorithmic bytes (each population and volume
        fraction read once and written once) over the step's time from the timed region's events
        (which bracket every launch of the step), and the same for each kernel of the step with its
        own algorithmic bytes and its library-event time."""
        kt = r["kt"]
        info = r["info"]
        bps = info["min_bytes_per_site"]
        step_ms = r["ms_step"]
        ach = bps * n / (step_ms * 1e-3) / 1e9
        traffic = captured_traffic(traffic_name, info["variant"]) if traffic_name else None
        per_kernel = {}
        for kind, (cnt, ms) in kt.items():
            kb = kernel_bytes(kind, info, prec)
            a = kb * n / (ms * 1e-3) / 1e9
            per_kernel[kind] = dict(launches=cnt, avg_ms=round(ms, 5), bytes_per_site=kb, achieved=round(a, 1),
                                    frac=round(a / hbm, 4))
        return dict(bound="hbm", kernel=" + ".join(sorted(kt)), variant=info["variant"],
                    launches_per_step=info["kernels_per_step"], bytes_per_site=bps, algorithmic_bytes=bps * n,
                    achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4), peak_source=peak_kind,
                    traffic=traffic, step_ms=round(step_ms, 5),
                    timing="CUDA events around the timed steps on the library stream",
                    per_kernel=per_kernel)

    def path_summary(r):
        mlups = ws * n / (r["ms_step"] * 1e-3) / 1e6
        eff = r["info"]["min_bytes_per_site"] * n / (r["ms_step"] * 1e-3) / 1e9
        return dict(value=round(mlups * N, 1), mlups=round(mlups, 1), ms_per_step=round(r["ms_step"], 5),
                    effective_gbs=round(eff, 1), effective_frac=round(eff / hbm, 4),
                    min_bytes_per_site=r["info"]["min_bytes_per_site"],
                    kernels={k: dict(launches=c, avg_ms=round(t, 5)) for k, (c, t) in r["kt"].items()})

    s32 = path_summary(r32)
    s64 = path_summary(results["fp64"])
    s64["roofline"] = roofline(results["fp64"], "fp64")
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
        "data": "synthetic (seeded Janus-drop layout, numpy PCG64)",
        "config": _config(ws),
        "mlups": s32["mlups"],
        "effective_gbs": s32["effective_gbs"],
        "effective_frac": s32["effective_frac"],
        "roofline": roofline(r32, "fp32", "traffic_step3d_janus256_N4"),
        "kernels": s32["kernels"],
        "fp64_path": s64,
        "e2e": {"value": round(e2e_val, 1), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": Ke,
                "how": "nfe_set_state (pinned host -> device), nfe_step(1), nfe_get_state (device -> pinned host)"},
        "gpu_launches": r32["info"]["kernels_per_step"] * r32["K"],
        "clocks": r32["clocks"].summary() if r32["clocks"] is not None else None,
    }
    for r in results.values():
        r["sim"].close()
    del results, sim
    torch.cuda.empty_cache()

    if not args.no_extras:
        line["extras"] = extras_measure(nfe, torch, stream, args, hbm, peak_kind)
        line["batched"] = batch_sweep_measure(nfe, torch, stream, args.batch_steps, hbm)
        line["coarsening"] = coarsening_measure(nfe, stream)
    if args.precision_study:
        line["precision_study"] = precision_study(nfe, stream)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def extras_measure(nfe, torch, stream, args, hbm, peak_kind):
    """The same time step on the other configurations, sizes and storage formats, each with the
    roofline of its step (algorithmic bytes per step over the step's device time)."""
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    cases = [
        ("janus 256^3 D3Q19 N=4", lambda: W.janus_3d(seed=1004), "f16", 20, False),
        ("janus 256^3 D3Q19 N=4", lambda: W.janus_3d(seed=1004), "bf16", 20, False),
        ("spinodal 512x512 D2Q9 N=4 (c2)", lambda: W.spinodal_2d(seed=1002), "fp32", 400, True),
        ("spinodal 4096x4096 D2Q9 N=4", lambda: W.spinodal_2d(nx=4096, ny=4096, seed=1012), "fp32", 60, False),
        ("spinodal 4096x4096 D2Q9 N=4", lambda: W.spinodal_2d(nx=4096, ny=4096, seed=1012), "f16", 60, False),
        ("spinodal 4096x4096 D2Q9 N=4", lambda: W.spinodal_2d(nx=4096, ny=4096, seed=1012), "bf16", 60, False),
        ("spinodal 4096x4096 D2Q9 N=4", lambda: W.spinodal_2d(nx=4096, ny=4096, seed=1012), "fp64", 6, False),
        ("spinodal 4096x4096 D2Q9 N=4, tau_g = 1.3 (stored g)",
         lambda: dict(W.spinodal_2d(nx=4096, ny=4096, seed=1012), tau_g=1.3), "fp32", 30, False),
        ("layered Poiseuille 32x32x192 D3Q19 N=7 (c3)", lambda: W.layered_poiseuille(), "fp32", 200, True),
        ("lens 64x64 D2Q9 N=3 (c1)", lambda: W.lens_2d(), "fp64", 400, True),
        ("porous channel 4096x1024 D2Q9 N=4 (4x4 posts every 16 sites, inlet, outflow)",
         lambda: W.porous_channel_2d(), "fp32", 60, False),
        ("porous block 256^3 D3Q19 N=4 (3^3 solid cubes every 10 sites, slab with a window, walls in z)",
         lambda: W.porous_3d(256, 256, 256, 4, walls=(False, False, True)), "fp32", 20, False),
    ]
    out = []
    for name, make, prec, K, fl in cases:
        q = make()
        nq = q["nx"] * q["ny"] * q["nz"]
        with nfe.Sim(q, prec, stream=stream.cuda_stream, scale_exp=10) as sx:
            sx.set_fields(q["C0"])
            if "geometry" in q:
                geo = q["geometry"]
                sx.set_geometry(geo["node"], geo["inlets"], geo["outflow"])
            with torch.cuda.stream(stream):
                sx.step(3)
            if fl:
                # L2-resident working set: a 256 MiB write before every timed step (cold L2)
                total = 0.0
                with torch.cuda.stream(stream):
                    evs = []
                    for _ in range(K):
                        flush.zero_()
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        sx.step(1)
                        b.record(stream)
                        evs.append((a, b))
                torch.cuda.synchronize()
                total = sum(a.elapsed_time(b) for a, b in evs)
                ms = total / K
            else:
                with torch.cuda.stream(stream):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    sx.step(K)
                    b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b) / K
            inf = sx.info()
        mlups = nq / (ms * 1e-3) / 1e6
        eff = inf["min_bytes_per_site"] * nq / (ms * 1e-3) / 1e9
        l2_resident = inf["min_bytes_per_site"] * nq < 129e6
        out.append(dict(workload=name, precision=prec, sites=nq, ms_per_step=round(ms, 5),
                        mlups=round(mlups, 1), mlups_x_n=round(mlups * q["N"], 1),
                        min_bytes_per_site=inf["min_bytes_per_site"], kernels_per_step=inf["kernels_per_step"],
                        variant=inf["variant"],
                        roofline=dict(bound="hbm", achieved=round(eff, 1), peak=hbm, unit="GB/s",
                                      frac=round(eff / hbm, 4), peak_source=peak_kind,
                                      note=("working set fits in L2: DRAM bytes are below the algorithmic bytes"
                                            if l2_resident else "algorithmic bytes per step / step time")),
                        l2="flushed before every step" if fl else "working set > L2, steps back to back"))
        del q
    del flush
    torch.cuda.empty_cache()
    return out


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


def precision_study(nfe, stream, n=256, steps=5000, radius=32.0):
    """The c4 precision study at its stated size: four Janus drops of radius 32 in 256^3, 5000
    steps, FP32 compute with FP32 / FP16 / BF16 storage of f against the FP64 path: volume-fraction
    error, Laplace-pressure error of each drop (mean P inside minus mean P in the matrix) and the
    momentum drift per site."""
    p = W.janus_3d(n=n, radius=radius, seed=1004)
    R = p["radius"]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    dists = [np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) for cx, cy, cz in p["centres"]]
    del x, y, z
    inside = [d < R - 4 for d in dists]
    matrix = np.all([d > R + 6 for d in dists], axis=0)
    del dists

    def run(prec):
        with nfe.Sim(p, prec, stream=stream.cuda_stream, scale_exp=10) as s:
            s.set_fields(p["C0"])
            s.step(steps)
            C, v, P = s.fields()
            d = s.diagnostics()
        dP = np.array([P[m].mean() - P[matrix].mean() for m in inside])
        return C, P, dP, np.abs(d["momentum"]).max() / n ** 3, d

    t0 = time.perf_counter()
    C64, P64, dP64, m64, d64 = run("fp64")
    out = {"workload": f"4 Janus drops {n}^3 (radius {R:g}), {steps} steps, FP32 compute vs the FP64 path",
           "fp64": {"momentum_per_site": m64, "laplace_dP": [float(v) for v in dP64],
                    "mass": [float(v) for v in d64["mass"]]}}
    for prec in ("fp32", "f16", "bf16"):
        C, P, dP, m, d = run(prec)
        out[prec] = {"max_abs_C_err": float(np.abs(C - C64).max()),
                     "max_rel_P_err": float(np.abs(P - P64).max() / np.abs(P64).max()),
                     "laplace_rel_err": float(np.abs(dP - dP64).max() / np.abs(dP64).max()),
                     "momentum_per_site": m,
                     "mass_rel_err": float(np.abs(d["mass"] - d64["mass"]).max() / np.abs(d64["mass"]).max())}
        del C, P
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def batch_sweep_measure(nfe, torch, stream, steps, hbm):
    """The 512-simulation lens/Janus sweep (D2Q9, N in {3,4,5}, FP32): one persistent launch
    for all steps, one batched launch per step, and one launch per simulation per step."""
    sims = W.batch_sweep(512, seed=1005)
    sites = sum(p["nx"] * p["ny"] for p in sims)
    site_n = sum(p["nx"] * p["ny"] * p["N"] for p in sims)
    bytes_step = sum(p["nx"] * p["ny"] * 2 * 4 * (8 + p["N"] - 1) for p in sims)
    out = {"workload": "512 D2Q9 lens/Janus simulations, edge in {64,96,128,192,256}, N in {3,4,5}, "
                       "sigma ~ U(0.004, 0.012), seed 1005+i, FP32", "sites": sites, "steps": steps,
           "algorithmic_bytes_per_step": bytes_step}
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
            eff = bytes_step / (ms * 1e-3) / 1e9
            out[name] = {"ms_per_step": round(ms, 4), "mlups": round(sites / (ms * 1e-3) / 1e6, 1),
                         "mlups_x_n": round(site_n / (ms * 1e-3) / 1e6, 1), "tile_y": inf["tile_y"],
                         "form": inf["form"], "grid": inf["grid"],
                         "roofline": {"bound": "hbm", "achieved": round(eff, 1), "peak": hbm, "unit": "GB/s",
                                      "frac": round(eff / hbm, 4)}}
        out["info"] = bt.info()
    # the same jobs, one launch per simulation per step
    singles = []
    for p in sims:
        s = nfe.Sim(p, "fp32", stream=stream.cuda_stream)
        s.set_fields(p["C0"])
        s.set_variant(1)
        singles.append(s)
    k = max(2, min(200, steps // 10))
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


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.  Each bench step is one
    time step of one periodic 32^3 cube of the 256^3 input per host core, all cubes in parallel
    (a bounded sample of the workload); same metric, unit and config as the library arm."""
    ws, rank = _dist()
    if rank != 0:
        return
    full = W.janus_3d(seed=1004)
    cores = os.cpu_count() or 1
    pool = OraclePool(sample_cubes(full, cores))
    del full
    try:
        for _ in range(args.warmup):
            pool.step(1)
        dt = pool.step(args.steps)
    finally:
        pool.close()
    val = pool.sites * args.steps * pool.N / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Janus-drop layout, numpy PCG64)",
            "config": _config(ws),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(val, 4), "unit": UNIT,
                             "sample": f"{args.steps} steps of {cores} periodic {SAMPLE_EDGE}^3 cubes of the 256^3 "
                                       f"input, one process per core"},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["nfe", "reference"], default="nfe")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads, sizes and formats")
    ap.add_argument("--batch-steps", type=int, default=5000, help="steps of the batched sweep (c5: 5000)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="form of the headline FP32 step (-1: the library's autotuner picks; a profiler "
                         "distorts the autotuner's trial timings, so profiled runs name the form)")
    ap.add_argument("--precision-study", action="store_true",
                    help="also run the c4 precision study at 256^3, radius 32, 5000 steps (a few minutes)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nfe(args)


if __name__ == "__main__":
    main()

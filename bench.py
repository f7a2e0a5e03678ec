"""Benchmark of the fused D3Q19 stream-collide step on one or more GB300s.

Workload (one bench "step" = one time step of the whole lattice): D3Q19 SRT
Taylor-Green vortex (the 2-D closed form of Sec. 4.2 extruded along z, an
exact 3-D flow) on a fully periodic 256^3 lattice (u0 = 0.05, tau = 0.53),
initial fields from the closed form at t = 0, A-B streaming, flag-free
periodic kernel -- the paper's benchmark box (Sec. 5: periodic cube, no
boundary nodes, 256^3).  The headline tier is FP32 arithmetic with FP16S
storage (`--format`); every other storage tier is measured on the same
workload in `per_format`, and the batched ensemble of lid-driven cavities
(512 cubes, edges 16..128, FP16S) against one launch per member in
`ensemble`.  Inputs are resident in HBM for `value`; `e2e` goes through the
C ABI with pinned host buffers.  Under torchrun each rank advances its own
replica of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPs/s per storage format vs HBM roofline; ensemble MLUPs/s vs per-launch"
PAPER_A100_FP16S = 15455.0   # MLUPs/s, Nvidia A100 40GB, FP32/FP16S, D3Q19 SRT 256^3 (appendix hardware table, Table 6)
TIERS = [  # (name, arithmetic, storage)
    ("FP64/FP64", "FP64", "FP64"), ("FP64/FP32", "FP64", "FP32"), ("FP32/FP32", "FP32", "FP32"),
    ("FP32/FP16", "FP32", "FP16"), ("FP32/FP16S", "FP32", "FP16S"), ("FP32/FP16C", "FP32", "FP16C"),
    ("FP32/P16_0S", "FP32", "P16_0S"), ("FP32/P16_1S", "FP32", "P16_1S"), ("FP32/P16_2C", "FP32", "P16_2C"),
    ("FP32/P16_0", "FP32", "P16_0"), ("FP32/P16_1", "FP32", "P16_1"),
]
BYTES_PER_POP = {"FP64": 8, "FP32": 4}


def pop_bytes(storage):
    return BYTES_PER_POP.get(storage, 2)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for n in ("lbm_kernels.cuh", "lbm_device.cuh"):
        with open(os.path.join(ROOT, "paper_2112_08926_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(tier):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "stream_collide_d3q19_tgv256_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == tier and parts[1] == want:
                return float(parts[2])
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def tg_fields(n):
    """Closed-form Taylor-Green vortex at t = 0 (Sec. 4.2), extruded along z."""
    import workloads as W
    return W.taylor_green_extruded(n, 0.05)


def make_lattice(P, n, arith, storage, scheme="AB", fields=None):
    g = P.Lattice(n, n, n, "D3Q19", "SRT", storage, arith, scheme, tau=0.53)
    if fields is not None:
        g.set_rho_u(*fields)
    return g


def max_over_ranks(dist, seconds, device):
    """The slowest rank's time (every rank gets it); `seconds` when not distributed."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, cells, steps, seconds):
    """Whole-job throughput: every rank advances its own replica of `cells`."""
    return world * cells * steps / seconds / 1e6


def time_steps(torch, g, steps):
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record()
    g.step(steps)
    s1.record()
    torch.cuda.synchronize()
    return s0.elapsed_time(s1) / 1e3


def cpu_baseline(n, storage, budget_s=10.0):
    """The oracle (FP32 arithmetic in the paper's order + the storage codec),
    as it stands, on a bounded sample: whole steps of the same lattice until
    ~budget_s of CPU time."""
    import oracle
    import workloads as W
    o = oracle.Lattice(n, n, n, "D3Q19", "SRT", "ORD32", storage, tau=0.53)
    o.set_rho_u(*W.taylor_green_extruded(n, 0.05))
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    k = max(1, min(50, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * k / dt / 1e6, "unit": "MLUPs/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{k} oracle steps (after 1 warm-up) of the same D3Q19 SRT TGV {n}^3 lattice, "
                      f"FP32 ordered arithmetic with {storage} storage",
            "cpu_model": cpu_model(), "one_core": oracle_one_core(storage=storage)}


def cpu_model():
    """The host CPU's model name (lscpu), else its architecture."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def oracle_one_core(n=64, storage="FP16S", budget_s=2.0):
    """The same oracle step on one thread, on an n^3 sample of the workload."""
    import oracle
    import workloads as W
    threads = oracle.threads()
    oracle.set_threads(1)
    try:
        o = oracle.Lattice(n, n, n, "D3Q19", "SRT", "ORD32", storage, tau=0.53)
        o.set_rho_u(*W.taylor_green_extruded(n, 0.05))
        t0 = time.perf_counter()
        o.step(1)
        k = max(1, min(50, int(budget_s / max(time.perf_counter() - t0, 1e-6))))
        t0 = time.perf_counter()
        o.step(k)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    return {"value": n ** 3 * k / dt / 1e6, "unit": "MLUPs/s", "cores": 1,
            "sample": f"{k} oracle steps of a {n}^3 D3Q19 SRT TGV lattice, FP32 ordered arithmetic, {storage} storage"}


def oracle_cavity(n, storage, tau, u_lid, budget_s=4.0):
    """The oracle on the same cavity (all host cores): MLUPs/s over a few steps."""
    import oracle
    import workloads as W
    o = oracle.Lattice(n, n, n, "D3Q19", "TRT", "ORD32", storage, tau=tau)
    flags, node_u = W.cavity(n, u_lid)
    o.set_geometry(flags, node_u)
    o.set_rho_u()
    t0 = time.perf_counter()
    o.step(1)
    k = max(1, min(20, int(budget_s / max(time.perf_counter() - t0, 1e-6))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * k / dt / 1e6, "cores": oracle.threads(), "steps": k}


def run_ensemble(P, torch, steps, warmup, count=512, seed=20211216):
    import workloads as W
    specs = W.ensemble_cavities(count=count, seed=seed)
    cells = sum(s.n ** 3 for s in specs)

    def build():
        mem = []
        for s in specs:
            g = P.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=s.tau)
            flags, node_u = W.cavity(s.n, s.u_lid)
            g.set_geometry(flags, node_u)
            g.set_rho_u()
            mem.append(g)
        return mem

    mem = build()
    e = P.Ensemble(mem)
    bx, by = e.autotune(trial_steps=3)
    scheme, kernel, layout = e.scheme(), e.variant(), e.layout()
    e.step(warmup)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record()
    e.step(steps)
    ev[1].record()
    e.step_each(warmup)
    torch.cuda.synchronize()
    ev[2].record()
    e.step_each(steps)
    ev[3].record()
    torch.cuda.synchronize()
    t_b = ev[0].elapsed_time(ev[1]) / 1e3
    t_e = ev[2].elapsed_time(ev[3]) / 1e3
    e.close()
    for g in mem:
        g.close()
    peak, _ = peaks()
    bpc = 2 * 19 * 2 + 1   # 16-bit populations read and written, own flag byte
    return {"workload": f"{count} D3Q19 SRT lid-driven cavities, edges U{{16..128}} (splitmix64 seed {seed}), "
                        f"tau U[0.51,0.9], lid U[0.02,0.1], FP32/FP16S, member layout, kernel, tile and streaming scheme autotuned",
            "cells": cells, "steps": steps, "tile": [bx, by], "scheme": scheme, "kernel": kernel, "layout": layout,
            "batched_mlups": cells * steps / t_b / 1e6, "per_launch_mlups": cells * steps / t_e / 1e6,
            "bytes_per_cell": bpc, "frac_hbm": bpc * cells * steps / t_b / 1e9 / peak,
            "per_launch_frac_hbm": bpc * cells * steps / t_e / 1e9 / peak,
            "speedup": t_e / t_b, "launches_per_step": {"batched": 2, "per_launch": 2 * count}}


def small_ensembles(P, torch, steps, warmup, edges=(32, 48, 64), total=256 ** 3):
    """Small lattices alone fill little of the GPU: for each edge n, one FP16S
    lid-driven cavity n^3 (D3Q19 SRT, CUDA graphs of 32 steps) against an
    ensemble of equal members with about `total` cells in all (member layout,
    kernel, tile and scheme autotuned), both timed with CUDA events."""
    import workloads as W
    peak, _ = peaks()
    bpc = 2 * 19 * 2 + 1
    rows = []
    for n in edges:
        count = max(1, total // n ** 3)

        def member():
            g = P.Lattice(n, n, n, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.6)
            flags, node_u = W.cavity(n, 0.1)
            g.set_geometry(flags, node_u)
            g.set_rho_u()
            return g

        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        one = member()
        one.step(64)
        torch.cuda.synchronize()
        ev[0].record(); one.step(steps); ev[1].record()
        torch.cuda.synchronize()
        t_one = ev[0].elapsed_time(ev[1]) / 1e3
        one.close()
        mem = [member() for _ in range(count)]
        e = P.Ensemble(mem)
        bx, by = e.autotune(trial_steps=3)
        e.step(max(warmup, 64))
        torch.cuda.synchronize()
        ev[0].record(); e.step(steps); ev[1].record()
        torch.cuda.synchronize()
        t_ens = ev[0].elapsed_time(ev[1]) / 1e3
        layout, kernel, scheme = e.layout(), e.variant(), e.scheme()
        e.close()
        for g in mem:
            g.close()
        cells = count * n ** 3
        rows.append({"edge": n, "members": count, "cells": cells, "steps": steps,
                     "single_mlups": n ** 3 * steps / t_one / 1e6,
                     "single_frac_hbm": bpc * n ** 3 * steps / t_one / 1e9 / peak,
                     "ensemble_mlups": cells * steps / t_ens / 1e6,
                     "ensemble_frac_hbm": bpc * cells * steps / t_ens / 1e9 / peak,
                     "tile": [bx, by], "layout": layout, "kernel": kernel, "scheme": scheme})
    return rows


def cavity_sweep(P, torch, steps, formats=("FP32", "FP16S", "FP16C"), re=1000.0, u_lid=0.1, only=None,
                 with_oracle=True):
    """D3Q19 TRT lid-driven cavities N^3 (wall shell included, lid z = N-1
    moving along +y, rho = 1, u = 0 at start, tau from Re = u_lid (N-2) / nu):
    FP32 storage up to 512^3, 16-bit up to 1024^3 (A-B below 768^3, in-place
    A-A from 768^3 on).  Algorithmic bytes per cell: 2 q s + 1 (own flag).
    At 128^3 and 256^3 the oracle's rate on the same cavity (all host cores,
    a few steps) is reported beside the GPU's."""
    import workloads as W
    peak, _ = peaks()
    rows = []
    for storage in formats:
        sizes = [64, 96, 128, 192, 256, 384, 512] + ([] if storage in ("FP32", "FP64") else [768, 1024])
        for n in sizes:
            if only and n not in only:
                continue
            scheme = "AA" if n >= 768 else "AB"
            tau = 0.5 + 3.0 * u_lid * (n - 2) / re
            g = P.Lattice(n, n, n, "D3Q19", "TRT", storage, "FP32", scheme, tau=tau)
            g.set_geometry(W.cavity_flags(n))
            g.set_nodes(*W.cavity_lid(n, u_lid))
            g.set_rho_u()
            g.step(5)
            dt = time_steps(torch, g, steps)
            m, e = g.reduce()
            info = g.info()
            g.close()
            cells = n ** 3
            b = 2 * 19 * pop_bytes(storage) + 1
            rows.append({"storage": storage, "n": n, "scheme": scheme, "tau": tau, "steps": steps,
                         "mlups": cells * steps / dt / 1e6, "gbs": b * cells * steps / dt / 1e9,
                         "frac_hbm": b * cells * steps / dt / 1e9 / peak, "bytes_per_cell": b,
                         "device_gb": info.device_bytes / 1e9, "kinetic_energy": e})
            if with_oracle and n in (128, 256) and storage != "FP64":
                rows[-1]["oracle"] = oracle_cavity(n, storage, tau, u_lid)
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return rows


def strouhal(t, uy, d, u):
    """St = f D / U from the mean spacing of upward zero crossings of u_y."""
    t, uy = np.asarray(t, dtype=np.float64), np.asarray(uy, dtype=np.float64)
    up = np.flatnonzero((uy[:-1] < 0) & (uy[1:] >= 0))
    if up.size < 2:
        return None
    tc = t[up] - uy[up] * (t[up + 1] - t[up]) / (uy[up + 1] - uy[up])   # linear interpolation
    return d / u / float(np.mean(np.diff(tc)))


def karman(P, torch, steps=50000, t0=20000, every=20, tiers=(("FP64", "FP64"), ("FP32", "FP32"), ("FP32", "FP16C"))):
    """D3Q19 SRT Karman vortex street, channel 1024 x 256 x 64 (Sec. 4.3 in a
    3-D channel): cylinder of radius 24 along z at x = 256, equilibrium
    inflow u = 0.05 at x = 0, zero-gradient outflow, free-slip side walls,
    Re = U D / nu = 250, no body force.  Per tier: Strouhal number from u_y
    probed at (352, 128, 32) over steps t0..steps, and the relative L2 of the
    final velocity field against the FP64 tier."""
    import workloads as W
    nx, ny, nz, r, u_in, re = 1024, 256, 64, 24, 0.05, 250.0
    tau = 0.5 + 3.0 * u_in * 2 * r / re
    flags, node_u, node_rho = W.karman_channel(nx, ny, nz, radius=r, cx=256, cy=128, u_in=u_in)
    fields = W.karman_initial_fields(nx, ny, nz, u_in=u_in)
    probe = np.array([352 + nx * (128 + ny * 32)], dtype=np.int64)
    out, ref = {}, None
    for arith, storage in tiers:
        g = P.Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, "AB", tau=tau)
        g.set_geometry(flags, node_u, node_rho)
        g.set_rho_u(*fields)
        g.step(t0)
        ts, uys = [], []
        t_start = time.perf_counter()
        for t in range(t0, steps, every):
            uys.append(float(g.rho_u_cells(probe)[2][0]))
            ts.append(t)
            g.step(every)
        torch.cuda.synchronize()
        _, ux, uy, uz = g.rho_u()
        g.close()
        u = np.stack([ux, uy, uz])
        if ref is None:
            ref = u
        out[f"{arith}/{storage}"] = {
            "strouhal": strouhal(ts, uys, 2 * r, u_in), "l2_u_vs_fp64": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
            "uy_probe_rms": float(np.sqrt(np.mean(np.square(uys)))), "tau": tau, "steps": steps,
            "seconds_sampled_part": time.perf_counter() - t_start}
        print(json.dumps({f"{arith}/{storage}": out[f"{arith}/{storage}"]}), file=sys.stderr, flush=True)
    return out


def collision_sweep(P, torch, steps, n=256):
    """SRT, TRT and MRT on the periodic Taylor-Green workload for the tiers of
    the paper's roofline comparison (Sec. 5: three collision operators per
    number format): MLUPs/s and the HBM fraction of each."""
    import workloads as W
    peak, _ = peaks()
    fields = W.taylor_green_extruded(n, 0.05)
    rows = []
    for arith, storage in (("FP64", "FP64"), ("FP32", "FP32"), ("FP32", "FP16S"), ("FP32", "FP16C")):
        for coll in ("SRT", "TRT", "MRT"):
            g = P.Lattice(n, n, n, "D3Q19", coll, storage, arith, "AB", tau=0.53)
            g.set_rho_u(*fields)
            g.step(5)
            st = max(10, steps // (8 if arith == "FP64" else 1))
            dt = time_steps(torch, g, st)
            b = 2 * 19 * pop_bytes(storage)
            rows.append({"tier": f"{arith}/{storage}", "collision": coll, "variant": g.variant(),
                         "mlups": n ** 3 * st / dt / 1e6, "frac_hbm": b * n ** 3 * st / dt / 1e9 / peak})
            g.close()
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return rows


def velset_sweep(P, torch, steps):
    """D2Q9, D3Q19 and D3Q27 SRT on the periodic Taylor-Green workload (the
    velocity sets of the paper's roofline, Sec. 5), 16.8 M cells each
    (4096^2 for D2Q9, 256^3 otherwise): MLUPs/s and the HBM fraction for
    FP32, FP16S and FP16C storage with FP32 arithmetic."""
    import workloads as W
    peak, _ = peaks()
    rows = []
    for vs, q, (nx, ny, nz) in (("D2Q9", 9, (4096, 4096, 1)), ("D3Q19", 19, (256, 256, 256)),
                                ("D3Q27", 27, (256, 256, 256))):
        fields = W.taylor_green_extruded(nx, 0.05, nz=nz, ny=ny)
        for storage in ("FP32", "FP16S", "FP16C"):
            g = P.Lattice(nx, ny, nz, vs, "SRT", storage, "FP32", "AB", tau=0.53)
            g.set_rho_u(*fields)
            g.step(5)
            dt = time_steps(torch, g, steps)
            cells, b = nx * ny * nz, 2 * q * pop_bytes(storage)
            rows.append({"velset": vs, "storage": storage, "variant": g.variant(), "cells": cells,
                         "mlups": cells * steps / dt / 1e6, "bytes_per_cell": b,
                         "frac_hbm": b * cells * steps / dt / 1e9 / peak})
            g.close()
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return rows


def bench_reference(args, rank, world, budget_s=150.0):
    """The oracle, as it stands, on the same workload as our arm: the periodic
    Taylor-Green vortex on 256^2 planes (D3Q19 SRT, FP32 ordered arithmetic,
    the storage format of the run).  Every step is one oracle step of the
    whole 256^3 lattice when the warm-up and timed steps fit about budget_s of
    host time; otherwise of a z-slab of the same planes (periodic in z), as
    many planes as fit, and the sample says how many."""
    if rank != 0:
        return
    import oracle
    import workloads as W
    n = args.size
    probe = oracle.Lattice(n, n, 4, "D3Q19", "SRT", "ORD32", args.format, tau=0.53)
    probe.set_rho_u(*[a[:4] for a in W.taylor_green_extruded(n, 0.05)])
    probe.step(1)
    t0 = time.perf_counter()
    probe.step(2)
    per_plane = (time.perf_counter() - t0) / 8
    del probe
    nz = int(max(1, min(n, budget_s / max(per_plane * (args.steps + args.warmup), 1e-9))))
    fields = [a[:nz] for a in W.taylor_green_extruded(n, 0.05)]
    o = oracle.Lattice(n, n, nz, "D3Q19", "SRT", "ORD32", args.format, tau=0.53)
    o.set_rho_u(*fields)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    cells = n * n * nz
    v = cells * args.steps / dt / 1e6
    what = f"the whole {n}^3 lattice" if nz == n else f"a {n}x{n}x{nz} z-slab of it (periodic in z)"
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3 * (n * n * n) / cells,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"D3Q19 SRT Taylor-Green vortex (2-D closed form extruded along z), "
                               f"periodic {n}^3, u0=0.05, tau=0.53",
                   "storage": args.format, "arithmetic": "FP32", "scheme": "AB"},
        "cpu_baseline": {"value": v, "unit": "MLUPs/s", "kind": "oracle", "cores": oracle.threads(),
                         "sample": f"each step one oracle step of {what} (FP32 ordered arithmetic, "
                                   f"{args.format} storage); ms_per_step scaled to the whole lattice"},
        "e2e": {"value": v, "unit": "MLUPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=int(os.environ.get("WORLD_SIZE", "1")))
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--format", default="FP16S")
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--scheme", default="AB", choices=["AB", "AA"])
    ap.add_argument("--no-sweep", action="store_true", help="headline tier only")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cavity-sweep", action="store_true",
                    help="only the D3Q19 TRT lid-driven cavity size sweep (one JSON line)")
    ap.add_argument("--cavity-sizes", default="", help="comma-separated subset of the sweep's edge lengths")
    ap.add_argument("--collisions", action="store_true",
                    help="only SRT / TRT / MRT per number format on the Taylor-Green workload")
    ap.add_argument("--velsets", action="store_true",
                    help="D2Q9 / D3Q19 / D3Q27 throughput per storage format instead of the default run")
    ap.add_argument("--karman", action="store_true",
                    help="only the Karman vortex street accuracy run (Strouhal number, L2 vs FP64)")
    ap.add_argument("--small-ensembles", action="store_true",
                    help="only small cavities alone against ensembles of equal members")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        bench_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2112_08926_gb300 as P

    if args.collisions:
        if rank == 0:
            print(json.dumps({"collisions": collision_sweep(P, torch, args.steps)}), flush=True)
        return

    if args.velsets:
        if rank == 0:
            print(json.dumps({"velsets": velset_sweep(P, torch, args.steps)}), flush=True)
        return

    if args.karman:
        if rank == 0:
            print(json.dumps({"karman": karman(P, torch)}), flush=True)
        return

    if args.small_ensembles:
        if rank == 0:
            print(json.dumps({"small_ensembles": small_ensembles(P, torch, args.steps, args.warmup)}), flush=True)
        return

    if args.cavity_sweep:
        if rank == 0:
            only = [int(v) for v in args.cavity_sizes.split(",")] if args.cavity_sizes else None
            rows = cavity_sweep(P, torch, args.steps, only=only)
            print(json.dumps({"cavity_sweep": rows, "peak_gbs": peaks()[0]}), flush=True)
        return

    n = args.size
    N = n ** 3
    fields = tg_fields(n)
    head_arith = "FP64" if args.format == "FP64" else "FP32"
    g = make_lattice(P, n, head_arith, args.format, args.scheme, fields)
    variant_used = g.variant()
    g.step(args.warmup)
    m0, _ = g.reduce()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clk:
        elapsed = time_steps(torch, g, args.steps)
    elapsed = max_over_ranks(dist, elapsed, "cuda")
    m1, e1 = g.reduce()
    value = job_mlups(world, N, args.steps, elapsed)
    ms = elapsed / args.steps * 1e3
    bpc = 2 * 19 * pop_bytes(args.format)
    peak, peak_kind = peaks()
    achieved = bpc * N / (elapsed / args.steps) / 1e9
    tier_name = f"{head_arith}/{args.format}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(tier_name), "peak_kind": peak_kind,
                "bytes_per_cell": bpc, "kernel": "stream-collide D3Q19 SRT %s A-B flag-free, variant %s" % (args.format, variant_used)}

    # end to end through the C ABI with pinned host buffers
    pin = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).pin_memory() for a in fields]
    outs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(4)]
    g.set_rho_u_ptr(*[p.data_ptr() for p in pin])
    g.step(args.warmup)
    g.get_rho_u_ptr(*[o.data_ptr() for o in outs])
    # the whole job (upload, K steps, readback) three times; the median job time
    jobs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_rho_u_ptr(*[p.data_ptr() for p in pin])
        g.step(args.steps)
        g.get_rho_u_ptr(*[o.data_ptr() for o in outs])
        torch.cuda.synchronize()
        jobs.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(dist, sorted(jobs)[1], "cuda")
    g.close()
    e2e = {"value": job_mlups(world, N, args.steps, e2e_t), "unit": "MLUPs/s",
           "h2d_bytes_per_step": 4 * N * 8 / args.steps, "d2h_bytes_per_step": 4 * N * 8 / args.steps}

    per_format, ens, cpu = None, None, None
    if rank == 0 and world == 1:
        if not args.no_sweep:
            per_format = {}
            for name, arith, storage in TIERS:
                steps = max(args.steps // (8 if arith == "FP64" else 2), 10)
                gg = make_lattice(P, n, arith, storage, "AB", fields)
                gg.step(args.warmup)
                dt = time_steps(torch, gg, steps)
                b = 2 * 19 * pop_bytes(storage)
                per_format[name] = {"mlups": N * steps / dt / 1e6, "gbs": b * N * steps / dt / 1e9,
                                    "frac_hbm": b * N * steps / dt / 1e9 / peak, "bytes_per_cell": b,
                                    "roofline_mlups": peak * 1e3 / b, "steps": steps,
                                    "variant": gg.variant(), "traffic": profiled_traffic(name)}
                gg.close()
            variants = {}
            for v in ("generic", "paired", "staged"):
                gg = make_lattice(P, n, head_arith, args.format, "AB", fields)
                gg.set_variant(v)
                if gg.variant() != v:
                    gg.close()
                    continue
                gg.step(args.warmup)
                steps = max(args.steps // 2, 10)
                dt = time_steps(torch, gg, steps)
                variants[v] = {"mlups": N * steps / dt / 1e6, "frac_hbm": bpc * N * steps / dt / 1e9 / peak}
                gg.close()
            per_format[f"{tier_name} kernel variants"] = variants
            gg = make_lattice(P, n, head_arith, args.format, "AA", fields)
            gg.step(args.warmup)
            steps = max(args.steps // 2, 10)
            dt = time_steps(torch, gg, steps)
            per_format[f"{tier_name} A-A"] = {"mlups": N * steps / dt / 1e6,
                                              "frac_hbm": bpc * N * steps / dt / 1e9 / peak,
                                              "bytes_per_cell": bpc, "steps": steps}
            gg.close()
        if not args.no_ensemble:
            ens = run_ensemble(P, torch, steps=500, warmup=args.warmup)
        if not args.no_cpu:
            cpu = cpu_baseline(n, args.format)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_A100_FP16S if args.format == "FP16S" else None,
        "baseline_ref": "paper appendix hardware table (Table 6), Nvidia A100 40GB, FP32/FP16S, D3Q19 SRT 256^3: 15455 MLUPs/s",
        "dtype": "f32" if head_arith == "FP32" else "f64", "data": "synthetic",
        "config": {"workload": f"D3Q19 SRT Taylor-Green vortex (2-D closed form extruded along z), "
                               f"periodic {n}^3, u0=0.05, tau=0.53",
                   "storage": args.format, "arithmetic": head_arith, "scheme": args.scheme,
                   "kernel": "flag-free periodic", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "clocks": clk.summary(), "e2e": e2e, "gpu_launches": args.steps,
        "check": {"mass_rel_drift": abs(m1 / m0 - 1), "kinetic_energy": e1},
        "cpu_baseline": cpu, "per_format": per_format, "ensemble": ens,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

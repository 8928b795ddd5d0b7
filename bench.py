#!/usr/bin/env python
"""Benchmark: LJ atom-steps/s of the FP32 pair loop with FP64 Velocity Verlet
on the large fcc solid (1,000,188 atoms, rc = 2.5, list cutoff 2.8, list
rebuilt every 10 steps, dt = 0.005), one B300.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LJ atom-steps/s (FP32 vs FP64) and classified atoms/s (MLP vs CNA, >=99.5% agree)"
UNIT = "atom-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=63, help="fcc cells per edge (63 -> 1,000,188 atoms)")
    ap.add_argument("--cpu-steps", type=int, default=10, help="oracle steps timed for the CPU baseline")
    ap.add_argument("--cpu-cells", type=int, default=44, help="fcc cells per edge of the CPU-baseline sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=200)
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def workload_desc(c, n):
    return {"workload": f"LJ fcc solid {c}^3 cells, {n} atoms, rho 0.8442, rc 2.5, list 2.8, rebuild every 10, "
                        f"dt 0.005, T 0.8, Gaussian noise 0.02",
            "atoms": n, "rc": 2.5, "r_list": 2.8, "rebuild_every": 10, "dt": 0.005,
            "pair_precision": "fp32 (Kahan sums)", "integration": "fp64",
            "l2": "inputs larger than L2 (neighbour list ~312 MB, positions 24 MB)",
            "cuda_graph": True, "energy_every": 10}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[3 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def lj_source_sha():
    h = hashlib.sha256()
    for name in ("md_kernels.cu", "md_kernels.cuh", "lj.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1704_03329_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_atom():
    """DRAM bytes per atom of the force kernel from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    p = os.path.join(ROOT, "profiles", "lj_force_fp32_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_sha") != lj_source_sha():
        return None
    return float(d["dram_bytes_per_atom"])


def cpu_baseline(c_cells, steps):
    """The oracle as it stands, single thread, on a bounded sample: the full
    workload for `steps` steps (including its list builds)."""
    import oracle
    from synth import configs
    c = configs.lj_solid(n_cells=c_cells)
    n = len(c["pos"])
    oracle.build()
    t0 = time.perf_counter()
    oracle.md_run(c["pos"], c["vel"], c["box"], steps, r_list=2.8, rebuild_every=10)
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 C oracle, {n} atoms x {steps} steps (set-up list build + rebuild every 10), "
                      f"{dt:.1f} s wall, 1 thread"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_cells, args.cpu_steps)
    from synth import configs
    n = len(configs.lj_solid(n_cells=args.cpu_cells)["pos"])
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.cpu_steps, "warmup": 0, "ms_per_step": n / cb["value"] * 1e3 if cb["value"] else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(args.cpu_cells, n), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1704_03329_b300 import lib as L
    from synth import configs

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    c = configs.lj_solid(seed=2 + rank, n_cells=args.cells)
    n = len(c["pos"])
    pos_h = torch.from_numpy(c["pos"]).pin_memory()
    vel_h = torch.from_numpy(c["vel"]).pin_memory()
    box = c["box"]
    ctx = L.Context(local)
    stream = torch.cuda.current_stream()

    def make_md(prec):
        return L.MD(ctx, [0, n], [box], r_list=2.8, rc=2.5, rebuild_every=10, max_nbr=128, prec=prec, energy_every=10)

    md = make_md(L.FP32)
    pos_d = pos_h.cuda()
    vel_d = vel_h.cuda()
    md.set_state(pos_d, vel_d)
    K, W = args.steps, args.warmup
    K = max(10, (K // 10) * 10)
    W = max(3, W)
    energies = torch.zeros((K, 2), dtype=torch.float64, device="cuda")
    md.run(W, None)
    ctx.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    sampler = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    k0 = ctx.kernel_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    md.run(K, energies)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.kernel_count() - k0
    clocks = sampler.stop()
    info = md.info()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n * K / (ms * 1e-3)

    # ---- force kernel alone: average launch duration ----------------------
    pairs, max_row = md.list_stats()
    R = 50
    md.forces()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(R):
        md.forces()
    f1.record(stream)
    torch.cuda.synchronize()
    f_ms = f0.elapsed_time(f1) / R
    alg_bytes = 36.0 * n + 4.0 * pairs  # cnt + own xq + float4 force + list entries
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (f_ms * 1e-3) / 1e9
    tpa = traffic_per_atom()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": (tpa * n if tpa is not None else None),
                "peak_source": peak_kind, "kernel": "k_lj_col32 (integrator pair loop, FP32, timed alone via ppmd_md_forces)",
                "kernel_ms": round(f_ms, 5), "algorithmic_bytes_per_launch": alg_bytes,
                "pairs_listed_per_atom": round(pairs / n, 2)}

    # ---- plain FP64 GPU path on the same workload -------------------------
    md64 = make_md(L.FP64)
    md64.set_state(pos_d, vel_d)
    md64.run(10)
    torch.cuda.synchronize()
    K64 = max(10, (args.fp64_steps // 10) * 10)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    md64.run(K64)
    g1.record(stream)
    torch.cuda.synchronize()
    value64 = n * K64 / (g0.elapsed_time(g1) * 1e-3)
    md64.close()

    # ---- end to end through the public API, host buffers ------------------
    md_e = make_md(L.FP32)
    pos_out = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    en_h = torch.empty((K, 2), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    pd = pos_h.to("cuda", non_blocking=True)
    vd = vel_h.to("cuda", non_blocking=True)
    md_e.set_state(pd, vd)
    md_e.run(K, energies)
    out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    md_e.get_state(out)
    pos_out.copy_(out, non_blocking=True)
    en_h.copy_(energies, non_blocking=True)
    barrier()
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * n * K / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 48.0 * n / K, "d2h_bytes_per_step": (24.0 * n + 16.0 * K) / K,
           "note": "pinned host positions+velocities in, set-up (sort, list, F(r0)), K steps, positions+energies out"}
    md_e.close()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(args.cpu_cells, args.cpu_steps)
    en = en_h.numpy()
    rows = en[9::10]
    drift = float((rows[-1].sum() - rows[0].sum()) / n) if len(rows) > 1 else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": workload_desc(args.cells, n),
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clocks,
            "fp64_gpu_path": {"value": value64, "unit": UNIT, "steps": K64,
                              "fp32_speedup": value / world / value64},
            "md_info": {"max_disp": info["max_disp"], "skin_warning": info["status"] == L.WARN_SKIN,
                        "total_energy_drift_per_atom": drift},
            "impl": "ours"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

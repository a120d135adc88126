"""Benchmark of the cubic Fokker-Planck closure on one or more GB300s.

A step is one pass of the closure pipeline over the Mach-10 cylinder-shaped
population (512 x 256 cells, ~12M particles, FP32 velocities): the moment
gather, the 9x9 assembly and the pivoted FP64 solve (fp_closure_exact,
FP32-moment mode).  Inputs are resident in HBM before the timed region;
the L2 is flushed (a 256 MB write) between timed steps, outside the step's
events.  `value` is closure cells/s over all ranks (weak scaling: every rank
closes its own seeded population, no collective on the data path).

Further keys: per-kernel timings and the roofline of the dominant kernel,
the exact FP64 path on the same cells, the end-to-end number through the
C ABI with host buffers, nvidia-smi clocks sampled during the timed region,
and the CPU oracle timed on host cores on a bounded sample.

--impl reference times the CPU oracle (the reference of this build) on the
same workload, a bounded sample per step.
"""

from __future__ import annotations

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

METRIC = "closure cells/s + particles/s (exact FP64, FP32-moment, surrogate) at stated C/Gamma error"
L2_FLUSH_BYTES = 256 << 20

# algorithmic work per unit ("Roofline accounting")
GATHER_BYTES_PER_PARTICLE_F32 = 12  # three f32 velocity components, read once
GATHER_BYTES_PER_CELL = 8 + 8 + 8 * 30  # offsets (one int64 per cell), tau is not read, moments written
SOLVE_BYTES_PER_CELL = 8 * 30 + 8 + 8 * 9 + 4  # moments + tau read, coeffs + flags written
SOLVE_FLOPS_PER_CELL = 658  # FP64 flops of assembly + elimination + back substitution (FMA = 2)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP64 FMA-chain peak measured on this machine's GB300 (152 SMs x ~2 FP64 FMA
# lanes per clock): 1.197 TFLOP/s.
FP64_PEAK_TFLOPS = 1.197


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        time.sleep(0.05)

    def summary(self):
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _population(name, seed):
    from paper_2606_15622_gb300 import populations as P
    return P.make(name, seed=seed)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2606_15622_gb300 import api

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    pop = _population(args.config, seed=3 + rank)
    n_cells, n_p = pop.n_cells, pop.n_particles
    v32 = torch.from_numpy(pop.v32).to(dev)
    v64 = torch.from_numpy(pop.v64).to(dev)
    off = torch.from_numpy(pop.offsets).to(dev)
    tau = torch.from_numpy(pop.tau).to(dev)
    mom = torch.empty((n_cells, 30), dtype=torch.float64, device=dev)
    coeffs = torch.empty((n_cells, 9), dtype=torch.float64, device=dev)
    flags = torch.empty((n_cells,), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    prm = api.default_params()
    stream = torch.cuda.current_stream()

    def step():
        api.fp_closure_exact(v32, off, tau, params=prm, prec="fp32", moments_out=mom, coeffs_out=coeffs,
                             flags_out=flags, stream=stream)

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(k):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    if args.only:
        # profiling mode: launch one kernel `steps` times (no timing output)
        fns = {"gather": lambda: api.fp_moments(v32, off, prec="fp32", moments_out=mom, stream=stream),
               "gather64": lambda: api.fp_moments(v64, off, prec="fp64", moments_out=mom, stream=stream),
               "solve": lambda: api.fp_closure_solve(mom, tau, params=prm, prec="fp32", coeffs_out=coeffs,
                                                     flags_out=flags, stream=stream)}
        api.fp_moments(v32, off, prec="fp32", moments_out=mom, stream=stream)
        for _ in range(args.steps):
            fns[args.only]()
        torch.cuda.synchronize()
        print(json.dumps({"profiled": args.only, "launches": args.steps, "config": pop.name}))
        return

    # ---- headline: the timed region ------------------------------------
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed(step, args.steps, 0)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = float(np.sum(times))
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    cells_per_s = ws * n_cells / (ms_per_step * 1e-3)
    parts_per_s = ws * n_p / (ms_per_step * 1e-3)

    # ---- per-kernel timings (the two halves, same stream) -------------------
    t_gather = timed(lambda: api.fp_moments(v32, off, prec="fp32", moments_out=mom, stream=stream), 10, 3)
    t_solve = timed(lambda: api.fp_closure_solve(mom, tau, params=prm, prec="fp32", coeffs_out=coeffs,
                                                 flags_out=flags, stream=stream), 10, 3)
    g_ms, s_ms = float(np.median(t_gather)), float(np.median(t_solve))
    peaks = _peaks()
    gather_bytes = GATHER_BYTES_PER_PARTICLE_F32 * n_p + GATHER_BYTES_PER_CELL * n_cells
    gather_gbs = gather_bytes / (g_ms * 1e-3) / 1e9
    solve_tflops = SOLVE_FLOPS_PER_CELL * n_cells / (s_ms * 1e-3) / 1e12
    kernels = {
        "gather_fp32": {"ms": g_ms, "bound": "hbm", "achieved": gather_gbs, "unit": "GB/s",
                        "peak": peaks["hbm_gbs"], "frac": gather_gbs / peaks["hbm_gbs"],
                        "algorithmic_bytes": gather_bytes},
        "solve_fp64": {"ms": s_ms, "bound": "alu", "achieved": solve_tflops, "unit": "TFLOP/s",
                       "peak": FP64_PEAK_TFLOPS, "frac": solve_tflops / FP64_PEAK_TFLOPS,
                       "algorithmic_flops": SOLVE_FLOPS_PER_CELL * n_cells},
    }
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    roofline = {"kernel": dom, "bound": dk["bound"], "achieved": round(dk["achieved"], 3), "peak": dk["peak"],
                "unit": dk["unit"], "frac": round(dk["frac"], 4), "traffic": None,
                "peak_src": peaks["src"] if dk["bound"] == "hbm" else "measured (FP64 FMA chain)"}

    # ---- the exact FP64 path on the same cells -------------------------------
    t64 = timed(lambda: api.fp_closure_exact(v64, off, tau, params=prm, prec="fp64", moments_out=mom,
                                             coeffs_out=coeffs, flags_out=flags, stream=stream), 5, 2)
    fp64_ms = float(np.median(t64))

    # ---- end to end through the C ABI with host buffers ----------------------
    h_v = torch.from_numpy(pop.v32).pin_memory()
    h_off = torch.from_numpy(pop.offsets).pin_memory()
    h_tau = torch.from_numpy(pop.tau).pin_memory()
    h_coeffs = torch.empty((n_cells, 9), dtype=torch.float64).pin_memory()
    h_flags = torch.empty((n_cells,), dtype=torch.int32).pin_memory()

    def e2e_step():
        v32.copy_(h_v, non_blocking=True)
        off.copy_(h_off, non_blocking=True)
        tau.copy_(h_tau, non_blocking=True)
        api.fp_closure_exact(v32, off, tau, params=prm, prec="fp32", moments_out=mom, coeffs_out=coeffs,
                             flags_out=flags, stream=stream)
        h_coeffs.copy_(coeffs, non_blocking=True)
        h_flags.copy_(flags, non_blocking=True)

    te = timed(e2e_step, max(3, args.steps), 2)
    e2e_ms = float(np.median(te))
    h2d = h_v.numel() * 4 + h_off.numel() * 8 + h_tau.numel() * 8
    d2h = h_coeffs.numel() * 8 + h_flags.numel() * 4

    out = {
        "metric": METRIC,
        "value": round(cells_per_s, 1),
        "unit": "cells/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 moments, f64 solve",
        "data": "synthetic (seeded Mach-10 cylinder-shaped population)",
        "config": {"workload": f"{pop.name}: {n_cells} cells, {n_p} particles per GPU",
                   "cells": n_cells, "particles": n_p, "velocities": "f32 SoA",
                   "prec": "fp32_moments", "eps2_hat": prm.eps2_hat,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "particles_per_s": round(parts_per_s, 1),
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in d.items()}
                    for k, d in kernels.items()},
        "roofline": roofline,
        "paths": {
            "exact_fp32_moments": {"ms": round(ms_per_step, 5), "cells_per_s": round(cells_per_s / ws, 1),
                                   "particles_per_s": round(parts_per_s / ws, 1)},
            "exact_fp64": {"ms": round(fp64_ms, 5), "cells_per_s": round(n_cells / (fp64_ms * 1e-3), 1),
                           "particles_per_s": round(n_p / (fp64_ms * 1e-3), 1), "velocities": "f64"},
        },
        "e2e": {"value": round(n_cells / (e2e_ms * 1e-3) * ws, 1), "unit": "cells/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 5)},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pop, budget_s=args.cpu_seconds)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def cpu_baseline(pop, budget_s=15.0, max_cells=None):
    """The oracle, as it stands, single-threaded on this host: moments +
    closure over consecutive blocks of cells until the time budget is used."""
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    done_cells = done_parts = 0
    blk = 4096
    start = 0
    while time.perf_counter() - t0 < budget_s and (max_cells is None or done_cells < max_cells):
        end = min(start + blk, pop.n_cells)
        a, b = int(pop.offsets[start]), int(pop.offsets[end])
        offs = pop.offsets[start:end + 1] - a
        m = O.moments(pop.v64[:, a:b], offs)
        O.closure(m, pop.tau[start:end])
        done_cells += end - start
        done_parts += b - a
        start = end % pop.n_cells
    el = time.perf_counter() - t0
    return {"value": round(done_cells / el, 1), "unit": "cells/s", "cores": 1, "kind": "oracle",
            "particles_per_s": round(done_parts / el, 1),
            "sample": f"{done_cells} cells ({done_parts} particles) of {pop.name} in {el:.1f} s, "
                      "FP64 moments + closure, 1 thread"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    pop = _population(args.config, seed=3)
    budget = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(pop, budget_s=budget / 4)
    per = [cpu_baseline(pop, budget_s=budget) for _ in range(args.steps)]
    value = float(np.median([p["value"] for p in per]))
    ms_per_step = pop.n_cells / value * 1e3
    out = {
        "metric": METRIC, "impl": "reference", "value": round(value, 1), "unit": "cells/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Mach-10 cylinder-shaped population)",
        "config": {"workload": f"{pop.name}: {pop.n_cells} cells, {pop.n_particles} particles (bounded sample per step)",
                   "cells": pop.n_cells, "particles": pop.n_particles},
        "cpu_baseline": {"value": round(value, 1), "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": per[0]["sample"]},
        "e2e": {"value": round(value, 1), "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cylinder", choices=["cylinder", "cavity", "couette"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["gather", "gather64", "solve"], default=None,
                    help="profiling mode: launch one kernel --steps times, print no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

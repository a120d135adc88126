"""Benchmark of the cubic Fokker-Planck closure pipeline on one or more GB300s.

Workload (per GPU): the Mach-10 cylinder-shaped population, 512 x 256 cells,
~12M particles, FP32 velocities, resident in HBM.  A step is one pass of the
whole hot path over that batch:
  1. exact closure, FP32 moments + FP64 pivoted solve   (fp_closure_exact)
  2. learned closure with exact fallback                 (fp_closure_surrogate)
  3. adjoint of sum(Y) to the moments and the velocities (fp_closure_backward)
  4. velocity update, Philox noise, in place             (fp_velocity_update)
The L2 is flushed (256 MB write) before every timed step, outside its events.
`value` = cells per second of that step over all ranks (weak scaling: every
rank runs its own seeded population, no collective on the data path).

Beside the headline: per-call and per-kernel timings with the roofline of the
dominant kernel; each path's own cells/s (exact FP64, FP32-moment, surrogate,
adjoint, velocity update, one training step); the learned closure on the
1,048,576-cell inference batch of held-out cells from the training
distributions, with its error against the exact closure and its fallback
rate; the end-to-end step through the C ABI with host buffers; nvidia-smi
clocks sampled during the timed region; and the CPU oracle timed on host
cores on a bounded sample.

--impl reference times the CPU oracle (the reference of the CUDA path) on the same
workload, a bounded sample per step.
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
# DRAM bytes (read + write) per launch on this workload, from one ncu capture
# of the current build of each kernel; None once a kernel has changed since
# DRAM bytes (read + write) of one launch in the ncu captures summarised under
# profiles/ (current kernels; a kernel changed since its capture has none)
NCU_DRAM_BYTES = {"velocity_update": 298.03e6, "gather_fp32": 175.77e6, "solve_fp64": 85.43e6,
                  "gather_fp64": 313.65e6}
ORACLE_BLOCK = 4096            # cells per block of the CPU oracle's timing
E2E_CHUNKS = 8                 # chunks of the host-resident step (copy / compute overlap)
WEIGHTS = os.path.join(ROOT, "paper_2606_15622_gb300", "weights", "surrogate_full.fpw")
WEIGHTS_LITE = os.path.join(ROOT, "paper_2606_15622_gb300", "weights", "surrogate_lite.fpw")

# algorithmic work per unit of each kernel
GATHER_BYTES_PER_PARTICLE = 12          # three FP32 components read once
GATHER_BYTES_PER_CELL = 8 + 8 * 31      # one offset read, the moment vector and <|c|^6> written
LITE_BYTES_PER_CELL = 8 + 8 * 14        # one offset read, the LITE moment vector written
VEL_BYTES_PER_PARTICLE = 24             # read + write three FP32 components
VEL_BYTES_PER_CELL = 8 + 8 * (3 + 1 + 3 + 9 + 1) + 4 + 4 + 8  # offset; U, theta, q, C, Gamma, tau; flags in/out; alpha
GATHER64_FLOPS_PER_PARTICLE = 61       # FP64 gather: 3 (mean) + 3 (centre) + 55 (26 monomial sums, FMA = 2)
SOLVE_MIXED_FP64_FLOPS_PER_CELL = 290  # mixed solve, FP64 part: the emitted entries (~150), b - A x (~135, FMA = 2), update
SOLVE_FLOPS_PER_CELL = 658              # FP64: assembly + elimination + back substitution (FMA = 2)
MLP_FLOPS_PER_CELL = 2 * (32 * 128 + 3 * 128 * 128 + 128 * 16)  # padded layer shapes
FP64_PEAK_TFLOPS = 1.197                # FP64 peak of a GB300, measured with independent DFMA chains


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


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
            time.sleep(0.3)
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
    from paper_2606_15622_gb300 import populations as P
    from paper_2606_15622_gb300 import surrogate as S

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    pop = _population(args.config, seed=3 + rank)
    n_cells, n_p = pop.n_cells, pop.n_particles
    v0 = torch.from_numpy(pop.v32).to(dev)          # pristine copy of M^0
    vb = [v0.clone(), torch.empty_like(v0)]          # M^n and M^{n+1}, swapped after every step
    cur = [0]
    v64 = torch.from_numpy(pop.v64).to(dev)
    off = torch.from_numpy(pop.offsets).to(dev)
    tau = torch.from_numpy(pop.tau).to(dev)
    mom = torch.empty((n_cells, 30), dtype=torch.float64, device=dev)
    m6 = torch.empty(n_cells, dtype=torch.float64, device=dev)
    coeffs = torch.empty((n_cells, 9), dtype=torch.float64, device=dev)
    flags = torch.empty((n_cells,), dtype=torch.int32, device=dev)
    flags_v = torch.empty_like(flags)                # the update's own copy (it adds FP_FLAG_ALPHA)
    coeffs_s = torch.empty_like(coeffs)
    flags_s = torch.empty_like(flags)
    gY = torch.ones((n_cells, 9), dtype=torch.float64, device=dev)
    gmom = torch.empty_like(mom)
    lu = torch.empty(api.lu_doubles(n_cells), dtype=torch.float64, device=dev)  # factors kept for the adjoint
    gv = torch.empty_like(v0)
    alpha = torch.empty(n_cells, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_r = torch.ones(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # weak scaling: the global problem is one population per rank; rank r owns
    # population r (its shard: no collective on the data path) and draws its
    # variates from its own counter range
    prm = api.default_params(particle_offset=rank << 40)
    # the gather -> solve -> adjoint chain is the critical path: its stream
    # gets the highest priority, so its blocks are dispatched first
    stream = torch.cuda.Stream(device=dev, priority=-3)
    torch.cuda.set_stream(stream)
    s_sur = torch.cuda.Stream(device=dev)            # learned closure
    s_vel = torch.cuda.Stream(device=dev)            # velocity update
    ev_mom, ev_coef, ev_sur, ev_vel = (torch.cuda.Event() for _ in range(4))
    sur = S.Surrogate.load(WEIGHTS, device=dev)
    s_ws = torch.empty(int(api.lib().fp_surrogate_workspace_bytes(n_cells)), dtype=torch.uint8, device=dev)
    step_idx = [0]

    def c_moments():
        # also <|c|^6>, so the velocity update reads the particles once
        api.fp_moments(vb[cur[0]], off, prec="fp32", moments_out=mom, stream=stream, m6_out=m6)

    def c_solve():
        # keeps its factors for the adjoint (fp_closure_backward(lu=...))
        api.fp_closure_solve(mom, tau, params=prm, prec="fp32", coeffs_out=coeffs, flags_out=flags, stream=stream,
                             lu_out=lu)

    def c_exact():
        # the exact closure as the step runs it: gather, then the solve that
        # also keeps its factors for the adjoint
        c_moments()
        c_solve()

    def c_surrogate(on=None):
        sur.closure(mom, tau, params=prm, prec="fp32", coeffs_out=coeffs_s, flags_out=flags_s, workspace=s_ws,
                    stream=on if on is not None else stream)

    def c_adjoint():
        api.fp_closure_backward(vb[cur[0]], off, tau, mom, coeffs, flags, gY, params=prm, grad_moments=gmom,
                                grad_v=gv, stream=stream, lu=lu)

    def c_velocity(on=None):
        # M^n -> M^{n+1} out of place: the adjoint still reads M^n meanwhile
        api.fp_velocity_update(vb[cur[0]], off, mom, coeffs, tau, flags_v, 0.1, params=prm, seed=1234,
                               step=step_idx[0], alpha_out=alpha, stream=on if on is not None else stream,
                               v_out=vb[1 - cur[0]], m6=m6)
        step_idx[0] += 1

    def c_velocity_call():
        flags_v.copy_(flags)
        c_velocity()

    calls = [("exact_closure", c_exact), ("surrogate_closure", c_surrogate), ("adjoint", c_adjoint),
             ("velocity_update", c_velocity_call)]

    def step():
        # Three streams.  The gather runs on the (high-priority) main stream;
        # the learned closure, which needs only the moments, starts beside the
        # FP64 solve; after the solve the velocity update (writes M^{n+1} to
        # the other buffer) and the FP64-bound adjoint (still reads M^n) run
        # side by side; all join before the step ends.
        c_moments()
        ev_mom.record(stream)
        s_sur.wait_event(ev_mom)
        c_surrogate(on=s_sur)
        ev_sur.record(s_sur)
        c_solve()
        ev_coef.record(stream)
        s_vel.wait_event(ev_coef)
        with torch.cuda.stream(s_vel):
            flags_v.copy_(flags)
        c_velocity(on=s_vel)
        ev_vel.record(s_vel)
        c_adjoint()
        stream.wait_event(ev_sur)
        stream.wait_event(ev_vel)
        cur[0] ^= 1

    def timed(fn, k, w, reset=None, clean=True):
        # L2 flush before each timed launch: a write larger than L2, then (clean)
        # a read larger than L2, so that the flush's dirty lines are written
        # back before the timed region instead of inside it; the step itself is
        # timed after the write alone (dirty lines drain inside it, as the
        # previous step's outputs would)
        for _ in range(w):
            if reset:
                reset()
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(k):
            if reset:
                reset()
            flush.fill_(1)
            if clean:
                flush_r.amax()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def reset_v():
        vb[0].copy_(v0)
        cur[0] = 0

    if args.only:
        # profiling mode: launch one call `steps` times (no bench line)
        fns = dict(calls)
        fns["gather"] = c_moments
        fns["solve"] = c_solve
        fns["gather64"] = lambda: api.fp_moments(v64, off, prec="fp64", moments_out=mom, stream=stream)
        fns["step"] = step
        c_exact()
        xf, _ = sur.features(mom, tau, params=prm)
        of = torch.empty((n_cells, 16), dtype=torch.float32, device=dev)
        fns["mlp"] = lambda: sur.forward(xf, standardized=False, out=of, stream=stream)
        cell_sorted = np.repeat(np.arange(n_cells), pop.counts)
        rng_cs = np.random.default_rng(17)
        moved = rng_cs.random(n_p) < 0.03
        c_near = np.where(moved, np.clip(cell_sorted + rng_cs.integers(-1, 2, n_p), 0, n_cells - 1), cell_sorted)
        c_near_d = torch.from_numpy(c_near.astype(np.int32)).to(dev)
        vs_b = torch.empty_like(v0)
        fns["sort"] = lambda: api.fp_sort_by_cell(c_near_d, n_cells, v=v0, v_sorted=vs_b, stream=stream)
        fns["collision"] = lambda: api.fp_collision_step(c_near_d, v0, n_cells, tau, 0.1, params=prm, prec="fp32",
                                                         v_out=vs_b, coeffs_out=coeffs, flags_out=flags,
                                                         stream=stream)
        lite = torch.empty((n_cells, api.NLITE), dtype=torch.float64, device=dev)
        fns["gather_lite"] = lambda: api.fp_moments_lite(vb[cur[0]], off, out=lite, stream=stream)
        if os.path.exists(WEIGHTS_LITE):
            sl = S.Surrogate.load(WEIGHTS_LITE, device=dev)
            fns["lite"] = lambda: (api.fp_moments_lite(vb[cur[0]], off, out=lite, stream=stream),
                                   sl.closure_lite(lite, tau, params=prm, coeffs_out=coeffs_s, flags_out=flags_s,
                                                   stream=stream))
        if args.only == "train":
            trs = S.Surrogate.load(WEIGHTS, device=dev)
            tr = S.Trainer(trs, batch=8192)
            ts = S.TrainingSet(P.training_cells(16384, seed=55), eps2_hat=prm.eps2_hat)
            xt = ts.inputs(trs)[:8192].contiguous()
            tt, at = ts.t[:8192].contiguous(), ts.aux[:8192].contiguous()
            fns["train"] = lambda: tr.step(xt, tt, at, 1.0 / 8192)
        for _ in range(args.steps):
            fns[args.only]()
        torch.cuda.synchronize()
        print(json.dumps({"profiled": args.only, "launches": args.steps, "config": pop.name}))
        return

    # ---- headline: the timed region -------------------------------------
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    reset_v()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed(step, args.steps, 0, clean=False)
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
    # the learned closure's flags of the last step (later legs reuse the buffer)
    step_fallback_rate = float(((flags_s & api.FLAG_FALLBACK) != 0).double().mean())
    step_range_rate = float(((flags_s & api.FLAG_RANGE) != 0).double().mean())
    step_energy_rate = float(((flags_s & api.FLAG_ENERGY) != 0).double().mean())

    # ---- per call, per kernel ------------------------------------------------
    peaks = _peaks()
    per_call = {name: float(np.median(timed(fn, 10, 2))) for name, fn in calls}
    t_gather = float(np.median(timed(c_moments, 10, 2)))
    t_vel = float(np.median(timed(c_velocity, 10, 2)))  # the update kernel alone (flags copy excluded)
    # the step's solve keeps the FP64 factors for the adjoint; without factors
    # FP32 moments take the mixed-precision solve
    t_solve = float(np.median(timed(lambda: api.fp_closure_solve(mom, tau, params=prm, prec="fp32",
                                                                 coeffs_out=coeffs, flags_out=flags, lu_out=lu,
                                                                 stream=stream), 10, 2)))
    t_solve_mixed = float(np.median(timed(lambda: api.fp_closure_solve(mom, tau, params=prm, prec="fp32",
                                                                       coeffs_out=coeffs, flags_out=flags,
                                                                       stream=stream), 10, 2)))
    x_feat, _ = sur.features(mom, tau, params=prm)
    out16 = torch.empty((n_cells, 16), dtype=torch.float32, device=dev)
    t_mlp = float(np.median(timed(lambda: sur.forward(x_feat, standardized=False, out=out16, stream=stream), 10, 2)))
    t_g64 = float(np.median(timed(lambda: api.fp_moments(v64, off, prec="fp64", moments_out=mom, stream=stream), 5, 2)))
    # the exact FP32-moment closure as a caller without the adjoint runs it:
    # gather + mixed-precision solve (no factors kept)
    t_exact32 = float(np.median(timed(lambda: api.fp_closure_exact(vb[cur[0]], off, tau, params=prm, prec="fp32",
                                                                   moments_out=mom, coeffs_out=coeffs,
                                                                   flags_out=flags, stream=stream), 10, 2)))
    gather_bytes = GATHER_BYTES_PER_PARTICLE * n_p + GATHER_BYTES_PER_CELL * n_cells
    vel_bytes = VEL_BYTES_PER_PARTICLE * n_p + VEL_BYTES_PER_CELL * n_cells

    def kern(ms_, bound, achieved, unit, peak, work):
        return {"ms": round(ms_, 5), "bound": bound, "achieved": round(achieved, 4), "unit": unit, "peak": peak,
                "frac": round(achieved / peak, 4), **work}

    kernels = {
        "gather_fp32": kern(t_gather, "hbm", gather_bytes / (t_gather * 1e-3) / 1e9, "GB/s", peaks["hbm_gbs"],
                            {"algorithmic_bytes": gather_bytes}),
        "solve_fp64": kern(t_solve, "alu", SOLVE_FLOPS_PER_CELL * n_cells / (t_solve * 1e-3) / 1e12, "TFLOP/s",
                           FP64_PEAK_TFLOPS, {"algorithmic_flops": SOLVE_FLOPS_PER_CELL * n_cells,
                                              "peak_note": "FP64 pipe, measured FMA chain"}),
        "velocity_update": kern(t_vel, "hbm", vel_bytes / (t_vel * 1e-3) / 1e9, "GB/s", peaks["hbm_gbs"],
                                {"algorithmic_bytes": vel_bytes}),
        "solve_mixed": kern(t_solve_mixed, "alu", SOLVE_MIXED_FP64_FLOPS_PER_CELL * n_cells / (t_solve_mixed * 1e-3) / 1e12,
                            "TFLOP/s", FP64_PEAK_TFLOPS,
                            {"algorithmic_flops": SOLVE_MIXED_FP64_FLOPS_PER_CELL * n_cells,
                             "peak_note": "FP64 part only (FP64 assembly of the residual, refinement); the FP32 "
                                          "factorisation and solves run on the FP32 pipe"}),
        "gather_fp64": kern(t_g64, "alu", GATHER64_FLOPS_PER_PARTICLE * n_p / (t_g64 * 1e-3) / 1e12, "TFLOP/s",
                            FP64_PEAK_TFLOPS, {"algorithmic_flops": GATHER64_FLOPS_PER_PARTICLE * n_p,
                                               "peak_note": "FP64 pipe, measured FMA chain; an FP64 add or multiply "
                                                            "takes the pipe slot of an FMA, and idle lanes of a warp "
                                                            "instruction take it too (ncu: FP64 pipe 89 % busy)"}),
        "mlp_forward": kern(t_mlp, "tensor", MLP_FLOPS_PER_CELL * n_cells / (t_mlp * 1e-3) / 1e12, "TFLOP/s",
                            peaks["bf16_tflops"], {"algorithmic_flops": MLP_FLOPS_PER_CELL * n_cells}),
    }
    dom = max(("gather_fp32", "solve_fp64", "velocity_update", "mlp_forward"), key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    roofline = {"kernel": dom, "bound": dk["bound"], "achieved": dk["achieved"], "peak": dk["peak"],
                "unit": dk["unit"], "frac": dk["frac"], "traffic": NCU_DRAM_BYTES.get(dom),
                "peak_src": "measured (FP64 FMA chain)" if dk["bound"] == "alu" else peaks["src"]}

    def q(x, p):
        return round(float(torch.quantile(x, p)), 6)

    # ---- the exact FP64 path on the same cells ----------------------------------
    t64 = float(np.median(timed(lambda: api.fp_closure_exact(v64, off, tau, params=prm, prec="fp64",
                                                             moments_out=mom, coeffs_out=coeffs, flags_out=flags,
                                                             stream=stream), 5, 2)))
    # ---- error of the learned closure on these cells against the exact FP64 closure --
    mom64, y64, fl64 = torch.empty_like(mom), torch.empty_like(coeffs), torch.empty_like(flags)
    api.fp_closure_exact(v64, off, tau, params=prm, prec="fp64", moments_out=mom64, coeffs_out=y64, flags_out=fl64,
                         stream=stream)
    torch.cuda.synchronize()
    sur_err = S.error_report(sur, mom64, tau, y64, fl64, prm.eps2_hat, params=prm)
    reset_v()   # M^0, the particles of the FP64 reference above
    c_exact()   # as deployed in the step: the learned closure on the FP32-moment gather's moments
    c_surrogate()
    torch.cuda.synchronize()
    t_ex64 = S.dimensionless(y64, mom64, tau)
    ok64 = fl64 == 0
    rel_dep = ((S.dimensionless(coeffs_s, mom64, tau) - t_ex64).norm(dim=1) / t_ex64.norm(dim=1))[ok64].float().cpu()
    sur_err["rel_err_closure_as_deployed_fp32_moments"] = {
        "median": round(float(rel_dep.median()), 7), "p95": round(float(torch.quantile(rel_dep, 0.95)), 7),
        "p99": round(float(torch.quantile(rel_dep, 0.99)), 7), "max": round(float(rel_dep.max()), 7)}
    c_exact()
    torch.cuda.synchronize()

    # ---- learned closure on the 1M-cell inference batch -------------------
    inf = P.training_cells(131072, seed=987654)          # held-out seeds of the training distributions
    iv = torch.from_numpy(inf.v64).to(dev)
    ioff = torch.from_numpy(inf.offsets).to(dev)
    itau = torch.from_numpy(inf.tau).to(dev)
    imom, iy_ex, ifl_ex = api.fp_closure_exact(iv, ioff, itau, params=prm, prec="fp64")
    iy_s, ifl_s = sur.closure(imom, itau, params=prm, prec="fp64")
    torch.cuda.synchronize()
    t_ex = S.dimensionless(iy_ex, imom, itau)
    t_s = S.dimensionless(iy_s, imom, itau)
    ok = ifl_ex == 0
    rel = ((t_s - t_ex).norm(dim=1) / t_ex.norm(dim=1))[ok].float().cpu()
    lin = torch.zeros_like(t_ex)
    lin[:, [0, 3, 5]] = -1.0
    rel_lin = ((lin - t_ex).norm(dim=1) / t_ex.norm(dim=1))[ok].float().cpu()
    # energy residual of the surrogate drift (exact closure: 0)
    ax = S.aux_moments(imom, itau)  # u^_ij, b^_i, s4^
    mult = torch.tensor([1, 2, 2, 1, 2, 1], dtype=torch.float64, device=dev)
    e = 1 + ((t_s[:, :6] * ax[:, :6] * mult).sum(1) + (t_s[:, 6:] * ax[:, 6:9]).sum(1) - prm.eps2_hat * ax[:, 9]) / 3
    reps = 8
    big_mom = imom.repeat(reps, 1).contiguous()
    big_tau = itau.repeat(reps).contiguous()
    nb = big_mom.shape[0]
    by = torch.empty((nb, 9), dtype=torch.float64, device=dev)
    bfl = torch.empty(nb, dtype=torch.int32, device=dev)
    bws = torch.empty(int(api.lib().fp_surrogate_workspace_bytes(nb)), dtype=torch.uint8, device=dev)
    t_sur_1m = float(np.median(timed(lambda: sur.closure(big_mom, big_tau, params=prm, prec="fp64", coeffs_out=by,
                                                         flags_out=bfl, workspace=bws, stream=stream), 10, 2)))
    t_ex_1m = float(np.median(timed(lambda: api.fp_closure_solve(big_mom, big_tau, params=prm, prec="fp64",
                                                                 coeffs_out=by, flags_out=bfl, stream=stream), 5, 2)))
    xb, _ = sur.features(big_mom, big_tau, params=prm)
    ob = torch.empty((nb, 16), dtype=torch.float32, device=dev)
    t_mlp_1m = float(np.median(timed(lambda: sur.forward(xb, standardized=False, out=ob, stream=stream), 10, 2)))
    fb_rate = float(((ifl_s & api.FLAG_FALLBACK) != 0).double().mean())

    # ---- the LITE path: low-order moment pass + network on 16 inputs --------
    lite_rep = None
    if os.path.exists(WEIGHTS_LITE):
        sl = S.Surrogate.load(WEIGHTS_LITE, device=dev)
        lite = torch.empty((n_cells, api.NLITE), dtype=torch.float64, device=dev)
        l_ws = torch.empty(int(api.lib().fp_surrogate_lite_workspace_bytes(n_cells)), dtype=torch.uint8, device=dev)

        def c_gather_lite():
            api.fp_moments_lite(vb[cur[0]], off, out=lite, stream=stream)

        def c_lite():
            c_gather_lite()
            sl.closure_lite(lite, tau, params=prm, coeffs_out=coeffs_s, flags_out=flags_s, workspace=l_ws,
                            stream=stream)

        t_gl = float(np.median(timed(c_gather_lite, 10, 2)))
        t_lite = float(np.median(timed(c_lite, 10, 2)))
        lite_bytes = GATHER_BYTES_PER_PARTICLE * n_p + LITE_BYTES_PER_CELL * n_cells
        kernels["gather_lite"] = kern(t_gl, "hbm", lite_bytes / (t_gl * 1e-3) / 1e9, "GB/s", peaks["hbm_gbs"],
                                      {"algorithmic_bytes": lite_bytes})
        torch.cuda.synchronize()
        lfb = float(((flags_s & api.FALLBACK_FLAGS) != 0).double().mean())
        lrng = float(((flags_s & api.FLAG_RANGE) != 0).double().mean())
        # accuracy on the held-out cells of the training distributions, beside the full-input network
        il = api.fp_moments_lite(iv, ioff)
        ly, lfl = sl.closure_lite(il, itau, params=prm)
        torch.cuda.synchronize()
        t_l = S.dimensionless(ly, imom, itau)
        rel_l = ((t_l - t_ex).norm(dim=1) / t_ex.norm(dim=1))[ok].float().cpu()
        lite_err = S.error_report(sl, mom64, tau, y64, fl64, prm.eps2_hat, params=prm,
                                  lite=api.fp_moments_lite(v64, off))
        # the coefficient-sensitivity probe of the cylinder study: 50 dropout passes at rate 0.2
        sens_ws = torch.empty(int(api.lib().fp_surrogate_sensitivity_workspace_bytes(n_cells)), dtype=torch.uint8,
                              device=dev)
        sens_o = torch.empty((n_cells, api.NSENS), dtype=torch.float64, device=dev)
        c_gather_lite()
        t_sens = float(np.median(timed(lambda: sl.sensitivity(lite, tau, n_passes=50, rate=0.2, seed=5, params=prm,
                                                              sens_out=sens_o, workspace=sens_ws, stream=stream),
                                       3, 1)))
        lite_rep = {"ms": round(t_lite, 5), "gather_lite_ms": round(t_gl, 5),
                    "sensitivity_probe": {"passes": 50, "rate": 0.2, "ms": round(t_sens, 4),
                                          "cell_passes_per_s": round(50 * n_cells / (t_sens * 1e-3), 1)},
                    "cells_per_s": round(n_cells / (t_lite * 1e-3), 1),
                    "speedup_vs_exact_fp32_moments": round(per_call["exact_closure"] / t_lite, 3),
                    "linear_drift_rate_cylinder": round(lfb, 5), "range_flag_rate_cylinder": round(lrng, 5),
                    "held_out_rel_err_vs_exact": {"median": q(rel_l, 0.5), "p95": q(rel_l, 0.95),
                                                  "max": round(float(rel_l.max()), 6)},
                    "full_input_network_rel_err": {"median": q(rel, 0.5), "p95": q(rel, 0.95)},
                    "error_vs_exact_fp64_cylinder": lite_err,
                    "note": "LITE moment pass (N, U, theta, u_ij, heat flux) + network on the 16 low-order "
                            "inputs; no exact fallback (flagged cells take the linear drift)"}

    # ---- collision step from particles in any order (sort + closure + update) --
    # "nearly sorted": the cell order of the previous step with 3 % of the
    # particles moved to a neighbouring cell; "shuffled": random order
    cell_sorted = np.repeat(np.arange(n_cells), pop.counts)
    rng_cs = np.random.default_rng(17)
    moved = rng_cs.random(n_p) < 0.03
    c_near = np.where(moved, np.clip(cell_sorted + rng_cs.integers(-1, 2, n_p), 0, n_cells - 1), cell_sorted)
    c_near_d = torch.from_numpy(c_near.astype(np.int32)).to(dev)
    shuf = rng_cs.permutation(n_p)
    c_shuf_d = torch.from_numpy(cell_sorted[shuf].astype(np.int32)).to(dev)
    sort_ws = torch.empty(int(api.lib().fp_sort_workspace_bytes(n_p, n_cells)), dtype=torch.uint8, device=dev)
    perm_b = torch.empty(n_p, dtype=torch.int32, device=dev)
    off_b = torch.empty(n_cells + 1, dtype=torch.int64, device=dev)
    vs_b = torch.empty_like(v0)
    t_sort_near = float(np.median(timed(lambda: api.fp_sort_by_cell(c_near_d, n_cells, v=v0, v_sorted=vs_b,
                                                                    perm_out=perm_b, offsets_out=off_b,
                                                                    workspace=sort_ws, stream=stream), 10, 2)))
    t_sort_shuf = float(np.median(timed(lambda: api.fp_sort_by_cell(c_shuf_d, n_cells, v=v0, v_sorted=vs_b,
                                                                    perm_out=perm_b, offsets_out=off_b,
                                                                    workspace=sort_ws, stream=stream), 10, 2)))
    cs_ws = torch.empty(int(api.lib().fp_collision_step_workspace_bytes(n_p, n_cells, api.V_F32, 1)),
                        dtype=torch.uint8, device=dev)
    cs_ws_ex = torch.empty(int(api.lib().fp_collision_step_workspace_bytes(n_p, n_cells, api.V_F32, 0)),
                           dtype=torch.uint8, device=dev)

    def c_collision(lite_net=None, cells=c_near_d):
        api.fp_collision_step(cells, v0, n_cells, tau, 0.1, params=prm, prec="fp32", net_lite=lite_net, seed=1234,
                              step=step_idx[0], v_out=vs_b, perm_out=perm_b, offsets_out=off_b, coeffs_out=coeffs,
                              flags_out=flags, workspace=cs_ws if lite_net is not None else cs_ws_ex, stream=stream)

    t_cs_ex = float(np.median(timed(lambda: c_collision(None), 10, 2)))
    t_cs_lite = float(np.median(timed(lambda: c_collision(sl.net()), 10, 2))) if lite_rep is not None else None
    collision_rep = {
        "input": "cylinder particles; nearly sorted = previous cell order with 3 % moved to a neighbouring cell",
        "sort_nearly_sorted_ms": round(t_sort_near, 5), "sort_shuffled_ms": round(t_sort_shuf, 5),
        "sort_particles_per_s": round(n_p / (t_sort_near * 1e-3), 1),
        "exact_step_ms": round(t_cs_ex, 5), "exact_step_particles_per_s": round(n_p / (t_cs_ex * 1e-3), 1),
        "lite_step_ms": round(t_cs_lite, 5) if t_cs_lite else None,
        "lite_step_particles_per_s": round(n_p / (t_cs_lite * 1e-3), 1) if t_cs_lite else None,
        "note": "one fp_collision_step call: stable radix sort by cell, velocity gather, moments, closure "
                "(exact FP32-moment / FP64 solve, or the learned closure on LITE inputs), velocity update"}

    # ---- adjoint on the cavity-shaped population (C4) -----------------------
    cav = P.cavity(seed=4)
    cv = torch.from_numpy(cav.v32).to(dev)
    coff, ctau = torch.from_numpy(cav.offsets).to(dev), torch.from_numpy(cav.tau).to(dev)
    cm, cy, cfl = api.fp_closure_exact(cv, coff, ctau, params=prm, prec="fp32")
    cg = torch.ones_like(cy)
    cgm = torch.empty_like(cm)
    cgv = torch.empty_like(cv)
    t_fwd_c4 = float(np.median(timed(lambda: api.fp_closure_exact(cv, coff, ctau, params=prm, prec="fp32",
                                                                  moments_out=cm, coeffs_out=cy, flags_out=cfl,
                                                                  stream=stream), 10, 2)))
    t_bwd_c4 = float(np.median(timed(lambda: api.fp_closure_backward(cv, coff, ctau, cm, cy, cfl, cg, params=prm,
                                                                     grad_moments=cgm, grad_v=cgv, stream=stream),
                                     10, 2)))

    # ---- one training step (batch 8192) ----------------------------------------
    import copy
    trs = S.Surrogate.load(WEIGHTS, device=dev)
    tr = S.Trainer(trs, batch=8192)
    ts = S.TrainingSet(P.training_cells(16384, seed=55), eps2_hat=prm.eps2_hat)
    xt = ts.inputs(trs)[:8192].contiguous()
    tt, at = ts.t[:8192].contiguous(), ts.aux[:8192].contiguous()
    t_train = float(np.median(timed(lambda: tr.step(xt, tt, at, 1.0 / 8192), 10, 3)))

    # ---- end to end through the C ABI with host buffers -------------------
    # fp_step_host: the same step on host-resident (pinned) velocities; the
    # cells are split into chunks whose copies overlap the others' compute
    h_v = torch.from_numpy(pop.v32).pin_memory()
    h_off = torch.from_numpy(pop.offsets).pin_memory()
    h_tau = torch.from_numpy(pop.tau).pin_memory()
    h_coeffs = torch.empty((n_cells, 9), dtype=torch.float64).pin_memory()
    h_flags = torch.empty((n_cells,), dtype=torch.int32).pin_memory()
    h_vout = torch.empty_like(h_v).pin_memory()
    hstep = api.HostStep(n_cells, n_p, dtype=torch.float32, surrogate=sur, adjoint=True, device=dev)

    def e2e_step():
        hstep(h_v, h_off, h_tau, h_vout, h_coeffs, h_flags, 0.1, params=prm, prec="fp32", seed=1234,
              step=step_idx[0], n_chunks=E2E_CHUNKS, stream=stream)
        step_idx[0] += 1

    te = timed(e2e_step, max(3, args.steps), 2)
    e2e_ms = float(np.median(te))
    h2d = h_v.numel() * 4 + h_off.numel() * 8 + h_tau.numel() * 8
    d2h = h_coeffs.numel() * 8 + h_flags.numel() * 4 + h_vout.numel() * 4
    # gather, solve; learned closure (one tcgen05 kernel) + its exact fallback; update; adjoint x2
    launches_per_step = 2 + 2 + 1 + 2

    out = {
        "metric": METRIC,
        "value": round(cells_per_s, 1),
        "unit": "cells/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "step_ms": step_stats(times),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 moments, f64 solve, bf16/f32 MLP",
        "data": f"synthetic (seeded population {pop.name}; no paper data)",
        "config": {"workload": f"{pop.name}: {n_cells} cells, {n_p} particles per GPU",
                   "step": "exact closure (FP32 moments, FP64 solve) + learned closure with exact fallback + "
                           "adjoint to moments and velocities + velocity update",
                   "cells": n_cells, "particles": n_p, "velocities": "f32 SoA", "eps2_hat": prm.eps2_hat,
                   "l2": "flushed before every timed step (256 MB write); before every per-call and per-kernel timing by a 256 MB write then a 256 MB read (no flush write-backs inside those timed regions)", "parallelism": f"replicas x{ws}",
                   "streams": "learned closure beside the FP64 solve; then velocity update (out of place) and "
                              "adjoint side by side; three streams"},
        "particles_per_s": round(parts_per_s, 1),
        "per_call_ms": {k: round(v, 5) for k, v in per_call.items()},
        "kernels": kernels,
        "roofline": roofline,
        "paths": {
            "exact_fp32_moments": {"ms": round(t_exact32, 5),
                                   "cells_per_s": round(n_cells / (t_exact32 * 1e-3), 1),
                                   "particles_per_s": round(n_p / (t_exact32 * 1e-3), 1),
                                   "solve": "mixed precision (FP32 factors, FP64 residual, one refinement; "
                                            "agrees with the FP64 solve to <= 4e-9 on the cylinder)",
                                   "with_factors_for_the_adjoint_ms": round(per_call["exact_closure"], 5),
                                   "error_vs_oracle": "<= 1e-4 relative, or kappa * 2^-24 on 7 of 131,021 "
                                                      "cylinder cells (parity coverage test)"},
            "exact_fp64": {"ms": round(t64, 5), "cells_per_s": round(n_cells / (t64 * 1e-3), 1),
                           "particles_per_s": round(n_p / (t64 * 1e-3), 1), "velocities": "f64",
                           "error_vs_oracle": "<= 1e-10 relative (parity tests)"},
            "surrogate_on_cylinder": {"ms": round(per_call["surrogate_closure"], 5),
                                      "fallback_rate": round(step_fallback_rate, 5),
                                      "range_flag_rate": round(step_range_rate, 5),
                                      "energy_flag_rate": round(step_energy_rate, 5),
                                      "error_vs_exact_fp64": sur_err,
                                      "note": "flags of the step's learned closure: cells outside the training "
                                              "box (range) or with a large energy residual are recomputed by the "
                                              "exact closure"},
            "surrogate_1M": {"cells": nb, "ms": round(t_sur_1m, 5), "cells_per_s": round(nb / (t_sur_1m * 1e-3), 1),
                             "mlp_forward_ms": round(t_mlp_1m, 5),
                             "exact_solve_same_moments_ms": round(t_ex_1m, 5),
                             "speedup_vs_exact_solve": round(t_ex_1m / t_sur_1m, 3),
                             "fallback_rate": round(fb_rate, 5),
                             "rel_err_vs_exact": {"median": q(rel, 0.5), "p95": q(rel, 0.95),
                                                  "max": round(float(rel.max()), 6)},
                             "rel_err_linear_closure": {"median": q(rel_lin, 0.5), "p95": q(rel_lin, 0.95)},
                             "energy_residual_abs": {"median": q(e.abs().float().cpu(), 0.5),
                                                     "max": round(float(e.abs().max()), 6)},
                             "inputs": "131072 held-out cells of the training distributions, tiled x8"},
            "lite_on_cylinder": lite_rep if lite_rep is not None else {"unavailable": "no LITE weight file"},
            "collision_step_cylinder": collision_rep,
            "adjoint_cavity": {"cells": cav.n_cells, "particles": cav.n_particles,
                               "forward_ms": round(t_fwd_c4, 5), "backward_ms": round(t_bwd_c4, 5),
                               "fwd_bwd_cells_per_s": round(cav.n_cells / ((t_fwd_c4 + t_bwd_c4) * 1e-3), 1)},
            "velocity_update": {"ms": round(per_call["velocity_update"], 5),
                                "particles_per_s": round(n_p / (per_call["velocity_update"] * 1e-3), 1)},
            "training_step": {"batch": 8192, "ms": round(t_train, 5),
                              "cells_per_s": round(8192 / (t_train * 1e-3), 1)},
        },
        "e2e": {"value": round(n_cells / (e2e_ms * 1e-3) * ws, 1), "unit": "cells/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 5),
                "api": f"fp_step_host, pinned host buffers, {E2E_CHUNKS} chunks",
                "results_to_host": "M^{n+1} velocities, exact-closure coefficients and flags; the adjoint's "
                                   "gradients and the learned closure's coefficients are computed in the step "
                                   "and stay on the device"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pop, budget_s=args.cpu_seconds, workers=args.cpu_workers)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def _oracle_block(v32, offs, tau):
    """One block of cells through the oracle as it stands: FP64 moments, exact
    closure and velocity update."""
    import oracle as O
    v = np.asarray(v32, dtype=np.float64)
    m = O.moments(v, offs)
    y, fl = O.closure(m, tau)
    O.velocity_update(v, offs, m, y, tau, fl, 0.1, seed=1234, step=0)


def _oracle_blocks(v32, offsets, tau, n_cells, blocks, budget_s, blk=ORACLE_BLOCK):
    """Runs the blocks of cells in `blocks` (indices of `blk`-cell blocks),
    cycling, until `budget_s` seconds have passed -> (cells, particles, s)."""
    t0 = time.perf_counter()
    cells = parts = 0
    i = 0
    while time.perf_counter() - t0 < budget_s:
        start = blocks[i % len(blocks)] * blk
        end = min(start + blk, n_cells)
        a, b = int(offsets[start]), int(offsets[end])
        _oracle_block(v32[:, a:b], np.asarray(offsets[start:end + 1]) - a, np.asarray(tau[start:end]))
        cells += end - start
        parts += b - a
        i += 1
    return cells, parts, time.perf_counter() - t0


_ORACLE_WORKER = {}


def _oracle_worker_init(folder):
    import oracle as O
    O.lib()
    for k in ("v", "off", "tau"):
        _ORACLE_WORKER[k] = np.load(os.path.join(folder, k + ".npy"), mmap_mode="r")


def _oracle_worker_ping(_):
    time.sleep(0.2)
    return os.getpid()


def oracle_share(w, n_workers, n_blocks):
    """The blocks process w of n_workers times: w, w + n_workers, ... (one
    block, w mod n_blocks, when there are more processes than blocks)."""
    return list(range(w % n_blocks, n_blocks, n_workers)) or [w % n_blocks]


def _oracle_worker_share(w, n_workers, t_start, budget_s):
    """Worker w's share of the blocks, from wall time t_start."""
    v, off, tau = _ORACLE_WORKER["v"], _ORACLE_WORKER["off"], _ORACLE_WORKER["tau"]
    n_cells = tau.shape[0]
    mine = oracle_share(w, n_workers, (n_cells + ORACLE_BLOCK - 1) // ORACLE_BLOCK)
    while time.time() < t_start:
        time.sleep(0.002)
    return _oracle_blocks(v, off, tau, n_cells, mine, budget_s)


class OracleCores:
    """The oracle as it stands on `workers` host processes at once, each over
    its own share of the population's cells.  The processes are started with
    the spawn method (nothing of the parent's CUDA state is inherited) and
    read the population from memory-mapped files."""

    def __init__(self, pop, workers):
        import multiprocessing as mp
        import tempfile
        self.workers = int(workers)
        self.folder = tempfile.mkdtemp(prefix="fp_oracle_")
        np.save(os.path.join(self.folder, "v.npy"), pop.v32)
        np.save(os.path.join(self.folder, "off.npy"), np.asarray(pop.offsets, dtype=np.int64))
        np.save(os.path.join(self.folder, "tau.npy"), np.asarray(pop.tau, dtype=np.float64))
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init,
                                                 initargs=(self.folder,))
        seen = set()
        for _ in range(20):  # until every process has started and loaded the oracle
            seen.update(self.pool.map(_oracle_worker_ping, range(self.workers), chunksize=1))
            if len(seen) >= self.workers:
                break

    def run(self, budget_s):
        """All processes at once for `budget_s` -> (cells/s, particles/s, cells, particles)
        summed over the processes."""
        t_start = time.time() + 0.2
        res = self.pool.starmap(_oracle_worker_share,
                                [(w, self.workers, t_start, budget_s) for w in range(self.workers)], chunksize=1)
        return (sum(c / t for c, _, t in res), sum(p / t for _, p, t in res), sum(c for c, _, _ in res),
                sum(p for _, p, _ in res))

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.folder, ignore_errors=True)


def host_cpu():
    """The host's CPU model (lscpu's model name, else /proc/cpuinfo's, else
    the machine type) and its online CPUs, for the CPU baseline's record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def step_stats(times_ms):
    """Median and best of the timed steps (ms), beside the mean the bench line
    reports as ms_per_step."""
    t = np.asarray(times_ms, dtype=np.float64)
    return {"median": round(float(np.median(t)), 5), "best": round(float(np.min(t)), 5)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(pop, budget_s=15.0, workers=None):
    """The oracle as it stands on this host: moments, exact closure and velocity
    update over blocks of cells for `budget_s` seconds, first on one thread
    (consecutive blocks), then on every host core at once (one process a core,
    each over its share of the blocks); `value` is the all-cores figure.  The
    learned closure and the adjoint have no CPU counterpart at this scale."""
    import oracle as O
    O.build()
    n_blocks = (pop.n_cells + ORACLE_BLOCK - 1) // ORACLE_BLOCK
    c1, p1, el = _oracle_blocks(pop.v32, pop.offsets, pop.tau, pop.n_cells, list(range(n_blocks)), budget_s)
    single = {"value": round(c1 / el, 1), "unit": "cells/s", "cores": 1, "particles_per_s": round(p1 / el, 1),
              "sample": f"{c1} cells ({p1} particles) of {pop.name} in {el:.1f} s"}
    workers = host_cores() if workers is None else workers
    if workers <= 1:
        return dict(single, kind="oracle", host=host_cpu(),
                    sample=single["sample"] + ": FP64 moments, exact closure and velocity update, 1 thread")
    cores = OracleCores(pop, workers)
    try:
        rate, prate, cn, pn = cores.run(budget_s)
    finally:
        cores.close()
    return {"value": round(rate, 1), "unit": "cells/s", "cores": workers, "kind": "oracle",
            "particles_per_s": round(prate, 1), "host": host_cpu(),
            "sample": f"{cn} cells ({pn} particles) of {pop.name} in {budget_s:.0f} s on {workers} processes, one a "
                      f"core, each over its share of {ORACLE_BLOCK}-cell blocks: FP64 moments, exact closure and "
                      "velocity update",
            "single_thread": single}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    pop = _population(args.config, seed=3)
    import oracle as O
    O.build()
    workers = host_cores() if args.cpu_workers is None else args.cpu_workers
    budget = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    cores = OracleCores(pop, workers)
    try:
        for _ in range(args.warmup):
            cores.run(budget / 4)
        per = [cores.run(budget) for _ in range(args.steps)]
    finally:
        cores.close()
    value = float(np.median([r[0] for r in per]))
    ms_per_step = pop.n_cells / value * 1e3
    sample = (f"{per[0][2]} cells ({per[0][3]} particles) of {pop.name} in {budget:.1f} s per step on {workers} "
              f"processes, one a core: FP64 moments, exact closure and velocity update")
    out = {
        "metric": METRIC, "impl": "reference", "value": round(value, 1), "unit": "cells/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": f"synthetic (seeded population {pop.name}; no paper data)",
        "config": {"workload": f"{pop.name}: {pop.n_cells} cells, {pop.n_particles} particles "
                               "(bounded sample per step)", "cells": pop.n_cells, "particles": pop.n_particles},
        "cpu_baseline": {"value": round(value, 1), "unit": "cells/s", "cores": workers, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
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
    ap.add_argument("--cpu-workers", type=int, default=None,
                    help="host processes for the oracle's all-cores timing (default: every core)")
    ap.add_argument("--only", default=None,
                    choices=["gather", "gather64", "solve", "exact_closure", "surrogate_closure", "adjoint",
                             "velocity_update", "step", "mlp", "gather_lite", "lite", "sort", "collision", "train"],
                    help="profiling mode: launch one call --steps times, print no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

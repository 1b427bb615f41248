#!/usr/bin/env python
"""Throughput of the composite spectral direct solver on GB300.

One step = the whole hot path on one problem: hps_build (leaf DtN maps and all
merges, Algorithm 1) followed by hps_solve of 16 right-hand sides (Algorithm 2
and the leaf post-process; in mixed precision also the iterative refinement
against the FP64 residual), on the convection-diffusion workload of 64 x 64
leaves, p = 16, q = 14 (1 048 576 collocation nodes).  Both precisions are
timed; the mixed one is the headline and the FP64 one is reported beside it.  Inputs (coefficients
and boundary data) are resident in HBM when the timed region starts; L2 is
flushed (a 512 MiB write) before every timed step.  Timing uses CUDA events on
the library's stream, max over ranks.  With --gpus N (torchrun), every rank
solves its own independent problem (replicas; weak scaling): there is no data
exchange between problems.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the only reference implementation of this method), on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build DOF/s and solves/s at rel err ≤1e-10: mixed+refine vs plain FP64, same GB300"
DOMAIN = (0.0, 1.0, 0.0, 1.0)
NX = NY = 64
P, Q, NRHS = 16, 14, 16
DOF = NX * NY * P * P
FP64_DFMA_PER_SM_CLK = 2
N_SM = 152


def workload_config(precision="fp64"):
    return {"workload": f"convection-diffusion c1=-100cos(4pi y), c2=100sin(4pi x) on [0,1]^2, "
                        f"{NX}x{NY} leaves, p={P}, q={Q}, {NRHS} RHS (20-mode Fourier data), "
                        f"build+solve, {precision}",
            "leaves": f"{NX}x{NY}", "p": P, "q": Q, "nrhs": NRHS, "dof": DOF,
            "precision": precision, "l2": "flushed before every timed step (512 MiB write)"}


def make_inputs(nx=NX, ny=NY, p=P, q=Q, nrhs=NRHS, seed0=0, xy=None, bxy=None):
    from paper_1307_2665_gb300 import inputs as I
    co = I.convection_diffusion(xy[..., 0], xy[..., 1])
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64)) for k, v in co.items()}
    f = np.ascontiguousarray(np.stack([I.fourier_boundary(seed0 + s, bxy[:, 0], bxy[:, 1], DOMAIN)
                                       for s in range(nrhs)]))
    return co, f


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def oracle_step(n, nrhs=NRHS):
    """One oracle solve (static condensation + sparse LU, FP64) of the same
    workload restricted to n x n leaves; returns seconds and DOF."""
    from oracle import hps_oracle as O
    from paper_1307_2665_gb300 import inputs as I
    prob = O.make_problem(DOMAIN, n, n, P, Q, I.convection_diffusion)
    bxy = O.boundary_points(prob)
    f = np.stack([I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], DOMAIN) for s in range(nrhs)], axis=1)
    t0 = time.perf_counter()
    O.solve_condensed(prob, f)
    return time.perf_counter() - t0, n * n * P * P


def cpu_baseline(n=32, reps=1):
    ts = []
    dof = 0
    for _ in range(reps):
        t, dof = oracle_step(n)
        ts.append(t)
    t = min(ts)
    return {"value": dof / t, "unit": "DOF/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n}x{n} leaves of the same field, p={P}, q={Q}, {NRHS} RHS: FP64 static "
                      f"condensation (per-leaf dense solves, BLAS on all cores) + SuperLU of the "
                      f"edge system (single-threaded); {t:.2f} s per solve"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.ref_leaves
    for _ in range(args.warmup):
        oracle_step(n)
    ts = []
    dof = 0
    for _ in range(args.steps):
        t, dof = oracle_step(n)
        ts.append(t)
    tot = sum(ts)
    value = dof * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(), sample_leaves=f"{n}x{n}"),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{n}x{n} leaves of the workload's field per step"},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- native
# ALU peaks of a GB300 at a given SM clock: FP64 is 2 DFMA per SM per clock
# (measured 1.198 TFLOP/s with 152 SMs at 1987 MHz), FP32 128 FFMA per SM per
# clock (measured 74.8 TFLOP/s at the same clock).
FP32_FFMA_PER_SM_CLK = 128


def alu_peak_tflops(name, sm_mhz):
    per = FP64_DFMA_PER_SM_CLK if "f64" in name else FP32_FFMA_PER_SM_CLK
    return N_SM * per * 2 * sm_mhz * 1e6 / 1e12, per


def roofline_of(stats, t_total_ms, sm_mhz):
    name, st = max(stats.items(), key=lambda kv: kv[1]["ms"])
    peak, per = alu_peak_tflops(name, sm_mhz)
    per_launch_flops = st["flops"] / max(st["launches"], 1)
    per_launch_s = st["ms"] / 1e3 / max(st["launches"], 1)
    achieved = per_launch_flops / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": f"{'FP64 DFMA' if per == FP64_DFMA_PER_SM_CLK else 'FP32 FFMA'}: "
                           f"{N_SM} SMs x {per}/clk x 2 flop x {sm_mhz:.0f} MHz (max SM clock; "
                           f"per-clock rate measured by an FMA probe on this pool)",
            "flops_per_launch": per_launch_flops, "launches": st["launches"],
            "ms_per_launch": per_launch_s * 1e3, "share_of_step": st["ms"] / max(t_total_ms, 1e-9)}


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_1307_2665_gb300 import hps
    from paper_1307_2665_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    build()  # no-op when up to date

    xy = hps.hps_cheb_nodes(DOMAIN, NX, NY, P)
    bxy = hps.hps_boundary_nodes_grid(DOMAIN, NX, NY, Q)
    co_h, f_h = make_inputs(xy=xy, bxy=bxy, seed0=NRHS * rank)
    co_d = {k: (None if v is None else torch.from_numpy(v).to(dev)) for k, v in co_h.items()}
    f_d = torch.from_numpy(f_h).to(dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    modes = {"fp64": hps.HPS_FP64, "mixed": hps.HPS_MIXED}
    if args.precision != "both":
        modes = {args.precision: modes[args.precision]}

    def step(prec, u_d, events=None, info=None):
        if events:
            events[0].record(stream)
        h = hps.hps_build(DOMAIN, NX, NY, P, Q, co_d, precision=prec, device_ptrs=True, stream=sp)
        if events:
            events[1].record(stream)
        hps.hps_solve(h, f_d, u_d, info=info, check=False)
        if events:
            events[2].record(stream)
        return h

    results = {}
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    for mname, prec in modes.items():
        u_d = torch.empty((NRHS, NX * NY, P, P), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            step(prec, u_d).close()
        torch.cuda.synchronize()
        hps.hps_profile_reset()
        hps.hps_profile_enable(True)
        launches0 = hps.hps_kernel_launches()
        t_build = t_solve = 0.0
        iters = []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            info = hps.SolveInfo()
            h = step(prec, u_d, ev, info)
            stream.synchronize()
            if info.status not in (hps.HPS_OK,):
                raise RuntimeError(f"{mname} solve status {info.status} (last update {info.last_update})")
            iters.append(info.iterations)
            t_build += ev[0].elapsed_time(ev[1])
            t_solve += ev[1].elapsed_time(ev[2])
            h.close()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches = hps.hps_kernel_launches() - launches0
        stats = hps.hps_profile_read()
        hps.hps_profile_enable(False)
        if world > 1:
            t = torch.tensor([t_build, t_solve], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_build, t_solve = t.tolist()
        results[mname] = {"t_build": t_build, "t_solve": t_solve, "iters": iters, "stats": stats,
                          "launches": launches, "u": u_d}
    clocks = sampler.stop() if rank == 0 else None
    head = "mixed" if "mixed" in results else "fp64"
    R = results[head]

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_steps = max(1, min(args.steps, 3))
    t_e2e = 0.0
    h2d = sum(v.nbytes for v in co_h.values() if v is not None) + f_h.nbytes
    d2h = NRHS * NX * NY * P * P * 8
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = hps.hps_build(DOMAIN, NX, NY, P, Q, co_h, precision=modes[head], device_ptrs=False,
                          stream=sp)
        u_h = hps.hps_solve(h, f_h, device_ptrs=False)
        e1.record(stream)
        stream.synchronize()
        t_e2e += e0.elapsed_time(e1)
        h.close()
    if world > 1:
        t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = t.item()
    assert np.isfinite(u_h).all()
    rel_diff = None
    if "mixed" in results and "fp64" in results:
        a, b = results["mixed"]["u"], results["fp64"]["u"]
        rel_diff = float((a - b).abs().max() / b.abs().max())

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0

    def summary(r):
        tt = r["t_build"] + r["t_solve"]
        return {"dof_per_s": world * DOF * args.steps / (tt / 1e3),
                "build_dof_per_s": world * DOF * args.steps / (r["t_build"] / 1e3),
                "solves_per_s": world * NRHS * args.steps / (r["t_solve"] / 1e3),
                "build_ms": r["t_build"] / args.steps, "solve_ms": r["t_solve"] / args.steps,
                "refine_iterations": r["iters"],
                "gpu_launches": int(r["launches"] // args.steps),
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] > 0 else 0.0}
                            for k, v in sorted(r["stats"].items(), key=lambda kv: -kv[1]["ms"])},
                "roofline": roofline_of(r["stats"], tt, sm_max)}

    summ = {k: summary(v) for k, v in results.items()}
    H = summ[head]
    t_total = R["t_build"] + R["t_solve"]
    line = {"metric": METRIC, "value": H["dof_per_s"], "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (FP32 leaves/lower merges, FP64 top merges and residual)"
            if head == "mixed" else "f64",
            "data": "synthetic", "config": workload_config(head),
            "build_dof_per_s": H["build_dof_per_s"], "solves_per_s": H["solves_per_s"],
            "build_ms": H["build_ms"], "solve_ms": H["solve_ms"],
            "clocks": clocks, "gpu_launches": H["gpu_launches"],
            "e2e": {"value": world * DOF * e2e_steps / (t_e2e / 1e3), "unit": "DOF/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": H["roofline"]}
    if "fp64" in summ and head != "fp64":
        F = summ["fp64"]
        line["fp64"] = {k: F[k] for k in ("dof_per_s", "build_dof_per_s", "solves_per_s",
                                          "build_ms", "solve_ms", "gpu_launches", "roofline")}
        line["speedup_mixed_over_fp64"] = {"step": H["dof_per_s"] / F["dof_per_s"],
                                           "build": H["build_dof_per_s"] / F["build_dof_per_s"],
                                           "solve": H["solves_per_s"] / F["solves_per_s"]}
        line["fp64"]["kernels"] = F["kernels"]
    line["rel_diff_mixed_vs_fp64"] = rel_diff
    line["refine_iterations"] = H["refine_iterations"]
    line["kernels"] = H["kernels"]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.ref_leaves)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-leaves", type=int, default=32,
                    help="leaves per side of the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: time FP64 and mixed, report mixed as the headline")
    ap.add_argument("--leaves", type=int, default=64,
                    help="leaves per side (64 is the benchmarked workload; smaller values are "
                         "for profiling captures)")
    args = ap.parse_args()
    global NX, NY, DOF
    NX = NY = args.leaves
    DOF = NX * NY * P * P
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())

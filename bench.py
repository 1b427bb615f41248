#!/usr/bin/env python
"""Throughput of the composite spectral direct solver on GB300.

One step = the whole hot path on one batch of input: hps_build (leaf DtN maps
and all merges, Algorithm 1) followed by the solve of every right-hand side
(Algorithm 2 and the leaf post-process; in mixed precision also the iterative
refinement against the FP64 residual).  Workloads (--workload):

  helmholtz256  (default) variable-speed Helmholtz, kappa = 80, 256 x 256
                leaves, p = 16, q = 14 (16.8 M nodes), 64 right-hand sides: the
                largest single-GPU configuration and the one specified in mixed
                precision
  convdiff64    convection-diffusion on [0,1]^2, 64 x 64 leaves, p = 16,
                q = 14 (1 048 576 collocation nodes), 16 right-hand sides
  batch64       64 independent problems of uneven size (n log-uniform in
                [8, 128]) and order (p in {12, 16, 20}, q = p - 2) with random
                smooth coefficient fields, 16 right-hand sides each, one batched
                build and solve
  post          post-processing on the helmholtz256 problem built in FP64 with
                its root DtN map T^1 (nbnd = 14336): T^1 applied to 1, 8 and 64
                data sets (Section 9.1's T_apply) and the solution evaluated at
                4 M random points (Section 5.3); one step = one T^1 apply to one
                data set
  serve         the request loop (include/hps_serve.h) on a Poisson stream

Both precisions are timed; the mixed one is the headline and the FP64 one is
reported beside it.  Inputs (coefficients and boundary data) are resident in
HBM when the timed region starts; L2 is flushed (a 512 MiB write) before every
timed step.  Timing uses CUDA events on the library's stream, max over ranks.
With --gpus N (torchrun), every rank solves its own independent input
(replicas; weak scaling): there is no data exchange between problems.

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
UNIT_SQ = (0.0, 1.0, 0.0, 1.0)
FP64_DFMA_PER_SM_CLK = 2
FP32_FFMA_PER_SM_CLK = 128
N_SM = 152
MAX_REFINE = 30  # refinement cap (tolerance 1e-11, plain refinement, leaf correction on: library defaults)


# ------------------------------------------------------------- workloads
class Workload:
    """A list of problems (domain, nx, ny, p, q, host coefficients, host f)
    plus a description.  One problem goes through hps_build / hps_solve, more
    through hps_build_batch / hps_solve_batch."""

    def __init__(self, name, desc, probs, nrhs, oracle_fn):
        self.name, self.desc, self.probs, self.nrhs = name, desc, probs, nrhs
        self.oracle_fn = oracle_fn  # coefficient function of the oracle sample
        self.dof = sum(pr["nx"] * pr["ny"] * pr["p"] ** 2 for pr in probs)
        self.leaves = sum(pr["nx"] * pr["ny"] for pr in probs)

    def config(self, precision):
        return dict(self.desc, precision=precision, dof=self.dof, nrhs=self.nrhs,
                    problems=len(self.probs), leaves_total=self.leaves,
                    l2="flushed before every timed step (512 MiB write)",
                    refinement="tol 1e-11 per RHS (or the next correction predicted below it), "
                               "plain refinement, cap 30; leaf operators corrected once in FP64")


def _problem(hps, I, dom, nx, ny, p, q, fn, nrhs, seed0):
    xy = hps.hps_cheb_nodes(dom, nx, ny, p)
    xs = xy[:nx, 0, :, 0].reshape(-1)
    ys = xy[::nx, :, 0, 1].reshape(-1)
    co = I.sample_on_leaf_grid(fn, xs, ys, nx, ny, p)
    del xy
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    f = np.ascontiguousarray(np.stack([I.fourier_boundary(seed0 + s, bxy[:, 0], bxy[:, 1], dom)
                                       for s in range(nrhs)]))
    return dict(domain=dom, nx=nx, ny=ny, p=p, q=q, coeffs=co, f=f)


def describe_workload(name, leaves, rank=0):
    """The workload's description (the JSON line's `config` core), its
    right-hand sides per problem and, for batch64, each problem's (n, p); no
    arrays are sampled, so both arms can name the same workload."""
    if name == "convdiff64":
        n = leaves or 64
        nrhs = 16
        desc = {"workload": f"convection-diffusion c1=-100cos(4pi y), c2=100sin(4pi x) on [0,1]^2, "
                            f"{n}x{n} leaves, p=16, q=14, {nrhs} RHS (20-mode Fourier data), "
                            f"build+solve", "leaves": f"{n}x{n}", "p": 16, "q": 14}
        return desc, nrhs, [(n, 16)]
    if name == "helmholtz256":
        n = leaves or 256
        nrhs = 64
        desc = {"workload": f"variable-speed Helmholtz -Lap u - 80^2 (1 - 0.5 exp(-|x-c|^2/0.02)) u = 0 "
                            f"on [0,1]^2, {n}x{n} leaves, p=16, q=14, {nrhs} RHS (20-mode Fourier "
                            f"data), build+solve", "leaves": f"{n}x{n}", "p": 16, "q": 14}
        return desc, nrhs, [(n, 16)]
    if name == "batch64":
        nprob = 64
        nmax = leaves or 128
        nrhs = 16
        rng = np.random.Generator(np.random.PCG64(20240 + rank))
        shapes = []
        for _ in range(nprob):
            n = int(round(np.exp(rng.uniform(np.log(8), np.log(nmax)))))
            shapes.append((n, int(rng.choice([12, 16, 20]))))
        desc = {"workload": f"{nprob} independent problems, n x n leaves with n log-uniform in "
                            f"[8, {nmax}], p in {{12, 16, 20}}, q = p - 2, random smooth c11, c22, "
                            f"c12, c1, c2 (c = 0), {nrhs} RHS each, one batched build+solve",
                "sizes": [n for n, _ in shapes], "orders": [p for _, p in shapes]}
        return desc, nrhs, shapes
    raise ValueError(name)


def make_workload(name, leaves, rank):
    from paper_1307_2665_gb300 import hps
    from paper_1307_2665_gb300 import inputs as I
    desc, nrhs, shapes = describe_workload(name, leaves, rank)
    if name == "convdiff64":
        (n, _), = shapes
        pr = _problem(hps, I, UNIT_SQ, n, n, 16, 14, I.convection_diffusion, nrhs, nrhs * rank)
        return Workload(name, desc, [pr], nrhs, I.convection_diffusion)
    if name == "helmholtz256":
        (n, _), = shapes
        pr = _problem(hps, I, UNIT_SQ, n, n, 16, 14, I.gaussian_bump_helmholtz, nrhs, nrhs * rank)
        return Workload(name, desc, [pr], nrhs, I.gaussian_bump_helmholtz)
    # batch64
    probs = []
    for k, (n, p) in enumerate(shapes):
        seed = 1000 * rank + k
        fn = (lambda s: (lambda x, y: I.random_smooth_operator(s, x, y)))(seed)
        probs.append(_problem(hps, I, UNIT_SQ, n, n, p, p - 2, fn, nrhs, 100 * seed))
    return Workload(name, desc, probs, nrhs, lambda x, y: I.random_smooth_operator(0, x, y))


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
def oracle_step(n, fn, nrhs=16):
    """One oracle solve (static condensation + sparse LU, FP64) of the
    workload's coefficient field on n x n leaves, p = 16, q = 14; returns
    seconds, DOF, the data f (nrhs, nbnd) and the oracle's solution
    (nrhs, n*n, p, p)."""
    from oracle import hps_oracle as O
    from paper_1307_2665_gb300 import inputs as I
    prob = O.make_problem(UNIT_SQ, n, n, 16, 14, fn)
    bxy = O.boundary_points(prob)
    f = np.stack([I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], UNIT_SQ) for s in range(nrhs)],
                 axis=1)
    t0 = time.perf_counter()
    sol = O.solve_condensed(prob, f)
    return time.perf_counter() - t0, n * n * 16 * 16, np.ascontiguousarray(f.T), sol.w


def cpu_baseline(fn, n=32, nrhs=16):
    """The oracle timed on a bounded sample of the workload; also returns the
    sample's data and oracle solution for the accuracy check."""
    t, dof, f, w = oracle_step(n, fn, nrhs)
    return ({"value": dof / t, "unit": "DOF/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{n}x{n} leaves of the workload's coefficient field, p=16, q=14, {nrhs} "
                       f"RHS: FP64 static condensation (per-leaf dense solves, BLAS on all "
                       f"cores) + SuperLU of the edge system (single-threaded); {t:.2f} s per "
                       f"solve"}, f, w)


def sample_vs_oracle(hps, fn, n, f, w_oracle):
    """The library on the oracle's sample (same field, data and leaf grid), in
    both precisions, against the oracle's solution element by element: max
    |u - u_oracle| / max |u_oracle| over every node of every right-hand side."""
    from paper_1307_2665_gb300 import inputs as I
    xy = hps.hps_cheb_nodes(UNIT_SQ, n, n, 16)
    co = I.sample_on_leaf_grid(fn, xy[:n, 0, :, 0].reshape(-1), xy[::n, :, 0, 1].reshape(-1),
                               n, n, 16)
    out = {"leaves": f"{n}x{n}", "nrhs": int(f.shape[0])}
    scale = float(np.max(np.abs(w_oracle)))
    for name, prec in (("fp64", hps.HPS_FP64), ("mixed", hps.HPS_MIXED)):
        h = hps.hps_build(UNIT_SQ, n, n, 16, 14, co, precision=prec, max_refine=MAX_REFINE)
        info = hps.SolveInfo()
        u = hps.hps_solve(h, f, info=info, check=False)
        h.close()
        out[f"max_rel_err_{name}"] = float(np.max(np.abs(u - w_oracle)) / scale)
        if prec == hps.HPS_MIXED:
            out["mixed_corrections"] = int(info.iterations)
    return out


def full_size_residual(W, u_by_mode, nrhs=2, seed=11, count=40):
    """The oracle's leaf-local FP64 check (E1, E2, shared-side continuity,
    Dirichlet data) of the benchmarked solutions at full size, on a fixed set
    of leaves (seeded sample plus the corners and the centre) and the first
    nrhs right-hand sides; only those leaves and their east and north
    neighbours are copied to the host."""
    from oracle import hps_oracle as O
    pr = W.probs[0]
    nx, ny, p = pr["nx"], pr["ny"], pr["p"]
    nl = nx * ny
    rng = np.random.default_rng(seed)
    leaves = sorted(set(rng.choice(nl, min(count, nl), replace=False).tolist()) |
                    {0, nx - 1, nx * (ny - 1), nl - 1, nx * (ny // 2) + nx // 2 - 1})
    need = sorted({m for l in leaves for m in (l, l + 1, l + nx) if m < nl})
    co = {k: (None if v is None else v.reshape(nl, p, p)) for k, v in pr["coeffs"].items()}
    prob = O.Problem(pr["domain"], nx, ny, p, pr["q"], co)
    k = min(nrhs, W.nrhs)
    out = {"leaves": len(leaves), "nrhs": k}
    for name, us in u_by_mode.items():
        w = np.zeros((k, nl, p, p))
        w[:, need] = us[0][:k, need].cpu().numpy()
        out[name] = {key: float(v) for key, v in O.sampled_residual(prob, w, pr["f"][:k],
                                                                    leaves).items()}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1307_2665_gb300 import inputs as I
    fn = {"convdiff64": I.convection_diffusion, "helmholtz256": I.gaussian_bump_helmholtz,
          "batch64": lambda x, y: I.random_smooth_operator(0, x, y)}[args.workload]
    n = args.ref_leaves
    for _ in range(args.warmup):
        oracle_step(n, fn)
    ts = []
    dof = 0
    for _ in range(args.steps):
        t, dof, _, _ = oracle_step(n, fn)
        ts.append(t)
    tot = sum(ts)
    value = dof * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(describe_workload(args.workload, args.leaves)[0],
                           sample=f"oracle on {n}x{n} leaves of the workload's coefficient "
                                  f"field, p=16, q=14, 16 RHS per step"),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{n}x{n} leaves of the workload's field per step"},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ ranks
def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time); the identity on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, units_per_rank, steps, t_ms):
    """Whole-job throughput: the units all ranks processed (each rank the same
    count, its own independent input) over the slowest rank's time."""
    return world * units_per_rank * steps / (t_ms / 1e3)


# ---------------------------------------------------------------- native
# ALU peaks of a GB300 at a given SM clock: FP64 is 2 DFMA per SM per clock
# (measured 1.198 TFLOP/s with 152 SMs at 1987 MHz), FP32 128 FFMA per SM per
# clock (measured 74.8 TFLOP/s at the same clock).
def alu_peak_tflops(name, sm_mhz):
    per = FP64_DFMA_PER_SM_CLK if "f64" in name else FP32_FFMA_PER_SM_CLK
    return N_SM * per * 2 * sm_mhz * 1e6 / 1e12, per


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an
# ncu capture of the same kernel's launch in the same workload step; a kernel
# changed since its capture has no entry.  leaf_resflux_tc<f64>: captured on
# 64 x 64 leaves with 64 right-hand sides (850.7 MB per launch, 3245 bytes per
# leaf and right-hand side) and scaled by the 16 times as many units of a
# 256 x 256 launch.  leaf_gj_inverse<f32>: captured on 64 x 64 leaves (4096
# matrices, 810.5 + 758.4 MB, 383 KB per leaf), scaled the same way.
TRAFFIC_PER_LAUNCH = {("helmholtz256", "leaf_resflux_tc<f64>"): 850.7e6 * 16,
                      ("helmholtz256", "leaf_gj_inverse<f32>"): (810.5e6 + 758.4e6) * 16}


def roofline_of(stats, t_total_ms, sm_mhz, workload=None):
    name, st = max(stats.items(), key=lambda kv: kv[1]["ms"])
    peak, per = alu_peak_tflops(name, sm_mhz)
    per_launch_flops = st["flops"] / max(st["launches"], 1)
    per_launch_s = st["ms"] / 1e3 / max(st["launches"], 1)
    achieved = per_launch_flops / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TRAFFIC_PER_LAUNCH.get((workload, name)),
            "peak_source": f"{'FP64 DFMA' if per == FP64_DFMA_PER_SM_CLK else 'FP32 FFMA'}: "
                           f"{N_SM} SMs x {per}/clk x 2 flop x {sm_mhz:.0f} MHz (max SM clock; "
                           f"per-clock rate measured on a GB300 by an FMA throughput probe)"
                           + ("; achieved counts the operation's FP64 flops, whose products "
                              "run as exact BF16 digit products on the tensor cores, so it "
                              "can exceed the FP64 pipe's peak" if "_tc<f64>" in name else ""),
            "flops_per_launch": per_launch_flops, "launches": st["launches"],
            "ms_per_launch": per_launch_s * 1e3, "share_of_step": st["ms"] / max(t_total_ms, 1e-9)}


class Runner:
    """Build and solve of a workload through the public binding."""

    def __init__(self, hps, W, dev):
        import torch
        self.hps, self.W = hps, W
        self.single = len(W.probs) == 1
        self.co_d = [{k: (None if v is None else torch.from_numpy(v).to(dev))
                      for k, v in pr["coeffs"].items()} for pr in W.probs]
        self.f_d = [torch.from_numpy(pr["f"]).to(dev) for pr in W.probs]
        self.u_d = [torch.empty((W.nrhs, pr["nx"] * pr["ny"], pr["p"], pr["p"]),
                                dtype=torch.float64, device=dev) for pr in W.probs]

    def build(self, prec, sp, host=False):
        hps, W = self.hps, self.W
        cos = [pr["coeffs"] for pr in W.probs] if host else self.co_d
        if self.single:
            pr = W.probs[0]
            return hps.hps_build(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"], cos[0],
                                 precision=prec, device_ptrs=not host, stream=sp,
                                 max_refine=MAX_REFINE)
        plist = [dict(pr, coeffs=c) for pr, c in zip(W.probs, cos)]
        return hps.hps_build_batch(plist, precision=prec, device_ptrs=not host, stream=sp,
                                   max_refine=MAX_REFINE)

    def solve(self, h, info, host=False):
        hps, W = self.hps, self.W
        if host:
            us = [np.empty((W.nrhs, pr["nx"] * pr["ny"], pr["p"], pr["p"])) for pr in W.probs]
            fs = [pr["f"] for pr in W.probs]
        else:
            us, fs = self.u_d, self.f_d
        if self.single:
            hps.hps_solve(h, fs[0], us[0], info=info, check=False)
        else:
            hps.hps_solve_batch(h, fs, us, info=info, check=False)
        return us


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

    W = make_workload(args.workload, args.leaves, rank)
    run = Runner(hps, W, dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    modes = {"fp64": hps.HPS_FP64, "mixed": hps.HPS_MIXED}
    if args.precision != "both":
        modes = {args.precision: modes[args.precision]}

    def step(prec, events=None, info=None):
        if events:
            events[0].record(stream)
        h = run.build(prec, sp)
        if events:
            events[1].record(stream)
        run.solve(h, info)
        if events:
            events[2].record(stream)
        return h

    results = {}
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    for mname, prec in modes.items():
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            step(prec).close()
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
            h = step(prec, ev, info)
            stream.synchronize()
            if info.status != hps.HPS_OK:
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
        t_build, t_solve = max_over_ranks([t_build, t_solve], dist, dev)
        results[mname] = {"t_build": t_build, "t_solve": t_solve, "iters": iters, "stats": stats,
                          "launches": launches, "u": [u.clone() for u in run.u_d]}
    clocks = sampler.stop() if rank == 0 else None
    head = "mixed" if "mixed" in results else "fp64"
    R = results[head]

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_steps = max(1, min(args.steps, 3))
    t_e2e = 0.0
    h2d = sum(v.nbytes for pr in W.probs for v in pr["coeffs"].values() if v is not None)
    h2d += sum(pr["f"].nbytes for pr in W.probs)
    d2h = W.nrhs * W.dof * 8
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = run.build(modes[head], sp, host=True)
        u_h = run.solve(h, None, host=True)
        e1.record(stream)
        stream.synchronize()
        t_e2e += e0.elapsed_time(e1)
        h.close()
    t_e2e, = max_over_ranks([t_e2e], dist, dev)
    assert all(np.isfinite(u).all() for u in u_h)
    rel_diff = None
    if "mixed" in results and "fp64" in results:
        rel_diff = max(float((a - b).abs().max() / b.abs().max())
                       for a, b in zip(results["mixed"]["u"], results["fp64"]["u"]))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0

    def summary(r):
        tt = r["t_build"] + r["t_solve"]
        return {"dof_per_s": job_rate(world, W.dof, args.steps, tt),
                "build_dof_per_s": job_rate(world, W.dof, args.steps, r["t_build"]),
                "solves_per_s": job_rate(world, W.nrhs * len(W.probs), args.steps, r["t_solve"]),
                "build_ms": r["t_build"] / args.steps, "solve_ms": r["t_solve"] / args.steps,
                "refine_iterations": r["iters"],
                "gpu_launches": int(r["launches"] // args.steps),
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] > 0 else 0.0}
                            for k, v in sorted(r["stats"].items(), key=lambda kv: -kv[1]["ms"])},
                "roofline": roofline_of(r["stats"], tt, sm_max, None if args.leaves else args.workload)}

    summ = {k: summary(v) for k, v in results.items()}
    H = summ[head]
    t_total = R["t_build"] + R["t_solve"]
    line = {"metric": METRIC, "value": H["dof_per_s"], "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (FP32 leaves/lower merges, FP64 top merges and residual)"
            if head == "mixed" else "f64",
            "data": "synthetic", "config": W.config(head),
            "build_dof_per_s": H["build_dof_per_s"], "solves_per_s": H["solves_per_s"],
            "build_ms": H["build_ms"], "solve_ms": H["solve_ms"],
            "clocks": clocks, "gpu_launches": H["gpu_launches"],
            "e2e": {"value": job_rate(world, W.dof, e2e_steps, t_e2e), "unit": "DOF/s",
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
    # accuracy of the benchmarked run: mixed against FP64 at full size, both
    # against the oracle's leaf-local FP64 residual at full size, and both
    # against the oracle's solution on the cpu_baseline sample
    acc = {"rel_diff_mixed_vs_fp64": rel_diff}
    if len(W.probs) == 1:
        acc["full_size_residual"] = full_size_residual(W, {k: v["u"] for k, v in results.items()})
    if world == 1 and not args.no_cpu_baseline:
        cb, fs, ws = cpu_baseline(W.oracle_fn, args.ref_leaves)
        line["cpu_baseline"] = cb
        acc["oracle_sample"] = sample_vs_oracle(hps, W.oracle_fn, args.ref_leaves, fs, ws)
    line["accuracy"] = acc
    line["kernels"] = H["kernels"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------- serving
def run_serve(args):
    """Request stream of the serving loop: Poisson arrivals, builds and solves
    on resident operators; reports latency percentiles and solves/s."""
    import threading

    import torch
    from paper_1307_2665_gb300 import hps
    from paper_1307_2665_gb300 import inputs as I
    from paper_1307_2665_gb300.build import build
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank != 0:  # replicas: each GPU would serve its own stream; one is measured
        return 0
    torch.cuda.set_device(local)
    build()
    nreq, rate = args.requests, args.rate
    rng = np.random.Generator(np.random.PCG64(7))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    kinds = (rng.random(nreq) < 0.1).astype(int)  # 1 = build
    kinds[:4] = 1  # the stream opens with builds
    nmax = args.leaves or 128
    builds, ops_inputs = [], []
    for i in np.nonzero(kinds)[0]:
        n = int(round(np.exp(rng.uniform(np.log(16), np.log(nmax)))))
        helm = len(builds) % 2 == 1
        kappa = float(rng.uniform(10, 60))
        fn = (lambda k: (lambda x, y: I.constant_helmholtz(x, y, k)))(kappa) if helm else I.laplace
        xy = hps.hps_cheb_nodes(UNIT_SQ, n, n, 16)
        co = I.sample_on_leaf_grid(fn, xy[:n, 0, :, 0].reshape(-1), xy[::n, :, 0, 1].reshape(-1),
                                   n, n, 16)
        del xy
        bxy = hps.hps_boundary_nodes_grid(UNIT_SQ, n, n, 14)
        bank = I.fourier_boundary_bank(1000 + len(builds), bxy[:, 0], bxy[:, 1], UNIT_SQ, 256)
        builds.append(int(i))
        ops_inputs.append((dict(domain=UNIT_SQ, nx=n, ny=n, p=16, q=14, coeffs=co), bank,
                           "helmholtz kappa=%.1f" % kappa if helm else "laplace"))
    nrhs_of = np.maximum(1, np.round(np.exp(rng.uniform(0, np.log(256), nreq)))).astype(int)
    pick = rng.random(nreq)
    prec = hps.HPS_MIXED if args.serve_precision == "mixed" else hps.HPS_FP64
    srv = hps.Server(workers=args.workers, max_rhs_per_solve=256)
    ids = [None] * nreq
    op_of_build = {}
    t0 = time.perf_counter()

    def submitter():
        done_builds = []
        bi = 0
        for i in range(nreq):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if kinds[i]:
                pr, bank, _ = ops_inputs[bi]
                ids[i] = srv.submit_build(pr, precision=prec, max_refine=MAX_REFINE)
                op_of_build[bi] = ids[i]
                bi += 1
            else:
                # a uniformly chosen resident operator (built and not evicted);
                # before the first build completes, any submitted one
                done_builds[:] = [b for b in op_of_build
                                  if srv.wait(op_of_build[b], 0.0).status == hps.HPS_OK]
                cand = done_builds or list(op_of_build)
                b = cand[int(pick[i] * len(cand))]
                bank = ops_inputs[b][1]
                k = int(nrhs_of[i])
                s0 = int((pick[i] * 7919) % (257 - k))
                ids[i] = srv.submit_solve(op_of_build[b], bank[s0:s0 + k])

    th = threading.Thread(target=submitter)
    th.start()
    lat_b, lat_s, rhs_done, t_last, failed, batched = [], [], 0, 0.0, 0, 0
    t_first = None
    iters = []
    for i in range(nreq):
        while ids[i] is None:
            time.sleep(0.0005)
        info = srv.wait(ids[i])
        lat = info.t_end - (info.t_submit)
        if info.status not in (hps.HPS_OK,):
            failed += 1
        if kinds[i]:
            lat_b.append(lat)
        else:
            lat_s.append(lat)
            rhs_done += info.nrhs
            batched += info.batch_rhs > info.nrhs
            iters.append(info.iterations)
            srv.release(ids[i])
        t_last = max(t_last, info.t_end)
        t_first = info.t_submit if t_first is None else min(t_first, info.t_submit)
    th.join()
    stats = srv.stats()
    srv.close()
    span = t_last - t_first  # server clock: first submission to last completion
    pct = lambda v, q: float(np.percentile(np.asarray(v) * 1e3, q)) if v else None
    line = {"metric": "serving: solves/s and p50/p99 latency (arrival to result), Poisson stream",
            "value": rhs_done / span, "unit": "RHS/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic",
            "dtype": "f32+f64 (mixed, refined to 1e-11)" if prec == hps.HPS_MIXED else "f64",
            "config": {"workload": f"{nreq} requests at {rate}/s, 10% builds (n log-uniform in "
                                   f"[16, {nmax}], p=16, q=14, Laplace / Helmholtz kappa~U[10,60]), "
                                   f"90% solves with nrhs log-uniform in [1, 256]",
                       "workers": args.workers, "max_rhs_per_solve": 256},
            "latency_ms": {"solve_p50": pct(lat_s, 50), "solve_p99": pct(lat_s, 99),
                           "build_p50": pct(lat_b, 50), "build_p99": pct(lat_b, 99),
                           "all_p50": pct(lat_s + lat_b, 50), "all_p99": pct(lat_s + lat_b, 99)},
            "requests_per_s": nreq / span, "span_s": span, "failed": failed,
            "coalesced_requests": int(batched), "refine_iterations_median": float(np.median(iters)),
            "server": stats}
    print(json.dumps(line), flush=True)
    return 0


def run_post(args):
    """T^1 apply and point evaluation on the 256 x 256 Helmholtz problem."""
    import torch
    from paper_1307_2665_gb300 import hps
    from paper_1307_2665_gb300.build import build
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank != 0:  # replicas: one GPU is measured
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    W = make_workload("helmholtz256", args.leaves, 0)
    pr = W.probs[0]
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    co_d = {k: (None if v is None else torch.from_numpy(v).to(dev)) for k, v in pr["coeffs"].items()}
    h = hps.hps_build(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"], co_d, device_ptrs=True,
                      stream=sp, form_root_dtn=True)
    n = hps.hps_boundary_count(pr["nx"], pr["ny"], pr["q"])
    f_all = torch.from_numpy(np.ascontiguousarray(pr["f"])).to(dev)
    K, Wm = max(args.steps, 1), max(args.warmup, 3)
    clk = ClockSampler(local)

    def timed(fn, reps):
        for _ in range(Wm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    clk.start()
    hps.hps_profile_reset()
    hps.hps_profile_enable(True)
    launches0 = hps.hps_kernel_launches()
    g1 = torch.empty((1, n), dtype=torch.float64, device=dev)
    f1 = f_all[:1].contiguous()
    t1 = timed(lambda: hps.hps_apply_dtn(h, f1, g1, device_ptrs=True), K)
    launches = (hps.hps_kernel_launches() - launches0) // (K + Wm)
    stats = hps.hps_profile_read()
    hps.hps_profile_enable(False)
    for k in (8, 64):
        fk = f_all[:k].contiguous()
        gk = torch.empty((k, n), dtype=torch.float64, device=dev)
        out[k] = timed(lambda: hps.hps_apply_dtn(h, fk, gk, device_ptrs=True), K)
    # point evaluation of one solution at 4 M random points
    u = torch.empty((1, pr["nx"] * pr["ny"], pr["p"], pr["p"]), dtype=torch.float64, device=dev)
    hps.hps_solve(h, f1, u, device_ptrs=True)
    npts = 4 * 1024 * 1024
    rng = np.random.default_rng(3)
    xy = torch.from_numpy(rng.random((npts, 2))).to(dev)
    vals = torch.empty((1, npts), dtype=torch.float64, device=dev)
    t_interp = timed(lambda: hps.hps_interpolate(h, u, xy, vals, device_ptrs=True), K)
    # the same number of points on a regular 2048 x 2048 grid (neighbouring
    # threads share leaves)
    g1d = (np.arange(2048) + 0.5) / 2048
    gx, gy = np.meshgrid(g1d, g1d)
    xyg = torch.from_numpy(np.ascontiguousarray(np.column_stack([gx.ravel(), gy.ravel()]))).to(dev)
    t_interp_grid = timed(lambda: hps.hps_interpolate(h, u, xyg, vals, device_ptrs=True), K)
    clocks = clk.stop()
    # end to end: host arrays, copies inside the call
    f1h = np.ascontiguousarray(pr["f"][:1])
    g1h = np.empty_like(f1h)
    t0 = time.perf_counter()
    for _ in range(K):
        hps.hps_apply_dtn(h, f1h, g1h, device_ptrs=False)
    t_e2e = (time.perf_counter() - t0) / K * 1e3
    h.close()
    mv = stats.get("dtn_matvec", {"ms": 0.0, "bytes": 0.0, "launches": 1})
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    per_launch_bytes = mv["bytes"] / max(mv["launches"], 1)
    per_launch_s = mv["ms"] / 1e3 / max(mv["launches"], 1)
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    line = {"metric": "T_apply: applications of the root DtN map T^1 per second (1 data set)",
            "value": 1e3 / t1, "unit": "applies/s", "n_gpus": 1, "steps": K, "warmup": Wm,
            "ms_per_step": t1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"T^1 of the helmholtz256 problem (nbnd = {n}, "
                                   f"{8.0 * n * n / 1e9:.2f} GB in FP64) applied to 20-mode Fourier "
                                   f"data; point evaluation at {npts} uniform random points "
                                   f"and at a regular 2048x2048 grid",
                       "l2": "inputs larger than L2 (T^1 is read from HBM every apply)"},
            "apply_ms": {"1": t1, "8": out[8], "64": out[64]},
            "interp_points_per_s": npts / (t_interp / 1e3), "interp_ms": t_interp,
            "interp_grid_points_per_s": npts / (t_interp_grid / 1e3),
            "gpu_launches": int(launches),
            "roofline": {"kernel": "dtn_matvec", "bound": "hbm", "achieved": achieved,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "e2e": {"value": 1e3 / t_e2e, "unit": "applies/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "clocks": clocks, "kernels": stats}
    if not args.no_cpu_baseline:  # the oracle's T^1 f: global sparse solve + boundary fluxes
        from oracle import hps_oracle as O
        from paper_1307_2665_gb300 import inputs as I
        ns = 16
        prob = O.make_problem(UNIT_SQ, ns, ns, 16, 14, I.gaussian_bump_helmholtz)
        xyb = O.boundary_points(prob)
        fs = I.fourier_boundary(0, xyb[:, 0], xyb[:, 1], UNIT_SQ)[None, :]
        t0 = time.perf_counter()
        O.dtn_apply(prob, fs)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "applies/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"one T^1 f by the FP64 oracle (sparse LU of the global "
                                          f"system + boundary fluxes) on {ns}x{ns} leaves, p=16, "
                                          f"q=14, not the full 256x256 problem"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="helmholtz256",
                    choices=["convdiff64", "helmholtz256", "batch64", "serve", "post"])
    ap.add_argument("--requests", type=int, default=2000, help="serve: stream length")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: arrivals per second")
    ap.add_argument("--workers", type=int, default=4, help="serve: concurrent device jobs")
    ap.add_argument("--serve-precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--ref-leaves", type=int, default=32,
                    help="leaves per side of the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: time FP64 and mixed, report mixed as the headline")
    ap.add_argument("--leaves", type=int, default=0,
                    help="leaves per side (batch64: largest side); 0 = the workload's own size. "
                         "Smaller values are for profiling captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "post":
        return run_post(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())

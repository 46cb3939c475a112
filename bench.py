"""Benchmark: Parareal for monolithic ALE-FSI on the 128 x 32 Q2 channel-with-bar
workload (83,525 dofs per state, T = 2, 64 slices x 32 fine shifted
Crank-Nicolson steps, FP64 throughout).

The line follows a continuing Parareal run (Sec. 3). The predictor sweep
(64 implicit-Euler steps) comes first, untimed; then one step = one Parareal
iteration (parareal_continue): the fine propagator of every slice not yet exact,
batched (32 steps of all those slices at once: residual, Jacobian,
multigrid-FGMRES Newton), then the corrected coarse sweep with the correction.
The first --warmup iterations are untimed, the next --steps are timed.
value = fine time-steps advanced per second over the timed steps. Each timed
step also copies the iterate in from pinned host memory and back out, and the
same loop gives the end-to-end figure. On this workload the iterates beyond the
exact front grow from iteration to iteration until a propagator's solve fails
(about iteration 23); that step ends the run, a new run starts from the
predictor, and the failed step stays in the timed total without advancing any
fine step.

Against the metric's accuracy: the serial fine solution of the whole interval
is computed first on the same GPU (timed: the serial single-slice figure), and
every iterate's slice-boundary error against it (v, u, p, Frobenius norm, Sec.
4.1) is reported with the iteration at which it reaches 1e-8, if it does, and
the run time to that point. A converged run of the 16 x 4 workload (8 slices x
16 fine steps), iterated to 1e-8, gives the time to that accuracy and the
speed-up over the serial fine solve on a workload small enough to converge in
the bench. The precision variants run the predictor and one iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Profiling aids (not the benchmark line): --unit fine_step times one batched
fine theta step of --slices slices of the same workload, --unit coarse_step
one single-slice coarse (theta = 1) step as in the sequential sweep, and
--kernel-table prints the per-kernel CUDA-event times of the last warm-up step
to stderr. --unit spmv times every kernel variant of the finest-level block
product (FP64, FP32, float pairs; row-list and row-tile kernels) on --slices
slices, each against the measured HBM bandwidth.

--unit batch measures the batch runner instead: the first --instances
problems of the seeded uneven batch (meshes 64x16 .. 192x48, random solid
shear modulus and inflow, 16 .. 32 slices of 16 fine steps over T = 1), one
Parareal iteration each, run concurrently by the library's worker threads with
the worker count chosen by the library's autotuner (its timed candidate runs
are the warm-up). value = fine time-steps of all problems per second.

--unit fine_step3d times one batched fine theta step of all 32 slices of that 3D
workload from their predictor states (profiling aid; kernel shares of the last
warm-up step in the line).

--unit parareal3d measures the 3D path (hexahedral Q2, 7 unknowns per node) on the
32 x 8 x 8 channel with the plate (131,495 dofs, T = 1, 32 slices x 16 fine steps): one
fsi3_parareal iteration per step, FP32 multigrid inside FP64 FGMRES and Newton.

N > 1 runs N independent replicas (one per GPU, one rank each): the path
does not shard, so there is no collective on the data path.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Parareal FSI time-steps/s, batched slices vs serial, at 1e-8 rel error"
UNIT = "fine time-steps/s"
# DRAM read + write bytes of one finest-level launch of the row-list FP64 block product (k_bsr_spmv<double>)
# over 8 slices, from the ncu captures summarised in profiles/fsi_spmv_128x32_ncu_full.md (451.4 MB) and
# profiles/fsi_spmv_variants_128x32_8slices_ncu.md (451.6 MB); set to None when that kernel changes.
SPMV_TRAFFIC_8_SLICES = 451.4e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--unit", default="parareal", choices=["parareal", "fine_step", "coarse_step", "spmv", "batch",
                                                           "parareal3d", "fine_step3d"])
    ap.add_argument("--instances", type=int, default=4,
                    help="--unit batch: the first K problems of the seeded 48-problem uneven batch")
    ap.add_argument("--slices", type=int, default=64, help="batch for --unit fine_step")
    ap.add_argument("--kernel-table", action="store_true")
    ap.add_argument("--no-precision-variant", action="store_true",
                    help="skip the precision-variant runs (FP32 solver or FP32 multigrid)")
    ap.add_argument("--no-small-converged", action="store_true",
                    help="skip the converged Parareal run of the 16 x 4 workload")
    ap.add_argument("--from-t", type=float, default=0.0,
                    help="--unit fine_step / coarse_step: start every slice from the state reached by coarse "
                         "steps from rest up to this time")
    ap.add_argument("--set", action="append", default=[], metavar="KEY=VALUE",
                    help="--unit fine_step / coarse_step: override a solver parameter of the context")
    return ap.parse_args()


def overrides(args):
    out = {}
    for kv in args.set:
        key, val = kv.split("=", 1)
        out[key] = float(val) if any(ch in val for ch in ".e") else int(val)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms_local, units_per_rank, dist=None, device=None):
    """Whole-job rate of independent replicas: the time is the maximum over
    ranks, the work the sum over ranks (every rank does units_per_rank)."""
    import torch
    world = 1
    ms = ms_local
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms / 1000.0)


def cpu_oracle_sample(processes=None):
    """The FP64 oracle on the host cores, laid out as the paper's CPU implementation
    runs Parareal (one slice per core): P concurrent single-threaded processes,
    each one fine shifted-CN step (k = 1/1024) of one slice of the 128 x 32
    workload from rest. value = P steps over the window in which they ran."""
    P = processes or max(1, min(os.cpu_count() or 1, 16))
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import fsi as of
from paper_1907_01252_gb300 import workloads as wl
w = wl.LARGE_128x32
mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
model = of.FSIModel(mesh, w.material, newton_tol=w.newton_tol)
U = np.zeros((mesh.n_nodes, 5))
k = w.k_fine
t0 = time.time()
U = model.step(U, 0.0, k, model.theta_fine(k))
t1 = time.time()
print(json.dumps({"start": t0, "end": t1, "newton": model.newton_counts}))
""" % ROOT
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(P)]
    res = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    window = max(r["end"] for r in res) - min(r["start"] for r in res)
    each = statistics.mean(r["end"] - r["start"] for r in res)
    return {"value": P / window, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": "%d concurrent single-threaded oracle processes (one slice per core, the paper's CPU "
                      "layout), each one fine theta step (k=1/1024, Newton to 1e-10, sparse LU) of one slice of "
                      "the 128x32 workload from rest; %.1f s window, %.1f s per step and process (%.4f steps/s "
                      "on one core)" % (P, window, each, 1.0 / each)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_sample()
    vals = [cpu_oracle_sample() for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fsi2d_q2_128x32_T2_64x32", "oracle_sample": vals[0]["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def bench_batch(args, torch, fsi, wl, dev):
    """One line for the batch runner (see the module docstring)."""
    ws = wl.uneven_batch()[:max(args.instances, 1)]
    batch = fsi.Batch(ws, max_iter=1)
    cands = [1, 2, 4, 8]
    best, secs = batch.autotune([c for c in cands if c <= 2 * len(ws)])
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    l0 = fsi.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = batch.run(best)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    units = sum(w.n_slices * w.m_fine for w in ws)
    value = units * args.steps / (ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": len(secs) + 1, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "uneven_batch_seed1907_first%d_of_48" % len(ws), "unit": "batch",
                       "problems": [{"name": w.name, "n_dofs": fsi.mesh_size(w)[1], "slices": w.n_slices,
                                     "mu_s": w.material.mu_s, "vbar": w.material.vbar,
                                     "seconds": r["seconds"], "worker": r["worker"],
                                     "fine_gmres": r["stats"]["fine"]["gmres_iters"]}
                                    for w, r in zip(ws, res)],
                       "step": "every problem: parareal_iterate with 1 iteration, problems concurrent",
                       "workers": best, "autotune_seconds": dict(zip(map(str, cands), secs)),
                       "one_worker_vs_best": secs[0] / min(secs)},
            "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": fsi.launch_count() - l0}
    print(json.dumps(line))


def bench_3d(args, torch, fsi, wl, dev):
    """One line for the 3D path (see the module docstring): one Parareal iteration of the
    32 x 8 x 8 channel workload per step, all 32 slices' fine solves batched."""
    w = wl.CHANNEL3D_32x8x8
    N = w.n_slices
    ctx = fsi.Context3D(w, max_batch=N, **overrides(args))
    U = torch.zeros((N + 1, ctx.n_dofs), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        U[1:].zero_()
        return ctx.fsi3_parareal(U, 1, 0.0)[1]

    for i in range(args.warmup):
        if i == args.warmup - 1:
            fsi.profile3(True)   # per-kernel CUDA-event times of the last warm-up step
        step()
    torch.cuda.synchronize()
    kernel_ms = {k: v for k, v in fsi.profile3_read().items() if v[1]}
    fsi.profile3(False)
    total = sum(v[0] for v in kernel_ms.values()) or 1.0
    shares = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / total, 4)}
              for k, v in sorted(kernel_ms.items(), key=lambda kv: -kv[1][0])}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    l0 = fsi.launch_count3()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = fsi.launch_count3() - l0
    value = N * w.m_fine * args.steps / (ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FP32 multigrid)", "data": "synthetic",
            "config": {"workload": w.name, "unit": "parareal3d", "n_dofs": ctx.n_dofs, "n_slices": N,
                       "m_fine": w.m_fine, "levels": ctx.n_levels, "nnzb": ctx.nnzb,
                       "step": "fsi3_parareal with 1 iteration from rest",
                       "fine_newton": st["fine"]["newton_iters"], "fine_gmres": st["fine"]["gmres_iters"],
                       "coarse_newton": st["coarse"]["newton_iters"], "coarse_gmres": st["coarse"]["gmres_iters"],
                       "l2": "inputs larger than L2 (Jacobian blocks 426 MB per slice)",
                       "kernels_last_warmup": shares},
            "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": launches}
    print(json.dumps(line))


def bench_3d_step(args, torch, fsi, wl, dev):
    """Profiling aid for the 3D path: the predictor sweep of the 32 x 8 x 8 workload
    (32 implicit-Euler steps, untimed), then one batched fine theta step (shifted
    Crank-Nicolson, k = 1/512) of all 32 slices from their predictor states per step.
    value = fine time-steps (slices x steps) per second."""
    w = wl.CHANNEL3D_32x8x8
    N = w.n_slices
    K = w.T / N
    k = K / w.m_fine
    c1 = fsi.Context3D(w, max_batch=1, **overrides(args))
    U = torch.zeros((N + 1, c1.n_dofs), dtype=torch.float64, device=dev)
    for i in range(N):
        c1.fsi3_coarse(U[i:i + 1], [i * K], U[i + 1:i + 2])
    c1.close()
    ctx = fsi.Context3D(w, max_batch=N, **overrides(args))
    stream = torch.cuda.current_stream(dev)
    t0 = [i * K for i in range(N)]
    theta = 0.5 + w.material.theta0 * k
    U0 = U[:N].contiguous()
    U1 = torch.empty_like(U0)
    for i in range(args.warmup):
        if i == args.warmup - 1:
            fsi.profile3(True)
        ctx.fsi3_theta_step(U0, t0, k, theta, U1)
    torch.cuda.synchronize()
    kernel_ms = {kk: v for kk, v in fsi.profile3_read().items() if v[1]}
    fsi.profile3(False)
    total = sum(v[0] for v in kernel_ms.values()) or 1.0
    shares = {kk: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / total, 4)}
              for kk, v in sorted(kernel_ms.items(), key=lambda kv: -kv[1][0])}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = fsi.launch_count3()
    stats = []
    _, sec = timed(stream, torch, lambda: [stats.append(ctx.fsi3_theta_step(U0, t0, k, theta, U1)[1])
                                           for _ in range(args.steps)])
    clk = clocks.stop()
    print(json.dumps({"metric": METRIC, "value": N * args.steps / sec, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sec / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f64 (FP32 multigrid)", "data": "synthetic",
                      "config": {"workload": w.name, "unit": "fine_step3d", "slices": N, "n_dofs": ctx.n_dofs,
                                 "nnzb": ctx.nnzb, "levels": ctx.n_levels, "k": k,
                                 "step": "one batched fine theta step of all slices from their predictor states",
                                 "newton_iters": [st["newton_iters"] for st in stats],
                                 "gmres_iters": [st["gmres_iters"] for st in stats],
                                 "kernels_last_warmup": shares},
                      "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
                      "gpu_launches": fsi.launch_count3() - l0}))
    ctx.close()


FIELDS = (("v", slice(0, 2)), ("u", slice(2, 4)), ("p", slice(4, 5)))


def rel_errors(Ua, Ur, N):
    """Largest relative error over the slice boundaries 1..N, per field (v, u, p),
    each boundary's field measured in the Frobenius norm (Sec. 4.1)."""
    A = Ua.view(N + 1, -1, 5)[1:]
    B = Ur.view(N + 1, -1, 5)[1:]
    out = {}
    for name, sl in FIELDS:
        num = (A[:, :, sl] - B[:, :, sl]).flatten(1).norm(dim=1)
        den = B[:, :, sl].flatten(1).norm(dim=1).clamp_min(1e-300)
        out[name] = float((num / den).max())
    return out


def load_peaks():
    """HBM copy bandwidth (GB/s) measured on this machine's GPUs, or the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def fp64_peak(torch, fsi, stream):
    """FP64 FMA throughput of this GPU in TFLOP/s, measured with the library's probe
    kernel (8 independent FMA chains per thread, 8 CTAs of 256 threads per SM)."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    blocks = 152 * 8
    fsi.fp64_probe(blocks, 2000, sink)   # warm-up
    best = 0.0
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        flops = fsi.fp64_probe(blocks, 20000, sink)
        b.record(stream)
        torch.cuda.synchronize()
        best = max(best, flops / (a.elapsed_time(b) / 1000.0) / 1e12)
    return best


def serial_fine(ctx, w, U, stream, torch):
    """The serial fine solution: slice after slice, one slice per fsi_fine call, on the
    GPU. U[0] holds the initial state; fills U[1..N]. Returns the seconds it took."""
    N = w.n_slices
    dt = w.T / N
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for i in range(N):
        ctx.fsi_fine(U[i:i + 1], [i * dt], U[i + 1:i + 2])
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0


def timed(stream, torch, fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return out, a.elapsed_time(b) / 1000.0


def converged_run(torch, fsi, w, dev, stream, tol=1e-8):
    """Parareal to the metric's accuracy on a small workload: one iteration at a time
    until the slice-boundary error against the serial fine solution is <= tol
    (at the latest at k = N, where the iterate is the serial solution). Times the
    whole run (predictor included) and the serial fine solve on the same GPU."""
    N = w.n_slices
    ctx = fsi.Context(w, max_batch=N)
    Us = torch.zeros((N + 1, ctx.n_dofs), dtype=torch.float64, device=dev)
    serial_fine(ctx, w, Us.clone(), stream, torch)   # warm-up (graph capture, tables)
    t_ser = serial_fine(ctx, w, Us, stream, torch)
    U = torch.zeros_like(Us)
    _, t = timed(stream, torch, lambda: ctx.parareal_iterate(U, 0, 0.0))
    errs = []
    while True:
        (_, st), ti = timed(stream, torch, lambda: ctx.parareal_continue(U, 1, 0.0))
        t += ti
        e = rel_errors(U, Us, N)
        errs.append(max(e.values()))
        if max(e.values()) <= tol or st["iterations"] >= N:
            break
    ctx.close()
    return {"workload": w.name, "n_slices": N, "m_fine": w.m_fine, "iterations_to_1e-8": len(errs),
            "max_rel_err_per_iteration": errs, "parareal_seconds": t, "serial_gpu_seconds": t_ser,
            "parareal_fine_steps_per_s": N * w.m_fine / t, "serial_gpu_fine_steps_per_s": N * w.m_fine / t_ser,
            "speedup_vs_serial": t_ser / t}


def bench_parareal(args, torch, fsi, wl, dev, dist, rank, world):
    """The bench line: one continuing Parareal run of the 128 x 32 workload, one
    iteration per step (see the module docstring)."""
    w = wl.LARGE_128x32
    N = w.n_slices
    dt = w.T / N
    stream = torch.cuda.current_stream(dev)
    hbm_gbs, hbm_src = load_peaks()
    ctx = fsi.Context(w, max_batch=N, **overrides(args))
    n = ctx.n_dofs

    # the serial fine solution of the whole interval on the same GPU (the metric's reference)
    Us = torch.zeros((N + 1, n), dtype=torch.float64, device=dev)
    t_serial = serial_fine(ctx, w, Us, stream, torch)

    # the run: predictor sweep, then W warm-up iterations (the last one finds the dominant kernel)
    U = torch.zeros((N + 1, n), dtype=torch.float64, device=dev)
    _, t_pred = timed(stream, torch, lambda: ctx.parareal_iterate(U, 0, 0.0))
    # One step: the next Parareal iteration of the current run. On this workload the
    # iterates beyond the exact front grow until a propagator's solve fails; such a
    # step ends the run, the run is restarted from the predictor, and the failed step
    # (with the restart) stays in the timed total while advancing nothing.
    runs = [{"run": 1, "predictor_seconds": t_pred, "ended": None}]
    steps = []       # every step: warm-up and timed
    saved = {}       # step index -> iterate after it (successful steps)
    names = fsi.kernel_names()
    hU = torch.empty((N + 1, n), dtype=torch.float64).pin_memory()

    def one_step(timed_step, host_copies):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        if host_copies:
            U.copy_(hU, non_blocking=True)
        e[1].record(stream)
        prev_it = steps[-1]["iteration"] if steps and steps[-1]["run"] == runs[-1]["run"] else 0
        rec = {"run": runs[-1]["run"], "timed": timed_step}
        try:
            if runs[-1]["ended"]:
                raise fsi.FsiError(fsi.FSI_EINVAL, "no run to continue: " + runs[-1]["ended"])
            _, st = ctx.parareal_continue(U, 1, 0.0)
            S = N - (st["iterations"] - 1) if st["iterations"] > prev_it else 0   # no iteration runs past N
            rec.update({"iteration": st["iterations"], "fine_slices": S, "fine_gmres": st["fine"]["gmres_iters"],
                        "coarse_gmres": st["coarse"]["gmres_iters"], "failed": None})
        except fsi.FsiError as err:
            rec.update({"iteration": prev_it + 1, "fine_slices": 0, "failed": {"code": err.code, "message": str(err)}})
            if not runs[-1]["ended"]:
                runs[-1]["ended"] = "iteration %d: %s" % (prev_it + 1, err)
                U[1:].zero_()
                try:
                    ctx.parareal_iterate(U, 0, 0.0)   # a new run: the predictor sweep
                    runs.append({"run": runs[-1]["run"] + 1, "predictor_seconds": None, "ended": None})
                except fsi.FsiError as err2:
                    runs.append({"run": runs[-1]["run"] + 1, "predictor_seconds": None,
                                 "ended": "predictor: %s" % err2})
        e[2].record(stream)
        if host_copies:
            hU.copy_(U, non_blocking=True)
        e[3].record(stream)
        if rec["failed"] is None:
            saved[len(steps)] = U.clone()
        rec["_ev"] = e
        steps.append(rec)

    for i in range(args.warmup):
        if i == args.warmup - 1:
            fsi.profile_enable(names)
        one_step(False, False)
        torch.cuda.synchronize()
    shares = {nm: fsi.profile_read(nm)[0] for nm in names}
    if not any(shares.values()):
        shares["k_bsr_spmv"] = 1.0
    dominant = max(shares, key=shares.get)
    total_ms = sum(shares.values())
    if args.kernel_table and rank == 0:
        print("kernel event times of the last warm-up iteration (ms, share, launches):", file=sys.stderr)
        for nm in sorted(shares, key=shares.get, reverse=True):
            if shares[nm] > 0:
                print("  %-20s %10.2f %6.2f%% %8d" % (nm, shares[nm], 100 * shares[nm] / total_ms,
                                                   fsi.profile_read(nm)[1]), file=sys.stderr)
    fsi.profile_enable([dominant])

    # timed region: K steps; every step copies the iterate in from pinned host memory and
    # back out, so the same loop gives the device and the end-to-end time
    hU.copy_(U)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = fsi.launch_count()
    for _ in range(args.steps):
        one_step(True, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = fsi.launch_count() - l0
    clk = clocks.stop()
    for rec in steps:
        e = rec.pop("_ev")
        rec["seconds"] = e[1].elapsed_time(e[2]) / 1000.0
        rec["e2e_seconds"] = e[0].elapsed_time(e[3]) / 1000.0
    timed_steps = [r for r in steps if r["timed"]]
    fine_units = sum(r["fine_slices"] * w.m_fine for r in timed_steps)
    dom_ms, dom_n, dom_flops = fsi.profile_read(dominant)
    dom_bytes = fsi.profile_read_bytes(dominant)
    fsi.profile_enable([])
    # FP64 peak of the ALU roofline: the unit counts and the SM clock (152 SMs x 2 FP64 FMA per clock x 2 flop,
    # at the median SM clock sampled during the timed region; the maximum clock if none was sampled). The
    # library's FMA probe kernel is reported beside it; it reaches less than the row-list product does.
    fp64_probe = fp64_peak(torch, fsi, stream)   # right after the timed region, at its clocks
    clk_mhz = clk.get("sm_mhz") or 2070.0
    fp64_tflops = 152 * 2 * 2 * clk_mhz * 1e6 / 1e12
    ms = 1000.0 * sum(r["seconds"] for r in timed_steps)
    if fine_units:
        ms, value = aggregate(ms, fine_units, dist, dev)
        e2e_ms, e2e_value = aggregate(1000.0 * sum(r["e2e_seconds"] for r in timed_steps), fine_units, dist, dev)
    else:
        value = e2e_value = None

    # error of every iterate against the serial fine solution; run time within its run
    reached = None
    t_run = {1: t_pred}
    for idx, rec in enumerate(steps):
        t_run[rec["run"]] = t_run.get(rec["run"], 0.0) + rec["seconds"]
        rec["run_seconds"] = t_run[rec["run"]]
        if idx in saved:
            rec["max_rel_err_vs_serial"] = rel_errors(saved[idx], Us, N)
            if reached is None and max(rec["max_rel_err_vs_serial"].values()) <= 1e-8:
                reached = rec
    ok_steps = [r for r in steps if "max_rel_err_vs_serial" in r]
    best = min(ok_steps, key=lambda r: max(r["max_rel_err_vs_serial"].values())) if ok_steps else None
    at_tol = {"tolerance": 1e-8, "reached": reached is not None,
              "iterations_run": len(ok_steps),
              "iteration_reached": reached["iteration"] if reached else None,
              "run_seconds_to_reach": reached["run_seconds"] if reached else None,
              "fine_steps_per_s_at_1e-8": (N * w.m_fine / reached["run_seconds"]) if reached else None,
              "smallest_error": best["max_rel_err_vs_serial"] if best else None,
              "smallest_error_iteration": best["iteration"] if best else None,
              "exact_at_iteration": N,
              "runs": runs,
              "note": "an iterate is exact (the serial fine solution) at k = N (Sec. 4.1); boundaries "
                      "1..k are exact after iteration k; a run ends when a propagator's solve fails on its "
                      "iterates (run_seconds include the run's predictor)"}
    first_ok = saved[min(saved)] if saved and 0 in saved else None
    last_saved = saved[max(saved)] if saved else U
    saved = {}


    # the dominant kernel's roofline over the timed region, and one isolated launch of it
    roof = {"kernel": dominant, "share_of_kernel_time_last_warmup": shares[dominant] / total_ms if total_ms else None}
    if dom_ms > 0 and dom_bytes > 0:
        gbs = dom_bytes / (dom_ms / 1000.0) / 1e9
        tfl = dom_flops / (dom_ms / 1000.0) / 1e12
        alu_frac = tfl / fp64_tflops
        hbm_frac = gbs / hbm_gbs
        roof.update({"bound": "alu" if alu_frac >= hbm_frac else "hbm",
                     "achieved": tfl if alu_frac >= hbm_frac else gbs,
                     "peak": fp64_tflops if alu_frac >= hbm_frac else hbm_gbs,
                     "unit": "TFLOP/s" if alu_frac >= hbm_frac else "GB/s",
                     "frac": max(alu_frac, hbm_frac),
                     "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_gbs, "frac": hbm_frac, "peak_source": hbm_src},
                     "fp64": {"achieved_tflops": tfl, "peak_tflops": fp64_tflops, "frac": alu_frac,
                              "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x %.0f MHz (median SM "
                                             "clock of the timed region)" % clk_mhz,
                              "probe_tflops": fp64_probe,
                              "probe_source": "measured in this run: the library's FP64 FMA probe kernel"},
                     "timed_launches": dom_n, "algorithmic_bytes": dom_bytes, "algorithmic_flops": dom_flops,
                     "traffic": None,
                     "traffic_note": "the timed launches mix levels and batch sizes; the per-launch DRAM traffic "
                                     "of the finest-level batched launch is in isolated_finest_launch"})
    elif dom_ms > 0 and dom_flops > 0:
        tfl = dom_flops / (dom_ms / 1000.0) / 1e12
        roof.update({"bound": "alu", "achieved": tfl, "peak": fp64_tflops, "unit": "TFLOP/s",
                     "frac": tfl / fp64_tflops, "traffic": None, "timed_launches": dom_n})
    iso = None
    if dominant == "k_bsr_spmv":
        t_old = [i * dt for i in range(N)]
        vals = ctx.fsi_jacobian(last_saved[1:], last_saved[:N], w.k_fine, 0.5 + w.material.theta0 * w.k_fine)
        x = last_saved[1:].contiguous()
        y = torch.empty_like(x)
        # the row-list kernel (the variant the library picks on this level at 64 slices), kernel time only
        ctx.fsi_bsr_spmv_variant(0, 0, vals, x, y)
        reps = 20
        fsi.profile_enable(["k_bsr_spmv"])
        for _ in range(reps):
            ctx.fsi_bsr_spmv_variant(0, 0, vals, x, y)
        torch.cuda.synchronize()
        ms_iso, n_iso, _ = fsi.profile_read("k_bsr_spmv")
        fsi.profile_enable([])
        nnzb = ctx.nnzb
        abytes = N * 8 * (25 * nnzb + 2 * n) + 4 * (nnzb + 2 * n // 5 + 1)
        sec = ms_iso / 1000.0 / n_iso
        iso = {"slices": N, "kernel": "k_bsr_spmv<double> (row list)", "ms": 1000 * sec, "algorithmic_bytes": abytes, "achieved_gbs": abytes / sec / 1e9,
               "hbm_frac": abytes / sec / 1e9 / hbm_gbs,
               "fp64_frac": 50.0 * nnzb * N / sec / 1e12 / fp64_tflops,
               "traffic": SPMV_TRAFFIC_8_SLICES * N / 8 if SPMV_TRAFFIC_8_SLICES else None,
               "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 8-slice finest-level "
                                 "launch, scaled by 8 (traffic grows with the slices)",
               "l2": "inputs larger than L2 (3.4 GB of blocks); back-to-back launches, kernel time from CUDA events"}
        del vals, x, y, t_old
    roof["isolated_finest_launch"] = iso

    # precision variants (config 3): the predictor and one iteration from the same start,
    # against the FP64 iterate after iteration 1 and the exact first boundary
    variants = []
    if not args.no_precision_variant and first_ok is not None:
        U1_64 = first_ok
        tip = wl.tip_node(w)
        desc = {1: "FP32 linear solver (FGMRES, multigrid, Vanka, operator; element contraction on the tensor cores, "
                   "BF16 split terms into FP32) inside the FP64 Newton loop (Newton tolerance 2e-12); FP64 "
                   "residual, J = det F, Parareal correction",
                2: "FP64 FGMRES preconditioned by an FP32 multigrid V-cycle (FP32 Vanka, transfers, level "
                   "operators); FP64 residual, J = det F, Parareal correction"}
        for prec in (1, 2):
            # precision 1: the Jacobian in FP32 (tensor-core contraction, FP32 tangent) makes Newton converge
            # linearly, so its iterate sits closer to the stopping test; at 1e-11 the first boundary's tip
            # displacement was 9e-8 off the FP64 iterate, at 2e-12 it is 2e-9
            ctxv = fsi.Context(w, max_batch=N, precision=prec, **({"newton_tol": 2e-12} if prec == 1 else {}))
            Uv = torch.zeros_like(U)
            (_, sv), tv = timed(stream, torch, lambda: ctxv.parareal_iterate(Uv, 1, 0.0))
            err = rel_errors(Uv, U1_64, N)
            a = Uv.view(N + 1, -1, 5)[1:, tip, 2:4]
            b = U1_64.view(N + 1, -1, 5)[1:, tip, 2:4]
            # per boundary, relative to the tip displacement at that boundary (the strictest reading: the
            # first boundaries, in the inflow ramp, have the smallest displacements), and relative to the
            # largest tip displacement of the trajectory
            err["tip_displacement"] = float(((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-300)).max())
            err["tip_displacement_rel_to_max"] = float((a - b).norm(dim=1).max() / b.norm(dim=1).max())
            b1 = rel_errors(Uv[:2].contiguous(), Us[:2].contiguous(), 1)
            variants.append({"precision": prec, "what": desc[prec], "step": "predictor + iteration 1",
                             "seconds": tv, "fine_steps_per_s": N * w.m_fine / tv,
                             "fp64_seconds_same_work": t_pred + steps[0]["seconds"],
                             "max_rel_err_vs_fp64_iterate": err, "boundary1_rel_err_vs_fp64_serial": b1,
                             "newton_fine": sv["fine"], "newton_coarse": sv["coarse"]})
            ctxv.close()
            del Uv

    small = None
    if not args.no_small_converged:
        small = converged_run(torch, fsi, wl.SMALL_16x4, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample()

    # the paper's speedup model, Eq. (eq:speedup), S = 1 / (r + (K / N)(1 + r)), with r the measured
    # cost of one coarse slice step (the predictor sweep / N) over one serial fine slice
    r = (t_pred / N) / (t_serial / N)
    model = {"r": r, "K": args.steps, "N": N, "S": 1.0 / (r + (args.steps / N) * (1.0 + r)),
             "note": "model speed-up with one processor per slice and K iterations"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / max(len(timed_steps), 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "steps_completed": sum(1 for r in timed_steps if r["failed"] is None),
                "config": {"workload": w.name, "unit": "parareal", "n_dofs": n, "n_slices": N,
                           "m_fine": w.m_fine, "m_coarse": w.m_coarse, "mg_levels": ctx.n_levels,
                           "step": "one Parareal iteration of a continuing run (parareal_continue): batched "
                                   "fine solves of every slice not yet exact, then the corrected coarse sweep. A "
                                   "step whose solve fails on the run's iterates ends the run and starts a new one "
                                   "(predictor sweep); it stays in the timed total and advances no fine step. "
                                   "value = fine time-steps advanced per second over all timed steps",
                           "l2": "inputs larger than L2 (3.4 GB of Jacobian values per batch)",
                           "overrides": overrides(args),
                           "solver": {"newton_tol": w.newton_tol, "newton_eta": w.newton_eta,
                                      "gmres_rtol_first": w.gmres_rtol_first, "gmres_rtol": w.gmres_rtol,
                                      "gmres_restart": w.gmres_restart},
                           "at_1e-8": at_tol,
                           "serial_gpu_seconds": t_serial,
                           "serial_gpu_fine_steps_per_s": N * w.m_fine / t_serial,
                           "batched_iterations_vs_serial_steps_per_s": value / (N * w.m_fine / t_serial),
                           "predictor_seconds": t_pred,
                           "iterations": steps,
                           "paper_speedup_model": model,
                           "converged_small_workload": small},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": hU.numel() * 8,
                        "d2h_bytes_per_step": hU.numel() * 8,
                        "note": "the same timed iterations, each with the iterate copied in from pinned host "
                                "memory and back out through the public API"},
                "clocks": clk, "precision_variants": variants, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    ctx.close()


def bench_spmv(args, torch, fsi, wl, dev):
    """Profiling aid: every variant of the finest-level block product of the 128 x 32
    workload (FP64, FP32 and float-pair values; the row-list kernel and the row-tile
    kernel at each tile height), --slices slices of Jacobians assembled at seeded
    random states. Per variant: --warmup untimed launches, then --steps launches
    whose kernel time comes from the library's CUDA events (the float-pair
    conversions of vals and x are launched too but not counted)."""
    import numpy as np
    w = wl.LARGE_128x32
    S = args.slices
    hbm_gbs, hbm_src = load_peaks()
    ctx = fsi.Context(w, max_batch=S, ff_operator=1)
    nn = ctx.n_dofs // 5
    U = torch.tensor(np.stack([wl.random_state(nn, 900 + s) for s in range(S)]).reshape(S, -1), dtype=torch.float64,
                     device=dev)
    x = torch.tensor(np.stack([wl.random_state(nn, 950 + s) for s in range(S)]).reshape(S, -1), dtype=torch.float64,
                     device=dev)
    vals = ctx.fsi_jacobian(U, U, w.k_fine, 0.5 + w.material.theta0 * w.k_fine)
    v32, x32 = vals.float(), x.float()
    nnzb, n = ctx.nnzb, ctx.n_dofs
    out = []
    for vt, name, kname, (v, xx) in ((0, "f64", "k_bsr_spmv", (vals, x)), (1, "f32", "k_bsr_spmv", (v32, x32)),
                                     (2, "float_pair", "k_bsr_spmv_ff", (vals, x))):
        vsz = 4 if vt == 1 else 8
        abytes = S * vsz * (25 * nnzb + 2 * n) + 4 * (nnzb + 2 * nn + 1)
        ref = None
        for rows in (0, 8, 16, 32, 64):
            try:
                y = ctx.fsi_bsr_spmv_variant(vt, rows, v, xx)
            except fsi.FsiError as err:
                out.append({"values": name, "tile_rows": rows, "skipped": str(err)})
                continue
            for _ in range(max(0, args.warmup - 1)):
                ctx.fsi_bsr_spmv_variant(vt, rows, v, xx, y)
            torch.cuda.synchronize()
            fsi.profile_enable([kname])
            for _ in range(args.steps):
                ctx.fsi_bsr_spmv_variant(vt, rows, v, xx, y)
            torch.cuda.synchronize()
            ms, cnt, fl = fsi.profile_read(kname)
            fsi.profile_enable([])
            same = True if ref is None else bool(torch.equal(y, ref))
            ref = y if ref is None else ref
            sec = ms / 1000.0 / cnt
            out.append({"values": name, "tile_rows": rows, "us_per_launch": 1e6 * sec,
                        "algorithmic_bytes": abytes, "achieved_gbs": abytes / sec / 1e9,
                        "hbm_frac": abytes / sec / 1e9 / hbm_gbs, "gflops": 50.0 * nnzb * S / sec / 1e9,
                        "same_bits_as_row_list": same})
    print(json.dumps({"unit": "spmv", "workload": w.name, "slices": S, "nnzb": nnzb, "n_dofs": n,
                      "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": hbm_src,
                      "l2": "inputs larger than L2 (%.2f GB of FP64 blocks)" % (S * nnzb * 200 / 1e9),
                      "variants": out}))
    ctx.close()


def bench_unit(args, torch, fsi, wl, dev, dist, rank, world):
    """Profiling aids: one batched fine theta step (--unit fine_step) or one
    single-slice coarse step (--unit coarse_step) of the 128 x 32 workload."""
    w = wl.LARGE_128x32
    if args.unit == "coarse_step":
        args.slices = 1
    ctx = fsi.Context(w, max_batch=args.slices, **overrides(args))
    n = ctx.n_dofs
    stream = torch.cuda.current_stream(dev)
    Uf = torch.zeros((args.slices, n), dtype=torch.float64, device=dev)
    tf = [0.0] * args.slices      # first step of the trajectory, from rest
    if args.from_t > 0:           # or from a developed state: coarse steps from rest up to from_t
        nc = max(1, int(round(args.from_t / w.k_coarse)))
        U1 = torch.zeros((1, n), dtype=torch.float64, device=dev)
        for i in range(nc):
            U1, _ = ctx.fsi_coarse(U1, [i * w.k_coarse])
        Uf[:] = U1
        tf = [nc * w.k_coarse] * args.slices
    kf = w.k_fine if args.unit == "fine_step" else w.k_coarse
    th = 0.5 + w.material.theta0 * kf if args.unit == "fine_step" else 1.0
    names = fsi.kernel_names()
    for i in range(args.warmup):
        if i == args.warmup - 1:
            fsi.profile_enable(names)
        ctx.fsi_theta_step(Uf, tf, kf, th)
    torch.cuda.synchronize()
    shares = {nm: fsi.profile_read(nm)[0] for nm in names}
    total_ms = sum(shares.values()) or 1.0
    fsi.profile_enable([])
    if args.kernel_table:
        print("kernel event times of the last warm-up step (ms, share, launches):", file=sys.stderr)
        for nm in sorted(shares, key=shares.get, reverse=True):
            if shares[nm] > 0:
                print("  %-20s %10.2f %6.2f%% %8d" % (nm, shares[nm], 100 * shares[nm] / total_ms,
                                                   fsi.profile_read(nm)[1]), file=sys.stderr)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    l0 = fsi.launch_count()
    print("launches before the timed steps: %d" % l0, file=sys.stderr)
    stats = []
    _, sec = timed(stream, torch, lambda: [stats.append(ctx.fsi_theta_step(Uf, tf, kf, th)[1]) for _ in range(args.steps)])
    clk = clocks.stop()
    value = args.slices * args.steps / sec
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1000 * sec / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": w.name, "unit": args.unit, "slices": args.slices,
                                 "overrides": overrides(args),
                                 "newton_iters": [st["newton_iters"] for st in stats],
                                 "gmres_iters": [st["gmres_iters"] for st in stats]},
                      "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
                      "gpu_launches": fsi.launch_count() - l0}))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_1907_01252_gb300 import build, fsi, workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build_library()
    if args.unit == "batch":
        bench_batch(args, torch, fsi, wl, dev)
    elif args.unit == "parareal3d":
        bench_3d(args, torch, fsi, wl, dev)
    elif args.unit == "fine_step3d":
        bench_3d_step(args, torch, fsi, wl, dev)
    elif args.unit == "spmv":
        bench_spmv(args, torch, fsi, wl, dev)
    elif args.unit in ("fine_step", "coarse_step"):
        bench_unit(args, torch, fsi, wl, dev, dist, rank, world)
    else:
        bench_parareal(args, torch, fsi, wl, dev, dist, rank, world)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

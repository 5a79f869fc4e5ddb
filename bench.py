#!/usr/bin/env python
"""Benchmark: time-to-solution of Improved Seed-CG on one GB300 (and the
oracle's CPU baseline), printed as one JSON line.

Workload (default): the 16^3x32 lattice (eps = 0.5, seed 2, kappa tuned to
cond(M) ~ 1e5), nrhs = 12 unit point sources b^j = D^dag eta^j, tol 1e-8 on
the FP64 true residual, PO every k = 10 iterations, RHS 1 run 2x past
convergence, mixed precision (FP32 dslash, bf16 V, FP64 scalars and
reliable updates).  One step = one seedcg_solve of all 12 systems (every
stage of the method: dslash, Lanczos + LU of T, PO, seeds, batched CG).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU; every rank solves its own copy
of the workload (replicas: the method has no exchange step between
independent problems), timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "large_16x16x16x32_nrhs12"
METRIC = "time-to-solution, all nrhs at rel. residual 1e-8 (s); dslash HBM GB/s vs peak"


# measured DRAM read + write bytes / algorithmic bytes of the PO step (projection + subtraction)
PO_DRAM_PER_ALG_BF16 = 1.01


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--precision", default=None, help="fp64 | mixed_v32 | mixed_vbf16")
    p.add_argument("--m-max", type=int, default=8000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-sample-iters", type=int, default=24)
    p.add_argument("--record-units", action="store_true",
                   help="write this run's work units (m, CG iterations) for the reference arm")
    p.add_argument("--no-compare", action="store_true",
                   help="skip the comparators reported beside the line (one plain FP64 seed-CG "
                        "solve and one standard batched CG from x0 = 0, both untimed by the line)")
    p.add_argument("--no-cpu-c1", action="store_true",
                   help="skip the end-to-end oracle run of the 8^3x16 workload on the host cores")
    p.add_argument("--oracle-c1-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--compare-classic", action="store_true",
                   help="also time classic repeated seeding (seed_mode 2, Section 1's comparison "
                        "variant) on the same workload, reported beside the line")
    p.add_argument("--tc-po", type=int, default=1, choices=[0, 1, 2],
                   help="with --only po: use_tensor_cores for the bf16 basis (0 SIMT, 1 default: "
                        "tcgen05 for the seeds only, 2 tcgen05 for the PO projection too)")
    p.add_argument("--sweep", default=None, choices=["m", "k", "kappa"],
                   help="Figs 1-2 / Table 1 of the paper on a synthetic field: CG matvecs of the "
                        "second right-hand side against the past-convergence factor (m) or the PO "
                        "period (k), first-RHS cost against k; 'kappa' scans --kappas. One JSON "
                        "line per setting (not a bench line)")
    p.add_argument("--kappa", type=float, default=None, help="with --sweep: kappa of the field")
    p.add_argument("--po-passes", type=int, default=1, choices=[1, 2],
                   help="with --sweep: Gram-Schmidt passes per PO step (2 = CGS2)")
    p.add_argument("--po-guard", type=int, default=1, choices=[0, 1],
                   help="with --sweep: 0 runs step 8 as printed, without the guard that ends "
                        "Lanczos when a PO step finds the basis far from orthonormal")
    p.add_argument("--kappas", default="", help="with --sweep kappa: comma-separated values")
    p.add_argument("--guess-eval", action="store_true",
                   help="learned initial guess on the workload's field: train on (b, x) pairs the "
                        "solver produces, then solve held-out Z2 sources from x0 = 0 and from the "
                        "learned x0 (iterations and time; one JSON line, not a bench line)")
    p.add_argument("--deflate-eval", type=int, default=0, metavar="NEV",
                   help="Ritz deflation at the workload's scale: after the solve, a new batch of "
                        "Z2 sources is solved from x0 = 0 and from the guess deflated with NEV "
                        "Ritz vectors (one JSON line, not a bench line)")
    p.add_argument("--train-pairs", type=int, default=2000)
    p.add_argument("--eval-pairs", type=int, default=64)
    p.add_argument("--epochs", type=int, default=10)
    p.add_argument("--lr", type=float, default=3e-3)
    p.add_argument("--eo", action="store_true",
                   help="the even-odd preconditioned system of Section 3 (A^dag A x_o = A^dag phi on "
                        "odd-site half vectors) on the same workload: its own JSON line with its PO "
                        "roofline, beside one full-lattice solve of the same sources (not a bench line)")
    p.add_argument("--only", default=None, choices=["dslash", "po", "guess", "cg"],
                   help="profiling aid: run only the 12-RHS dslash timing, one solve capped "
                        "at --m-max Lanczos iterations (re-orthogonalisation kernels), --steps "
                        "forward passes of the learned guess, or the workload's systems by "
                        "batched CG from zero (no stored basis: a few GB on the device)")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: a bounded sample of the same workload, scaled by work units
# ---------------------------------------------------------------------------
def oracle_unit_costs(workload, sample_iters: int):
    """Time the oracle (as it stands) on the workload's own field and sources:
    `sample_iters` Lanczos iterations of Algorithm 1 with literal seeding of all
    right-hand sides, one re-orthogonalisation against that many stored
    vectors, and a few CG iterations.  Returns per-unit seconds."""
    import numpy as np
    from oracle.seedcg import cg, periodic_reorth, seed_lanczos
    from oracle.wilson import WilsonOperator
    from paper_0901_3512_gb300 import workloads as W
    f = workload.fields[0]
    op = WilsonOperator(f.dims, f.gauge(), W.kappa_for(f.name))
    eta = workload.sources_for(0)
    B = np.stack([op.Ddag(e) for e in eta]).reshape(len(eta), -1)
    t0 = time.perf_counter()
    res = seed_lanczos(op.M, B, None, workload.tol, sample_iters, 0)
    t_lz = (time.perf_counter() - t0) / max(res.m, 1)
    V = np.array(res.V)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    fvec = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    Vw = np.zeros((V.shape[0] + 1, op.n), dtype=np.complex128)
    Vw[:V.shape[0]] = V
    t0 = time.perf_counter()
    periodic_reorth(Vw, V.shape[0] + 1, v, fvec, 1)
    t_po_row = (time.perf_counter() - t0) / (2 * V.shape[0] + 1)
    ncg = 4
    t0 = time.perf_counter()
    cg(op.M, B[1], None, 1e-30, ncg)
    t_cg = (time.perf_counter() - t0) / (ncg + 2)
    return {"t_lanczos_iter": t_lz, "t_po_row": t_po_row, "t_cg_iter": t_cg,
            "sample": f"{res.m} Lanczos iterations with literal seeding of {len(eta)} RHS, "
                      f"one PO against {V.shape[0]} vectors, {ncg} CG iterations, on the "
                      f"{'x'.join(map(str, f.dims))} field"}


def oracle_estimate(costs, m, k, cg_iters_total, nrhs):
    po_rows = sum(i - 1 for i in range(k, m + 1, k)) * 2 + (m // k if k else 0) if k else 0
    return m * costs["t_lanczos_iter"] + po_rows * costs["t_po_row"] + cg_iters_total * costs["t_cg_iter"]


C1_WORKLOAD = "small_8x8x8x16_nrhs12"


def oracle_c1_worker():
    """Run the oracle, as it stands, end to end on the 8^3x16 twelve-point-source
    workload (Algorithm 1 with blocked Eq. (1) seeds, then CG for every system
    above tol) and print one JSON line.  Runs in its own process on the cores it
    was given, so that it can proceed while the GPU arm measures."""
    import numpy as np
    from oracle.seedcg import improved_seed_cg
    from oracle.wilson import WilsonOperator
    from paper_0901_3512_gb300 import workloads as W
    wl = W.WORKLOADS[C1_WORKLOAD]
    f = wl.fields[0]
    op = WilsonOperator(f.dims, f.gauge(), W.kappa_for(f.name))
    eta = wl.sources_for(0)
    B = np.stack([op.Ddag(e) for e in eta]).reshape(len(eta), -1)
    t0 = time.perf_counter()
    r = improved_seed_cg(op.M, B, None, wl.tol, 6000, wl.reorth_period, wl.past_factor,
                         seed_mode="blocked")
    t = time.perf_counter() - t0
    print(json.dumps({"seconds": t, "m_conv": int(r.seed.m_conv), "m": int(r.seed.m),
                      "iters": [int(i) for i in r.iters],
                      "max_true_resid": float(np.max(r.true_resid))}), flush=True)


def start_oracle_c1():
    """Start the end-to-end oracle run of the 8^3x16 workload in a child process
    (a fresh interpreter, started before this process touches the GPU) pinned to
    every host core but the first two, which stay with the GPU arm's launches."""
    cores = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else []
    use = cores[2:] if len(cores) > 4 else cores
    env = dict(os.environ)
    n = str(max(len(use), 1))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = n
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    pre = None
    if use and hasattr(os, "sched_setaffinity"):
        def pre():
            os.sched_setaffinity(0, use)
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-c1-worker"],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                            preexec_fn=pre, cwd=ROOT)
    return proc, len(use) if use else os.cpu_count()


def finish_oracle_c1(handle, timeout_s: float = 900.0):
    proc, cores = handle
    try:
        out, err = proc.communicate(timeout=timeout_s)
    except subprocess.TimeoutExpired:
        proc.kill()
        proc.communicate()
        return {"workload": C1_WORKLOAD, "error": f"did not finish within {timeout_s:.0f} s",
                "cores": cores}
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    if proc.returncode != 0 or not lines:
        return {"workload": C1_WORKLOAD, "error": (err or out).strip().splitlines()[-1:] or "failed",
                "cores": cores}
    d = json.loads(lines[-1])
    d.update({"workload": C1_WORKLOAD, "cores": cores, "kind": "oracle", "unit": "s",
              "sample": "the whole 8^3x16 twelve-point-source solve (Algorithm 1 + Eq. (1) "
                        "seeds + CG), end to end, concurrently with the GPU arm"})
    return d


# ---------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------
def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _config(args, wl, world: int) -> dict:
    """The single-field workload's config, shared by our arm and the reference arm."""
    from paper_0901_3512_gb300 import workloads as W
    f = wl.fields[0]
    return {"workload": args.workload, "lattice": list(f.dims), "nrhs": wl.nrhs[0],
            "sources": wl.sources, "tol": wl.tol, "reorth_period": wl.reorth_period,
            "past_factor": wl.past_factor, "precision": args.precision or wl.precision,
            "kappa": W.kappa_for(f.name),
            "l2": "inputs larger than L2 (the stored basis V is tens of GB)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_0901_3512_gb300 import workloads as W
    wl = W.WORKLOADS[args.workload]
    units_path = os.path.join(ROOT, "paper_0901_3512_gb300", "workload_units.json")
    units = json.load(open(units_path)).get(args.workload) if os.path.exists(units_path) else None
    if units is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          "no recorded work-unit counts for this workload"}))
        return
    vals = []
    costs = None
    for _ in range(args.warmup):
        oracle_unit_costs(wl, max(4, args.cpu_sample_iters // 4))
    t_all = time.perf_counter()
    for _ in range(args.steps):
        costs = oracle_unit_costs(wl, args.cpu_sample_iters)
        vals.append(oracle_estimate(costs, units["m"], wl.reorth_period, units["cg_iters_total"],
                                    sum(wl.nrhs)))
    wall = time.perf_counter() - t_all
    v = statistics.median(vals)
    cores = os.cpu_count()
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": _config(args, wl, world) if len(wl.fields) == 1 else
                     {"workload": args.workload, "nrhs": sum(wl.nrhs), "tol": wl.tol,
                      "reorth_period": wl.reorth_period, "past_factor": wl.past_factor},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                            "sample": costs["sample"] + "; scaled by the recorded work units "
                            f"(m={units['m']}, CG iterations={units['cg_iters_total']})"},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """Several uneven gauge fields in one seedcg_batch_solve (one step = one call)."""
    import torch

    from paper_0901_3512_gb300 import replicas, seedcg, workloads as W
    world, rank, local = _dist()
    replicas.init("nccl", torch.device("cuda", local))
    torch.cuda.set_device(local)
    wl = W.WORKLOADS[args.workload]
    prec = args.precision or wl.precision
    solvers, Bs, Xs = [], [], []
    for i, f in enumerate(wl.fields):
        s = seedcg.Solver(f.dims, f.gauge(), W.kappa_for(f.name), precision=prec,
                          past_factor=wl.past_factor, m_max=args.m_max)
        eta = torch.from_numpy(wl.sources_for(i)).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        solvers.append(s)
        Bs.append(B)
        Xs.append(torch.zeros_like(B))
    hs = [s.h for s in solvers]
    for _ in range(args.warmup):
        seedcg.seedcg_batch_solve(hs, Bs, Xs, wl.tol, 0, wl.reorth_period)
    torch.cuda.synchronize()
    replicas.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = seedcg.seedcg_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        code, infos = seedcg.seedcg_batch_solve(hs, Bs, Xs, wl.tol, 0, wl.reorth_period)
    e1.record()
    torch.cuda.synchronize()
    replicas.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, torch.device("cuda", local))
    if rank != 0:
        replicas.finish()
        return
    out = {"metric": METRIC, "value": replicas.job_seconds_per_solve(ms / 1000.0, world), "unit": "s",
           "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": prec, "data": "synthetic",
           "config": {"workload": args.workload,
                      "fields": [{"lattice": list(f.dims), "nrhs": n, "kappa": W.kappa_for(f.name)}
                                 for f, n in zip(wl.fields, wl.nrhs)],
                      "sources": wl.sources, "tol": wl.tol, "reorth_period": wl.reorth_period},
           "valid": code == 0 and all(max(i["true_resid"]) <= wl.tol for i in infos),
           "fields": [{"m_conv": i["m_conv"], "m": i["m"], "cg_iters_max": i["cg_iters_max"],
                       "max_true_resid": max(i["true_resid"]), "ms_lanczos": i["ms_lanczos"],
                       "ms_po": i["ms_po"]} for i in infos],
           "ms_cg_batched": infos[0]["ms_cg"], "clocks": clocks,
           "gpu_launches": seedcg.seedcg_kernel_launches() - l0}
    print(json.dumps(out))
    for s in solvers:
        s.close()
    replicas.finish()


BATCH_WORKLOAD = "batch3_uneven_nrhs24_12_6"


def batch3_once():
    """The three uneven gauge fields (8^3x16 / 12^3x24 / 16^3x32, Z2 sources 24 / 12 / 6) in one
    seedcg_batch_solve in the workload's own precision (FP32 iteration, FP64 reliable updates):
    one warm-up call (autotuning), one timed call."""
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[BATCH_WORKLOAD]
    prec = wl.precision
    solvers, Bs, Xs = [], [], []
    for i, f in enumerate(wl.fields):
        sv = seedcg.Solver(f.dims, f.gauge(), W.kappa_for(f.name), precision=prec,
                           past_factor=wl.past_factor, m_max=4000)
        eta = torch.from_numpy(wl.sources_for(i)).cuda()
        B = torch.empty_like(eta)
        sv.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        solvers.append(sv)
        Bs.append(B)
        Xs.append(torch.zeros_like(B))
    hs = [sv.h for sv in solvers]
    seedcg.seedcg_batch_solve(hs, Bs, Xs, wl.tol, 0, wl.reorth_period, allow_not_converged=True)
    for x in Xs:
        x.zero_()
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record()
    code, infos = seedcg.seedcg_batch_solve(hs, Bs, Xs, wl.tol, 0, wl.reorth_period, allow_not_converged=True)
    eb.record()
    torch.cuda.synchronize()
    out = {"workload": BATCH_WORKLOAD, "precision": prec, "seconds": ea.elapsed_time(eb) / 1000.0,
           "status": code, "systems": sum(wl.nrhs),
           "fields": [{"lattice": list(f.dims), "nrhs": n, "m_conv": i["m_conv"], "m": i["m"],
                       "cg_iters_max": i["cg_iters_max"], "max_true_resid": max(i["true_resid"])}
                      for f, n, i in zip(wl.fields, wl.nrhs, infos)],
           "ms_cg_batched": infos[0]["ms_cg"]}
    for sv in solvers:
        sv.close()
    del Bs, Xs
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_0901_3512_gb300 import replicas, seedcg, workloads as W

    world, rank, local = _dist()
    c1 = None
    all_cores = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_cpu_c1:
        c1 = start_oracle_c1()
        if all_cores and len(all_cores) > 4:
            os.sched_setaffinity(0, all_cores[:2])
    replicas.init("nccl", torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or wl.precision
    kappa = W.kappa_for(f.name)
    nrhs = wl.nrhs[0]
    gauge = f.gauge()
    s = seedcg.Solver(f.dims, gauge, kappa, precision=prec, past_factor=wl.past_factor,
                      m_max=args.m_max)
    eta = torch.from_numpy(wl.sources_for(0)).to(dev)
    B = torch.empty_like(eta)
    s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
    X = torch.zeros_like(B)
    stream = torch.cuda.current_stream(dev)
    k = wl.reorth_period

    barrier = replicas.barrier

    for _ in range(args.warmup):
        s.solve(B, X, wl.tol, 0, k, stream=stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = seedcg.seedcg_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        code, info = s.solve(B, X, wl.tol, 0, k, stream=stream)
        infos.append((code, info))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = seedcg.seedcg_kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = replicas.max_over_ranks(ms, dev)
    code, info = infos[-1]
    ok = all(c == 0 for c, _ in infos) and max(info["true_resid"]) <= wl.tol

    # ---- the dominant kernel group: periodic re-orthogonalisation against V ----
    peaks, peak_kind = _peaks()
    vol = int(np.prod(f.dims))
    n = 12 * vol
    vbytes = {"fp64": 16, "mixed_v32": 8, "mixed_vbf16": 4}[prec]
    m = info["m"]
    po_rows = sum(i - 1 for i in range(k, m + 1, k)) if k else 0
    po_alg_bytes = 2 * po_rows * n * vbytes  # V_{1:i-1} read by the projection and the update
    po_s = info["ms_po"] / 1000.0
    po_gbs = po_alg_bytes / po_s / 1e9 if po_s > 0 else None
    # DRAM bytes per algorithmic byte of the PO kernels, from the 1-pass ncu window of this
    # workload's PO launches; only for the configuration measured
    traffic = (round(PO_DRAM_PER_ALG_BF16 * po_alg_bytes)
               if prec == "mixed_vbf16" and args.workload == "large_16x16x16x32_nrhs12" else None)
    roofline = {"bound": "hbm", "achieved": po_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (po_gbs / peaks["hbm_gbs"]) if po_gbs else None, "traffic": traffic,
                "traffic_unit": "bytes per solve",
                "kernel": "periodic re-orthogonalisation (V^dag [v,f] projection + [v,f] -= V c)",
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_solve": po_alg_bytes, "ms_per_solve": info["ms_po"]}

    # ---- the 12-RHS dslash alone (the metric's second part) ----
    dslash = None
    try:
        ms_d = s.time_dslash(prec=1, n=nrhs, reps=20, stream=stream)
        bytes_site = nrhs * 2 * 12 * 8 + 4 * 9 * 8  # FP32: spinors in + out, 4 links per site
        gbs = bytes_site * vol / (ms_d / 1000.0) / 1e9
        dslash = {"kernel": "multi-RHS Wilson dslash, FP32, n=%d" % nrhs, "ms": ms_d,
                  "achieved_gbs": gbs, "frac": gbs / peaks["hbm_gbs"],
                  "algorithmic_bytes_per_site": bytes_site, "l2": "flushed before each launch"}
    except Exception as e:  # timing helper missing in an old build
        dslash = {"error": str(e)}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        Bh = B.cpu().pin_memory()
        Xh = torch.zeros_like(Bh).pin_memory()
        s.solve(Bh, Xh, wl.tol, 0, k)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.solve(Bh, Xh, wl.tol, 0, k)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        nb = Bh.numel() * Bh.element_size()
        e2e = {"value": replicas.job_seconds_per_solve(replicas.max_over_ranks(e2e_s, dev), world),
               "unit": "s", "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}

    fp64_cmp = None
    cg_only_cmp = None
    eo_cmp = None
    batch_cmp = None
    if not args.no_compare and rank == 0 and args.workload == DEFAULT_WORKLOAD:
        # the same 12 systems by standard batched CG from x0 = 0 (no Lanczos, no seeds):
        # what seeding buys on this field (untimed by the line)
        s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max, seed_mode=3)
        Xc = torch.zeros_like(B)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        cc, ic = s.solve(B, Xc, wl.tol, 0, k, stream=stream, allow_not_converged=True)
        eb.record(stream)
        torch.cuda.synchronize()
        tcg = ea.elapsed_time(eb) / 1000.0
        cg_only_cmp = {"seconds": tcg, "status": cc, "iters": ic["iters"],
                       "max_true_resid": max(ic["true_resid"]),
                       "reliable_updates": ic["reliable_updates"],
                       "seeded_over_cg_only_time": (ms_max / 1000.0) / tcg}
        s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max)
        del Xc
        # the even-odd system of Section 3 on the same sources (one warm-up, one timed solve)
        Xe = torch.zeros_like(eta)
        seedcg.seedcg_solve_eo(s.h, eta, Xe, wl.tol, 0, k, stream=stream, allow_not_converged=True)
        Xe.zero_()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        ce, ie = seedcg.seedcg_solve_eo(s.h, eta, Xe, wl.tol, 0, k, stream=stream, allow_not_converged=True)
        eb.record(stream)
        torch.cuda.synchronize()
        te = ea.elapsed_time(eb) / 1000.0
        eo_cmp = {"seconds": te, "status": ce, "m_conv": ie["m_conv"], "m": ie["m"],
                  "cg_iters_max": ie["cg_iters_max"], "ms_po": ie["ms_po"], "ms_cg": ie["ms_cg"],
                  "max_true_resid": max(ie["true_resid"]), "max_true_resid_D": max(ie["true_resid_D"]),
                  "speedup_over_full_lattice": (ms_max / 1000.0) / te}
        del Xe
        # one plain FP64 Improved Seed-CG solve of the same systems on the GPU, for the
        # mixed-precision speed-up (the stored FP64 basis takes ~100 GB: the mixed solver's
        # basis is released first)
        s.close()
        torch.cuda.empty_cache()
        s64 = seedcg.Solver(f.dims, gauge, kappa, precision="fp64", past_factor=wl.past_factor,
                            m_max=5000)
        X64 = torch.zeros_like(B)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        c64, i64 = s64.solve(B, X64, wl.tol, 0, k, stream=stream, allow_not_converged=True)
        eb.record(stream)
        torch.cuda.synchronize()
        t64 = ea.elapsed_time(eb) / 1000.0
        fp64_cmp = {"seconds": t64, "status": c64, "m_conv": i64["m_conv"], "m": i64["m"],
                    "iters": i64["iters"], "max_true_resid": max(i64["true_resid"]),
                    "ms_po": i64["ms_po"], "ms_cg": i64["ms_cg"],
                    "speedup_mixed_over_fp64": t64 / (ms_max / 1000.0)}
        s64.close()
        del X64
        torch.cuda.empty_cache()
        batch_cmp = batch3_once()

    classic_cmp = None
    if args.compare_classic and rank == 0:
        torch.cuda.empty_cache()
        sc = seedcg.Solver(f.dims, gauge, kappa, precision=prec, m_max=args.m_max, seed_mode=2)
        Xc = torch.zeros_like(B)
        sc.solve(B, Xc, wl.tol, 0, k, stream=stream, allow_not_converged=True)   # warm-up
        Xc.zero_()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        cc, ic = sc.solve(B, Xc, wl.tol, 0, k, stream=stream, allow_not_converged=True)
        eb.record(stream)
        torch.cuda.synchronize()
        tc = ea.elapsed_time(eb) / 1000.0
        classic_cmp = {"seconds": tc, "status": cc, "iters": ic["iters"],
                       "matvecs_total": int(sum(ic["matvecs"])),
                       "max_true_resid": max(ic["true_resid"]), "ms_po": ic["ms_po"],
                       "speedup_improved_over_classic": tc / (ms_max / 1000.0)}
        sc.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c1_res = finish_oracle_c1(c1) if c1 is not None else None
        c1 = None
        if all_cores:
            os.sched_setaffinity(0, all_cores)
        costs = oracle_unit_costs(wl, args.cpu_sample_iters)
        cg_total = sum(info["iters"]) - m
        est = oracle_estimate(costs, m, k, cg_total, nrhs)
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": costs["sample"] + f"; scaled to this run's work units (m={m}, "
                         f"{len(range(k, m + 1, k))} PO steps, {cg_total} CG iterations)",
               "per_unit_s": {kk: costs[kk] for kk in ("t_lanczos_iter", "t_po_row", "t_cg_iter")},
               "value_kind": "extrapolated to this workload from the timed sample"}
        if c1_res is not None:
            cpu["measured_c1"] = c1_res

    if args.record_units and rank == 0:
        units_path = os.path.join(ROOT, "paper_0901_3512_gb300", "workload_units.json")
        table = json.load(open(units_path)) if os.path.exists(units_path) else {}
        table[args.workload] = {"m": m, "m_conv": info["m_conv"],
                                "cg_iters_total": sum(info["iters"]) - m,
                                "precision": prec, "recorded_by": "bench.py --record-units"}
        with open(units_path, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)

    if rank == 0:
        out = {"metric": METRIC, "value": replicas.job_seconds_per_solve(ms_max / 1000.0, world), "unit": "s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None,
               "dtype": {"fp64": "f64", "mixed_v32": "f32+c64V+f64", "mixed_vbf16": "f32+bf16V+f64"}[prec],
               "data": "synthetic",
               "config": _config(args, wl, world),
               "valid": ok,
               "solve": {"m_conv": info["m_conv"], "m": m, "po_count": info["po_count"],
                         "cg_iters_max": info["cg_iters_max"], "iters": info["iters"],
                         "max_true_resid": max(info["true_resid"]),
                         "reliable_updates": info["reliable_updates"],
                         "ms_lanczos": info["ms_lanczos"], "ms_po": info["ms_po"],
                         "ms_seed": info["ms_seed"], "ms_cg": info["ms_cg"]},
               "roofline": roofline, "dslash": dslash, "clocks": clocks,
               "gpu_launches": launches // max(args.steps, 1) * args.steps,
               "e2e": e2e, "cpu_baseline": cpu}
        if fp64_cmp:
            out["fp64_plain"] = fp64_cmp
        if cg_only_cmp:
            out["cg_only"] = cg_only_cmp
        if eo_cmp:
            out["even_odd"] = eo_cmp
        if batch_cmp:
            out["batch3_uneven"] = batch_cmp
        if classic_cmp is not None:
            out["classic_seeding"] = classic_cmp
        print(json.dumps(out))
    s.close()
    if c1 is not None and cpu is None:
        finish_oracle_c1(c1, 1.0)
    replicas.finish()


def run_eo(args):
    """Section 3's even-odd system on the workload: time-to-solution of seedcg_solve_eo for all
    right-hand sides (binding residual of A^dag A x_o = b, the original system's residual
    reported), the PO roofline on half-length rows, and one full-lattice solve beside it."""
    import numpy as np
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or wl.precision
    kappa = W.kappa_for(f.name)
    gauge = f.gauge()
    k = wl.reorth_period
    s = seedcg.Solver(f.dims, gauge, kappa, precision=prec, past_factor=wl.past_factor, m_max=args.m_max)
    eta = torch.from_numpy(wl.sources_for(0)).cuda()
    X = torch.zeros_like(eta)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        seedcg.seedcg_solve_eo(s.h, eta, X, wl.tol, 0, k, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    l0 = seedcg.seedcg_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        code, info = seedcg.seedcg_solve_eo(s.h, eta, X, wl.tol, 0, k, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = seedcg.seedcg_kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    peaks, peak_kind = _peaks()
    vol = int(np.prod(f.dims))
    n = 12 * vol // 2
    vbytes = {"fp64": 16, "mixed_v32": 8, "mixed_vbf16": 4}[prec]
    m = info["m"]
    po_rows = sum(i - 1 for i in range(k, m + 1, k)) if k else 0
    po_alg = 2 * po_rows * n * vbytes
    po_gbs = po_alg / (info["ms_po"] / 1000.0) / 1e9 if info["ms_po"] > 0 else None
    # the same sources on the full lattice, for comparison
    B = torch.empty_like(eta)
    s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
    Xf = torch.zeros_like(B)
    s.solve(B, Xf, wl.tol, 0, k, stream=stream)
    Xf.zero_()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    cf, inf_full = s.solve(B, Xf, wl.tol, 0, k, stream=stream)
    eb.record(stream)
    torch.cuda.synchronize()
    full_s = ea.elapsed_time(eb) / 1000.0
    out = {"mode": "even_odd", "metric": METRIC, "value": ms / 1000.0, "unit": "s", "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "dtype": {"fp64": "f64", "mixed_v32": "f32+c64V+f64", "mixed_vbf16": "f32+bf16V+f64"}[prec],
           "data": "synthetic", "config": dict(_config(args, wl, 1), system="A^dag A x_o = A^dag phi (odd sites)"),
           "valid": code == 0 and max(info["true_resid"]) <= wl.tol,
           "solve": {"m_conv": info["m_conv"], "m": m, "po_count": info["po_count"],
                     "cg_iters_max": info["cg_iters_max"], "iters": info["iters"],
                     "max_true_resid": max(info["true_resid"]),
                     "max_true_resid_D": max(info["true_resid_D"]),
                     "ms_lanczos": info["ms_lanczos"], "ms_po": info["ms_po"], "ms_seed": info["ms_seed"],
                     "ms_cg": info["ms_cg"]},
           "roofline": {"bound": "hbm", "achieved": po_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": po_gbs / peaks["hbm_gbs"] if po_gbs else None, "traffic": None,
                        "kernel": "periodic re-orthogonalisation against the half-length basis",
                        "peak_kind": peak_kind, "algorithmic_bytes_per_solve": po_alg,
                        "ms_per_solve": info["ms_po"]},
           "full_lattice": {"seconds": full_s, "status": cf, "m_conv": inf_full["m_conv"], "m": inf_full["m"],
                            "ms_po": inf_full["ms_po"], "ms_cg": inf_full["ms_cg"],
                            "cg_iters_max": inf_full["cg_iters_max"],
                            "po_bytes_per_solve": 2 * sum(i - 1 for i in range(k, inf_full["m"] + 1, k)) * 2 * n * vbytes,
                            "speedup_eo_over_full": full_s / (ms / 1000.0)},
           "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(out))
    s.close()


def run_only(args):
    """Small runs of single kernels for ncu captures (not bench lines)."""
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or wl.precision
    s = seedcg.Solver(f.dims, f.gauge(), W.kappa_for(f.name), precision=prec,
                      past_factor=wl.past_factor, m_max=args.m_max)
    if args.only == "dslash":
        ms = s.time_dslash(prec=1, n=wl.nrhs[0], reps=max(args.steps, 1))
        print(json.dumps({"only": "dslash", "ms": ms}))
    elif args.only == "guess":
        seedcg.seedcg_guess_set_weights(s.h, W.guess_weights(7))
        eta = torch.from_numpy(W.z2_sources(f.dims, 1, f.seed, f.field_index, stream=100)).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        X0 = torch.zeros_like(B)
        seedcg.seedcg_guess_predict(s.h, B, X0)                # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(args.steps, 1)):
            seedcg.seedcg_guess_predict(s.h, B, X0)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"only": "guess", "ms_per_forward": e0.elapsed_time(e1) / max(args.steps, 1)}))
    elif args.only == "cg":
        eta = torch.from_numpy(wl.sources_for(0)).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        X = torch.zeros_like(B)
        s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max, seed_mode=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        code, info = s.solve(B, X, wl.tol, 0, wl.reorth_period, allow_not_converged=True)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"only": "cg", "status": code, "seconds": e0.elapsed_time(e1) / 1000.0,
                          "iters": info["iters"], "max_true_resid": max(info["true_resid"])}))
    else:
        eta = torch.from_numpy(wl.sources_for(0)).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        X = torch.zeros_like(B)
        s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max,
                      stop_after_seed=1, use_tensor_cores=args.tc_po)
        code, info = s.solve(B, X, wl.tol, 0, wl.reorth_period, allow_not_converged=True)
        print(json.dumps({"only": "po", "m": info["m"], "ms_po": info["ms_po"],
                          "po_count": info["po_count"]}))
    s.close()


def run_sweep(args):
    """The paper's parameter studies (Section 3, Figs 1-2, Table 1) on a synthetic field: two
    point sources (spin 1, colours 1 and 2); the second system's CG matvecs after seeding
    against standard CG from zero, as m (past factor) and k (PO period) vary."""
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or "mixed_v32"
    gauge = f.gauge()
    eta_all = W.point_sources(f.dims, 2)

    def run(kappa, pf, k, nrhs=2):
        s = seedcg.Solver(f.dims, gauge, kappa, precision=prec, past_factor=pf, m_max=args.m_max,
                          po_passes=args.po_passes, po_guard=args.po_guard)
        eta = torch.from_numpy(eta_all[2 - nrhs:]).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        X = torch.zeros_like(B)
        s.solve(B, X, wl.tol, 0, k, allow_not_converged=True)      # warm-up (autotuning)
        X.zero_()
        code, info = s.solve(B, X, wl.tol, 0, k, allow_not_converged=True)
        s.close()
        return code, info

    def plain_cg(kappa):
        # the second system alone, no past-convergence: D-Lanczos == CG from zero
        code, info = run(kappa, 1.0, 0, nrhs=1)
        return info["m_conv"] if info["m_conv"] else info["iters"][0]

    if args.sweep == "kappa":
        for kap in [float(x) for x in args.kappas.split(",") if x]:
            cg0 = plain_cg(kap)
            code, info = run(kap, 2.0, 10)
            print(json.dumps({"sweep": "kappa", "kappa": kap, "plain_cg_iters_rhs2": cg0,
                              "m_conv": info["m_conv"], "m": info["m"],
                              "seeded_cg_iters_rhs2": info["iters"][1], "status": code}), flush=True)
        return
    kappa = args.kappa if args.kappa is not None else W.kappa_for(f.name)
    cg0 = plain_cg(kappa)
    base = {"workload": args.workload, "lattice": list(f.dims), "kappa": kappa, "precision": prec,
            "po_passes": args.po_passes, "po_guard": args.po_guard,
            "tol": wl.tol, "plain_cg_iters_rhs2": cg0, "plain_cg_matvecs_rhs2": 2 * cg0}
    settings = ([(pf, 10) for pf in (1.0, 1.2, 1.4, 1.6, 2.0)] if args.sweep == "m"
                else [(1.4, k) for k in (10, 100, 200, 250, 0)])
    for pf, k in settings:
        code, info = run(kappa, pf, k)
        print(json.dumps(dict(base, sweep=args.sweep, past_factor=pf, k=k, m_conv=info["m_conv"],
                              m=info["m"], po_count=info["po_count"],
                              cg_iters_rhs2=info["iters"][1], matvecs_rhs2=info["matvecs"][1],
                              matvecs_rhs1=info["matvecs"][0],
                              ms_rhs1=round(info["ms_lanczos"], 2), ms_po=round(info["ms_po"], 2),
                              true_resid=[float(x) for x in info["true_resid"]], status=code)),
              flush=True)


def run_guess_eval(args):
    """The learned initial guess at the workload's scale: training pairs (b = D^dag eta,
    x = M^-1 b) from the solver on seeded Z2 sources, Adam training by the library's own
    kernels, then held-out Z2 sources solved from x0 = 0 and from the learned x0."""
    import numpy as np
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or wl.precision
    kappa = W.kappa_for(f.name)
    chunk = 12
    ntr = max(chunk, args.train_pairs // chunk * chunk)
    nev = max(chunk, args.eval_pairs // chunk * chunk)
    s = seedcg.Solver(f.dims, f.gauge(), kappa, precision=prec, past_factor=1.0, m_max=args.m_max)
    vol = int(np.prod(f.dims))
    Btr = torch.empty((ntr, vol, 4, 3), dtype=torch.complex128, device="cuda")
    Xtr = torch.zeros_like(Btr)
    t0 = time.time()
    for c in range(ntr // chunk):
        eta = torch.from_numpy(W.z2_sources(f.dims, chunk, f.seed, f.field_index, stream=100 + c)).cuda()
        sl = slice(c * chunk, (c + 1) * chunk)
        s.apply(seedcg.OP_DDAG, eta, Btr[sl], prec=0, multi=1)
        code, _ = s.solve(Btr[sl], Xtr[sl], wl.tol, 0, wl.reorth_period)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    seedcg.seedcg_guess_set_weights(s.h, W.guess_weights(7))
    t0 = time.time()
    loss = seedcg.seedcg_guess_train(s.h, Btr, Xtr, args.epochs, 8, args.lr)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del Btr, Xtr
    res = {"zero": {"iters": [], "ms": 0.0}, "guess": {"iters": [], "ms": 0.0}}
    val_loss = []
    for c in range(nev // chunk):
        eta = torch.from_numpy(W.z2_sources(f.dims, chunk, f.seed, f.field_index, stream=500 + c)).cuda()
        B = torch.empty_like(eta)
        s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
        for mode, use in (("zero", 0), ("guess", 1)):
            s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max, use_guess=use)
            X = torch.zeros_like(B)
            code, info = s.solve(B, X, wl.tol, 0, wl.reorth_period)
            res[mode]["iters"] += info["iters"]
            res[mode]["ms"] += info["ms_total"]
            res[mode]["max_true_resid"] = max(res[mode].get("max_true_resid", 0.0), max(info["true_resid"]))
            if use:
                val_loss.append(seedcg.seedcg_guess_loss_grad(s.h, B, X, want_grad=False)[0])
    out = {"mode": "guess_eval", "workload": args.workload, "lattice": list(f.dims), "kappa": kappa,
           "precision": prec, "train_pairs": ntr, "eval_pairs": nev, "epochs": args.epochs, "lr": args.lr,
           "train_loss": loss, "heldout_loss": float(np.mean(val_loss)),
           "s_data": round(t_data, 1), "s_train": round(t_train, 1),
           "iters_total_zero": int(sum(res["zero"]["iters"])),
           "iters_total_guess": int(sum(res["guess"]["iters"])),
           "ms_solve_zero": round(res["zero"]["ms"], 1), "ms_solve_guess": round(res["guess"]["ms"], 1),
           "max_true_resid": max(res["zero"]["max_true_resid"], res["guess"]["max_true_resid"])}
    print(json.dumps(out))
    s.close()


def run_deflate_eval(args):
    """Later right-hand sides on the same field: the Seed-CG solve of a new batch
    from x0 = 0 against the same solve from the Ritz-deflated guess of the first
    solve's basis."""
    import time
    import torch
    from paper_0901_3512_gb300 import seedcg, workloads as W
    wl = W.WORKLOADS[args.workload]
    f = wl.fields[0]
    prec = args.precision or wl.precision
    s = seedcg.Solver(f.dims, f.gauge(), W.kappa_for(f.name), precision=prec, past_factor=wl.past_factor,
                      m_max=args.m_max)
    eta = torch.from_numpy(wl.sources_for(0)).cuda()
    B = torch.empty_like(eta)
    s.apply(seedcg.OP_DDAG, eta, B, prec=0, multi=1)
    X = torch.zeros_like(B)
    code, info = s.solve(B, X, wl.tol, 0, wl.reorth_period)
    eta2 = torch.from_numpy(W.z2_sources(f.dims, wl.nrhs[0], f.seed, f.field_index, stream=900)).cuda()
    B2 = torch.empty_like(eta2)
    s.apply(seedcg.OP_DDAG, eta2, B2, prec=0, multi=1)
    X0 = torch.zeros_like(B2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta = seedcg.seedcg_deflate_guess(s.h, args.deflate_eval, B2, X0)
    torch.cuda.synchronize()
    t_defl = time.perf_counter() - t0
    runs = {}
    for mode, x0 in (("zero", torch.zeros_like(B2)), ("deflated", X0.clone())):
        s.set_options(precision=prec, past_factor=wl.past_factor, m_max=args.m_max,
                      x0_given=1 if mode == "deflated" else 0)
        c, i = s.solve(B2, x0, wl.tol, 0, wl.reorth_period)
        runs[mode] = {"status": c, "ms_total": round(i["ms_total"], 1), "m": i["m"],
                      "iters_total": int(sum(i["iters"])), "max_true_resid": max(i["true_resid"])}
    print(json.dumps({"mode": "deflate_eval", "workload": args.workload, "precision": prec, "nev": args.deflate_eval,
                      "first_solve_m": info["m"], "ritz_values_lowest": [float(t) for t in theta[:4]],
                      "s_deflation": round(t_defl, 3), "new_batch": runs}))
    s.close()


def main():
    args = _args()
    if args.oracle_c1_worker:
        oracle_c1_worker()
        return
    if args.deflate_eval:
        run_deflate_eval(args)
        return
    if args.guess_eval:
        run_guess_eval(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.only:
        run_only(args)
        return
    if args.eo:
        run_eo(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif len(__import__("paper_0901_3512_gb300.workloads", fromlist=["W"]).WORKLOADS[args.workload].fields) > 1:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

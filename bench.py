#!/usr/bin/env python3
"""Benchmark of the GB300 AA-PDHG hot path; prints ONE JSON line.

A step is one AA-PDHG loop iteration (Alg. 2): x-step and y-step of T with the
fused KKT / residual epilogues, the memory pass with the incremental Gram row,
the safeguard and the m x m solve, and the AA mix with projection.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|medium|tiny]
  python bench.py --impl reference ...   (the FP64 CPU oracle as the reference arm)

value      iterations/s of the whole job (sum over ranks; replicas: one LP per
           rank, no data-path collective), inputs resident in HBM.
e2e        the same metric through the public API from pinned host buffers:
           create (host CSR -> device), power-iteration step size, K
           iterations, read back x and y; per-step bytes = session bytes / K.
roofline   the dominant kernel (CUDA events on the solver's stream) against
           the measured HBM copy bandwidth.
cpu_baseline  the FP64 CPU oracle on a bounded sample of the same LP.
time_to_1e-4  seconds to KKT <= 1e-4 for AA-PDHG and plain PDHG (tiny, the
           preconditioned medium LP, and the large LP under an iteration cap).
batched_to_1e-4, p99_latency  the 256-LP batch solved to KKT <= 1e-4: solves/s,
           per-LP p50 / p99 time from submission to result, and the FP64
           single-LP solver one LP at a time on a sample, for comparison.
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

METRIC = "time-to-1e-4 KKT & iters/s vs plain PDHG on 1 GB300; SpMV HBM GB/s; p99 latency"
UNIT = "iters/s"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "large": dict(method="aa", mem=20, precision="mixed",
                  desc="2M x 5M CSR, ~50M nnz, Chung-Lu power-law row/col degrees (exponent "
                       "2.1), N(0,1)*lognormal(0,3) per row, 20% '>=' rows, bounds [0,U(1,100)] "
                       "with 10% free; AA-PDHG m=20, FP32 SpMV/iterates + FP64-accurate "
                       "Gram/solve/safeguard/KKT"),
    "banded": dict(method="aa", mem=20, precision="mixed",
                   desc="diagnostic: the large sizes (2M x 5M, 50M nnz) with banded structure (row i "
                        "holds 25 consecutive columns), values/senses/bounds as large; the "
                        "half-steps' streaming ceiling when gathers share cache lines; AA-PDHG m=20, "
                        "mixed precision"),
    "medium": dict(method="aa", mem=10, precision="mixed",
                   desc="100k x 300k CSR, ~2M nnz, log-normal row lengths (median 7, max 2000), "
                        "N(0,1)*lognormal(0,2) per row, 70/30 '='/'>=' rows, bounds [0,U(1,100)] "
                        "with 10% free; AA-PDHG m=10, mixed precision"),
    "tiny": dict(method="aa", mem=5, precision="fp64",
                 desc="200 x 500 CSR, 10 nnz/row, N(0,1), '=' rows, 0<=x<=10; AA-PDHG m=5, FP64"),
    "serve": dict(method="aa", mem=10, precision="mixed",
                  desc="served stream: Poisson arrivals, LPs as in the batched workload but with "
                       "rows log-uniform in [500, 200k], tolerance 1e-4 or 1e-6 (FP64 cohorts) per "
                       "request; continuous batching into cohorts admitted by free HBM; AA-PDHG "
                       "m=10 with Ruiz x10 + Pock-Chambolle per LP"),
    "batch": dict(method="aa", mem=10, precision="mixed",
                  desc="256 independent LPs, rows log-uniform in [1k, 50k], cols 2.5x rows, "
                       "lognormal row lengths (mean 8), N(0,1)*lognormal(0,2) per row, 30% '>=' "
                       "rows, bounds [0,U(1,100)] with 10% free; packed block-diagonal, Ruiz x10 + "
                       "Pock-Chambolle per LP, AA-PDHG m=10 mixed precision, solved to 1e-4 "
                       "relative KKT (tested every 64 iterations)"),
}


# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device="cuda"):
    """The ranks' values summed (units that differ between ranks, e.g. LPs solved)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(world, units_per_rank, t_max_ms):
    """Units of all ranks per second of the slowest rank (replicas: weak scaling)."""
    return world * units_per_rank / (t_max_ms / 1e3)


def make_problem(workload, rank, scale=1.0):
    import lpgen
    seed = lpgen.SEED_BASE + {"tiny": 1, "medium": 2, "large": 3, "banded": 5}[workload] + 1000 * rank
    if scale != 1.0 and workload == "large":
        return lpgen.large(seed=seed, m=int(2_000_000 * scale), n=int(5_000_000 * scale),
                           z=int(50_000_000 * scale))
    if scale != 1.0 and workload == "banded":
        return lpgen.banded(seed=seed, m=int(2_000_000 * scale), n=int(5_000_000 * scale))
    if scale != 1.0 and workload == "medium":
        return lpgen.medium(seed=seed, m=int(100_000 * scale), n=int(300_000 * scale))
    return lpgen.WORKLOADS[workload](seed=seed)


def problem_bytes(P):
    return int(8 * (P.m + 1) + 12 * P.nnz + P.m + 8 * (P.m + 3 * P.n))


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_bytes(P, s_v, kind, M, iters, accepted, use_sum, prev_acc):
    """Algorithmic HBM bytes of `iters` launches of a kernel kind (see the design
    notes for the per-unit figures): matrix values + int32 indices, compulsory
    gathers once, every vector read or written once (row metadata not counted)."""
    n, m, Z = P.n, P.m, P.nnz
    N = n + m
    if kind == "xstep":
        return iters * (Z * (s_v + 4) + s_v * m + 7 * s_v * n)
    if kind == "ystep":
        return iters * (Z * (s_v + 4) + 2 * s_v * n + 6 * s_v * m)
    if kind == "memory":
        return (iters * N * s_v * 7 + prev_acc * N * s_v) if M > 0 else 0
    if kind == "gram":          # an AA attempt reads the M memory columns and g^k
        return accepted * N * s_v * (M + 1) if M > 0 else 0
    if kind == "mix":
        return accepted * N * s_v * 8 + use_sum * N * s_v
    return 0


# ---------------------------------------------------------------------------
def time_to_tolerance(args, P_large, rank, stream, barrier):
    """Wall-clock seconds to KKT <= 1e-4 (KKT tested every 64 iterations; the
    time starts at the first iterate call, after the layout and task-shape
    tuners) for AA-PDHG and
    plain PDHG on the same GPU in the same precision:
      tiny   200 x 500, FP64, AA m = 5, no scaling (the plain-method workload);
      medium 100k x 300k, mixed, AA m = 10, Ruiz x10 + Pock-Chambolle and the
             primal weight update every 3000 iterations (Sec. 5.2 set-up);
      large  2M x 5M, mixed, AA m = 20, the same set-up, capped at
             --ttt-large-iters iterations (the unscaled LP stays far from 1e-4).
    Each entry gives the iterations, the AA steps, the final KKT, and seconds
    (null when the cap came first)."""
    from paper_2508_08062_gb300 import Solver
    cases = [("tiny_fp64", make_problem("tiny", rank), "fp64", False, 0, 5, 200000),
             ("medium_preconditioned_U_P3000", make_problem("medium", rank), "mixed", True, 3000,
              10, 200000)]
    if args.workload in ("large", "banded"):
        cases.append((f"{args.workload}_preconditioned_U_P3000", P_large, "mixed", True, 3000, 20,
                      args.ttt_large_iters))
    out = {}
    for name, Q, prec, scale, period, mem, cap in cases:
        res = {"m": Q.m, "n": Q.n, "nnz": Q.nnz, "precision": prec, "memory": mem,
               "preconditioning": "Ruiz x10 + Pock-Chambolle" if scale else "none",
               "primal_weight_period": period, "iteration_cap": cap}
        with Solver(Q, precision=prec, stream=stream) as s:
            if scale:
                s.set_scaling(10, True)
            nrm = s.estimate_norm(100, seed=1)
            s.set_steps(0.9 / nrm, 0.9 / nrm)
            if Q.nnz > 1_000_000:
                s.autotune_layout()
            s.autotune()
            for meth in ("aa", "pdhg"):
                s.set_method(meth, mem=mem if meth == "aa" else 0, D=10.0, eps=1.0)
                if period:
                    s.set_primal_weight(period=period)
                barrier()
                t0 = time.perf_counter()
                conv, its = s.iterate(cap, tol=1e-4, kkt_every=64)
                barrier()
                dt = time.perf_counter() - t0
                cc = s.counters()
                res[meth] = {"converged": conv, "seconds": dt if conv else None, "iterations": its,
                             "seconds_run": dt, "aa_steps": cc["aa_steps"], "kkt": s.get_kkt()["kkt"]}
        out[name] = res
    return out


def batched_to_tolerance(args, rank, stream, barrier):
    """The 256-LP batch (the batched workload's LPs, seeded per rank) solved to
    KKT <= 1e-4 inside the default line: mixed precision, AA m = 10, Ruiz x10 +
    Pock-Chambolle and the primal weight update every 3000 iterations per LP,
    layouts and task shapes tuned first.  Every LP is submitted at the batch
    start, so its time to tolerance is its latency from submission to result
    (64-iteration granularity); p50 / p99 are over the LPs that converged.
    Beside it, the FP64 single-LP solver on a stratified sample of the same
    LPs, one at a time with the same set-up and cap (solves/s of solver time,
    converged LPs only)."""
    import lpgen
    from paper_2508_08062_gb300 import BatchSolver, Solver
    M, kkt_every, tol, period, cap = WORKLOADS["batch"]["mem"], 64, 1e-4, 3000, args.batch_max_iters
    members = lpgen.batch(seed=lpgen.SEED_BASE + 4 + 1000 * rank)
    nprob = len(members)

    def prepare(b):
        b.set_scaling(10, True)
        nrm = b.estimate_norms(100, seed=1)
        b.set_steps(0.9 / nrm, 0.9 / nrm)
        b.set_method("aa", mem=M, D=10.0, eps=1.0)
        b.set_primal_weight(period=period)

    with BatchSolver(members, precision="mixed", stream=stream) as b:
        prepare(b)
        b.autotune_layout()
        b.autotune()
        b.iterate(3 * kkt_every, tol=tol, kkt_every=kkt_every)     # graphs, clocks
        b.reset()
        barrier()
        t0 = time.perf_counter()
        done_at = np.full(nprob, np.nan)
        its = 0
        while its < cap:
            conv, n = b.iterate(kkt_every, tol=tol, kkt_every=kkt_every)
            its += n
            st = b.status()
            done_at[(st[:, 4] == 1) & np.isnan(done_at)] = time.perf_counter() - t0
            if conv or n == 0:
                break
        barrier()
        wall = time.perf_counter() - t0
        st = b.status()
        kk = b.get_kkt()
    solved = int(st[:, 4].sum())
    fin = done_at[~np.isnan(done_at)]

    order = np.argsort([P.m for P in members])
    pick = order[np.linspace(0, nprob - 1, 4).astype(int)]
    times, iters, ok = [], [], 0
    for p in pick:
        with Solver(members[p], precision="fp64", stream=stream) as s:
            s.set_scaling(10, True)
            nrm = s.estimate_norm(100, seed=1)
            s.set_steps(0.9 / nrm, 0.9 / nrm)
            s.set_method("aa", mem=M, D=10.0, eps=1.0)
            s.set_primal_weight(period=period)
            barrier()
            t1 = time.perf_counter()
            c, n = s.iterate(cap, tol=tol, kkt_every=kkt_every)
            barrier()
            times.append(time.perf_counter() - t1)
            iters.append(int(n))
            ok += int(c)
    single = ok / float(np.sum(times))          # converged solves per second of solver time
    rate = solved / wall
    return {"nprob": nprob, "rows": int(sum(P.m for P in members)),
            "cols": int(sum(P.n for P in members)), "nnz": int(sum(P.nnz for P in members)),
            "precision": "mixed", "memory": M, "preconditioning": "Ruiz x10 + Pock-Chambolle",
            "primal_weight_period": period, "iteration_cap": cap, "kkt_every": kkt_every,
            "solved": solved, "wall_s": wall, "solves_per_s": rate, "batch_iterations": int(its),
            "time_to_tol_s": {"p50": float(np.percentile(fin, 50)) if len(fin) else None,
                              "p99": float(np.percentile(fin, 99)) if len(fin) else None},
            "kkt_max": float(np.max(kk[:, 3])),
            "single_lp_fp64_one_at_a_time": {
                "solves_per_s": single, "sample_rows": [int(members[p].m) for p in pick],
                "sample_seconds": [round(t, 4) for t in times], "sample_iterations": iters,
                "sample_converged": ok},
            "speedup_vs_single_fp64": rate / single if single > 0 else None}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_08062_gb300 import Solver

    wl = WORKLOADS[args.workload]
    P = make_problem(args.workload, rank, args.scale)
    s_v = 4 if wl["precision"] == "mixed" else 8
    M = wl["mem"]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    s = Solver(P, precision=wl["precision"], stream=stream)
    if args.precondition:
        s.set_scaling(10, True)
    nrm = s.estimate_norm(100, seed=1)
    tau = sig = 0.9 / nrm
    s.set_steps(tau, sig)
    s.set_method(wl["method"], mem=M, D=10.0, eps=1.0)
    if args.primal_weight:
        s.set_primal_weight(period=args.primal_weight)
    kkt_every = 64
    layout = s.autotune_layout()  # slice width limit and long-row chunk of K', K, with their task shapes
    tuning = s.autotune()        # task shapes of the two half-steps on that layout

    dev_uuid = str(torch.cuda.get_device_properties(local).uuid)
    dev_id = ("GPU-" + dev_uuid) if not dev_uuid.startswith("GPU-") else dev_uuid
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_id) as clk:
        # warm-up (the sampler starts here so that it is running when timing starts)
        s.iterate(args.warmup, tol=0.0, kkt_every=kkt_every)
        time.sleep(0.5)
        s.iterate(args.warmup, tol=0.0, kkt_every=kkt_every)
        c0 = s.counters()
        l0 = s.launch_count()
        barrier()
        ev0.record(stream)
        s.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = s.launch_count() - l0
    c1 = s.counters()
    t_max = max_over_ranks(ms, world)
    value = whole_job_rate(world, args.steps, t_max)

    # per-kernel CUDA-event pass (same loop, instrumented), for the roofline
    if args.profile_region == "timed":   # the region an ncu capture with --profile-from-start off sees
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
    s.profile_kernels(True)
    cp0 = s.counters()
    s.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
    cp1 = s.counters()
    prof = s.kernel_profile()
    s.profile_kernels(False)
    if args.profile_region == "timed":
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
    acc_p = cp1["aa_steps"] - cp0["aa_steps"]
    it_p = cp1["iters"] - cp0["iters"]
    kern = {}
    peak, peak_src = measured_peak()
    for kind, d in prof.items():
        if not d["launches"]:
            continue
        b = kernel_bytes(P, s_v, kind, M, d["launches"], acc_p, acc_p * M, acc_p)
        gbs = b / (d["total_ms"] / 1e3) / 1e9 if d["total_ms"] > 0 else None
        kern[kind] = dict(launches=d["launches"], avg_us=1e3 * d["total_ms"] / d["launches"],
                          share=None, alg_bytes_per_launch=b / d["launches"], gbs=gbs,
                          frac_of_measured_hbm=(gbs / peak) if gbs else None)
    tot = sum(d["total_ms"] for d in prof.values())
    for kind in kern:
        kern[kind]["share"] = prof[kind]["total_ms"] / tot if tot else None
        kern[kind]["traffic"] = committed_traffic(args.workload, kind, args.scale)
    dom = max(kern, key=lambda k: prof[k]["total_ms"])
    traffic = committed_traffic(args.workload, dom, args.scale)
    roofline = {"bound": "hbm", "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["frac_of_measured_hbm"], "traffic": traffic,
                "kernel": dom, "peak_source": peak_src,
                "alg_bytes_per_launch": kern[dom]["alg_bytes_per_launch"]}

    # plain PDHG on the same GPU, same precision
    s.set_method("pdhg", mem=0)
    s.iterate(args.warmup, tol=0.0, kkt_every=kkt_every)
    barrier()
    ev0.record(stream)
    s.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
    ev1.record(stream)
    barrier()
    pd_ms = ev0.elapsed_time(ev1)
    kk = s.get_kkt()

    # the AA branch every iteration (safeguard always passing): times the m x m
    # solve and the mix, which the paper's D = 10 rarely reaches on this LP
    # (a short pass from a fresh start: without the safeguard the run may
    # diverge on a badly scaled LP, which is the method's behaviour, not a fault)
    aa_every = None
    n_ae = min(args.steps, 40)
    ae_warm = 5
    if wl["method"] != "pdhg":
        from paper_2508_08062_gb300 import AAPDHGError
        try:
            # each pass restarts from u^0 (set_method resets the run), so a run
            # never exceeds ae_warm + n_ae forced steps
            s.set_method(wl["method"], mem=M, D=1e30, eps=1.0)
            s.iterate(ae_warm, tol=0.0, kkt_every=kkt_every)
            ca0 = s.counters()
            barrier()
            ev0.record(stream)
            s.iterate(n_ae, tol=0.0, kkt_every=kkt_every)
            ev1.record(stream)
            barrier()
            ae_ms = ev0.elapsed_time(ev1)
            ca1 = s.counters()
            s.set_method(wl["method"], mem=M, D=1e30, eps=1.0)
            s.iterate(ae_warm, tol=0.0, kkt_every=kkt_every)
            if args.profile_region == "forced":    # every iteration attempts the AA step here
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStart()
            s.profile_kernels(True)
            cq0 = s.counters()
            s.iterate(n_ae, tol=0.0, kkt_every=kkt_every)
            cq1 = s.counters()
            if args.profile_region == "forced":
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
        except AAPDHGError as exc:
            aa_every = {"error": str(exc), "note": "safeguard D = 1e30 diverged"}
    if wl["method"] != "pdhg" and aa_every is None:
        prof2 = s.kernel_profile()
        s.profile_kernels(False)
        acc2 = cq1["aa_steps"] - cq0["aa_steps"]
        k2 = {}
        for kind, d in prof2.items():
            if not d["launches"]:
                continue
            b = kernel_bytes(P, s_v, kind, M, d["launches"], acc2, acc2 * M, acc2)
            gbs = b / (d["total_ms"] / 1e3) / 1e9 if d["total_ms"] > 0 else None
            k2[kind] = dict(avg_us=1e3 * d["total_ms"] / d["launches"], gbs=gbs,
                            frac_of_measured_hbm=(gbs / peak) if gbs else None)
        aa_every = {"iters_per_s": n_ae / (ae_ms / 1e3), "ms_per_iter": ae_ms / n_ae, "iters": n_ae,
                    "aa_steps": ca1["aa_steps"] - ca0["aa_steps"],
                    "ls_failures": ca1["ls_failures"] - ca0["ls_failures"], "kernels": k2,
                    "note": "safeguard D = 1e30: the AA step is attempted every iteration; "
                            "two passes of 5 + %d iterations from u^0" % n_ae}

    libspmv = library_spmv(P) if args.library_spmv else None

    # end to end through the public API from pinned host buffers
    import lpgen
    pin = {}
    for name in ("row_ptr", "col_idx", "val", "sense", "q", "c", "l", "u"):
        a = np.ascontiguousarray(getattr(P, name))
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        pin[name] = t.numpy()
    Pp = lpgen.Problem(P.m, P.n, **pin)
    barrier()
    t0 = time.perf_counter()
    with Solver(Pp, precision=wl["precision"], stream=stream) as s2:
        if args.precondition:
            s2.set_scaling(10, True)
        nrm2 = s2.estimate_norm(100, seed=1)
        s2.set_steps(0.9 / nrm2, 0.9 / nrm2)
        s2.set_method(wl["method"], mem=M, D=10.0, eps=1.0)
        s2.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
        x, y = s2.get_iterate()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    polls = (args.steps + 63) // 64 + 2
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": problem_bytes(P) / args.steps,
           "d2h_bytes_per_step": (8 * (P.n + P.m) + 56 * polls) / args.steps,
           "session": "create from pinned host CSR (validation, renumbering, H2D) + 100 "
                      "power iterations + K iterations + x,y read back"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ox, oy = cpu_baseline(P, wl, tau, sig, args.workload, precondition=args.precondition)
        if wl["precision"] == "mixed":
            # the same iterations on the GPU from u^0: how far the mixed-precision
            # iterate is from the FP64 oracle's
            s.set_method(wl["method"], mem=M, D=10.0, eps=1.0)
            s.iterate(cpu["iterations"], tol=0.0, kkt_every=kkt_every)
            gx, gy = s.get_iterate()
            u, r = np.concatenate([gx, gy]), np.concatenate([ox, oy])
            cpu["mixed_error_vs_oracle"] = {
                "iterations": cpu["iterations"],
                "rel_err": float(np.linalg.norm(u - r) / np.linalg.norm(r)),
                "note": "||u_gpu^k - u_oracle^k|| / ||u_oracle^k|| at k = iterations, from u^0"}
    s.close()

    # time to KKT <= 1e-4 (tested every 64 iterations) for AA-PDHG and plain PDHG
    ttt = None if (args.no_ttt or args.scale != 1.0) else time_to_tolerance(args, P, rank, stream, barrier)
    # the 256-LP batch to KKT <= 1e-4: solves/s and per-LP latency
    batched = None
    if not args.no_ttt and args.scale == 1.0 and args.workload == "large":
        batched = batched_to_tolerance(args, rank, stream, barrier)
    p99 = None
    if batched and batched["time_to_tol_s"]["p99"] is not None:
        p99 = {"value": batched["time_to_tol_s"]["p99"], "unit": "s",
               "source": "256-LP batch solved to KKT <= 1e-4, all LPs submitted at its start: "
                         "per-LP time from submission to result, over the LPs that converged"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if wl["precision"] == "mixed" else "f64",
            "data": "synthetic (seeded generator, known optimum; one LP per rank)",
            "config": {"workload": args.workload, "desc": wl["desc"], "m": P.m, "n": P.n,
                       "nnz": P.nnz, "scale": args.scale, "memory": M,
                       "preconditioning": "Ruiz x10 + Pock-Chambolle" if args.precondition else "none", "method": wl["method"],
                       "primal_weight_period": args.primal_weight,
                       "precision": wl["precision"], "kkt_every": kkt_every,
                       "layout": {"x": list(layout["x"]), "y": list(layout["y"]),
                                  "candidates_us": [[c["sell_max"], c["long_chunk"], round(c["x_us"], 1),
                                                     round(c["y_us"], 1)] for c in layout["candidates"]]},
                       "task_shapes": {"x": tuning["shape_x"], "y": tuning["shape_y"],
                                       "x_us": [round(v, 1) for v in tuning["x_us"]],
                                       "y_us": [round(v, 1) for v in tuning["y_us"]]},
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (no flush)" if P.nnz * 16 > 129e6 else
                             "inputs fit in L2 (not flushed: back-to-back iterations)"},
            "roofline": roofline, "kernels": kern,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "aa_steps": c1["aa_steps"] - c0["aa_steps"],
            "plain_pdhg": {"iters_per_s": args.steps / (pd_ms / 1e3), "ms_per_iter": pd_ms / args.steps},
            "aa_every_step": aa_every,
            "kkt_after_run": kk["kkt"],
            "library_spmv": libspmv,
            "time_to_1e-4": ttt,
            "batched_to_1e-4": batched,
            "p99_latency": p99,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def library_spmv(P, reps=20):
    """Context for the half-steps: a plain FP32 CSR SpMV (K v and K' w) by the
    vendor library (torch.sparse CSR with int32 indices, which calls cuSPARSE)
    on the same matrix, in the caller's order and with rows and columns sorted
    by degree (the order the half-steps use).  Reports the average time per
    product over `reps` CUDA-event-timed launches after 3 warm-up launches and
    the plain SpMV's bytes (values, indices, row pointers, x once, y) per
    second.  Not part of the solver: the fused half-steps also apply the prox
    operators and accumulate ||g||."""
    import scipy.sparse as sp
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    K = sp.csr_matrix((P.val.astype(np.float32), P.col_idx, P.row_ptr), shape=(P.m, P.n))
    deg_r = np.diff(P.row_ptr)
    deg_c = np.bincount(P.col_idx, minlength=P.n)
    pr = np.argsort(-deg_r, kind="stable")
    pc = np.argsort(-deg_c, kind="stable")
    Ks = K[pr][:, pc].tocsr()
    Ks.sort_indices()
    out = {"library": "cuSPARSE SpMV via torch.sparse_csr_tensor (FP32 values, int32 indices)",
           "reps": reps}
    for order, A in (("caller", K), ("degree_sorted", Ks)):
        for name, M in (("K_v", A), ("KT_w", A.T.tocsr())):
            M.sort_indices()
            t = torch.sparse_csr_tensor(
                torch.from_numpy(M.indptr.astype(np.int32)), torch.from_numpy(M.indices.astype(np.int32)),
                torch.from_numpy(M.data), size=M.shape, check_invariants=True).to(dev)
            v = torch.randn(M.shape[1], device=dev)
            for _ in range(3):
                r = torch.mv(t, v)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                r = torch.mv(t, v)
            e1.record()
            torch.cuda.synchronize()
            us = 1e3 * e0.elapsed_time(e1) / reps
            b = 8 * M.nnz + 4 * (M.shape[0] + 1) + 4 * M.shape[1] + 4 * M.shape[0]
            out[f"{order}_{name}"] = {"avg_us": us, "gbs": b / us / 1e3}
            del t, v, r
    torch.cuda.empty_cache()
    return out


KERNEL_FILES = {"xstep": ("common.cuh", "spmv.cuh"), "ystep": ("common.cuh", "spmv.cuh"),
                "memory": ("common.cuh", "anderson.cuh"), "mix": ("common.cuh", "anderson.cuh"),
                "gram": ("common.cuh", "anderson.cuh"),
                "batch:xstep": ("common.cuh", "spmv.cuh", "batch.cuh"),
                "batch:ystep": ("common.cuh", "spmv.cuh", "batch.cuh"),
                "batch:memory": ("common.cuh", "anderson.cuh", "batch.cuh")}


def committed_traffic(workload, kind, scale):
    """DRAM bytes per launch of a kernel kind from the committed ncu figures
    (profiles/traffic.json, full-size launch), or None when the workload is
    scaled, no figure exists, or the kernel's sources changed since the
    capture."""
    if scale != 1.0:
        return None
    try:
        tf = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    ent = tf.get(workload, {}).get(kind)
    key = "batch:" + kind if workload == "batch" else kind
    if not ent or key not in KERNEL_FILES or ent.get("kernel_sources") != kernel_source_hash(key):
        return None
    return ent["dram_bytes_per_launch"]


def kernel_source_hash(kind):
    """Hash of the source files a kernel kind is built from (staleness check of
    the committed ncu traffic figures)."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2508_08062_gb300", "csrc")
    for f in KERNEL_FILES[kind]:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


def cpu_baseline(P, wl, tau, sig, workload, budget_s=20.0, precondition=False):
    """The FP64 oracle as it stands, single-threaded, on the same LP: S AA-PDHG
    iterations timed end to end (including its one initial T application)."""
    from oracle import oracle as O
    lp = O.OracleLP.from_problem(P)
    if precondition:
        lp = O.scaled_lp(lp, *O.scaling(lp, 10, True))
    prm = O.Params(method={"aa": 1, "faa": 2, "pdhg": 0}[wl["method"]], mem=wl["mem"], tau=tau,
                   sigma=sig, D=10.0, eps=1.0)
    t0 = time.perf_counter()
    O.solve(lp, prm, 1)
    t1 = time.perf_counter() - t0
    S = int(max(2, min(1000, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    r = O.solve(lp, prm, S)
    ts = time.perf_counter() - t0
    x, y = r.x, r.y
    if precondition:             # x = Dc x~, y = Dr y~
        dr, dc = O.scaling(O.OracleLP.from_problem(P), 10, True)
        x, y = dc * x, dr * y
    return ({"value": S / ts, "unit": UNIT, "cores": 1, "kind": "oracle", "iterations": S,
             "sample": f"{S} FP64 oracle iterations ({wl['method']}, m={wl['mem']}) on the same "
                       f"{workload} LP from its start (includes the initial T), 1 thread"}, x, y)


def run_batch(args):
    """The batched workload: solves/s at 1e-4 relative KKT of the packed batch,
    against FP64 single-LP AA-PDHG solving the same LPs one at a time."""
    import torch
    import torch.distributed as dist
    import lpgen

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_08062_gb300 import BatchSolver, Solver

    wl = WORKLOADS["batch"]
    M, kkt_every, tol = wl["mem"], 64, 1e-4
    members = lpgen.batch(seed=lpgen.SEED_BASE + 4 + 1000 * rank, scale=args.scale)
    nprob = len(members)
    Ztot = sum(P.nnz for P in members)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def prepare(b):
        b.set_scaling(10, True)
        nrm = b.estimate_norms(100, seed=1)
        b.set_steps(0.9 / nrm, 0.9 / nrm)
        b.set_method("aa", mem=M, D=10.0, eps=1.0)
        if args.primal_weight:
            b.set_primal_weight(period=args.primal_weight)

    b = BatchSolver(members, precision="mixed", stream=stream)
    prepare(b)
    layout = b.autotune_layout()   # slice width limit and long-row chunk of the packed K', K
    tuning = b.autotune()
    dev_uuid = str(torch.cuda.get_device_properties(local).uuid)
    dev_id = ("GPU-" + dev_uuid) if not dev_uuid.startswith("GPU-") else dev_uuid
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_id) as clk:
        b.iterate(max(args.warmup, 3) * kkt_every, tol=tol, kkt_every=kkt_every)   # graphs, clocks
        b.reset()
        l0 = b.launch_count()
        barrier()
        t0 = time.perf_counter()
        ev0.record(stream)
        done_at = np.full(nprob, np.nan)
        its = 0
        while its < args.batch_max_iters:
            conv, n = b.iterate(kkt_every, tol=tol, kkt_every=kkt_every)
            its += n
            st = b.status()
            now = time.perf_counter() - t0
            done_at[(st[:, 4] == 1) & np.isnan(done_at)] = now
            if conv or n == 0:
                break
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = b.launch_count() - l0
    st = b.status()
    solved = int(st[:, 4].sum())
    t_max = max_over_ranks(ms, world)
    # each rank solves its own batch: the LPs all ranks solved over the slowest rank's time
    value = sum_over_ranks(solved, world) / (t_max / 1e3)
    kk = b.get_kkt()

    # throughput with every member active (tol = 0) and the roofline
    b.reset()
    b.iterate(kkt_every, tol=0.0, kkt_every=kkt_every)
    if args.profile_region:              # the region an ncu capture with --profile-from-start off sees
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
    b.profile_kernels(True)
    b.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
    prof = b.kernel_profile()
    b.profile_kernels(False)
    if args.profile_region:
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
    barrier()
    ev0.record(stream)
    b.iterate(args.steps, tol=0.0, kkt_every=kkt_every)
    ev1.record(stream)
    barrier()
    thr_ms = ev0.elapsed_time(ev1)
    st2 = b.status()
    peak, peak_src = measured_peak()

    class _Packed:   # the packed LP's sizes for the per-kernel byte formulas
        pass
    PK = _Packed()
    PK.n = sum((P.n + 3) // 4 * 4 for P in members)
    PK.m = sum((P.m + 3) // 4 * 4 for P in members)
    PK.nnz = Ztot
    acc = int(st2[:, 1].sum())
    kern = {}
    for kind, d in prof.items():
        if not d["launches"] or kind == "kkt":
            continue
        bts = kernel_bytes(PK, 4, kind, M, d["launches"], 0, 0, 0) if kind not in ("mix", "gram") else None
        gbs = bts / (d["total_ms"] / 1e3) / 1e9 if bts else None
        kern[kind] = dict(launches=d["launches"], avg_us=1e3 * d["total_ms"] / d["launches"],
                          alg_bytes_per_launch=(bts / d["launches"]) if bts else None, gbs=gbs,
                          frac_of_measured_hbm=(gbs / peak) if gbs else None)
    tot = sum(d["total_ms"] for d in prof.values())
    for kind in kern:
        kern[kind]["share"] = prof[kind]["total_ms"] / tot if tot else None
        kern[kind]["traffic"] = committed_traffic("batch", kind, args.scale)
    dom = max((k for k in kern if kern[k]["gbs"]), key=lambda k: prof[k]["total_ms"])
    roofline = {"bound": "hbm", "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["frac_of_measured_hbm"], "kernel": dom,
                "traffic": committed_traffic("batch", dom, args.scale),
                "peak_source": peak_src, "alg_bytes_per_launch": kern[dom]["alg_bytes_per_launch"]}
    b.close()

    # end to end through the public API: create from host arrays, scaling,
    # step sizes, solve to 1e-4, read every x, y back
    barrier()
    t0 = time.perf_counter()
    with BatchSolver(members, precision="mixed", stream=stream) as b2:
        prepare(b2)
        conv2, its2 = b2.iterate(args.batch_max_iters, tol=tol, kkt_every=kkt_every)
        solved2 = int(b2.status()[:, 4].sum())
        b2.get_iterate()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": sum_over_ranks(solved2, world) / e2e_s, "unit": "solves/s",
           "h2d_bytes_per_step": sum(problem_bytes(P) for P in members) / max(its2, 1),
           "d2h_bytes_per_step": (8 * sum(P.n + P.m for P in members)) / max(its2, 1),
           "session": "create from host CSR of 256 LPs (validation, renumbering, packing, H2D) "
                      "+ scaling + 100 power iterations + solve to 1e-4 + x,y read back"}

    # baseline: FP64 single-LP AA-PDHG, one LP at a time, on a stratified sample
    single = None
    if args.single_sample > 0:
        order = np.argsort([P.m for P in members])
        pick = order[np.linspace(0, nprob - 1, min(args.single_sample, nprob)).astype(int)]
        times, iters, ok = [], [], 0
        for p in pick:
            with Solver(members[p], precision="fp64", stream=stream) as s:
                s.set_scaling(10, True)
                nrm = s.estimate_norm(100, seed=1)
                s.set_steps(0.9 / nrm, 0.9 / nrm)
                s.set_method("aa", mem=M, D=10.0, eps=1.0)
                if args.primal_weight:
                    s.set_primal_weight(period=args.primal_weight)
                barrier()
                t0 = time.perf_counter()
                c, n = s.iterate(args.batch_max_iters, tol=tol, kkt_every=kkt_every)
                barrier()
                times.append(time.perf_counter() - t0)
                iters.append(n)
                ok += int(c)
        est = float(np.sum(times)) * nprob / len(pick)
        # converged solves per second of solver time (the same measure as the batch's value)
        single = {"solves_per_s": (ok / len(pick)) * nprob / est, "sample": [int(p) for p in pick],
                  "sample_rows": [int(members[p].m) for p in pick],
                  "sample_seconds": [round(t, 4) for t in times], "sample_iterations": iters,
                  "sample_converged": ok, "estimated_seconds_all": est,
                  "note": "FP64 single-LP solver (same scaling, step rule, AA m=10, primal weight "
                          "setting, KKT every 64, same iteration cap), solve time per LP, stratified "
                          "by size; time for all = mean x 256; solves/s counts converged LPs only"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(members, st, M, pw_period=args.primal_weight)

    if rank == 0:
        fin = done_at[~np.isnan(done_at)]
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": int(its), "warmup": max(args.warmup, 3) * kkt_every,
            "ms_per_step": t_max / max(its, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded generator, known optimum per LP; one batch per rank)",
            "config": {"workload": "batch", "desc": wl["desc"], "nprob": nprob,
                       "primal_weight_period": args.primal_weight,
                       "rows": int(sum(P.m for P in members)), "cols": int(sum(P.n for P in members)),
                       "nnz": int(Ztot), "scale": args.scale, "memory": M, "kkt_every": kkt_every,
                       "tol": tol, "parallelism": f"replicas{world}",
                       "task_shapes": {"x": tuning["shape_x"], "y": tuning["shape_y"],
                                       "x_us": [round(v, 1) for v in tuning["x_us"]],
                                       "y_us": [round(v, 1) for v in tuning["y_us"]]},
                       "layout": {"x": list(layout["x"]), "y": list(layout["y"]),
                                  "candidates_us": [[c["sell_max"], c["long_chunk"], round(c["x_us"], 1),
                                                     round(c["y_us"], 1)] for c in layout["candidates"]]},
                       "l2": "inputs larger than L2 (no flush)"},
            "solved": solved, "batch_iterations": int(its),
            "member_iterations": {"p50": float(np.median(st[:, 0])), "max": int(st[:, 0].max()),
                                  "sum": int(st[:, 0].sum())},
            "time_to_tol_s": {"p50": float(np.percentile(fin, 50)) if len(fin) else None,
                              "p99": float(np.percentile(fin, 99)) if len(fin) else None,
                              "note": "per LP, from the batch start, at 64-iteration granularity"},
            "kkt_max": float(np.max(kk[:, 3])),
            "throughput_all_active": {"batch_iters_per_s": args.steps / (thr_ms / 1e3),
                                      "member_iters_per_s": nprob * args.steps / (thr_ms / 1e3)},
            "roofline": roofline, "kernels": kern,
            "single_lp_fp64_one_at_a_time": single,
            "speedup_vs_single_fp64": (value / single["solves_per_s"]) if single else None,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serve(args):
    """The served stream: Poisson arrivals at --rate LPs/s for --duration s of
    arrivals (drawn from a pool of distinct instances), served with continuous
    batching; the queue then drains for at most --drain s.  Against a FIFO
    replay of the same stream through the FP64 single-LP solver, with service
    times measured per (instance, tolerance) on a sample."""
    import torch
    import lpgen
    from paper_2508_08062_gb300 import Server, Solver

    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WORKLOADS["serve"]
    M = wl["mem"]
    rng = np.random.default_rng(lpgen.SEED_BASE + 5 + 1000 * rank)
    sizes = np.rint(np.exp(rng.uniform(np.log(500), np.log(200_000), args.pool))).astype(int)
    sizes = np.maximum(4, np.rint(sizes * args.scale).astype(int))
    pool = [lpgen.batch_member(lpgen.SEED_BASE * 1000 + 5000 + i, int(m)) for i, m in enumerate(sizes)]
    n_req = int(rng.poisson(args.rate * args.duration))
    arrivals = np.sort(rng.uniform(0.0, args.duration, n_req))
    which = rng.integers(0, len(pool), n_req)
    tols = np.where(rng.random(n_req) < 0.5, 1e-4, 1e-6)
    stream_desc = {"requests": n_req, "rate_per_s": args.rate, "arrival_window_s": args.duration,
                   "pool": len(pool), "pool_rows": [int(m) for m in sizes], "drain_limit_s": args.drain}

    dev_uuid = str(torch.cuda.get_device_properties(local).uuid)
    dev_id = ("GPU-" + dev_uuid) if not dev_uuid.startswith("GPU-") else dev_uuid
    ids = []
    with Server(method="aa", mem=M, max_cohorts=args.max_cohorts,
                max_cohort_size=args.cohort_size, max_iters=args.serve_max_iters) as srv:
        if args.primal_weight:
            srv.set_primal_weight(period=args.primal_weight)
        with ClockSampler(dev_id) as clk:
            t0 = time.perf_counter()
            k = 0
            while True:
                now = time.perf_counter() - t0
                while k < n_req and arrivals[k] <= now:
                    ids.append(srv.submit(pool[which[k]], float(tols[k])))
                    k += 1
                running, waiting = srv.step()
                if k == n_req and running == 0 and waiting == 0:
                    break
                if now > args.duration + args.drain:
                    break
                if running == 0 and waiting == 0 and k < n_req:
                    time.sleep(max(0.0, min(arrivals[k] - now, 0.01)))
            wall = time.perf_counter() - t0
        res = [srv.result(i) for i in ids]
    states = [r["state"] for r in res]
    done = [r for r in res if r["state"] == "converged"]
    lat = np.array([r["t_done"] - r["t_submit"] for r in done])
    per_tol = {}
    for tv in (1e-4, 1e-6):
        sel = [r for r, t in zip(res, tols[:len(res)]) if t == tv and r["state"] == "converged"]
        per_tol[str(tv)] = len(sel)
    # each rank serves its own stream: all ranks' solves over the slowest rank's wall time
    value = sum_over_ranks(len(done), world) / max_over_ranks(wall, world)

    # FIFO replay through the FP64 single-LP solver: service time per
    # (instance, tolerance) measured on a sample of the pool
    base = None
    if args.single_sample > 0:
        order = np.argsort(sizes)
        pick = order[np.linspace(0, len(pool) - 1, min(args.single_sample, len(pool))).astype(int)]
        svc = {}
        stream = torch.cuda.current_stream()
        for p in pick:
            for tv in (1e-4, 1e-6):
                with Solver(pool[p], precision="fp64", stream=stream) as s1:
                    s1.set_scaling(10, True)
                    nrm = s1.estimate_norm(100, seed=1)
                    s1.set_steps(0.9 / nrm, 0.9 / nrm)
                    s1.set_method("aa", mem=M, D=10.0, eps=1.0)
                    if args.primal_weight:
                        s1.set_primal_weight(period=args.primal_weight)
                    torch.cuda.synchronize()
                    ts = time.perf_counter()
                    c, n_it = s1.iterate(args.serve_max_iters, tol=tv, kkt_every=64)
                    torch.cuda.synchronize()
                    svc[(int(p), tv)] = (time.perf_counter() - ts, bool(c))
        # instances outside the sample take the service time of the nearest sampled size
        def service(i, tv):
            q = int(pick[np.argmin(np.abs(np.log(sizes[pick]) - np.log(sizes[i])))])
            return svc[(q, tv)]
        t_free, lat_b, ok_b = 0.0, [], 0
        for a, i, tv in zip(arrivals, which, tols):
            d, c = service(int(i), float(tv))
            start = max(t_free, a)
            t_free = start + d
            if c:
                lat_b.append(t_free - a)
                ok_b += 1
        lat_b = np.array(lat_b)
        base = {"solves_per_s": ok_b / t_free if t_free > 0 else None, "makespan_s": t_free,
                "converged": ok_b,
                "p50_s": float(np.percentile(lat_b, 50)) if len(lat_b) else None,
                "p99_s": float(np.percentile(lat_b, 99)) if len(lat_b) else None,
                "sample": [int(p) for p in pick],
                "note": "FIFO replay of the same arrivals through the FP64 single-LP solver "
                        "(same scaling, step rule, AA m=10, iteration cap); service times "
                        "measured per (sampled instance, tolerance), nearest sampled size for "
                        "the others"}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": len(ids), "warmup": 0, "ms_per_step": 1e3 * wall / max(len(done), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded generator, known optimum per LP)",
        "config": {"workload": "serve", "desc": wl["desc"], **stream_desc,
                   "max_cohorts": args.max_cohorts, "cohort_size": args.cohort_size,
                   "max_iters_per_lp": args.serve_max_iters, "scale": args.scale,
                   "primal_weight_period": args.primal_weight},
        "completed": {s_: states.count(s_) for s_ in set(states)},
        "converged_by_tol": per_tol, "wall_s": wall,
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency": float(np.percentile(lat, 99)) if len(lat) else None,
        "sequential_fp64_single_lp": base,
        "clocks": clk.summary(),
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None,
                "session": "every request from host arrays through the public server API, "
                           "results read back: the value is already end to end"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline_batch(members, st, M, budget_s=20.0, pw_period=0):
    """The FP64 oracle as it stands on one median-size member of the batch
    (scaled as the GPU run scales it), timed for a bounded number of AA-PDHG
    iterations; solves/s of the batch are then estimated from the oracle's
    time per iteration and nonzero (x each member's nonzeros) and the
    iteration counts the GPU run needed per member."""
    from oracle import oracle as O
    from scipy.sparse.linalg import svds
    import scipy.sparse as sp
    order = np.argsort([P.m for P in members])
    p = int(order[len(order) // 2])
    P = members[p]
    lp = O.OracleLP.from_problem(P)
    S = O.scaled_lp(lp, *O.scaling(lp, 10, True))
    K = sp.csr_matrix((S.v, S.ci.astype(np.int64), S.rp), shape=(P.m, P.n))
    tau = 0.9 / svds(K, k=1, return_singular_vectors=False, random_state=0, maxiter=200, tol=1e-3)[0]
    prm = O.Params(method=1, mem=M, tau=tau, sigma=tau, D=10.0, eps=1.0, pw_period=pw_period)
    t0 = time.perf_counter()
    O.solve(S, prm, 10)
    t1 = (time.perf_counter() - t0) / 10
    n_it = int(max(10, min(100000, budget_s / max(t1, 1e-7))))
    t0 = time.perf_counter()
    O.solve(S, prm, n_it)
    per_it = (time.perf_counter() - t0) / n_it
    per_nnz_it = per_it / max(P.nnz, 1)
    est = sum(per_nnz_it * Q.nnz * max(int(st[q, 0]), 1) for q, Q in enumerate(members))
    return {"value": len(members) / est, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_it} FP64 oracle AA-PDHG iterations (m={M}) on batch member {p} "
                      f"({P.m}x{P.n}, {P.nnz} nnz, scaled); batch time estimated as oracle "
                      f"seconds per iteration per nonzero x each member's nonzeros x the "
                      f"iterations it needed on the GPU"}


def run_reference_batch(args):
    """Reference arm of the batched workload: the FP64 oracle solving members
    (stratified by size, smallest first) to 1e-4 until its time budget is
    spent; solves/s normalised to the batch's mean nonzeros per LP."""
    import lpgen
    from oracle import oracle as O
    from scipy.sparse.linalg import svds
    import scipy.sparse as sp
    members = lpgen.batch(scale=args.scale)
    order = np.argsort([P.m for P in members])
    pick = sorted(order[np.linspace(0, len(members) - 1, 16).astype(int)], key=lambda q: members[q].m)
    budget = float(os.environ.get("REF_BUDGET_S", "120"))
    t0 = time.perf_counter()
    done, nnz_done = 0, 0
    for q in pick:
        P = members[q]
        lp = O.OracleLP.from_problem(P)
        S = O.scaled_lp(lp, *O.scaling(lp, 10, True))
        K = sp.csr_matrix((S.v, S.ci.astype(np.int64), S.rp), shape=(P.m, P.n))
        tau = 0.9 / svds(K, k=1, return_singular_vectors=False, random_state=0, maxiter=200,
                         tol=1e-3)[0]
        r = O.solve(S, O.Params(method=1, mem=10, tau=tau, sigma=tau), 100000, tol=1e-4,
                    kkt_every=64)
        if r.status != 0:
            continue
        done += 1
        nnz_done += P.nnz
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    mean_all = np.mean([P.nnz for P in members])
    v = (done / dt) * ((nnz_done / max(done, 1)) / mean_all) if done else 0.0
    sample = (f"{done} batch members (stratified by size, smallest first) solved to 1e-4 by the "
              f"FP64 oracle in {dt:.1f} s, 1 thread; rate scaled by their mean nnz / the batch's")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 1,
            "steps": done, "warmup": 0, "ms_per_step": 1e3 * dt / max(done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "batch", "desc": WORKLOADS["batch"]["desc"]},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    if args.workload in ("batch", "serve"):
        return run_reference_batch(args)
    wl = WORKLOADS[args.workload]
    P = make_problem(args.workload, 0, args.scale)
    from scipy.sparse.linalg import svds
    import scipy.sparse as sp
    K = sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))
    nrm = svds(K, k=1, return_singular_vectors=False, random_state=0, maxiter=200, tol=1e-3)[0] \
        if min(P.m, P.n) > 2 else np.linalg.norm(K.toarray(), 2)
    tau = sig = 0.9 / nrm
    budget = float(os.environ.get("REF_BUDGET_S", "120"))
    cb, _, _ = cpu_baseline(P, wl, tau, sig, args.workload, budget_s=budget)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": world, "steps": int(cb["sample"].split()[0]), "warmup": 0,
            "requested_steps": args.steps, "requested_warmup": args.warmup,
            "ms_per_step": 1e3 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "m": P.m, "n": P.n,
                       "nnz": P.nnz, "memory": wl["mem"], "method": wl["method"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttt", action="store_true",
                    help="skip the time-to-1e-4 legs (AA-PDHG and plain PDHG to KKT <= 1e-4, and "
                         "the 256-LP batch to KKT <= 1e-4)")
    ap.add_argument("--ttt-large-iters", type=int, default=4096,
                    help="iteration cap of the time-to-1e-4 leg on the large LP")
    ap.add_argument("--precondition", action="store_true",
                    help="Ruiz (10 passes) + Pock-Chambolle diagonal scaling before the step size")
    ap.add_argument("--profile-region", nargs="?", const="timed", default=None,
                    choices=["timed", "forced"],
                    help="bracket with cudaProfilerStart/Stop the per-kernel CUDA-event pass of "
                         "the AA loop (timed, the default) or of the pass with the AA step "
                         "attempted every iteration (forced)")
    ap.add_argument("--primal-weight", type=int, default=0,
                    help="primal weight update every this many iterations (0: off; paper: 3000)")
    ap.add_argument("--batch-max-iters", type=int, default=100000,
                    help="batch workload: iteration cap of the solve to 1e-4")
    ap.add_argument("--single-sample", type=int, default=16,
                    help="batch workload: LPs solved one at a time by the FP64 single-LP solver")
    ap.add_argument("--rate", type=float, default=200.0, help="serve workload: arrivals per s")
    ap.add_argument("--duration", type=float, default=1.0,
                    help="serve workload: seconds of arrivals (the queue then drains)")
    ap.add_argument("--drain", type=float, default=120.0,
                    help="serve workload: at most this many seconds after the last arrival")
    ap.add_argument("--pool", type=int, default=16, help="serve workload: distinct LP instances")
    ap.add_argument("--max-cohorts", type=int, default=4)
    ap.add_argument("--cohort-size", type=int, default=64)
    ap.add_argument("--serve-max-iters", type=int, default=100000)
    ap.add_argument("--library-spmv", action="store_true",
                    help="single-LP workloads: also time the vendor library's plain SpMV on K, K'")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload's m, n, nnz (profiling captures only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

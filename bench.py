#!/usr/bin/env python
"""Benchmark: power-series Newton steps/s on one GB300 (and N replicas).

Workload: quad double, complex, n = 64 polynomials in 64 unknowns plus t, 64
monomials per polynomial of total degree <= 4 over <= 4 variables, unit-modulus
coefficients, truncation degree d = 64 (seeded synthetic system; the start point
x0 solves the system at t = 0).  A step is one Newton step on the truncated
power series: evaluate and differentiate, Householder QR of A_0, block
Toeplitz forward substitution, update.  Steps continue the Newton iteration
from x0 (the work per step does not depend on x).

Timing: W untimed warm-up steps, then exactly K steps, each bracketed by CUDA
events on the launching stream, L2 flushed (256 MB write) between steps outside
the events; barrier + synchronize around the timed region; max over ranks.
For N > 1 every rank runs its own replica (the single system does not shard);
--form batched instead splits its batch over the ranks by LPT cost.

--impl reference times the CPU oracle (oracle/, plain C, OpenMP over the
paper's jobs) on the host cores for the same workload and metric.
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
sys.path.insert(0, ROOT)

METRIC = "power-series Newton steps/s (qd, n=64, d=64); FP64-pipe % of peak; err vs oracle"
WORKLOAD = ("quad double complex, n=64 polynomials (+t), 64 monomials each of degree <= 4 over <= 4 variables, "
            "truncation degree d=64, seed 1")
CFG = 1
# the other seeded workloads (--config): the small double double case and the
# octo double real n = 128 case (the shape of the paper's 128-dimensional runs)
OTHER_WORKLOADS = {
    0: ("power-series Newton steps/s (dd, n=3, d=8); FP64-pipe % of peak; err vs oracle",
        "double double complex, n=3 polynomials (+t), 4 monomials each of degree <= 2 over 1-2 variables, "
        "truncation degree d=8, seed {seed}"),
    2: ("power-series Newton steps/s (od, n=128, d=32); FP64-pipe % of peak; err vs oracle",
        "octo double real, n=128 polynomials (+t), 32 monomials each of degree <= 3 over <= 3 variables, "
        "truncation degree d=32, seed {seed}"),
}


def metric_and_workload(cfg: int, seed: int):
    if cfg == CFG:
        return METRIC, WORKLOAD.replace("seed 1", f"seed {seed}")
    m, w = OTHER_WORKLOADS[cfg]
    return m, w.format(seed=seed)

# Table 1 of the paper: double operations per md add / mul (sum of the +,-,*,/ columns)
TABLE1 = {2: (20, 23), 3: (35, 209), 4: (89, 336), 5: (122, 554), 8: (269, 1742), 10: (397, 3089)}

# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 lanes per SM per
# cycle x 2.07 GHz (the nominal 1.25 TFLOP/s counting an FMA as two flops).
FP64_PEAK_INSTR = 152 * 2 * 2.07e9
# DRAM bytes (read + write) per launch of the series-product kernel at this
# workload: ncu dram__bytes_read.sum + dram__bytes_write.sum of the three
# launches of one step, averaged (8.74 + 32.11 + 9.06 MB), captured on the
# kernel as it stands; it must be retaken (or set to None) whenever that
# kernel changes.
CONV_TRAFFIC_BYTES_PER_LAUNCH = 16.64e6


# ----------------------------------------------------------------- op model
def fp64_instr_counts(K: int) -> dict:
    """FP64 instructions of the library's md algorithms (TwoSum = 3, TwoProd = 2,
    FastTwoSum = 3, plain op = 1), common path of the renormalisation."""
    ts, tp, fts = 3, 2, 3

    def renorm(m):
        # bottom-up m-1 TwoSums; top-down: K-1 TwoSums, then plain adds for the rest
        return (m - 1) * ts + (K - 1) * ts + (m - 1 - (K - 1))

    if K == 1:
        add = mul = 1
        muld = 1
    elif K == 2:
        add = 2 * ts + 2 * fts + 2
        mul = tp + 2 + 2 + fts
        muld = tp + 2 + fts
    else:
        add = ts * (K * (K + 1) // 2) + (K - 1) + renorm(K + 1)
        n_ts = sum(n * (n + 1) for n in range(K))
        level_k = (K - 1) + ((K - 2) + K + K * (K - 1))  # K-1 products, adds of products, lows, carries
        mul = tp * (K * (K + 1) // 2) + ts * n_ts + level_k + renorm(K + 1)
        muld = tp * K + ts * (K * (K - 1) // 2) + (K - 1) + renorm(K + 1)
    return {"add": add, "mul": mul, "mul_d": muld}


def complex_mac_instr(K: int, P: int) -> tuple:
    c = fp64_instr_counts(K)
    if P == 1:
        return c["mul"], c["add"]
    return 4 * c["mul"] + 2 * c["add"], 2 * c["add"]


def conv_schedule_counts(s) -> int:
    """Number of series products in the evaluation schedule of system s."""
    n = s.n
    total = 0
    for i in range(n):
        for _, pairs in s.monomials(i):
            xs = [(v, e) for v, e in pairs if v != n]
            m = len(xs)
            fch = sum(e - 1 for _, e in xs)
            F = max(fch - 1, 0)  # first factor is a copy
            Funit = fch == 0
            sp = (m - 1) + max(m - 2, 0) + max(m - 2, 0) if m >= 2 else 0
            g = 0 if (Funit or m == 0) else 1
            dq = 0
            if not Funit:
                dq = m if m >= 2 else (0 if m == 0 else 0)
            total += F + sp + g + dq
    return total


def step_fp64_model(s) -> dict:
    """FP64 instructions of one Newton step of system s: the series products
    exactly (the md algorithms' counts), the rest from the operation counts of
    the accumulation, the QR with Q^H, the back substitution, the block
    Toeplitz update and W r_k (complex multiply-adds; reductions as adds)."""
    P, K, n, d = s.planes, s.limbs, s.n, s.degree
    cm, ca = complex_mac_instr(K, P)
    mac = cm + ca
    D1 = d + 1
    conv = conv_schedule_counts(s) * (D1 * (D1 + 1) // 2 * cm + d * D1 // 2 * ca)
    contrib = sum(1 + len([v for v, _ in pairs if v != n]) for i in range(s.N) for _, pairs in s.monomials(i))
    accum = contrib * D1 * mac
    qr = sum(((n - j - 1) + n) * (n - j) * 2 * mac for j in range(n))
    backsub = sum((c + 1) * n for c in range(n)) * (2 * cm + ca)
    update = n * n * d * D1 // 2 * mac + D1 * n * n * mac
    return {"conv": conv, "accum": accum, "qr": qr, "backsub": backsub, "update": update,
            "total": conv + accum + qr + backsub + update}


# ------------------------------------------------------------------ clocks# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group("gloo")
    return dist


def reduce_max(dist, v: float) -> float:
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle leg
def oracle_steps_per_s(s, steps: int, warmup: int, want_x: bool = False, threads: int = 0):
    """The oracle's Newton steps on the host: all cores (OpenMP, threads = 0)
    or the given number of threads (restored to all cores afterwards)."""
    import oracle

    orc = oracle.Oracle(threads=threads or os.cpu_count() or 1)
    try:
        x = s.x0.copy()
        for _ in range(warmup):
            x, _ = orc.newton_step(s, x)
        t0 = time.perf_counter()
        for _ in range(steps):
            x, _ = orc.newton_step(s, x)
        dt = time.perf_counter() - t0
        used = orc.threads()
    finally:
        if threads:
            orc.lib.orc_set_threads(os.cpu_count() or 1)
    if want_x:
        return steps / dt, used, dt, x
    return steps / dt, used, dt


def err_vs_oracle(got, want) -> float:
    """max over degrees k of max_i |got_ik - want_ik| / max_i |want_ik|, each
    md number summed exactly over its limbs ([P][K][n][d+1] arrays)."""
    from math import fsum

    P, _, n, D1 = want.shape
    worst = 0.0
    for k in range(D1):
        diff = scale = 0.0
        for i in range(n):
            dd = [fsum(list(got[p, :, i, k]) + [-v for v in want[p, :, i, k]]) for p in range(P)]
            ww = [fsum(want[p, :, i, k]) for p in range(P)]
            diff = max(diff, sum(v * v for v in dd) ** 0.5)
            scale = max(scale, sum(v * v for v in ww) ** 0.5)
        if scale > 0:
            worst = max(worst, diff / scale)
    return worst


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import mdgen

    s = mdgen.config_system(args.config, args.seed)
    metric, workload = metric_and_workload(args.config, args.seed)
    v, cores, dt = oracle_steps_per_s(s, args.steps, args.warmup)
    line = {"impl": "reference", "metric": metric, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "arm": "CPU oracle (plain C, OpenMP over polynomials and RHS updates)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full Newton steps of the workload after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- main leg
def tune_factor_sms(md, sysd, x, ws, nrm, flags, dev):
    """MD_FLAG_AUTOTUNE of the single step: the calls that time the candidate
    SM counts of the factorisation (untimed here, before the warm-up); from
    the call after them the plan runs the fastest count."""
    import torch

    if flags & md.FLAG_AUTOTUNE:
        for _ in range(16):
            md.newton_step(sysd, x, ws, nrm, flags=flags)
            torch.cuda.synchronize(dev)
        if md.plan_factor_sms(sysd, flags) <= 0:
            raise RuntimeError("the factorisation's SM count was not tuned")


def run_product(args):
    import numpy as np
    import torch

    import mdgen
    import paper_2012_06607_gb300 as md

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world)
    dev = torch.device("cuda", local)
    s = mdgen.config_system(args.config, args.seed)
    metric, workload = metric_and_workload(args.config, args.seed)
    P, K, n, d = s.planes, s.limbs, s.n, s.degree
    sysd = md.DeviceSystem(s, device=dev)
    flags = (md.FLAG_OZAKI if args.update == "split" else 0) | (md.FLAG_LU if args.factor == "lu" else 0)
    if not args.no_autotune:
        flags |= md.FLAG_AUTOTUNE
    wsb = sysd.workspace_bytes(flags)
    ws = md.workspace(wsb, device=dev)
    x = md.to_device(s.x0, dev)
    nrm = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    tune_factor_sms(md, sysd, x, ws, nrm, flags, dev)
    for _ in range(args.warmup):
        md.newton_step(sysd, x, ws, nrm, flags=flags)
    torch.cuda.synchronize(dev)
    assert md.device_status(ws) == 0

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    md.profile_read()  # drop anything recorded before
    md.profile_enable(True)
    evs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        md.newton_step(sysd, x, ws, nrm, flags=flags)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    md.profile_enable(False)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    status = md.device_status(ws)
    prof = md.profile_read()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = reduce_max(dist, sum(step_ms))
    value = world * args.steps / (total_ms / 1e3)
    launches = sum(c for _, c in prof.values())

    # roofline of the dominant kernel (largest total time)
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_launches) = dom
    cmul_i, cadd_i = complex_mac_instr(K, P)
    nconv = conv_schedule_counts(s)
    conv_instr = nconv * ((d + 1) * (d + 2) // 2 * cmul_i + d * (d + 1) // 2 * cadd_i)
    t1 = TABLE1[K]
    paper_mul = (4 * t1[1] + 2 * t1[0]) if P == 2 else t1[1]
    paper_add = 2 * t1[0] if P == 2 else t1[0]
    conv_paper = nconv * ((d + 1) * (d + 2) // 2 * paper_mul + d * (d + 1) // 2 * paper_add)
    conv_ms, conv_launches = prof.get("conv_stage", (float("nan"), 0))
    # the timed region ran args.steps steps: conv_ms and conv_launches cover all of them
    achieved = args.steps * conv_instr / (conv_ms / 1e3) if conv_ms > 0 else None
    if args.update == "split" and K >= 3:
        # the split form's products run on the integer pipe: the FP64 count of
        # the md algorithms does not measure them (ncu figures of that kernel:
        # profiles/conv_stage_fx_qd_n64_d64.md)
        achieved = None
    roofline = {"bound": "alu", "kernel": "conv_stage", "achieved": achieved / 1e12 if achieved else None,
                "peak": FP64_PEAK_INSTR / 1e12, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_INSTR if achieved else None,
                "traffic": CONV_TRAFFIC_BYTES_PER_LAUNCH if args.update == "md" and args.config == CFG else None,
                "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                "counted": "FP64 instructions of the md algorithms (an fma counts once)" if achieved else
                           "not counted: the split form's series products run on 32-bit word slices (integer pipe)",
                "launches_in_timed_region": conv_launches, "avg_launch_ms": conv_ms / max(conv_launches, 1),
                "dominant_by_time": dom_name,
                "paper_ops_per_s": args.steps * conv_paper / (conv_ms / 1e3) if conv_ms > 0 else None,
                "algorithmic_fp64_per_step": conv_instr}
    line = {"metric": metric, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "l2": "flushed between steps (256 MB write outside the events)",
                       "parallelism": f"replicas x{world}", "workspace_bytes": wsb,
                       "update": ("split products: series products on 32-bit word slices (integer pipe), "
                                  "update on 8-bit slices (BF16 tensor pipe)") if args.update == "split"
                       else "md arithmetic",
                       "factor": "LU with partial pivoting" if args.factor == "lu" else "Householder QR",
                       "factor_sms": "autotuned over 16 untimed calls before the warm-up (MD_FLAG_AUTOTUNE)"
                       if not args.no_autotune else "4 (default)"},
            "roofline": roofline, "gpu_launches": launches, "clocks": clk, "device_status": status,
            "kernel_ms": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "wall_s_timed_region": wall, "dx_norm_last": float(nrm[0].item()),
            # relative to the size of the last coefficient of x (the solution series
            # has a small radius of convergence, so its degree-d coefficients are large)
            "dx_rel_last": float(nrm[0].item()) / max(float(torch.sqrt(x[0, 0, :, d] ** 2 + x[P - 1, 0, :, d] ** 2
                                                                          if P == 2 else x[0, 0, :, d] ** 2).max().item()),
                                                      1e-300)}

    # end to end through the C ABI with host buffers: H2D of x, step, D2H of x and norms
    xh = torch.from_numpy(s.x0.copy()).pin_memory()
    outh = torch.empty_like(xh).pin_memory()
    nh = torch.empty(2, dtype=torch.float64).pin_memory()
    e_ms = []
    for it in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        x.copy_(xh, non_blocking=True)
        md.newton_step(sysd, x, ws, nrm, flags=flags)
        outh.copy_(x, non_blocking=True)
        nh.copy_(nrm, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
        xh.copy_(outh)
    e_total = reduce_max(dist, sum(e_ms))
    line["e2e"] = {"value": world * args.steps / (e_total / 1e3), "unit": "steps/s",
                   "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(outh.numel() * 8 + 16)}

    # the other update form on the same GPU, same workload and timing (context,
    # not the headline): the split-product update against md arithmetic
    if args.update == "md" and not args.no_other_form:
        oflags = md.FLAG_OZAKI | (flags & (md.FLAG_LU | md.FLAG_AUTOTUNE))
        ows = md.workspace(sysd.workspace_bytes(oflags), device=dev)
        xo = md.to_device(s.x0, dev)
        tune_factor_sms(md, sysd, xo, ows, nrm, oflags, dev)
        for _ in range(args.warmup):
            md.newton_step(sysd, xo, ows, nrm, flags=oflags)
        torch.cuda.synchronize(dev)
        o_ms = []
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            md.newton_step(sysd, xo, ows, nrm, flags=oflags)
            b.record(stream)
            o_ms.append((a, b))
        torch.cuda.synchronize(dev)
        assert md.device_status(ows) == 0
        o_total = reduce_max(dist, sum(a.elapsed_time(b) for a, b in o_ms))
        line["other_forms"] = {"split_product_form": {
            "form": "MD_FLAG_OZAKI: series products on 32-bit word slices (integer pipe), block Toeplitz "
                    "update on 8-bit slices (BF16 tensor pipe), exact accumulation; the plain QR and W",
            "value": world * args.steps / (o_total / 1e3), "unit": "steps/s", "ms_per_step": o_total / args.steps,
            "speedup_vs_md": total_ms / o_total}}
        del ows, xo
        if world == 1:
            # the other two forms of the method on the same GPU: the n = 256
            # quad double solve (plain vs split-product update) and the batched
            # form with its per-system launch loop
            line["other_forms"]["solve_qd_n256_d16_cond1e8"] = measure_solve3(args, with_err=not args.no_cpu_baseline)
            bl = measure_batched(args, args.other_batch, 0, 1, local, None, with_loop=True,
                                 err_sample=0 if args.no_cpu_baseline else 8)
            line["other_forms"]["batched"] = {k: bl[k] for k in (
                "metric", "value", "unit", "ms_per_iteration", "system_steps_per_s", "latency_ms_p50",
                "latency_ms_p99", "latency_ms_max", "loop_ms_per_iteration", "speedup_vs_loop",
                "shared_sm_only_ms_per_iteration", "split_product_form", "roofline", "err_vs_oracle", "systems",
                "limb_counts",
                "phases_of_slowest_system")}
            torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, dt, x_orc = oracle_steps_per_s(s, 1, 0, want_x=True)
        vs, cs, _ = oracle_steps_per_s(s, 1, 0, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                "sample": "1 full Newton step of the workload from x0 (host cores, OpenMP)",
                                "serial": {"value": vs, "unit": "steps/s", "cores": cs,
                                           "sample": "the same step on one thread"}}
        # the same step on the GPU (outside the timed region), against the oracle's
        x1 = md.to_device(s.x0, dev)
        md.newton_step(sysd, x1, ws, nrm, flags=flags)
        torch.cuda.synchronize()
        e = err_vs_oracle(x1.cpu().numpy(), x_orc)
        eps = 2.0 ** (-52 * s.limbs)
        line["err_vs_oracle"] = {"max_rel": e, "max_rel_over_eps": e / eps, "eps": eps,
                                 "measure": "one step from x0; per degree, max_i |x_gpu - x_oracle| / max_i |x_oracle|"}
        sp = line.get("other_forms", {}).get("split_product_form")
        if sp is not None:  # the split-product form's step from x0 against the same oracle step
            sflags = md.FLAG_OZAKI | (flags & (md.FLAG_LU | md.FLAG_AUTOTUNE))
            sws = md.workspace(sysd.workspace_bytes(sflags), device=dev)
            x2 = md.to_device(s.x0, dev)
            md.newton_step(sysd, x2, sws, nrm, flags=sflags)
            torch.cuda.synchronize()
            e2 = err_vs_oracle(x2.cpu().numpy(), x_orc)
            sp["err_vs_oracle"] = {"max_rel": e2, "max_rel_over_eps": e2 / eps, "eps": eps,
                                   "measure": line["err_vs_oracle"]["measure"]}
            del sws, x2
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------- the other forms
def run_solve3(args):
    """Linearized solve, quad double real n=256 d=16, cond(A_0) = 1e8: plain
    block Toeplitz update against the split-product (Ozaki) update."""
    line = measure_solve3(args, with_err=not args.no_cpu_baseline)
    print(json.dumps(line), flush=True)
    return 0


def measure_solve3(args, with_err: bool) -> dict:
    """The plain and split-product solves of the n = 256, d = 16 quad double
    system (condition 1e8) on the same GPU: solves/s, the update's time per
    solve, the kernels, and (with_err) each form's largest per-degree error
    against the oracle, relative to the largest coefficient of that degree."""
    import numpy as np
    import torch

    import mdgen
    import paper_2012_06607_gb300 as md

    A, b = mdgen.solve_config3(args.seed)
    K, n, d = 4, 256, 16
    Ad, bd = md.to_device(A), md.to_device(b)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for name, flags in (("plain", 0), ("ozaki", md.FLAG_OZAKI)):
        ws = md.workspace(md.linsolve_workspace_bytes(K, False, n, d, flags))
        dx = torch.empty_like(bd)
        for _ in range(args.warmup):
            md.linsolve(K, False, Ad, bd, ws, dx, flags=flags)
        torch.cuda.synchronize()
        md.profile_read()
        md.profile_enable(True)
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            md.linsolve(K, False, Ad, bd, ws, dx, flags=flags)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        md.profile_enable(False)
        prof = md.profile_read()
        assert md.device_status(ws) == 0
        res[name] = {"ms_per_solve": statistics.mean(a.elapsed_time(b) for a, b in evs),
                     "kernel_ms_per_solve": {k: round(v[0] / args.steps, 3) for k, v in
                                             sorted(prof.items(), key=lambda kv: -kv[1][0])},
                     "dx": dx.cpu().numpy()}
    err = {}
    if with_err:
        import oracle

        from math import fsum
        orc = oracle.Oracle(threads=os.cpu_count() or 1)
        t0 = time.perf_counter()
        want = orc.linsolve(K, False, A, b)
        cpu_solve_s = time.perf_counter() - t0
        for name in ("plain", "ozaki"):
            got = res[name]["dx"]
            e = []
            for k in range(d + 1):
                diff = max(abs(fsum(list(got[0, :, i, k]) + [-v for v in want[0, :, i, k]])) for i in range(n))
                scale = max(abs(want[0, 0, i, k]) for i in range(n))
                e.append(diff / scale)
            err[name] = {"max_rel": max(e), "max_rel_over_eps": max(e) / 2.0 ** (-52 * K)}
        err["cpu_baseline"] = {"value": 1.0 / cpu_solve_s, "unit": "solves/s", "cores": orc.threads(),
                               "kind": "oracle", "sample": "one solve (host cores, OpenMP)"}
    upd = {name: sum(v for k, v in res[name]["kernel_ms_per_solve"].items()
                     if k in ("rhs_partial", "rhs_finish", "oz_split", "oz_update")) for name in res}
    return {"metric": "linearized block Toeplitz solves/s (qd real, n=256, d=16, cond(A_0)=1e8)",
            "unit": "solves/s", "form": "plain vs split-product",
            "value_plain": 1e3 / res["plain"]["ms_per_solve"], "value_ozaki": 1e3 / res["ozaki"]["ms_per_solve"],
            "speedup_solve": res["plain"]["ms_per_solve"] / res["ozaki"]["ms_per_solve"],
            "update_ms_plain": upd["plain"], "update_ms_ozaki": upd["ozaki"],
            "speedup_update": upd["plain"] / max(upd["ozaki"], 1e-9),
            "err_vs_oracle": err or None,
            "err_measure": "per degree, max_i |dx_gpu - dx_oracle| / max_i |dx_oracle|; eps = 2^-208; "
                           "cond(A_0) = 1e8 bounds both forms' forward error alike",
            "kernel_ms_plain": res["plain"]["kernel_ms_per_solve"],
            "kernel_ms_ozaki": res["ozaki"]["kernel_ms_per_solve"], "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic", "dtype": "f64 (quad double); bf16 slices for the split products"}


# The paper's octo double schedule (Table 2): truncation degrees 8, 16, 24,
# 32 with at most 5, 6, 12 and 16 iterations, tolerance 1e-32 on the update.
RUN_DEGREES = (8, 16, 24, 32)
RUN_MAX_ITER = (5, 6, 12, 16)
# the seconds of those runs in Table 2 (88 threads, cyclic 128-roots surface)
PAPER_TABLE2_OD_SECONDS = {8: 128, 16: 472, 24: 1934, 32: 4400}


def run_driver(args):
    """Newton with degree continuation through md_newton_series_run on the
    octo double n = 128 system (config 2, the shape of the paper's Table 2
    runs) under the paper's octo double schedule, plain and split-product
    form: seconds per run, iterations per level, the final update norms.
    The paper's Table 2 times (88 Xeon threads, cyclic 128-roots surface) are
    quoted beside it as context; the oracle's first level is the CPU sample."""
    import numpy as np
    import torch

    import mdgen
    import paper_2012_06607_gb300 as md

    s = mdgen.config_system(2, args.seed)
    sysd = md.DeviceSystem(s)
    sched = md.schedule(RUN_DEGREES, RUN_MAX_ITER, tol=1e-32)
    forms = {}
    for name, flags in (("plain", 0), ("split_product", md.FLAG_OZAKI)):
        ws = md.workspace(md.newton_run_workspace_bytes(sysd, sched, flags))
        for _ in range(max(args.warmup, 1)):  # plans and first launches of every level
            x = md.to_device(s.x0)
            md.newton_run(sysd, x, ws, sched, flags=flags)
        torch.cuda.synchronize()
        secs = []
        rep = None
        for _ in range(args.steps):
            x = md.to_device(s.x0)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            rep = md.newton_run(sysd, x, ws, sched, flags=flags)
            b.record()
            b.synchronize()
            secs.append(a.elapsed_time(b) / 1e3)
        assert md.device_status(ws) == 0
        forms[name] = {"seconds_per_run": statistics.median(secs), "levels_done": rep["levels_done"],
                       "iterations": rep["iterations"], "converged": rep["converged"],
                       "dx_norm_last": rep["dx_norm"][-1] if rep["dx_norm"] else None}
        del ws
    line = {"metric": "Newton runs with degree continuation (od real, n=128, d 8->16->24->32)", "form": "run",
            "value": forms["plain"]["seconds_per_run"], "unit": "s", "higher_is_better": False,
            "plain": forms["plain"], "split_product": forms["split_product"],
            "speedup_split": forms["plain"]["seconds_per_run"] / forms["split_product"]["seconds_per_run"],
            "schedule": {"degrees": list(RUN_DEGREES), "max_iter": list(RUN_MAX_ITER), "tol": 1e-32},
            "paper_table2_octo_double_s": {**{str(k): v for k, v in PAPER_TABLE2_OD_SECONDS.items()},
                                           "note": "88 threads of two Xeon E5-2699, cyclic 128-roots surface "
                                                   "(another system): context, not the same workload"},
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "f64 (octo double)"}
    if not args.no_cpu_baseline:
        import oracle

        orc = oracle.Oracle(threads=os.cpu_count() or 1)
        t0 = time.perf_counter()
        _, crep = orc.newton_run(s, RUN_DEGREES[:1], RUN_MAX_ITER[:1], 1e-32, 1.0)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": cpu_s, "unit": "s", "cores": orc.threads(), "kind": "oracle",
                                "sample": f"the first level only (d = 8, {crep['iterations']} iterations)"}
    print(json.dumps(line), flush=True)
    return 0


def run_ladder(args):
    """The cost of higher precision (Section 2, Table 1): the Newton step of
    the same system (the headline workload, its exact coefficients re-expanded
    into K limbs) at every precision K in {1, 2, 3, 4, 5, 8, 10}."""
    import torch

    import mdgen
    import paper_2012_06607_gb300 as md

    base = mdgen.config_system(CFG, args.seed)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    per = {}
    for K in (1, 2, 3, 4, 5, 8, 10):
        s = base if K == base.limbs else base.with_limbs(K)
        sysd = md.DeviceSystem(s)
        ws = md.workspace(sysd.workspace_bytes())
        x = md.to_device(s.x0)
        for _ in range(args.warmup):
            md.newton_step(sysd, x, ws)
        torch.cuda.synchronize()
        md.profile_read()
        md.profile_enable(True)
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            md.newton_step(sysd, x, ws)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        md.profile_enable(False)
        prof = md.profile_read()
        assert md.device_status(ws) == 0
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        cmul_i, cadd_i = complex_mac_instr(K, s.planes)
        nconv = conv_schedule_counts(s)
        d = s.degree
        conv_instr = nconv * ((d + 1) * (d + 2) // 2 * cmul_i + d * (d + 1) // 2 * cadd_i)
        conv_ms = prof.get("conv_stage", (float("nan"), 0))[0] / args.steps
        # the split-product form at the same precision (K >= 2): step and
        # series-product times
        split = None
        if K >= 2:
            oflags = md.FLAG_OZAKI
            ows = md.workspace(sysd.workspace_bytes(oflags))
            for _ in range(args.warmup):
                md.newton_step(sysd, x, ows, flags=oflags)
            torch.cuda.synchronize()
            md.profile_read()
            md.profile_enable(True)
            oevs = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                md.newton_step(sysd, x, ows, flags=oflags)
                e1.record(stream)
                oevs.append((e0, e1))
            torch.cuda.synchronize()
            md.profile_enable(False)
            oprof = md.profile_read()
            assert md.device_status(ows) == 0
            oms = statistics.mean(a.elapsed_time(b) for a, b in oevs)
            ocv = oprof.get("conv_stage_fx", oprof.get("conv_stage", (float("nan"), 0)))[0] / args.steps
            split = {"ms_per_step": oms, "conv_ms_per_step": ocv, "speedup_vs_md": ms / oms,
                     "conv_speedup_vs_md": conv_ms / ocv if ocv > 0 else None}
            del ows
        t1 = TABLE1.get(K)
        per[K] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "conv_ms_per_step": conv_ms, "split_product_form": split,
                  "conv_fp64_instr_per_step": conv_instr,
                  "conv_fp64_frac_of_peak": conv_instr / (conv_ms / 1e3) / FP64_PEAK_INSTR if conv_ms > 0 else None,
                  "table1_ops_per_complex_mac": (4 * t1[1] + 4 * t1[0]) if t1 else None}
        del ws, sysd, x
        torch.cuda.empty_cache()
    dd = per[2]["ms_per_step"]
    for K in per:
        per[K]["time_vs_dd"] = per[K]["ms_per_step"] / dd
    line = {"metric": "power-series Newton steps/s per precision (n=64, d=64, complex)", "form": "precision ladder",
            "unit": "steps/s", "per_limbs": per, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": WORKLOAD.replace("quad double", "K-limb") + " (same exact coefficients)",
                       "l2": "flushed between steps"},
            "data": "synthetic", "dtype": "f64 (K limbs)"}
    print(json.dumps(line), flush=True)
    return 0


def run_elementwise(args):
    """Elementwise md add and mul on arrays far larger than L2 (512 MB per
    input limb set), at every precision: HBM GB/s and FP64 instruction rate,
    each against its peak, to show where the md arithmetic stops being
    memory-bound."""
    import torch

    import paper_2012_06607_gb300 as md

    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    res = {}
    for K in (1, 2, 3, 4, 8, 10):
        count = (512 << 20) // (8 * K)
        x = torch.rand((1, K, count), dtype=torch.float64, device="cuda")
        y = torch.rand((1, K, count), dtype=torch.float64, device="cuda")
        x[:, 1:] *= 2.0 ** -60
        y[:, 1:] *= 2.0 ** -60
        z = torch.empty_like(x)
        c = fp64_instr_counts(K)
        for op in ("add", "mul"):
            for _ in range(2):
                md.elementwise(op, K, False, x, y, out=z)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record()
            for _ in range(reps):
                md.elementwise(op, K, False, x, y, out=z)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = 3 * 8 * K * count / (ms / 1e3) / 1e9
            instr = c[op] * count / (ms / 1e3)
            res[f"K{K}_{op}"] = {"ms": ms, "gb_per_s": gbs, "hbm_frac": gbs / hbm, "fp64_instr_per_s": instr,
                                 "fp64_frac": instr / FP64_PEAK_INSTR,
                                 "bound": "hbm" if gbs / hbm > instr / FP64_PEAK_INSTR else "alu"}
        del x, y, z
        torch.cuda.empty_cache()
    line = {"metric": "elementwise md add / mul, real, 512 MB per input limb set", "form": "elementwise",
            "per_op": res, "hbm_peak_gbs": hbm, "hbm_peak_source": "measured" if peaks else "fallback",
            "fp64_peak_instr_per_s": FP64_PEAK_INSTR, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def batched_shard(systems, rank: int, world: int):
    """This rank's systems of the batch: the LPT partition of the host cost
    estimates over the ranks (every rank computes the same partition; no
    communication).  Returns (indices of this rank, the whole partition)."""
    import paper_2012_06607_gb300 as md

    if world <= 1:
        return list(range(len(systems))), [list(range(len(systems)))]
    parts = md.shard_lpt(md.batched_job_costs(systems), world)
    return sorted(parts[rank]), parts


def run_batched(args):
    """2048 complex systems, n ~ U{8..64}, d ~ U{8..32}, double double / quad
    double: one persistent launch per precision class per Newton iteration
    (autotuned, replayed from a CUDA graph) against a per-system launch loop.
    With N ranks the batch is split by LPT over the GPUs (strong scaling; no
    collective on the data path) and the iteration time is the slowest
    rank's."""
    rank, world, local = dist_env()
    dist = dist_init(world)
    line = measure_batched(args, args.batch, rank, world, local, dist, with_loop=not args.no_loop,
                           err_sample=0 if args.no_cpu_baseline else 8)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_batched(args, count, rank, world, local, dist, with_loop: bool, err_sample: int) -> dict:
    """One batched Newton iteration over `count` systems of the batched
    workload (this rank's LPT shard): iterations/s, per-system latency, the
    same step with every CTA sharing SMs, the phases of the slowest system
    against the SM's FP64 rate, a per-system launch loop (with_loop), and the
    first step from x0 of `err_sample` systems (largest n first, both
    precisions) against the oracle's step."""
    import numpy as np
    import torch

    import mdgen
    import paper_2012_06607_gb300 as md

    if world > 1:
        torch.cuda.set_device(local)
    all_systems = mdgen.batch_systems(args.seed, count=count)
    if len(all_systems) < world:
        raise SystemExit(f"--batch {count} leaves ranks without systems at {world} GPUs")
    mine, _ = batched_shard(all_systems, rank, world)
    systems = [all_systems[i] for i in mine]
    sds = [md.DeviceSystem(s) for s in systems]
    flags = md.FLAG_AUTOTUNE | md.FLAG_GRAPH
    # room for both forms (the split-product form adds fixed-point copies)
    ws = md.workspace(max(md.batched_workspace_bytes(sds, flags),
                          md.batched_workspace_bytes(sds, flags | md.FLAG_OZAKI)))
    xs = [md.to_device(s.x0) for s in systems]
    nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
    times = torch.zeros((len(systems), 2), dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    sample = []
    if err_sample > 0 and rank == 0:
        by_size = sorted(range(len(systems)), key=lambda i: -systems[i].n * (systems[i].degree + 1))
        for K in (2, 4):
            sample += [i for i in by_size if systems[i].limbs == K][:err_sample // 2]
    first = {}
    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            md.newton_step_batched(sds, xs, ws, nrm, times, flags=flags, stream=stream)
            if w == 0:
                stream.synchronize()
                first = {i: xs[i].cpu().numpy() for i in sample}
        torch.cuda.synchronize()
        ms = []
        lat = []
        for _ in range(args.steps):
            if dist is not None:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            md.newton_step_batched(sds, xs, ws, nrm, times, flags=flags, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            t = times.cpu().numpy()
            lat.append((t[:, 1] - t[:, 0]) / 1e6)
        torch.cuda.synchronize()
        # the same step with every CTA sharing SMs, one class after another
        # (no whole-SM systems, one stream)
        sflags = flags | md.FLAG_SERIAL
        md.newton_step_batched(sds, xs, ws, nrm, None, flags=sflags, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        md.newton_step_batched(sds, xs, ws, nrm, None, flags=sflags, stream=stream)
        e1.record(stream)
        e1.synchronize()
        serial_ms = e0.elapsed_time(e1)
        # the split-product form (series products on 32-bit word slices), its
        # own plan, tuning and graph on the same buffers; its first step from
        # x0 for the error sample
        oflags = flags | md.FLAG_OZAKI
        for _ in range(max(args.warmup, 2)):
            md.newton_step_batched(sds, xs, ws, nrm, None, flags=oflags, stream=stream)
        oz_ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            md.newton_step_batched(sds, xs, ws, nrm, None, flags=oflags, stream=stream)
            e1.record(stream)
            e1.synchronize()
            oz_ms.append(e0.elapsed_time(e1))
        oz_first = {}
        if sample:
            for x, sy in zip(xs, systems):
                x.copy_(torch.from_numpy(np.ascontiguousarray(sy.x0, dtype=np.float64)))
            md.newton_step_batched(sds, xs, ws, nrm, None, flags=oflags, stream=stream)
            stream.synchronize()
            oz_first = {i: xs[i].cpu().numpy() for i in sample}
        # one more step (not timed) with a global-timer stamp after every phase
        ptimes = torch.zeros((len(systems), md.PHASE_STAMPS), dtype=torch.int64, device="cuda")
        md.newton_step_batched(sds, xs, ws, nrm, ptimes, flags=flags | md.FLAG_PHASE_TIMES, stream=stream)
        torch.cuda.synchronize()
        optimes = torch.zeros_like(ptimes)
        md.newton_step_batched(sds, xs, ws, nrm, optimes, flags=oflags | md.FLAG_PHASE_TIMES, stream=stream)
        torch.cuda.synchronize()
    assert md.device_status(ws) == 0
    lat = np.concatenate(lat)
    it_ms = reduce_max(dist, sum(ms) / len(ms))
    oz_it_ms = reduce_max(dist, sum(oz_ms) / len(oz_ms))
    # phases of the slowest system, against the SM's share of the FP64 peak
    pt = ptimes.cpu().numpy().astype(np.float64)
    plat = pt[:, -1] - pt[:, 0]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    slow = int(np.argmax(plat))
    ph = dict(zip(md.PHASE_NAMES, np.diff(pt[slow]) / 1e6))
    opt = optimes.cpu().numpy().astype(np.float64)
    oph = dict(zip(md.PHASE_NAMES, np.diff(opt[slow]) / 1e6))
    m = step_fp64_model(systems[slow])
    per_sm = FP64_PEAK_INSTR / sms
    spans = {"products": (m["conv"], ph["products"]), "accumulation": (m["accum"], ph["accumulation"]),
             "qr": (m["qr"], ph["qr_setup"] + ph["householder_qr"]), "w": (m["backsub"], ph["rinv"] + ph["w"]),
             "degree_loop": (m["update"], ph["degree_loop"])}
    phases = {"system": {"index": slow, "n": systems[slow].n, "d": systems[slow].degree, "limbs": systems[slow].limbs},
              "ms": {k: round(float(v), 3) for k, v in ph.items()},
              "fraction_of_sm_fp64_peak": {k: round(float(c / (t / 1e3) / per_sm), 3) for k, (c, t) in spans.items()
                                           if t > 0},
              "sm_busy_fraction": float(plat.sum() / (sms * (pt[:, -1].max() - pt[:, 0].min()))),
              "counted": "FP64 instructions of the bench's model per phase; stamps from MD_FLAG_PHASE_TIMES"}
    # per-system launch loop on the same systems (plain single-system steps)
    loop_ms = None
    if with_loop and world == 1:
        wmax = max(sd.workspace_bytes() for sd in sds)
        ws1 = md.workspace(wmax)
        xs1 = [md.to_device(s.x0) for s in systems]
        for i, sd in enumerate(sds[:4]):
            md.newton_step(sd, xs1[i], ws1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, sd in enumerate(sds):
            md.newton_step(sd, xs1[i], ws1)
        torch.cuda.synchronize()
        loop_ms = (time.perf_counter() - t0) * 1e3
    kinds = {}
    for s in all_systems:
        kinds[s.limbs] = kinds.get(s.limbs, 0) + 1
    models = [step_fp64_model(s) for s in all_systems]
    fp64 = {k: sum(m[k] for m in models) for k in models[0]}
    err = None
    if first:
        import oracle

        from math import fsum
        orc = oracle.Oracle(threads=os.cpu_count() or 1)
        worst = []
        cpu_s = 0.0

        def rel_over_eps(s, got, want):
            P, K, n, d = s.planes, s.limbs, s.n, s.degree
            rel = 0.0
            for k in range(d + 1):
                diff = max(math.hypot(*[fsum(list(got[p, :, j, k]) + [-v for v in want[p, :, j, k]]) for p in range(P)])
                           for j in range(n))
                scale = max(math.hypot(*[fsum(want[p, :, j, k]) for p in range(P)]) for j in range(n))
                rel = max(rel, diff / max(scale, 1e-300))
            return rel / 2.0 ** (-52 * K)

        for i, got in first.items():
            s = systems[i]
            t0 = time.perf_counter()
            want, _ = orc.newton_step(s, s.x0)
            cpu_s += time.perf_counter() - t0
            w = {"n": s.n, "d": s.degree, "limbs": s.limbs, "max_rel_over_eps": rel_over_eps(s, got, want)}
            if i in oz_first:
                w["split_form_max_rel_over_eps"] = rel_over_eps(s, oz_first[i], want)
            worst.append(w)
        err = {"systems": worst, "max_rel_over_eps": max(w["max_rel_over_eps"] for w in worst),
               "split_form_max_rel_over_eps": max(w.get("split_form_max_rel_over_eps", 0.0) for w in worst),
               "cpu_baseline": {"value": len(worst) / cpu_s, "unit": "system steps/s", "cores": orc.threads(),
                                "kind": "oracle", "sample": "the sampled systems' first steps (the largest n of "
                                                            "each precision; host cores, OpenMP)"},
               "measure": "first step from x0; per degree, max_i |x_gpu - x_oracle| / max_i |x_oracle|, "
                          "in units of eps_K = 2^(-52K)"}
    line = {"metric": f"batched Newton iterations/s ({len(all_systems)} systems, n~U{{8..64}}, d~U{{8..32}}, dd/qd, "
                      "complex)",
            "unit": "iterations/s", "value": 1e3 / it_ms, "ms_per_iteration": it_ms, "err_vs_oracle": err,
            "system_steps_per_s": len(all_systems) * 1e3 / it_ms, "n_gpus": world,
            "scaling": "strong" if world > 1 else "weak",
            "parallelism": f"LPT shards of the batch x{world}" if world > 1 else "one GPU",
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_max": float(lat.max()),
            "shared_sm_only_ms_per_iteration": serial_ms,
            "split_product_form": {"flags": "MD_FLAG_OZAKI: series products and update chunk sums on 32-bit word slices",
                                   "ms_per_iteration": oz_it_ms, "value": 1e3 / oz_it_ms, "unit": "iterations/s",
                                   "speedup_vs_md": it_ms / oz_it_ms,
                                   "phases_ms_of_the_same_system": {k: round(float(v), 3) for k, v in oph.items()}},
            "phases_of_slowest_system": phases,
            "loop_ms_per_iteration": loop_ms,
            "speedup_vs_loop": (loop_ms / it_ms) if loop_ms else None,
            "systems": len(all_systems), "systems_on_rank0": len(systems), "limb_counts": kinds,
            "workspace_gib": ws.numel() / 2 ** 30,
            "roofline": {"bound": "alu", "achieved": fp64["total"] / (it_ms / 1e3) / 1e12,
                         "peak": world * FP64_PEAK_INSTR / 1e12, "unit": "TFLOP/s",
                         "frac": fp64["total"] / (it_ms / 1e3) / (world * FP64_PEAK_INSTR),
                         "counted": "FP64 instructions per iteration: series products exact, solve modelled",
                         "fp64_instr_per_iteration": fp64},
            "steps": args.steps, "warmup": args.warmup, "flags": "autotune+graph", "data": "synthetic",
            "dtype": "f64 (double double / quad double)"}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=7)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--impl", default="product", choices=["product", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-form", action="store_true", help="skip timing the split-product update beside md")
    ap.add_argument("--no-autotune", action="store_true",
                    help="single step: keep the default SM count of the factorisation (no MD_FLAG_AUTOTUNE)")
    ap.add_argument("--form", default="plain", choices=["plain", "solve3", "batched", "ladder", "elementwise", "run"],
                    help="plain: the Newton-step benchmark; solve3: plain vs split-product solve; "
                         "batched: 2048-system batched step vs a per-system loop; ladder: the headline step at every precision; elementwise: md add/mul HBM vs FP64 bound; run: Newton with the paper's octo double degree continuation, plain and split form")
    ap.add_argument("--update", default="md", choices=["md", "split"],
                    help="block Toeplitz update of the plain form: md arithmetic or split-product")
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--other-batch", type=int, default=2048,
                    help="systems of the batched form measured beside the plain step (other_forms)")
    ap.add_argument("--factor", default="qr", choices=["qr", "lu"], help="factorisation of A_0 in the plain form")
    ap.add_argument("--config", type=int, default=CFG, choices=[0, 1, 2],
                    help="workload of the plain and reference forms: 1 (default, the headline), 0 or 2")
    ap.add_argument("--no-loop", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "solve3":
        return run_solve3(args)
    if args.form == "batched":
        return run_batched(args)
    if args.form == "ladder":
        return run_ladder(args)
    if args.form == "run":
        return run_driver(args)
    if args.form == "elementwise":
        return run_elementwise(args)
    return run_product(args)


if __name__ == "__main__":
    sys.exit(main())

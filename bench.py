#!/usr/bin/env python
"""Benchmark of the Strassen-fused FP64 GEMM on GB300 (one JSON line on rank 0).

Workload (default): m = n = k = 8192, FP64, A, B, C i.i.d. uniform[-1, 1] from fixed
seeds, C += A*B (accumulate mode), 2-level ABC Strassen.  One step = one
strassen_gemm call through the C ABI on inputs resident in HBM (1.5 GB of operands,
larger than the 129 MB L2, so no flush is needed between steps).

Metric: effective GFLOPS = 2mnk / t * 1e-9 (the paper's Eq. for effective GFLOPS).
Also reported: the library's classical FP64 kernel on the same inputs (the
comparator), the same product with one and three levels, an end-to-end figure with
host buffers, the roofline of the FP64 product
kernel against the FP64 pipe, SM clocks sampled during the timed region, and the CPU
oracle timed on a bounded sample.

Multi-GPU: the path does not shard into a collective; N ranks run N independent
replicas ("replicas only"), value = total effective flops of all ranks / the slowest
rank's time.

--impl reference times the CPU oracle (textbook recursive Strassen, plain C, one
thread) on a bounded sample of the same workload (m = n = k = 1024 per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "effective GFLOPS (2mnk/t) Strassen vs classical GEMM, 1 GB300, rel err ≤1e-12"
UNIT = "GFLOP/s"
# FP64 pipe peak: 2 FMA lanes (4 flops) per clock per SM x 152 SMs x 2070 MHz max clock.
FP64_PEAK_GFLOPS = 4 * 152 * 2070e6 / 1e9
CPU_SAMPLE_N = 2048
REF_SAMPLE_N = 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--levels", type=int, default=2)
    ap.add_argument("--variant", default="ABC")
    ap.add_argument("--dtype", default="f64", choices=["f64", "oz_bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-levels", action="store_true", help="skip the other level counts (1 and 3 levels)")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_flops(m, n, k, levels):
    """FP64-pipe flops of the method: 7^L products of 2 h_m h_n h_k multiply-add flops
    (Sections 3.1-3.2).  The extra additions of the performance model's T_a (Section
    4.2) are not on the FP64 pipe here (operand sums on the integer pipe, C updates as
    L2 atomics): see model_flops."""
    P = 1 << levels
    hm, hn, hk = -(-m // P), -(-n // P), -(-k // P)
    return 7 ** levels * 2.0 * hm * hn * hk


def model_flops(m, n, k, levels):
    """The paper's arithmetic count T_a / tau_a (Section 4.2): the products plus two flops
    per extra addition of A and B blocks and per C update, with the term counts of the
    L-level table."""
    from paper_1605_01078_gb300 import strassen_plan_table
    P = 1 << levels
    hm, hn, hk = -(-m // P), -(-n // P), -(-k // P)
    tab = strassen_plan_table(levels)
    a_adds = sum(len(p[0]) - 1 for p in tab)
    b_adds = sum(len(p[1]) - 1 for p in tab)
    c_upd = sum(len(p[2]) for p in tab) if levels > 0 else 0
    return algorithmic_flops(m, n, k, levels) + 2.0 * (a_adds * hm * hk + b_adds * hk * hn + c_upd * hm * hn)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# The sources the FP64 product kernel is compiled from (its recorded traffic is valid
# only while they are unchanged).
KERNEL_SOURCES = ("fp64_gemm.cu", "int_fadd.h", "plan_tables.h")


def kernel_source_sha256():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1605_01078_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch of the FP64 product kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "fp64_strassen_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            a, b = line.split("=", 1)
            rec[a.strip()] = b.strip()
    if rec.get("kernel_source_sha256") != kernel_source_sha256():
        return None
    try:
        return float(rec["dram_bytes_per_launch_8192_2L_ABC"])
    except (KeyError, ValueError):
        return None


def bench_batched(sg, W, torch, reps=3):
    """256 FP64 problems, m, n, k log-uniform in [256, 4096] (seed 0), levels and block
    tiles chosen by the library, in one batched call (one persistent launch per tile)
    captured in a CUDA graph; against a loop of 256 classical launches on the same
    operands."""
    shapes = W.loguniform_shapes(256, seed=0, lo=256, hi=4096)
    mats = [(W.uniform_device(m, k, 1000 + i), W.uniform_device(k, n, 2000 + i), W.uniform_device(m, n, 3000 + i))
            for i, (m, n, k) in enumerate(shapes)]
    arr = (sg.strassen_problem * len(mats))()
    for i, (A, B, C) in enumerate(mats):
        arr[i] = sg.strassen_problem(A.shape[0], B.shape[1], A.shape[1], A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                     A.stride(0), B.stride(0), C.stride(0), -1, sg.STRASSEN_AUTO)
    flops = sum(2.0 * m * n * k for (m, n, k) in shapes)
    stream = torch.cuda.current_stream()
    assert sg.strassen_gemm_batched(len(mats), arr, 0, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        assert sg.strassen_gemm_batched(len(mats), arr, 0, torch.cuda.current_stream().cuda_stream) == 0
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / 1e3 / reps
    for A, B, C in mats:
        sg.classical(A, B, C)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        for A, B, C in mats:
            sg.classical(A, B, C)
    e1.record()
    torch.cuda.synchronize()
    t_loop = e0.elapsed_time(e1) / 1e3 / reps
    # the same batched call with every problem classical: isolates the launch from the level choice
    for i in range(len(mats)):
        arr[i].levels = 0
        arr[i].variant = sg.STRASSEN_ABC
    g0 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g0):
        assert sg.strassen_gemm_batched(len(mats), arr, 0, torch.cuda.current_stream().cuda_stream) == 0
    g0.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        g0.replay()
    e1.record()
    torch.cuda.synchronize()
    t_graph0 = e0.elapsed_time(e1) / 1e3 / reps
    return {"workload": "256 FP64 problems, m,n,k log-uniform in [256,4096] (seed 0), one batched call (one persistent "
                        "launch per block tile) in a CUDA graph",
            "value": flops / t_graph / 1e9, "unit": UNIT, "ms": t_graph * 1e3,
            "all_classical_batched": {"value": flops / t_graph0 / 1e9, "ms": t_graph0 * 1e3},
            "loop_of_classical": {"value": flops / t_loop / 1e9, "ms": t_loop * 1e3, "launches": len(mats)},
            "speedup_vs_loop": t_loop / t_graph}


def bench_split_precision(sg, W, torch, n=8192, err_n=4096, reps=3):
    """Split-precision FP64 emulation (BF16 digit slices on the tensor cores): effective
    GFLOP/s at n^3 for 0, 1, 2 levels and at (2n)^3 for level 0, and the max-norm error
    against the library's
    plain FP64 classical result (normwise: / (||A||_inf max|B|)) for inputs
    u * 2^round(N(0, sigma)) at err_n^3."""
    out = {"workload": f"m=n=k={n} FP64 via BF16 slices, A,B,C uniform[-1,1]", "levels": {}}
    A, B, C = W.uniform_device(n, n, 11), W.uniform_device(n, n, 12), W.uniform_device(n, n, 13)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for L in (0, 1, 2):
        sg.gemm(A, B, C, levels=L, dtype="oz_bf16")
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sg.gemm(A, B, C, levels=L, dtype="oz_bf16")
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        out["levels"][str(L)] = {"value": 2.0 * n ** 3 / t / 1e9, "unit": UNIT, "ms": t * 1e3}
    del A, B, C
    # the larger square size of the split-precision workload, classical slices
    n2 = 2 * n
    A, B, C = W.uniform_device(n2, n2, 14), W.uniform_device(n2, n2, 15), W.uniform_device(n2, n2, 16)
    sg.gemm(A, B, C, levels=0, dtype="oz_bf16")
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        sg.gemm(A, B, C, levels=0, dtype="oz_bf16")
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    out[f"n{n2}_level0"] = {"value": 2.0 * n2 ** 3 / t / 1e9, "unit": UNIT, "ms": t * 1e3}
    del A, B, C
    errs = {}
    for sigma in (0, 4, 10):
        A = torch.from_numpy(W.scaled(err_n, err_n, 21, sigma)).cuda()
        B = torch.from_numpy(W.scaled(err_n, err_n, 22, sigma)).cuda()
        ref = torch.zeros((err_n, err_n), dtype=torch.float64, device="cuda")
        sg.classical(A, B, ref)
        den = float(torch.max(torch.sum(torch.abs(A), dim=1))) * float(torch.max(torch.abs(B)))
        row = {}
        for L in (0, 1, 2):
            Cz = torch.zeros_like(ref)
            sg.gemm(A, B, Cz, levels=L, dtype="oz_bf16")
            torch.cuda.synchronize()
            row[str(L)] = float(torch.max(torch.abs(Cz - ref))) / den
        errs[str(sigma)] = row
    out["error_vs_fp64_classical"] = {"n": err_n, "by_sigma_then_levels": errs}
    return out


def level_error(sg, torch, A, B, C, stream, levels, variant="ABC"):
    """max|C_L - C_0| / (||A||_inf max|B|) of one call against the library's classical
    result on the same inputs (the normwise reading of the tolerance)."""
    ref = C.clone()
    sg.classical(A, B, ref)
    got = C.clone()
    sg.gemm(A, B, got, levels=levels, variant=variant, stream=stream)
    torch.cuda.synchronize()
    den = float(A.abs().sum(dim=1).max()) * float(B.abs().max())
    err = float((got - ref).abs().max()) / den
    del ref, got
    return err


def bench_other_levels(sg, torch, A, B, C, stream, levels_list, variant="ABC", reps=3):
    """The same product with other level counts (on the same resident inputs): effective
    GFLOP/s and the FP64 pipe fraction of each (CUDA events per call), and the max-norm
    error of one call against the library's classical result on the same C
    (max|C_L - C_0| / (||A||_inf max|B|))."""
    m, k = A.shape
    n = B.shape[1]
    out = {}
    for lv in levels_list:
        err = level_error(sg, torch, A, B, C, stream, lv, variant)
        sg.gemm(A, B, C, levels=lv, variant=variant, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            sg.gemm(A, B, C, levels=lv, variant=variant, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        t = statistics.median(a.elapsed_time(b) / 1e3 for a, b in ev)
        alg = algorithmic_flops(m, n, k, lv) / t / 1e9
        out[str(lv)] = {"value": 2.0 * m * n * k / t / 1e9, "unit": UNIT, "ms": t * 1e3,
                        "variant": variant, "algorithmic_gflops": alg, "frac": alg / FP64_PEAK_GFLOPS,
                        "err_vs_classical": err}
    return out


def cpu_oracle_effective(n, levels, reps=1):
    import numpy as np
    import oracle
    import workloads as W
    A, B = W.uniform(n, n, 0), W.uniform(n, n, 1)
    C = W.uniform(n, n, 2)
    oracle.build()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.strassen(A, B, C, levels)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return 2.0 * n ** 3 / best / 1e9, best


def max_over_ranks(seconds, dist, device):
    """The slowest rank's time (all ranks call it; without a process group, the local
    time)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_step, steps, world, seconds):
    """Whole-job throughput of N replicas: every rank does `steps` steps of
    `flops_per_step`; the job takes the slowest rank's `seconds`."""
    return flops_per_step * steps * world / seconds / 1e9


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    import workloads as W
    n = REF_SAMPLE_N
    A, B, C = W.uniform(n, n, 0), W.uniform(n, n, 1), W.uniform(n, n, 2)
    oracle.build()
    for _ in range(args.warmup):
        oracle.strassen(A, B, C, args.levels)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.strassen(A, B, C, args.levels)
    dt = time.perf_counter() - t0
    val = 2.0 * n ** 3 * args.steps / dt / 1e9
    sample = f"m=n=k={n} {args.levels}-level textbook Strassen per step (oracle, plain C, 1 thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"square m=n=k={args.n} FP64 {args.levels}-level {args.variant} Strassen, C += A*B"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import paper_1605_01078_gb300 as sg
    import workloads as W

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    m = n = k = args.n
    L, variant = args.levels, args.variant
    sg.load_library()
    A = torch.from_numpy(W.uniform(m, k, 100 + rank)).cuda()
    B = torch.from_numpy(W.uniform(k, n, 200 + rank)).cuda()
    C = torch.from_numpy(W.uniform(m, n, 300 + rank)).cuda()
    stream = torch.cuda.current_stream()

    def step():
        sg.gemm(A, B, C, levels=L, variant=variant, dtype=args.dtype, stream=stream)

    launches_per_step = 1 if (L == 0 or variant.upper() == "ABC") else None
    if args.dtype == "oz_bf16":
        launches_per_step = 5  # split rows, column maxima, split columns, slice products, recombine + scatter
    elif launches_per_step is None:
        nprod = 7 ** L
        launches_per_step = nprod * (2 if variant.upper() == "AB" else 4)

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    per_launch = [a.elapsed_time(b) / 1e3 for a, b in ev]
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    eff_flops = 2.0 * m * n * k
    value = job_gflops(eff_flops, args.steps, ws, elapsed)

    # Comparator: the library's classical kernel on the same inputs.
    cls_steps = max(2, args.steps // 3)
    sg.classical(A, B, C)
    barrier()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(cls_steps):
        sg.classical(A, B, C)
    c1.record(stream)
    barrier()
    cls_val = eff_flops * cls_steps / (c0.elapsed_time(c1) / 1e3) / 1e9

    # End to end through the public API with pinned host buffers: every step copies its
    # inputs A, B, C host -> device and reads its result C back, pipelined on two copy
    # streams (the next step's inputs load while this step computes; double buffers).
    e2e = None
    if not args.no_e2e:
        hA, hB, hC = A.cpu().pin_memory(), B.cpu().pin_memory(), C.cpu().pin_memory()
        hOut = [torch.empty_like(hC).pin_memory() for _ in range(2)]
        bufs = [(torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)) for _ in range(2)]
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        e_steps = max(3, args.steps)

        def e2e_run(steps):
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_comp = [torch.cuda.Event() for _ in range(2)]
            ev_out = [torch.cuda.Event() for _ in range(2)]
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(h2d)

            def load(i):
                b = i % 2
                if i >= 2:
                    h2d.wait_event(ev_comp[b])   # step i-2 no longer reads this buffer
                dA, dB, dC = bufs[b]
                with torch.cuda.stream(h2d):
                    if i >= 2:
                        h2d.wait_event(ev_out[b])  # and its result has been read back
                    dA.copy_(hA, non_blocking=True)
                    dB.copy_(hB, non_blocking=True)
                    dC.copy_(hC, non_blocking=True)
                ev_in[b].record(h2d)

            load(0)
            for i in range(steps):
                b = i % 2
                if i + 1 < steps:
                    load(i + 1)
                stream.wait_event(ev_in[b])
                dA, dB, dC = bufs[b]
                sg.gemm(dA, dB, dC, levels=L, variant=variant, stream=stream)
                ev_comp[b].record(stream)
                d2h.wait_event(ev_comp[b])
                with torch.cuda.stream(d2h):
                    hOut[b].copy_(dC, non_blocking=True)
                ev_out[b].record(d2h)
            h2d.wait_event(ev_out[(steps - 1) % 2])
            h2d.wait_event(ev_comp[(steps - 1) % 2])
            t1.record(h2d)
            t1.synchronize()
            return t0.elapsed_time(t1) / 1e3

        e2e_run(2)
        barrier()
        et = max_over_ranks(e2e_run(e_steps), dist, "cuda")
        barrier()
        e2e = {"value": job_gflops(eff_flops, e_steps, ws, et), "unit": UNIT,
               "h2d_bytes_per_step": int(3 * 8 * m * n), "d2h_bytes_per_step": int(8 * m * n),
               "steps": e_steps, "pipelined": "inputs of step i+1 copied while step i computes (two buffers)"}
        del bufs

    err_headline = None
    if args.dtype == "f64" and rank == 0 and m <= 8192:
        err_headline = level_error(sg, torch, A, B, C, stream, L, variant)
    levels_other = None
    small = None
    if not args.no_levels and args.dtype == "f64" and rank == 0:
        levels_other = bench_other_levels(sg, torch, A, B, C, stream, [lv for lv in (1, 2, 3) if lv != L])
        # the small square case: m = n = k = 1024, one-level ABC, C = 0
        As, Bs = W.uniform_device(1024, 1024, 0), W.uniform_device(1024, 1024, 1)
        Cs = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
        small = {"workload": "m=n=k=1024, one-level ABC, C = 0 (uniform[-1,1])"}
        small.update(bench_other_levels(sg, torch, As, Bs, Cs, stream, [1], reps=20)["1"])
        del As, Bs, Cs

    batched = None
    if not args.no_batched and rank == 0:
        batched = bench_batched(sg, W, torch)
    split = None
    if not args.no_split and rank == 0:
        split = bench_split_precision(sg, W, torch)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    alg = algorithmic_flops(m, n, k, L)
    launch_s = statistics.mean(per_launch)
    achieved = alg / launch_s / 1e9
    if args.dtype == "oz_bf16":
        # tensor-core work of the slice products: 28 digit pairs x 2 h_m h_n h_k x 7^L
        P = 1 << L

        def padded(d, q):  # ceil(d / 2^L) rounded up to the tile edge q
            h = -(-d // P)
            return -(-h // q) * q

        hmp, hnp, hkp = padded(m, 128), padded(n, 256), padded(k, 64)
        mma = 28 * 2.0 * hmp * hnp * hkp * 7 ** L / launch_s / 1e12
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"bound": "tensor", "achieved": mma, "peak": bf16, "unit": "TFLOP/s", "frac": mma / bf16,
                "traffic": None, "kernel": "whole split-precision call (split, oz_gemm, recombine)",
                "peak_note": "measured BF16 dense peak (burst); per call, not per kernel"}
    else:
        roof = None
    roof = roof or {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS,
            "traffic": recorded_traffic() if (L == 2 and variant.upper() == "ABC" and m == 8192) else None,
            "kernel": "fp64_strassen_kernel",
            "peak_note": "FP64 pipe: 4 flop/clk/SM x 152 SMs x 2070 MHz (derived); DFMA probe measured 1200 GFLOP/s"}
    cpu = None
    if not args.no_cpu_baseline:
        cv, ct = cpu_oracle_effective(CPU_SAMPLE_N, L)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"m=n=k={CPU_SAMPLE_N} {L}-level textbook Strassen (plain C, 1 thread), {ct:.1f} s"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"square m=n=k={m} FP64 {L}-level {variant} Strassen, C += A*B (accumulate), "
                               f"A,B,C uniform[-1,1]" + (" (products as BF16 digit slices)" if args.dtype != "f64" else ""),
                   "m": m, "n": n, "k": k, "levels": L, "variant": variant, "products": args.dtype,
                   "parallelism": f"replicas{ws}", "l2": "inputs larger than L2 (3 x 8 m n bytes)"},
        "classical": {"value": cls_val, "unit": UNIT, "speedup": value / ws / cls_val},
        "err_vs_classical": err_headline,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "other_levels": levels_other,
        "small_square": small,
        "batched": batched,
        "split_precision": split,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

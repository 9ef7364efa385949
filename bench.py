#!/usr/bin/env python
"""Benchmark of the Strassen-fused FP64 GEMM on GB300 (one JSON line on rank 0).

Workload (default): m = n = k = 16384, FP64, A, B, C i.i.d. uniform[-1, 1] from fixed
seeds, C += A*B (accumulate mode), 2-level ABC Strassen -- the largest square size of
the FP64 shape sweep.  One step = one strassen_gemm call through the C ABI on inputs
resident in HBM (6 GB of operands, larger than the 129 MB L2, so no flush is needed
between steps).

Metric: effective GFLOPS = 2mnk / t * 1e-9 (the paper's effective GFLOPS, Section 4.2).
Also reported: the library's classical FP64 kernel on the same inputs (the comparator),
the same call with STRASSEN_FLAG_DETERMINISTIC (owner schedule), the strict max-norm
error max|C - C_exact| / (max|A| max|B|) and the Frobenius error of one call on sampled
entries next to the textbook Strassen's (the CPU leg computes the exact entries with
Dot2 and the textbook ones with the oracle), the one- and three-level products at
8192^3, an end-to-end figure with host buffers, the roofline of the FP64 product kernel
against the FP64 pipe, SM clocks sampled during the timed region, the batched and
split-precision workloads, and the CPU oracle timed on all host cores and on one.

Multi-GPU: the path does not shard into a collective; N ranks run N independent
replicas ("replicas only"), value = total effective flops of all ranks / the slowest
rank's time.

--impl reference times the CPU oracle (textbook recursive Strassen, plain C, OpenMP
timing build on all host cores) on a bounded sample of the workload (m = n = k = 4096
per step).
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
CPU_SAMPLE_N = 4096       # all host cores
CPU_SAMPLE_N_1CORE = 2048
REF_SAMPLE_N = 4096
ERR_SAMPLES = 4096        # sampled entries for the error figures


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--levels", type=int, default=2)
    ap.add_argument("--variant", default="ABC")
    ap.add_argument("--dtype", default="f64", choices=["f64", "oz_bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-levels", action="store_true", help="skip the other level counts (1 and 3 levels)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the sampled error figures")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="only time the CPU oracle (1 core and all cores, n = 1024..8192) and print the table")
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
KERNEL_SOURCES = ("fp64_gemm.cu", "int_fadd.h", "plan_tables.h", "internal.h")


def kernel_source_sha256():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1605_01078_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def recorded_traffic(n, levels, variant):
    """DRAM bytes per launch of the FP64 product kernel for this workload from the
    committed ncu summary, if it was taken on the current kernel source (else None)."""
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
        return float(rec[f"dram_bytes_per_launch_{n}_{levels}L_{variant.upper()}"])
    except (KeyError, ValueError):
        return None


def timed_calls(torch, fn, reps, stream):
    """Median seconds of `reps` calls of fn() (CUDA events on the launching stream),
    after one untimed call."""
    fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) / 1e3 for a, b in ev)


# ---------------------------------------------------------------- CPU leg (oracle)

def cpu_leg_errors(A, B, C0, got, rows, cols, levels):
    """The CPU leg's accuracy figures for one GPU call C = C0 + A B whose entries
    (rows, cols) are `got`: the exact entries (Dot2, rounded once) and the textbook
    recursive Strassen's entries (the oracle, entry by entry) on the same samples.
    strict = max|C - C_exact| / (max|A| max|B|); frobenius = ||C - C_exact||_F /
    (||A||_F ||B||_F), its numerator estimated from the samples."""
    import numpy as np
    import oracle
    oracle.build()
    exact = oracle.gemm_sampled(A, B, C0, rows, cols)
    den = float(np.max(np.abs(A))) * float(np.max(np.abs(B)))
    m, n = C0.shape
    fro_den = float(np.linalg.norm(A)) * float(np.linalg.norm(B))

    def figures(vals):
        e = np.abs(vals - exact)
        return float(np.max(e)) / den, float(np.sqrt(m * n * np.mean(e * e))) / fro_den

    strict, fro = figures(got)
    out = {"strict": strict, "frobenius": fro, "samples": int(rows.size),
           "tolerance": 1e-13 if levels <= 1 else 1e-12}
    if levels > 0:
        tb = oracle.strassen_sampled(A, B, C0, rows, cols, levels)
        out["textbook_strict"], out["textbook_frobenius"] = figures(tb)
    return out


def cpu_oracle_effective(n, levels, threads, reps=1):
    """Effective GFLOP/s of the oracle's textbook Strassen (OpenMP timing build) at n^3
    on `threads` host threads, best of `reps`."""
    import oracle
    import workloads as W
    A, B, C = W.uniform(n, n, 0), W.uniform(n, n, 1), W.uniform(n, n, 2)
    oracle.build_timing()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.strassen_timed(A, B, C, levels, threads)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return 2.0 * n ** 3 / best / 1e9, best


def cpu_baseline(levels):
    """The oracle on all host cores (4096^3) and on one core (2048^3)."""
    import oracle
    cores = oracle.host_cores()
    v, t = cpu_oracle_effective(CPU_SAMPLE_N, levels, cores)
    v1, t1 = cpu_oracle_effective(CPU_SAMPLE_N_1CORE, levels, 1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"m=n=k={CPU_SAMPLE_N} {levels}-level textbook Strassen (plain C, -O3, OpenMP over the rows "
                      f"of each classical leaf product) on {cores} host cores, {t:.1f} s",
            "one_core": {"value": v1, "unit": UNIT, "cores": 1,
                         "sample": f"m=n=k={CPU_SAMPLE_N_1CORE} {levels}-level textbook Strassen, 1 thread, "
                                   f"{t1:.1f} s"}}


def cpu_sweep():
    """1 core and all cores up to 4096, all cores at 8192: one line per row."""
    import oracle
    cores = oracle.host_cores()
    rows = []
    for n in (1024, 2048, 4096, 8192):
        for L in (0, 1, 2):
            for th in ((1, cores) if n <= 4096 else (cores,)):
                if th == 1 and n == 4096 and L == 0:
                    continue  # about a minute on one core; the 2-level row covers the size
                v, t = cpu_oracle_effective(n, L, th)
                row = {"n": n, "levels": L, "threads": th, "gflops": v, "seconds": t}
                print(json.dumps(row), flush=True)
                rows.append(row)
    return rows


# ---------------------------------------------------------------- GPU side sections

def bench_batched(sg, W, torch, reps=3):
    """256 FP64 problems, m, n, k log-uniform in [256, 4096] (seed 0), levels and block
    tiles chosen by the library, in one batched call captured in a CUDA graph; against
    a loop of 256 classical launches and a loop of 256 automatic single calls on the
    same operands."""
    shapes = W.loguniform_shapes(256, seed=0, lo=256, hi=4096)
    mats = [(W.uniform_device(m, k, 1000 + i), W.uniform_device(k, n, 2000 + i), W.uniform_device(m, n, 3000 + i))
            for i, (m, n, k) in enumerate(shapes)]
    arr = (sg.strassen_problem * len(mats))()
    for i, (A, B, C) in enumerate(mats):
        arr[i] = sg.strassen_problem(A.shape[0], B.shape[1], A.shape[1], A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                     A.stride(0), B.stride(0), C.stride(0), -1, sg.STRASSEN_AUTO)
    flops = sum(2.0 * m * n * k for (m, n, k) in shapes)
    stream = torch.cuda.current_stream()

    def graph_of(problems):
        assert sg.strassen_gemm_batched(len(mats), problems, 0, stream.cuda_stream) == 0
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            assert sg.strassen_gemm_batched(len(mats), problems, 0, torch.cuda.current_stream().cuda_stream) == 0
        g.replay()
        torch.cuda.synchronize()
        return g

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    g = graph_of(arr)
    t_graph = timed(g.replay)
    t_loop = timed(lambda: [sg.classical(A, B, C) for A, B, C in mats])
    t_auto = timed(lambda: [sg.gemm(A, B, C, levels=-1, variant="AUTO") for A, B, C in mats])
    # the same batched call with every problem classical: isolates the launch from the level choice
    for i in range(len(mats)):
        arr[i].levels = 0
        arr[i].variant = sg.STRASSEN_ABC
    g0 = graph_of(arr)
    t_graph0 = timed(g0.replay)
    return {"workload": "256 FP64 problems, m,n,k log-uniform in [256,4096] (seed 0), one batched call in a CUDA "
                        "graph, levels and tiles chosen by the library",
            "value": flops / t_graph / 1e9, "unit": UNIT, "ms": t_graph * 1e3,
            "all_classical_batched": {"value": flops / t_graph0 / 1e9, "ms": t_graph0 * 1e3},
            "loop_of_classical": {"value": flops / t_loop / 1e9, "ms": t_loop * 1e3, "launches": len(mats)},
            "loop_of_auto_calls": {"value": flops / t_auto / 1e9, "ms": t_auto * 1e3, "calls": len(mats)},
            "speedup_vs_loop": t_loop / t_graph}


def bench_syrk(sg, W, torch, n=8192, k=8192, reps=3):
    """The level-3 BLAS user: C = A A^T + C on the lower triangle (strassen_dsyrk) at
    n x k, effective GFLOP/s = n (n + 1) k / t (the flops of the triangle), with the
    selector's Strassen plans on the off-diagonal blocks and with classical products only
    (levels 0)."""
    A, C = W.uniform_device(n, k, 41), W.uniform_device(n, n, 42)
    s = torch.cuda.current_stream()
    out = {"workload": f"DSYRK lower, n={n}, k={k}, A, C uniform[-1,1], C += A A^T on the triangle"}
    for name, lv in (("auto", -1), ("two_levels", 2), ("classical", 0)):
        t = timed_calls(torch, lambda: sg.dsyrk(A, C, levels=lv, stream=s), reps, s)
        out[name] = {"value": n * (n + 1.0) * k / t / 1e9, "unit": UNIT, "ms": t * 1e3}
    del A, C
    torch.cuda.empty_cache()
    return out


def split_tensor_flops(m, n, k, L):
    """Tensor-core work of the slice products: 28 digit pairs x 2 h_mp h_np h_kp x 7^L
    (padded block edges: 128 rows of A, 256 columns of B, 64 of k)."""
    P = 1 << L

    def padded(d, q):
        h = -(-d // P)
        return -(-h // q) * q

    return 28 * 2.0 * padded(m, 128) * padded(n, 256) * padded(k, 64) * 7 ** L


def bench_split_precision(sg, W, torch, sizes=(8192, 16384), err_n=8192, reps=3, with_errors=True):
    """Split-precision FP64 emulation (BF16 digit slices on the tensor cores): effective
    GFLOP/s for 0, 1, 2 levels at each size, the per-stage times of one call
    (strassen_profile_split_precision) with the slice-product kernel's tensor-pipe
    fraction of the measured BF16 peak, and the errors against the exact product
    (Dot2-sampled, the CPU leg) for inputs u * 2^round(N(0, sigma)) at err_n^3."""
    import numpy as np
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    bf16_sustained = float(peaks.get("bf16_tflops_sustained", bf16))
    out = {"workload": "m=n=k in {8192, 16384} FP64 via BF16 digit slices, A,B,C uniform[-1,1]", "sizes": {}}
    stream = torch.cuda.current_stream()
    for n in sizes:
        A, B, C = W.uniform_device(n, n, 11), W.uniform_device(n, n, 12), W.uniform_device(n, n, 13)
        row = {}
        for L in (0, 1, 2):
            t = timed_calls(torch, lambda: sg.gemm(A, B, C, levels=L, dtype="oz_bf16", stream=stream), reps, stream)
            ms = sg.strassen_profile_split_precision(n, n, n, A.data_ptr(), n, B.data_ptr(), n, C.data_ptr(), n, L,
                                                     stream.cuda_stream)
            tf = split_tensor_flops(n, n, n, L) / (ms[1] / 1e3) / 1e12
            # a slice-product launch of 100 ms or more, one of a run of such calls, runs
            # under the power cap: its denominator is the sustained peak
            long_launch = ms[1] >= 100.0
            peak = bf16_sustained if long_launch else bf16
            row[str(L)] = {"value": 2.0 * n ** 3 / t / 1e9, "unit": UNIT, "ms": t * 1e3,
                           "stage_ms": {"splits": ms[0], "slice_products": ms[1], "recombine_scatter": ms[2]},
                           "oz_gemm_roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                                "frac": tf / peak, "frac_of_burst": tf / bf16,
                                                "peak_note": "measured BF16 dense peak (%s), MEASURED_PEAKS.json"
                                                % ("sustained" if long_launch else "burst")}}
        out["sizes"][str(n)] = row
        del A, B, C
        torch.cuda.empty_cache()
    if with_errors:
        import oracle
        errs = {}
        rows, cols = W.sample_indices(err_n, err_n, 2048, 5)
        ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
        for sigma in (0, 4, 10):
            Ah, Bh = W.scaled(err_n, err_n, 21, sigma), W.scaled(err_n, err_n, 22, sigma)
            A, B = torch.from_numpy(Ah).cuda(), torch.from_numpy(Bh).cuda()
            # CPU leg: the exact entries (Dot2, rounded once)
            exact = oracle.gemm_sampled(Ah, Bh, None, rows, cols)
            den = float(np.max(np.abs(Ah))) * float(np.max(np.abs(Bh)))
            den_norm = float(np.max(np.sum(np.abs(Ah), axis=1))) * float(np.max(np.abs(Bh)))
            fro_den = float(np.linalg.norm(Ah)) * float(np.linalg.norm(Bh))

            def figures(vals):
                e = np.abs(vals - exact)
                return {"strict": float(np.max(e)) / den, "normwise": float(np.max(e)) / den_norm,
                        "frobenius": float(np.sqrt(err_n * err_n * np.mean(e * e))) / fro_den}

            per = {}
            for L, dt in ((0, "f64"), (0, "oz_bf16"), (1, "oz_bf16"), (2, "oz_bf16")):
                Cz = torch.zeros((err_n, err_n), dtype=torch.float64, device="cuda")
                sg.gemm(A, B, Cz, levels=L, dtype=dt)
                got = Cz[ri, ci].cpu().numpy()
                del Cz
                per["fp64_classical" if dt == "f64" else str(L)] = figures(got)
            errs[str(sigma)] = per
            del A, B
        out["error_vs_exact"] = {"n": err_n, "samples": int(rows.size), "by_sigma_then_levels": errs,
                                 "norms": "strict: max|C - C_exact| / (max|A| max|B|); normwise: / (||A||_inf max|B|); "
                                          "frobenius: ||C - C_exact||_F / (||A||_F ||B||_F), numerator from the "
                                          "samples; C_exact from Dot2 (the CPU leg)"}
    return out


def bench_other_levels(sg, torch, W, n, levels_list, variant="ABC", reps=3, accuracy=True):
    """The same product at n^3 with other level counts on their own resident inputs
    (seeds 100-102, uniform[-1, 1], accumulate mode): effective GFLOP/s and FP64-pipe
    fraction (CUDA events per call), and the sampled strict error of one call next to
    the textbook Strassen's."""
    Ah, Bh, Ch = W.uniform(n, n, 100), W.uniform(n, n, 101), W.uniform(n, n, 102)
    A, B, C0 = torch.from_numpy(Ah).cuda(), torch.from_numpy(Bh).cuda(), torch.from_numpy(Ch).cuda()
    C = C0.clone()  # the timed calls accumulate into C; the error checks start from C0
    stream = torch.cuda.current_stream()
    rows, cols = W.sample_indices(n, n, ERR_SAMPLES // 2, 7)
    ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    out = {}
    for lv in levels_list:
        err = None
        if accuracy:
            C1 = C0.clone()
            sg.gemm(A, B, C1, levels=lv, variant=variant, stream=stream)
            got = C1[ri, ci].cpu().numpy()
            del C1
            err = cpu_leg_errors(Ah, Bh, Ch, got, rows, cols, lv)
        t = timed_calls(torch, lambda: sg.gemm(A, B, C, levels=lv, variant=variant, stream=stream), reps, stream)
        alg = algorithmic_flops(n, n, n, lv) / t / 1e9
        out[str(lv)] = {"value": 2.0 * n ** 3 / t / 1e9, "unit": UNIT, "ms": t * 1e3, "n": n,
                        "variant": variant, "algorithmic_gflops": alg, "frac": alg / FP64_PEAK_GFLOPS,
                        "error": err}
    del A, B, C, C0
    torch.cuda.empty_cache()
    return out


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
    cores = oracle.host_cores()
    A, B, C = W.uniform(n, n, 0), W.uniform(n, n, 1), W.uniform(n, n, 2)
    oracle.build_timing()
    for _ in range(args.warmup):
        oracle.strassen_timed(A, B, C, args.levels, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.strassen_timed(A, B, C, args.levels, cores)
    dt = time.perf_counter() - t0
    val = 2.0 * n ** 3 * args.steps / dt / 1e9
    sample = (f"m=n=k={n} {args.levels}-level textbook Strassen per step (oracle, plain C, -O3, OpenMP over the rows "
              f"of each classical leaf product, {cores} host cores)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"square m=n=k={args.n} FP64 {args.levels}-level {args.variant} Strassen, C += A*B"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_sweep:
        cpu_sweep()
        return 0
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
    # The shipped learned selector, loaded as a user of the package loads it: every
    # automatic plan below (levels -1, AUTO) is its choice where it is enabled (FP64).
    from paper_1605_01078_gb300 import tune
    selector = tune.load_default_selector()
    Ah, Bh, Ch = W.uniform(m, k, 100 + rank), W.uniform(k, n, 200 + rank), W.uniform(m, n, 300 + rank)
    A, B, C = torch.from_numpy(Ah).cuda(), torch.from_numpy(Bh).cuda(), torch.from_numpy(Ch).cuda()
    stream = torch.cuda.current_stream()

    def step():
        sg.gemm(A, B, C, levels=L, variant=variant, dtype=args.dtype, stream=stream)

    launches_per_step = 1 if (L == 0 or variant.upper() == "ABC") else None
    if args.dtype == "oz_bf16":
        launches_per_step = 5  # split rows, column maxima, split columns, slice products, recombine + scatter
    elif launches_per_step is None:
        nprod = 7 ** L
        launches_per_step = nprod * (2 if variant.upper() == "AB" else 4)

    # Accuracy of one call from the initial C (sampled entries; the CPU leg computes the
    # exact and the textbook entries), before the timed steps change C.
    accuracy = None
    if not args.no_accuracy and rank == 0:
        rows, cols = W.sample_indices(m, n, ERR_SAMPLES, 7)
        ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
        C1 = C.clone()
        sg.gemm(A, B, C1, levels=L, variant=variant, dtype=args.dtype, stream=stream)
        got = C1[ri, ci].cpu().numpy()
        del C1
        accuracy = {"one_call": got}

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

    # Comparators on the same inputs: the library's classical kernel, and the same call
    # with STRASSEN_FLAG_DETERMINISTIC (owner schedule: bitwise repeatable).
    cls_t = timed_calls(torch, lambda: sg.classical(A, B, C, stream=stream), 2, stream)
    cls_val = eff_flops / cls_t / 1e9
    det = None
    if args.dtype == "f64" and L > 0:
        det_t = timed_calls(torch, lambda: sg.gemm(A, B, C, levels=L, variant=variant, stream=stream,
                                                   deterministic=True), 2, stream)
        det = {"value": eff_flops / det_t / 1e9, "unit": UNIT, "ms": det_t * 1e3,
               "flag": "STRASSEN_FLAG_DETERMINISTIC (owner schedule)"}

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
                sg.gemm(dA, dB, dC, levels=L, variant=variant, dtype=args.dtype, stream=stream)
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
        del bufs, hA, hB, hC, hOut
    del A, B, C
    torch.cuda.empty_cache()

    levels_other = None
    small = None
    if not args.no_levels and args.dtype == "f64" and rank == 0:
        levels_other = bench_other_levels(sg, torch, W, 8192, [1, 2, 3], accuracy=not args.no_accuracy)
        # the small square case: m = n = k = 1024, one-level ABC, C = 0
        As, Bs = W.uniform_device(1024, 1024, 0), W.uniform_device(1024, 1024, 1)
        Cs = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
        small = {"workload": "m=n=k=1024, one-level ABC, C = 0 (uniform[-1,1])"}
        t = timed_calls(torch, lambda: sg.gemm(As, Bs, Cs, levels=1, stream=stream), 20, stream)
        small.update({"value": 2.0 * 1024 ** 3 / t / 1e9, "unit": UNIT, "ms": t * 1e3,
                      "frac": algorithmic_flops(1024, 1024, 1024, 1) / t / 1e9 / FP64_PEAK_GFLOPS})
        del As, Bs, Cs

    batched = None
    if not args.no_batched and rank == 0:
        batched = bench_batched(sg, W, torch)
    syrk = None
    if not args.no_levels and args.dtype == "f64" and rank == 0:
        syrk = bench_syrk(sg, W, torch)
    split = None
    if not args.no_split and rank == 0:
        split = bench_split_precision(sg, W, torch, with_errors=not args.no_accuracy)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    if accuracy is not None:
        accuracy = cpu_leg_errors(Ah, Bh, Ch, accuracy["one_call"], rows, cols, L if args.dtype == "f64" else 0)
    alg = algorithmic_flops(m, n, k, L)
    launch_s = statistics.mean(per_launch)
    achieved = alg / launch_s / 1e9
    if args.dtype == "oz_bf16":
        mma = split_tensor_flops(m, n, k, L) / launch_s / 1e12
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"bound": "tensor", "achieved": mma, "peak": bf16, "unit": "TFLOP/s", "frac": mma / bf16,
                "traffic": None, "kernel": "whole split-precision call (split, oz_gemm, recombine)",
                "peak_note": "measured BF16 dense peak (burst); per call, not per kernel"}
    else:
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": recorded_traffic(m, L, variant) if m == n == k else None,
                "algorithmic_bytes": algorithmic_bytes(m, n, k, L),
                "kernel": "fp64_strassen_kernel",
                "peak_note": "FP64 pipe: 4 flop/clk/SM x 152 SMs x 2070 MHz (derived); DFMA probe measured 1200 GFLOP/s"}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(L)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"square m=n=k={m} FP64 {L}-level {variant} Strassen, C += A*B (accumulate), "
                               f"A,B,C uniform[-1,1]" + (" (products as BF16 digit slices)" if args.dtype != "f64" else ""),
                   "m": m, "n": n, "k": k, "levels": L, "variant": variant, "products": args.dtype,
                   "parallelism": f"replicas{ws}", "l2": "inputs larger than L2 (3 x 8 m n bytes)"},
        "classical": {"value": cls_val, "unit": UNIT, "speedup": value / ws / cls_val},
        "deterministic": det,
        "error": accuracy,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "other_levels": levels_other,
        "small_square": small,
        "batched": batched,
        "syrk": syrk,
        "split_precision": split,
        "selector": {"loaded": "shipped network (data/selector_gb300.json)",
                     "enabled_for": [name for d, name in ((0, "f64"), (2, "oz_bf16"))
                                     if selector["use_for_dtype"].get(str(d))]},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def algorithmic_bytes(m, n, k, levels):
    """Minimum HBM bytes of one ABC launch with every operand term read once per product
    and every C update a read and a write: 3^L (mk + kn) 8 B + 3^L mn 16 B (the table
    has 12^L terms per operand over 4^L blocks, 3^L blocks' worth per product family)."""
    return 3 ** levels * (m * k + k * n) * 8.0 + 3 ** levels * m * n * 16.0


if __name__ == "__main__":
    sys.exit(main())

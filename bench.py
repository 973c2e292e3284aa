"""Benchmark of the FP32-accurate GEMM path on one GB300 (or N replicas).

One step = one call g3_gemm(F32_3XBF16) on the square FP32 problem
m = n = k = 16384, alpha = 1, beta = 0.5, uniform [-1, 1] inputs from seed 0:
the hi/lo split pre-pass of both operands (packing) followed by one persistent
tcgen05 kernel (blocking, TMA staging, 3 MMAs per k-step, alpha/beta epilogue).
The inputs (1 GiB per operand) exceed the 129 MB L2, so no flush is needed
between steps.  The plain FP32 SIMT kernel is timed on the same problem for the
speedup, and both results are checked on sampled rows against the binary64
oracle.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--size S] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the problem has
no exchange step): value = total flops of all ranks / max elapsed over ranks.
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

METRIC = "GEMM TFLOPS & % dtype peak; 3xBF16-FP32 vs SIMT-FP32 speedup at equal error"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
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
        os.unlink(self.f.name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sample(p, target_s=12.0, max_rows=4096):
    """Time the binary64 oracle on a bounded sample: whole rows of C."""
    import oracle
    A64 = p.A.astype(np.float64)
    B64 = p.B.astype(np.float64)
    rows = 16
    t0 = time.perf_counter()
    oracle.gemm(A64[:rows], B64, None, 1.0, 0.0)
    dt = time.perf_counter() - t0
    more = int(min(max_rows, max(rows, rows * (target_s / max(dt, 1e-3)))))
    sel = np.arange(rows, rows + more) % p.m
    t0 = time.perf_counter()
    oracle.gemm(A64, B64, p.C, p.alpha, p.beta, rows=sel)
    dt = time.perf_counter() - t0
    flops = 2.0 * more * p.n * p.k
    return {"value": flops / dt / 1e12, "unit": "TFLOPS", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{more} full rows of C of the {p.m}x{p.n}x{p.k} problem, binary64, {dt:.1f} s"}


def square_config(n):
    """The headline workload's config object, identical in both arms."""
    return {"workload": f"square FP32 GEMM m=n=k={n}, alpha=1, beta=0.5, uniform [-1,1], seed 0",
            "l2": "inputs 1 GiB/operand > L2, no flush", "flops_per_step": 2.0 * n * n * n}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the same workload.

    Each step computes a bounded sample of whole rows of C -- by default 8 rows
    per host thread, so that every core has several rows and the oracle runs
    at the rate the cpu_baseline leg of the GPU arm reports."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2310_20347_gb300 import synth
    import oracle
    oracle.build()
    p = synth.uniform_problem(args.size, args.size, args.size, seed=0, alpha=1.0, beta=0.5)
    A64 = p.A.astype(np.float64)
    B64 = p.B.astype(np.float64)
    cores = oracle.max_threads()
    rows_per_step = args.ref_rows if args.ref_rows > 0 else 8 * cores
    for w in range(args.warmup):
        oracle.gemm(A64, B64, p.C, 1.0, 0.5, rows=np.arange(rows_per_step) % p.m)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.gemm(A64, B64, p.C, 1.0, 0.5, rows=(np.arange(rows_per_step) + s * rows_per_step) % p.m)
    dt = time.perf_counter() - t0
    flops = 2.0 * rows_per_step * p.n * p.k * args.steps
    val = flops / dt / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": square_config(args.size),
            "method": "binary64 CPU oracle (plain triple loop, OpenMP over rows of C)",
            "cpu_baseline": {"value": val, "unit": "TFLOPS", "cores": cores, "kind": "oracle",
                             "sample": f"{rows_per_step} full rows of C per step ({rows_per_step // max(cores, 1)} "
                                       f"per host thread), binary64"},
            "e2e": {"value": val, "unit": "TFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Dense tensor peaks of GB300 from NVIDIA's datasheet (per GPU, no sparsity),
# reported beside the measured-peak fractions.
NOMINAL_TFLOPS = {"bf16": 2250.0, "fp8": 4500.0, "tf32": 1125.0}

# Sources of the headline kernel (its device code and launcher).  A
# DRAM-traffic record taken with ncu is reported as the roofline's "traffic"
# only while these files hash to the recorded value and the member and size
# match the record.
TRAFFIC_SOURCES = ("csrc/tc_gemm.cuh", "csrc/ptx.cuh", "csrc/sched.cuh", "csrc/tc_family_tu.cuh",
                   "csrc/tc_family_3xbf16.cu", "csrc/api.cu")
TRAFFIC_RECORD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                              "tc_gemm_3xbf16_16384_dram.md")


def kernel_sources_hash():
    """SHA-256 of the headline kernel's sources with comments and whitespace
    removed: the code the DRAM-traffic record was taken with."""
    import hashlib
    import re
    pkg = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2310_20347_gb300")
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(pkg, rel)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def recorded_traffic(member, n):
    """DRAM bytes per launch from the ncu record, or (None, why)."""
    try:
        text = open(TRAFFIC_RECORD).read()
    except OSError:
        return None, "no ncu record"
    rec = {}
    for line in text.splitlines():
        if ":" in line and line.split(":", 1)[0].strip() in ("member", "size", "sources_sha256",
                                                             "dram_bytes_per_launch"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("member") != member or rec.get("size") != str(n):
        return None, "ncu record is for another member or size"
    if rec.get("sources_sha256") != kernel_sources_hash():
        return None, "kernel sources changed since the ncu record"
    return float(rec["dram_bytes_per_launch"]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _kernel_ms(lib, fn, reps, flush):
    """Mean device time of the library's main kernel over `reps` calls of fn,
    with an L2 flush (a write larger than L2) before every call."""
    import torch
    lib.g3_kernel_timing(True)
    lib.g3_kernel_time_ms(reset=True)
    for _ in range(reps):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    ms, n = lib.g3_kernel_time_ms(reset=True)
    lib.g3_kernel_timing(False)
    return ms / max(n, 1)


def _rotating_graph_ms(calls, nrep):
    """Mean device time per call of `calls` (one per rotating operand set, each
    already run once) issued back to back from a CUDA graph."""
    import torch
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for i in range(nrep):
                calls[i % len(calls)]()
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / nrep


def _traffic_floor_ms(lib, read_bytes, write_bytes, nrep=None):
    """Per-call time of the library's streaming yardstick moving read_bytes in
    and write_bytes out in the same proportion (g3_stream_traffic), back to
    back from a CUDA graph over rotating buffers that together exceed 4x L2:
    the floor of any kernel with that memory traffic."""
    import torch
    r16, w16 = -(-int(read_bytes) // 16) * 16, -(-int(write_bytes) // 16) * 16
    sets = max(2, min(64, -(-(512 << 20) // (r16 + w16))))
    bufs = [(torch.empty(r16, dtype=torch.uint8, device="cuda"), torch.empty(w16, dtype=torch.uint8, device="cuda"))
            for _ in range(sets)]
    calls = [lambda a=a, b=b: lib.g3_stream_traffic(a.data_ptr(), r16, b.data_ptr(), w16,
                                                    torch.cuda.current_stream().cuda_stream) for a, b in bufs]
    for c in calls:
        assert c() == 0
    torch.cuda.synchronize()
    ms = _rotating_graph_ms(calls, nrep or max(40, 2 * sets))
    del bufs
    return ms


def _call_ms(fn, reps, flush):
    """Mean device time of whole calls (all their launches), L2 flushed between."""
    import torch
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0, e1 = _events()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


# When a list, _line appends each workload's result here instead of printing
# it (the default run collects the other configurations into its own line).
_COLLECT = None


def _line(args, metric_value, unit, config, extra):
    line = {"metric": METRIC, "value": metric_value, "unit": unit, "n_gpus": 1, "steps": args.reps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic", "config": config}
    line.update(extra)
    if _COLLECT is not None:
        _COLLECT.append(line)
        return
    print(json.dumps(line), flush=True)


def _stored(A, B, which):
    """A and B as the GEMM reads them: stored transposed where `which` names
    them ('a', 'b', 'ab'), with the matching trans_a / trans_b flags."""
    ta, tb = "a" in which, "b" in which
    return (A.t().contiguous() if ta else A, B.t().contiguous() if tb else B, {"trans_a": ta, "trans_b": tb})


def run_workload(args):
    """The non-headline configurations, one JSON line each."""
    import torch

    import oracle
    import paper_2310_20347_gb300 as pkg
    from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_F64, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_INT16, G3_TF32, _lib, synth,
                                        torch_api)
    torch.cuda.set_device(0)
    pkg.load()
    peaks, peak_src = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    bf16_peak = float(peaks["bf16_tflops"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dev = "cuda"

    def sample_err(got_rows, rows, A, B, C, alpha, beta, quantA=None, quantB=None):
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        ref = oracle.gemm(A64, B64, C, alpha, beta, rows=rows)
        D = oracle.absprod(A64, B64, alpha, rows=rows)
        if C is not None and beta != 0.0:
            D = D + np.abs(beta * C[rows].astype(np.float64))
        e = {"gate": float(np.max(np.abs(got_rows - ref) / np.maximum(D, 1e-300)))}
        if quantA is not None:
            Aq, Bq = quantA.astype(np.float64), quantB.astype(np.float64)
            refq = oracle.gemm(Aq, Bq, C, alpha, beta, rows=rows)
            Dq = oracle.absprod(Aq, Bq, alpha, rows=rows)
            e["kernel"] = float(np.max(np.abs(got_rows - refq) / np.maximum(Dq, 1e-300)))
        return e

    if args.workload == "plain":
        # the plain method alone: FP32 SIMT C := A*B at m = n = k = 512 (uniform
        # [-1, 1], seed 0, beta = 0), every element checked against the
        # binary64 oracle; FFMA-bound, so the roofline is the FP32 CUDA-core rate
        n = 512
        p = synth.uniform_problem(n, n, n, seed=0)
        A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
        C = torch.empty(n, n, dtype=torch.float32, device=dev)
        fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_F32)
        fn()
        torch.cuda.synchronize()
        got = C.cpu().numpy().astype(np.float64)
        A64, B64 = p.A.astype(np.float64), p.B.astype(np.float64)
        t0 = time.perf_counter()
        ref = oracle.gemm(A64, B64, None, 1.0, 0.0)
        cpu_s = time.perf_counter() - t0
        err = float(np.max(np.abs(got - ref) / np.maximum(oracle.absprod(A64, B64, 1.0), 1e-300)))
        for _ in range(args.warmup):
            fn()
        ms = _call_ms(fn, args.reps, flush)
        kms = _kernel_ms(_lib, fn, args.reps, flush)
        flops = 2.0 * n ** 3
        _, _, splits, _ = _lib.g3_plan_query(n, n, n, G3_F32)
        sm_mhz = 2070.0
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        _line(args, flops / ms / 1e9, "TFLOPS",
              {"workload": "plain FP32 GEMM C := A*B, m=n=k=512, uniform [-1, 1], seed 0, beta=0",
               "path": f"FP32 SIMT kernel (the plain method): 64 x 64 CTA tiles, 4 x 4 micro-tiles, k cut over a "
                       f"cluster of {splits} CTAs summed through distributed shared memory",
               "flush": "256 MB L2 flush before every call"},
              {"dtype": "f32", "ms": ms, "kernel_ms": kms, "err": {"gate_all_elements": err},
               "roofline": {"bound": "alu", "achieved": flops / kms / 1e9, "peak": fp32_peak, "unit": "TFLOP/s",
                            "frac": flops / kms / 1e9 / fp32_peak, "traffic": None,
                            "peak_source": "152 SMs x 128 FP32 FMA/clock x 2 x 2.07 GHz (maximum SM clock)",
                            "algorithmic": "2 n^3 FP32 flops per call"},
               "cpu_baseline": {"value": flops / cpu_s / 1e12, "unit": "TFLOPS", "cores": oracle.max_threads(),
                                "kind": "oracle", "sample": f"the whole 512^3 product in binary64, {cpu_s:.3f} s"}})
        return

    if args.workload == "simt":
        # the plain method alone at m = n = k = dsize (uniform [-1, 1], seed 0,
        # beta 0): the FP32 SIMT kernel on the CUDA cores, L2 flushed between calls
        n = args.dsize
        p = synth.uniform_problem(n, n, n, seed=0)
        A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
        C = torch.empty(n, n, dtype=torch.float32, device=dev)
        fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_F32, config=args.config)
        fn()
        torch.cuda.synchronize()
        rows = np.array([0, n // 2, n - 1])
        err = sample_err(C[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64), rows, p.A, p.B, None,
                         1.0, 0.0)
        for _ in range(args.warmup):
            fn()
        kms = _kernel_ms(_lib, fn, args.reps, flush)
        flops = 2.0 * n ** 3
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        _line(args, flops / kms / 1e9, "TFLOPS",
              {"workload": f"plain FP32 GEMM m=n=k={n}, uniform [-1, 1], seed 0, beta=0",
               "path": "FP32 SIMT kernel (the plain method)", "flush": "256 MB L2 flush before every call"},
              {"dtype": "f32", "kernel_ms": kms, "err": err,
               "roofline": {"bound": "alu", "achieved": flops / kms / 1e9, "peak": fp32_peak, "unit": "TFLOP/s",
                            "frac": flops / kms / 1e9 / fp32_peak, "traffic": None,
                            "peak_source": "152 SMs x 128 FP32 FMA/clock x 2 x 2.07 GHz (maximum SM clock)",
                            "algorithmic": "2 n^3 FP32 flops per call"}})
        return

    if args.workload == "streamk":
        # Stream-K tail (split_k = G3_SPLIT_STREAM_K) against the plain walk on
        # shapes whose tiles leave the last wave partly idle: whole calls (L2
        # flushed between them) and the GEMM kernel alone
        from paper_2310_20347_gb300 import G3_SPLIT_STREAM_K
        out = []
        for kind, n in (("3xbf16", 2048), ("bf16", 4096), ("int8", 8192)):
            g = torch.Generator(device=dev).manual_seed(n)
            if kind == "3xbf16":
                A = torch.rand(n, n, device=dev, generator=g) * 2 - 1
                B = torch.rand(n, n, device=dev, generator=g) * 2 - 1
                C = torch.rand(n, n, device=dev, generator=g) * 2 - 1
                dt, alpha, beta = G3_F32_3XBF16, 1.0, 0.5
            elif kind == "bf16":
                A = torch.randn(n, n, device=dev, generator=g).bfloat16()
                B = torch.randn(n, n, device=dev, generator=g).bfloat16()
                C = torch.empty(n, n, device=dev)
                dt, alpha, beta = G3_BF16, 1.0, 0.0
            else:
                A = torch.randint(-128, 128, (n, n), dtype=torch.int8, device=dev, generator=g)
                B = torch.randint(-128, 128, (n, n), dtype=torch.int8, device=dev, generator=g)
                C = torch.empty(n, n, dtype=torch.int32, device=dev)
                dt, alpha, beta = G3_INT8, 1, 0
            st, cfg, _, _ = _lib.g3_plan_query(n, n, n, dt)
            res = {"kind": kind, "n": n, "member": _lib.g3_family_describe(cfg)}
            for name, sk in (("plain", 1), ("stream_k", G3_SPLIT_STREAM_K)):
                fn = lambda: torch_api.gemm(A, B, C, alpha, beta, dtype=dt, split_k=sk)
                for _ in range(args.warmup):
                    fn()
                ms = _call_ms(fn, args.reps, flush)
                _lib.g3_kernel_timing(True)
                _lib.g3_kernel_time_ms(reset=True)
                for _ in range(args.reps):
                    flush.zero_()
                    fn()
                torch.cuda.synchronize()
                kms, kn = _lib.g3_kernel_time_ms(reset=True)
                _lib.g3_kernel_timing(False)
                res[name] = {"call_ms": ms, "gemm_kernel_ms": kms / max(kn, 1)}
            res["call_ratio"] = res["plain"]["call_ms"] / res["stream_k"]["call_ms"]
            out.append(res)
            del A, B, C
            torch.cuda.empty_cache()
        _line(args, out[0]["call_ratio"], "x",
              {"workload": "stream-K tail vs plain tile walk: FP32-accurate 2048^3 (beta 0.5), BF16 4096^3, "
                           "INT8 8192^3; planner's member, L2 flushed between calls"},
              {"dtype": "mixed", "cases": out})
        return

    if args.workload == "sweep":
        out = []
        for n in synth.SQUARE_SWEEP:
            p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C0 = torch.from_numpy(p.C).to(dev)
            C = C0.clone()
            rows = np.array([0, n // 2, n - 1])
            res = {"n": n}
            for name, dt in (("3xbf16", G3_F32_3XBF16), ("simt", G3_F32)):
                C.copy_(C0)
                torch_api.gemm(A, B, C, 1.0, 0.5, dtype=dt)
                torch.cuda.synchronize()
                got = C[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
                err = sample_err(got, rows, p.A, p.B, p.C, 1.0, 0.5)["gate"]
                reps = max(2, min(args.reps, 3 if (dt == G3_F32 and n >= 8192) else args.reps))
                for _ in range(2):
                    torch_api.gemm(A, B, C, 1.0, 0.5, dtype=dt)
                ms = _call_ms(lambda: torch_api.gemm(A, B, C, 1.0, 0.5, dtype=dt), reps, flush)
                res[name] = {"ms": ms, "tflops": 2.0 * n ** 3 / ms / 1e9, "rel_err": err}
            res["speedup"] = res["simt"]["ms"] / res["3xbf16"]["ms"]
            out.append(res)
            del A, B, C, C0
            torch.cuda.empty_cache()
        _line(args, out[-1]["3xbf16"]["tflops"], "TFLOPS",
              {"workload": "square FP32 sweep m=n=k in 1024..16384, alpha=1, beta=0.5, uniform [-1,1], "
                           "3xBF16 vs SIMT (whole calls incl. the split pre-pass), L2 flushed between calls"},
              {"dtype": "f32", "sweep": out})
        return

    if args.workload in ("im2col", "im2col-fp8", "im2col-int8"):
        kind = {"im2col": "bf16", "im2col-fp8": "fp8", "im2col-int8": "int8"}[args.workload]
        shapes = [(f"L{l}", m, n, k) for (l, m, n, k) in synth.im2col_shapes(16)]
        shapes += [(f"b1:{m}x{n}x{k}", m, n, k) for (m, n, k) in synth.IM2COL_BATCH1_EXAMPLES]
        if args.only:
            shapes = [s for s in shapes if s[0] in args.only.split(",")]
        per, tot_ms, tot_bytes, tot_flops, worst, tot_floor = [], 0.0, 0.0, 0.0, {}, 0.0
        tuned = {}
        if args.tune:
            # per-shape selection (the paper's Section 8.4 search): time every
            # family member x split-K for each layer shape before measuring it
            g3dt = {"bf16": G3_BF16, "fp8": G3_FP8_E4M3, "int8": G3_INT8}[kind]
            _lib.g3_tune_cache_clear()
            for (name, m, n, k) in shapes:
                st, cfg, sk, tms = _lib.g3_autotune(m, n, k, g3dt)
                tuned[name] = {"member": cfg, "split_k": sk, "ms": tms, "status": st}
        for li, (name, m, n, k) in enumerate(shapes):
            seed = li + 1
            if kind == "int8":
                p = synth.int8_problem(m, n, k, seed=seed)
                A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
                C = torch.empty(m, n, dtype=torch.int32, device=dev)
                fn = lambda: torch_api.gemm(A, B, C, 1, 0, dtype=G3_INT8)
                esz, csz = 1, 4
            else:
                p = synth.normal_problem(m, n, k, seed=seed)
                A32, B32 = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
                C = torch.empty(m, n, dtype=torch.float32, device=dev)
                if kind == "bf16":
                    A, B = torch_api.convert_bf16(A32), torch_api.convert_bf16(B32)
                    fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_BF16)
                    esz = 2
                else:
                    (A, sa), (B, sb) = torch_api.quantize_fp8(A32), torch_api.quantize_fp8(B32)
                    fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=sa, scale_b=sb)
                    esz = 1
                del A32, B32
                csz = 4
            fn()
            torch.cuda.synchronize()
            rows = np.array([0, m // 2, m - 1])
            got = C[torch.from_numpy(rows).to(dev)].cpu().numpy()
            if kind == "int8":
                ref = oracle.gemm_i8(p.A, p.B, rows=rows)
                err = {"exact": bool(np.array_equal(got.astype(np.int64), ref))}
            elif kind == "bf16":
                err = sample_err(got.astype(np.float64), rows, p.A, p.B, None, 1.0, 0.0,
                                 oracle.round_bf16(p.A), oracle.round_bf16(p.B))
            elif args.compact:
                # the gate only: the kernel check against the oracle's own
                # quantisation of every operand is the parity tests' job
                err = sample_err(got.astype(np.float64), rows, p.A, p.B, None, 1.0, 0.0)
            else:
                oqa, osa = oracle.fp8_quantize(p.A)
                oqb, osb = oracle.fp8_quantize(p.B)
                err = sample_err(got.astype(np.float64), rows, p.A, p.B, None, 1.0, 0.0,
                                 oracle.e4m3_decode(oqa).astype(np.float64) * osa,
                                 oracle.e4m3_decode(oqb).astype(np.float64) * osb)
            for _ in range(args.warmup):
                fn()
            nbytes = esz * (m * k + k * n) + csz * m * n
            # Rotating copies of the operands, together >= 4x L2, called back to
            # back: every call reads inputs that left L2 long ago, and no other
            # kernel runs between the GEMMs (as in a network's layer sequence).
            sets = max(1, min(64, -(-(512 << 20) // nbytes)))
            copies = [(A.clone(), B.clone(), torch.empty_like(C)) for _ in range(sets - 1)] + [(A, B, C)]
            if kind == "int8":
                calls = [lambda a=a, b=b, c=c: torch_api.gemm(a, b, c, 1, 0, dtype=G3_INT8) for a, b, c in copies]
            elif kind == "bf16":
                calls = [lambda a=a, b=b, c=c: torch_api.gemm(a, b, c, 1.0, 0.0, dtype=G3_BF16)
                         for a, b, c in copies]
            else:
                calls = [lambda a=a, b=b, c=c: torch_api.gemm(a, b, c, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=sa,
                                                              scale_b=sb) for a, b, c in copies]
            nrep = max(args.reps, 2 * sets)
            for i in range(sets):
                calls[i]()
            torch.cuda.synchronize()
            # kernel-only device time (events around each GEMM kernel), eager calls
            kms = None
            if not args.compact:
                _lib.g3_kernel_timing(True)
                _lib.g3_kernel_time_ms(reset=True)
                for i in range(nrep):
                    calls[i % sets]()
                torch.cuda.synchronize()
                kms_tot, kn = _lib.g3_kernel_time_ms(reset=True)
                _lib.g3_kernel_timing(False)
                kms = kms_tot / max(kn, 1)
            # whole calls back to back, replayed from a CUDA graph (no host
            # overhead between the GEMMs, as in a captured network)
            gs = torch.cuda.Stream()
            gs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(gs):
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=gs):
                    for i in range(nrep):
                        calls[i % sets]()
            torch.cuda.synchronize()
            graph.replay()
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / nrep
            del graph
            # cold single call after an L2 flush, for reference
            cold_ms = None if args.compact else _call_ms(fn, 5, flush)
            del copies, calls
            flops = 2.0 * m * n * k
            st, cfg, sk, rs = _lib.g3_plan_query(m, n, k, {"bf16": G3_BF16, "fp8": G3_FP8_E4M3,
                                                           "int8": G3_INT8}[kind])
            # the same bytes, in the same read/write proportion, through the
            # streaming yardstick: the floor of this layer's memory traffic
            floor_ms = _traffic_floor_ms(_lib, esz * (m * k + k * n), csz * m * n)
            per.append({"shape": name, "m": m, "n": n, "k": k, "ms": ms, "kernel_ms": kms, "cold_call_ms": cold_ms,
                        "rotating_sets": sets,
                        "tflops": flops / ms / 1e9, "gbs": nbytes / ms / 1e6, "hbm_frac": nbytes / ms / 1e6 / hbm,
                        "traffic_floor_ms": floor_ms, "frac_of_traffic_floor": floor_ms / ms,
                        "member": _lib.g3_family_describe(cfg) if cfg >= 0 else None, "split_k": sk, "err": err})
            if name.startswith("L"):
                tot_ms += ms
                tot_bytes += nbytes
                tot_flops += flops
                tot_floor += floor_ms
            for kk, v in err.items():
                worst[kk] = (worst.get(kk, 0.0) if kk != "exact" else True)
                worst[kk] = (worst[kk] and v) if kk == "exact" else max(worst[kk], v)
            del A, B, C
            torch.cuda.empty_cache()
        gbs = tot_bytes / tot_ms / 1e6
        _line(args, tot_flops / tot_ms / 1e9, "TFLOPS",
              {"workload": f"20 ResNet50 v1.5 im2col GEMMs (Table 1 transposed, batch 16) + 3 batch-1 layers, "
                           f"{kind} inputs, {'int32' if kind == 'int8' else 'fp32'} C, alpha=1, beta=0; "
                           f"whole calls, back to back, replayed from a CUDA graph (ms); kernel_ms: the GEMM "
                           f"kernel alone (CUDA events, eager)",
               "l2": "rotating operand copies, together >= 512 MiB (4x L2), per shape; cold_call_ms: one "
                     "call after a 256 MiB L2 flush"},
              {"dtype": kind, "total_ms_20_layers": tot_ms, "worst_err": worst, "autotuned": bool(args.tune),
               "traffic_floor_ms_20_layers": tot_floor,
               "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                            "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
                            "frac_of_traffic_floor": tot_floor / tot_ms,
                            "traffic_floor": "the 20 layers' bytes, each layer in its own read/write proportion, "
                                             "through the streaming yardstick (g3_stream_traffic), back to back "
                                             "from a CUDA graph over rotating buffers",
                            "algorithmic": f"{'1' if kind != 'bf16' else '2'} B per A/B element + 4 B per C "
                                           f"element, summed over the 20 layers"},
               "per_shape": per})
        return

    if args.workload in ("int8", "fp8", "bf16", "fp16", "tf32", "3xtf32", "fp64", "int16"):
        n = args.dsize if args.workload not in ("fp64", "int16") else min(args.dsize, 4096)
        if args.workload == "int16":
            rng = np.random.default_rng(0)
            p = synth.Problem(n, n, n, 1, 0, rng.integers(-(1 << 15), 1 << 15, (n, n)).astype(np.int16),
                              rng.integers(-(1 << 15), 1 << 15, (n, n)).astype(np.int16), None)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C = torch.empty(n, n, dtype=torch.int64, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1, 0, dtype=G3_INT16)
        elif args.workload == "fp64":
            rng = np.random.default_rng(0)
            p = synth.Problem(n, n, n, 1.0, 0.0, rng.uniform(-1, 1, (n, n)), rng.standard_normal((n, n)), None)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C = torch.empty(n, n, dtype=torch.float64, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_F64)
        elif args.workload == "3xtf32":
            # the second FP32-accurate mode, on the headline's inputs (uniform,
            # beta = 0.5 with C)
            p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C0 = torch.from_numpy(p.C).to(dev)
            C = C0.clone()
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.5, dtype=G3_F32_3XTF32, config=args.config)
        elif args.workload == "tf32":
            p = synth.normal_problem(n, n, n, seed=0)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C = torch.empty(n, n, dtype=torch.float32, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_TF32, config=args.config)
        elif args.workload == "fp16":
            p = synth.normal_problem(n, n, n, seed=0)
            A, B, tkw = _stored(torch.from_numpy(p.A).to(dev).half(), torch.from_numpy(p.B).to(dev).half(), args.trans)
            C = torch.empty(n, n, dtype=torch.float32, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP16, config=args.config, **tkw)
        elif args.workload == "bf16":
            p = synth.normal_problem(n, n, n, seed=0)
            A, B, tkw = _stored(torch_api.convert_bf16(torch.from_numpy(p.A).to(dev)), torch_api.convert_bf16(
                torch.from_numpy(p.B).to(dev)), args.trans)
            C = torch.empty(n, n, dtype=torch.float32, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_BF16, config=args.config, **tkw)
        elif args.workload == "int8":
            p = synth.int8_problem(n, n, n, seed=0)
            A, B = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            C = torch.empty(n, n, dtype=torch.int32, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1, 0, dtype=G3_INT8, config=args.config)
        else:
            p = synth.normal_problem(n, n, n, seed=0)
            A32, B32 = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.B).to(dev)
            (A, sa), (B, sb) = torch_api.quantize_fp8(A32), torch_api.quantize_fp8(B32)
            A, B, tkw = _stored(A, B, args.trans)
            C = torch.empty(n, n, dtype=torch.float32, device=dev)
            fn = lambda: torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=sa, scale_b=sb,
                                        config=args.config, **tkw)
        fn()
        torch.cuda.synchronize()
        rows = np.array([0, n // 2, n - 1])
        got = C[torch.from_numpy(rows).to(dev)].cpu().numpy()
        if args.workload == "int8":
            err = {"exact": bool(np.array_equal(got.astype(np.int64), oracle.gemm_i8(p.A, p.B, rows=rows)))}
        elif args.workload == "int16":
            err = {"exact": bool(np.array_equal(got.astype(np.int64), oracle.gemm_i16(p.A, p.B, rows=rows)))}
        elif args.workload == "3xtf32":
            err = sample_err(got.astype(np.float64), rows, p.A, p.B, p.C, 1.0, 0.5)
            C.copy_(C0)
        else:
            err = sample_err(got.astype(np.float64), rows, p.A, p.B, None, 1.0, 0.0)
        for _ in range(args.warmup):
            fn()
        ms = _call_ms(fn, args.reps, flush)
        kms = _kernel_ms(_lib, fn, args.reps, flush)
        flops = 2.0 * n ** 3
        if args.workload == "int16":
            # int64 multiply-adds of widened int16 products on the CUDA cores;
            # against 152 SMs x 64 int32 multiplies per clock x 2.07 GHz x 2
            int_peak = 152 * 64 * 2.07e9 * 2 / 1e12
            _line(args, flops / ms / 1e9, "TOPS",
                  {"workload": f"int16 GEMM m=n=k={n}, alpha=1, beta=0, uniform int16",
                   "path": "INT16 SIMT kernel, int64 accumulation (64 x 64 CTA tiles, 4 x 4 micro-tiles)"},
                  {"dtype": "int16", "ms": ms, "kernel_ms": kms, "err": err,
                   "roofline": {"bound": "alu", "achieved": flops / kms / 1e9, "peak": int_peak, "unit": "TOP/s",
                                "frac": flops / kms / 1e9 / int_peak, "traffic": None,
                                "peak_source": "152 SMs x 64 int32 multiplies/clock x 2.07 GHz x 2 ops",
                                "algorithmic": "2 n^3 integer ops per call"}})
            return
        if args.workload == "fp64":
            # FP64 FMAs on the CUDA cores: against the nominal FP64 rate
            _line(args, flops / ms / 1e9, "TFLOPS",
                  {"workload": f"fp64 GEMM m=n=k={n}, alpha=1, beta=0, A uniform [-1, 1], B normal(0, 1)",
                   "path": "FP64 SIMT kernel (64 x 64 CTA tiles, 4 x 4 register micro-tiles)"},
                  {"dtype": "f64", "ms": ms, "kernel_ms": kms, "err": err,
                   "roofline": {"bound": "alu", "achieved": flops / kms / 1e9, "peak": 1.25, "unit": "TFLOP/s",
                                "frac": flops / kms / 1e9 / 1.25, "traffic": None,
                                "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)",
                                "algorithmic": "2 n^3 FP64 flops per call"}})
            return
        tensor_peak = bf16_peak * {"fp8": 2.0, "tf32": 0.5, "3xtf32": 0.5}.get(args.workload, 1.0)
        tensor_flops = flops * (3.0 if args.workload == "3xtf32" else 1.0)   # three TF32 products per term
        _line(args, flops / ms / 1e9, "TOPS" if args.workload == "int8" else "TFLOPS",
              {"workload": f"{args.workload} GEMM m=n=k={n}, alpha=1, "
                           + ("beta=0.5, uniform [-1, 1]" if args.workload == "3xtf32" else "beta=0")
                           + (f", stored transposed: {'A (k x m) ' if 'a' in args.trans else ''}"
                              f"{'B (n x k)' if 'b' in args.trans else ''}, read in place" if args.trans else ""),
               "path": {"int8": "exact: int8 -> bf16 pre-pass, k-chunks of 1024 on the BF16 tensor path, "
                                "int32 split-K reduce (tcgen05 kind::i8 does not exist on sm_103a)",
                        "fp8": "tcgen05 kind::f8f6f4 E4M3, per-tensor scales",
                        "bf16": "tcgen05 kind::f16 BF16, FP32 accumulation",
                        "fp16": "tcgen05 kind::f16 FP16, FP32 accumulation",
                        "tf32": "TF32 rounding pre-pass + tcgen05 kind::tf32, FP32 accumulation",
                        "3xtf32": "FP32-accurate: hi/lo TF32 split pre-pass + 3 tcgen05 kind::tf32 products "
                                  "(main and correction accumulators)"}[args.workload]},
              {"dtype": args.workload, "ms": ms, "kernel_ms": kms, "err": err,
               "roofline": {"bound": "tensor", "achieved": tensor_flops / kms / 1e9, "peak": tensor_peak,
                            "unit": "TFLOP/s", "frac": tensor_flops / kms / 1e9 / tensor_peak, "traffic": None,
                            "peak_source": f"{peak_src} bf16 burst" + {
                                "fp8": " x 2 (fp8 nominal ratio)",
                                "tf32": " x 0.5 (tf32 nominal ratio)",
                                "3xtf32": " x 0.5 (tf32 nominal ratio)"}.get(args.workload, ""),
                            "frac_of_nominal": tensor_flops / kms / 1e9 / NOMINAL_TFLOPS[
                                {"fp8": "fp8", "tf32": "tf32", "3xtf32": "tf32"}.get(args.workload, "bf16")],
                            "algorithmic": "2 n^3 per call (INT8: of the main kernel's bf16 work; "
                                           "3xTF32: 3 x 2 n^3 tf32 tensor flops)"}})
        return

    if args.workload == "conv":
        # the Table 1 layers with C % 64 == 0 as implicit-GEMM convolutions
        # (NHWC bf16 activations, RSCK weights, NPQK fp32 output), batch 16
        per, tot_ms, tot_kms, tot_bytes, tot_flops, worst = [], 0.0, 0.0, 0.0, 0.0, 0.0
        for geo in synth.RESNET50_CONV:
            if geo["C"] % 64 or (args.only and f"L{geo['layer']}" not in args.only.split(",")):
                continue
            H, C, K, R, st, pd = geo["H"], geo["C"], geo["K"], geo["R"], geo["stride"], geo["pad"]
            rng = np.random.default_rng(geo["layer"])
            xh = rng.standard_normal((16, H, H, C)).astype(np.float32)
            wh = (rng.standard_normal((R, R, C, K)) / np.sqrt(R * R * C)).astype(np.float32)
            x = torch.from_numpy(xh).to(dev).to(torch.bfloat16)
            w = torch.from_numpy(wh).to(dev).to(torch.bfloat16)
            P = (H + 2 * pd - R) // st + 1
            y = torch.empty(16, P, P, K, dtype=torch.float32, device=dev)
            fn = lambda: torch_api.conv2d(x, w, y, (st, st), (pd, pd))
            fn()
            torch.cuda.synchronize()
            xq, wq = x[:1].float().cpu().numpy(), w.float().cpu().numpy()
            want = oracle.conv2d_nhwc(xq, wq, (st, st), (pd, pd))[0]
            D = oracle.conv2d_nhwc(np.abs(xq), np.abs(wq), (st, st), (pd, pd))[0]
            err = float(np.max(np.abs(y[0].cpu().numpy() - want) / np.maximum(D, 1e-300)))
            flops = 2.0 * 16 * P * P * K * R * R * C
            nbytes = 2.0 * (16 * H * H * C + R * R * C * K) + 4.0 * 16 * P * P * K
            # rotating operand sets (together >= 512 MiB, 4x L2) replayed back to
            # back from a CUDA graph, as the layers of a captured network run
            sets = max(1, min(64, -(-(512 << 20) // int(nbytes))))
            copies = [(x.clone(), w.clone(), torch.empty_like(y)) for _ in range(sets - 1)] + [(x, w, y)]
            calls = [lambda a=a, b=b, c=c: torch_api.conv2d(a, b, c, (st, st), (pd, pd)) for a, b, c in copies]
            for c_ in calls:
                c_()
            torch.cuda.synchronize()
            nrep = max(args.reps, 2 * sets)
            ms = _rotating_graph_ms(calls, nrep)
            kms = _kernel_ms(_lib, fn, args.reps, flush)
            cold_ms = _call_ms(fn, 5, flush)
            del copies, calls
            cfg = _lib.g3_plan_query(16 * P * P, K, R * R * C, G3_BF16)
            per.append({"layer": geo["layer"], "N": 16, "H": H, "C": C, "K": K, "R": R, "stride": st, "pad": pd,
                        "ms": ms, "kernel_ms": kms, "cold_call_ms": cold_ms, "rotating_sets": sets,
                        "tflops": flops / ms / 1e9, "gbs": nbytes / ms / 1e6,
                        "hbm_frac": nbytes / ms / 1e6 / hbm, "member": _lib.g3_family_describe(cfg[1]),
                        "split_k": cfg[2], "err": err})
            tot_ms += ms
            tot_kms += kms
            tot_bytes += nbytes
            tot_flops += flops
            worst = max(worst, err)
            del x, w, y
        _line(args, tot_flops / tot_ms / 1e9, "TFLOPS",
              {"workload": "19 ResNet-50 v1.5 convolution layers of Table 1 (C % 64 == 0), batch 16, as "
                           "implicit GEMMs (TMA im2col loads of NHWC bf16 activations, no im2col matrix), "
                           "fp32 NHWC output; whole calls back to back, replayed from a CUDA graph (ms); "
                           "kernel_ms: the GEMM kernel alone (CUDA events, eager, L2 flushed)",
               "l2": "rotating operand copies, together >= 512 MiB (4x L2), per layer; cold_call_ms: one call "
                     "after a 256 MiB L2 flush"},
              {"dtype": "bf16", "total_ms": tot_ms, "total_kernel_ms": tot_kms, "worst_err": worst,
               "roofline": {"bound": "hbm", "achieved": tot_bytes / tot_ms / 1e6, "peak": hbm, "unit": "GB/s",
                            "frac": tot_bytes / tot_ms / 1e6 / hbm, "traffic": None,
                            "peak_source": f"{peak_src} hbm_gbs",
                            "algorithmic": "activations and weights read once (2 B), output written once (4 B)"},
               "per_layer": per})
        return

    if args.workload in ("grouped", "grouped-3xbf16", "grouped-fp8"):
        dt = {"grouped": G3_BF16, "grouped-3xbf16": G3_F32_3XBF16, "grouped-fp8": G3_FP8_E4M3}[args.workload]
        shapes = synth.grouped_shapes(1000, seed=0)
        probs = []
        masters = {}
        flops = 0.0
        rng = np.random.default_rng(0)
        for gi, (m, n, k) in enumerate(shapes):
            a32 = (rng.standard_normal((m, k)) / np.sqrt(k)).astype(np.float32)
            b32 = rng.standard_normal((k, n)).astype(np.float32)
            if dt == G3_FP8_E4M3:
                lda, ldb = -(-k // 16) * 16, -(-n // 16) * 16      # 16-byte rows for TMA
                (qa, sa), (qb, sb) = torch_api.quantize_fp8(torch.from_numpy(a32).to(dev)), torch_api.quantize_fp8(
                    torch.from_numpy(b32).to(dev))
                A = torch.zeros(m, lda, dtype=torch.uint8, device=dev)[:, :k]
                B = torch.zeros(k, ldb, dtype=torch.uint8, device=dev)[:, :n]
                A.copy_(qa)
                B.copy_(qb)
                C = torch.empty(m, n, device=dev)
                probs.append((A, B, C, 1.0, 0.0, float(sa.item()), float(sb.item())))
                if gi % 50 == 0:
                    masters[gi] = (a32, b32)
                flops += 2.0 * m * n * k
                continue
            lda, ldb = -(-k // 8) * 8, -(-n // 8) * 8      # 16-byte rows for TMA
            if dt == G3_BF16:
                A = torch.zeros(m, lda, dtype=torch.bfloat16, device=dev)[:, :k]
                B = torch.zeros(k, ldb, dtype=torch.bfloat16, device=dev)[:, :n]
            else:
                A = torch.zeros(m, lda, dtype=torch.float32, device=dev)[:, :k]
                B = torch.zeros(k, ldb, dtype=torch.float32, device=dev)[:, :n]
            A.copy_(torch.from_numpy(a32))
            B.copy_(torch.from_numpy(b32))
            C = torch.empty(m, n, device=dev)
            probs.append((A, B, C, 1.0, 0.0))
            flops += 2.0 * m * n * k
        tuned_buckets, tune_s = 0, 0.0
        if args.tune:
            # per-bucket selection of the tile height (g3_autotune_grouped):
            # one timing per (log2 m, log2 n, log2 k) bucket of the batch
            _lib.g3_tune_cache_clear()
            t0 = time.perf_counter()
            seen = set()
            for (m, n, k) in shapes:
                key = tuple(int(np.ceil(np.log2(x))) for x in (m, n, k))
                if key not in seen:
                    seen.add(key)
                    _lib.g3_autotune_grouped(m, n, k, dt)
            tuned_buckets, tune_s = len(seen), time.perf_counter() - t0
        plan = torch_api.GroupedPlan(probs, dt)
        heights = [_lib.g3_grouped_plan_describe(plan.plan, i)[1] for i in range(len(probs))]
        plan.execute()
        torch.cuda.synchronize()
        errs, nonfinite = [], 0
        for gi in range(0, 1000, 50):
            A, B, C = probs[gi][:3]
            # the gate: against the FP32 masters (FP8), or the operands the GPU got
            a, b = masters[gi] if dt == G3_FP8_E4M3 else (A.float().cpu().numpy(), B.float().cpu().numpy())
            rows = np.arange(min(4, a.shape[0]))
            got = C.cpu().numpy()[rows].astype(np.float64)
            nonfinite += int(np.count_nonzero(~np.isfinite(got)))
            errs.append(sample_err(got, rows, a, b, None, 1.0, 0.0)["gate"])
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                plan.execute(stream=s)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            g.replay()
        grouped_ms = _call_ms(g.replay, args.reps, flush)
        kms = _kernel_ms(_lib, plan.execute, args.reps, flush)

        def per_call():
            for pr in probs:
                A, B, C, a, b = pr[:5]
                if dt == G3_FP8_E4M3:   # the scales folded into alpha, as the plan does
                    torch_api.gemm(A, B, C, a * pr[5] * pr[6], b, dtype=dt)
                else:
                    torch_api.gemm(A, B, C, a, b, dtype=dt)

        per_call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps_eager = 1 if args.compact else 3
        for _ in range(reps_eager):
            per_call()
        torch.cuda.synchronize()
        eager_ms = (time.perf_counter() - t0) * 1e3 / reps_eager
        s2 = torch.cuda.Stream()
        s2.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s2):
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2, stream=s2):
                per_call()
        torch.cuda.synchronize()
        g2.replay()
        graph_calls_ms = _call_ms(g2.replay, max(3, args.reps // 4), flush)
        extra = {}
        if dt == G3_F32_3XBF16:
            # the same batch split inside the grouped kernels (G3_GROUPED_SPLIT_IN_KERNEL)
            fz = torch_api.GroupedPlan(probs, dt, split_in_kernel=True)
            fz.execute()
            torch.cuda.synchronize()
            s3 = torch.cuda.Stream()
            s3.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s3):
                g3 = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g3, stream=s3):
                    fz.execute(stream=s3)
            torch.cuda.synchronize()
            g3.replay()
            extra = {"split_in_kernel_graph_ms": _call_ms(g3.replay, args.reps, flush)}
            fz.close()
        # algorithmic bytes: each operand read once in its input format, C written once
        es = {G3_BF16: 2, G3_F32_3XBF16: 4, G3_FP8_E4M3: 1}[dt]
        alg_bytes = float(sum(es * (m * k + k * n) + 4 * m * n for (m, n, k) in shapes))
        peaks, peak_src = load_peaks()
        hbm = float(peaks["hbm_gbs"])
        extra["roofline"] = {"bound": "hbm", "achieved": alg_bytes / grouped_ms / 1e6, "peak": hbm, "unit": "GB/s",
                             "frac": alg_bytes / grouped_ms / 1e6 / hbm, "traffic": None,
                             "peak_source": f"{peak_src} copy bandwidth",
                             "algorithmic": f"{alg_bytes / 1e9:.3f} GB: A and B once in the input format "
                                            f"({es} B per element), C written once (4 B)"}
        _line(args, flops / grouped_ms / 1e9, "TFLOPS",
              {"workload": f"1000 GEMMs, m,n,k log-uniform in [16,1024] (seed 0), "
                           f"{ {G3_BF16: 'bf16', G3_F32_3XBF16: '3xbf16 (fp32 in/out)', G3_FP8_E4M3: 'fp8 e4m3 with per-problem scales'}[dt] }, fp32 C, beta=0",
               "l2": "flushed before every replay"},
              {"dtype": {G3_BF16: "bf16", G3_F32_3XBF16: "bf16x3->f32", G3_FP8_E4M3: "fp8"}[dt], "total_gflop": flops / 1e9,
               "grouped_graph_ms": grouped_ms, "grouped_kernel_ms": kms,
               "per_call_eager_wall_ms": eager_ms, "per_call_graph_ms": graph_calls_ms,
               "speedup_vs_eager": eager_ms / grouped_ms, "speedup_vs_graph_of_calls": graph_calls_ms / grouped_ms,
               "max_rel_err_sampled": float(np.max(np.array(errs))), "nonfinite_sampled": nonfinite,
               "autotuned": bool(args.tune), "tuned_buckets": tuned_buckets, "tune_s": round(tune_s, 1),
               "tile_heights": {str(h): heights.count(h) for h in sorted(set(heights))}, **extra})
        plan.close()
        return


# The other configurations, measured compactly (fewer repetitions, no cold or
# eager-only passes) after the headline step and reported in its JSON line
# under "configs", each with its own clock sample.
OTHER_CONFIGS = (
    ("1_plain_fp32_512", "plain"),
    ("3_im2col_bf16", "im2col"),
    ("3_im2col_bf16_autotuned", "im2col+tune"),
    ("4_grouped_bf16", "grouped"),
    ("4_grouped_3xbf16", "grouped-3xbf16"),
    ("5_bf16_8192", "bf16"),
    ("5_bf16_8192_transposed", "bf16+trans"),
    ("5_fp8_8192", "fp8"),
    ("5_int8_8192", "int8"),
    ("5_im2col_fp8", "im2col-fp8"),
    ("5_im2col_int8", "im2col-int8"),
)


def _summary(line):
    """The figures of one configuration's line that the default line carries."""
    keep = {"value": line["value"], "unit": line["unit"]}
    rf = line.get("roofline")
    if rf:
        keep["roofline"] = {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac", "frac_of_traffic_floor")
                            if k in rf}
    for k in ("ms", "kernel_ms", "err", "worst_err", "total_ms_20_layers", "traffic_floor_ms_20_layers",
              "grouped_graph_ms", "grouped_kernel_ms", "split_in_kernel_graph_ms",
              "per_call_graph_ms", "per_call_eager_wall_ms", "speedup_vs_eager", "speedup_vs_graph_of_calls",
              "max_rel_err_sampled", "nonfinite_sampled", "total_gflop", "autotuned"):
        if k in line:
            keep[k] = line[k]
    if "per_shape" in line:
        keep["per_shape"] = [{"shape": r["shape"], "us": round(r["ms"] * 1e3, 2), "hbm_frac": round(r["hbm_frac"], 3),
                              "floor_us": round(r["traffic_floor_ms"] * 1e3, 2), "member": r["member"],
                              "split_k": r["split_k"]} for r in line["per_shape"]]
    keep["workload"] = line["config"].get("workload")
    return keep


def other_configs(args, gpu_index):
    global _COLLECT
    import copy
    out = {}
    for key, wl in OTHER_CONFIGS:
        a = copy.copy(args)
        tune, trans = wl.endswith("+tune"), wl.endswith("+trans")
        a.workload, a.reps, a.compact, a.only, a.tune, a.config, a.dsize = wl.split("+")[0], 10, True, "", tune, -1, 8192
        a.trans = "ab" if trans else ""
        _COLLECT = []
        clk = Clocks(gpu_index)
        clk.start()
        t0 = time.perf_counter()
        err = None
        try:
            run_workload(a)
        except Exception as e:  # noqa: BLE001 -- reported in the line, the headline stands
            err = f"{type(e).__name__}: {e}"
        wall = time.perf_counter() - t0
        c = clk.stop()
        lines, _COLLECT = _COLLECT, None
        entry = _summary(lines[0]) if lines else {"error": err or "no result"}
        entry["clocks"] = c
        entry["wall_s"] = round(wall, 1)
        out[key] = entry
        if tune:
            from paper_2310_20347_gb300 import _lib
            _lib.g3_tune_cache_clear()   # later configurations use the planner again
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--impl", default="g3", choices=["g3", "reference"])
    ap.add_argument("--ref-rows", type=int, default=0, help="reference arm: rows of C per step (0: 8 per host thread)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--simt-steps", type=int, default=3)
    ap.add_argument("--config", type=int, default=-1, help="force a member of the kernel family")
    ap.add_argument("--workload", default="square",
                    choices=["square", "sweep", "plain", "simt", "streamk", "im2col", "im2col-fp8", "im2col-int8", "int8", "fp8", "bf16", "fp16", "tf32", "3xtf32", "fp64", "int16", "conv",
                             "grouped", "grouped-3xbf16", "grouped-fp8"],
                    help="square (default) is the headline step; the others measure the remaining "
                         "configurations and print one JSON line each")
    ap.add_argument("--dsize", type=int, default=8192, help="int8 / fp8 / bf16 workloads: m = n = k")
    ap.add_argument("--trans", default="", choices=["", "a", "b", "ab"],
                    help="bf16 / fp16 / fp8 workloads: operands stored transposed (A k x m, B n x k), read in place")
    ap.add_argument("--print-kernel-hash", action="store_true",
                    help="print the hash of the headline kernel's sources (for the DRAM-traffic record) and exit")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--only", default="", help="im2col workloads: comma-separated layer names (e.g. L1,L12)")
    ap.add_argument("--tune", action="store_true",
                    help="im2col workloads: autotune every shape first; grouped workloads: every size bucket")
    ap.add_argument("--no-configs", action="store_true",
                    help="default run: skip the compact measurements of the other configurations")
    args = ap.parse_args()
    args.compact = False
    args.warmup = max(args.warmup, 3)
    if args.print_kernel_hash:
        print(kernel_sources_hash())
        return
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "square":
        return run_workload(args)

    import torch

    world, rank, local = dist_setup(args.gpus)
    import paper_2310_20347_gb300 as pkg
    from paper_2310_20347_gb300 import G3_F32, G3_F32_3XBF16, _lib, synth, torch_api
    pkg.load()
    n = args.size
    p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
    A = torch.from_numpy(p.A).cuda()
    B = torch.from_numpy(p.B).cuda()
    C0 = torch.from_numpy(p.C).cuda()
    C = C0.clone()
    stream = torch.cuda.current_stream()
    flops = 2.0 * n * n * n

    def step(dtype, out):
        cfg = args.config if dtype == G3_F32_3XBF16 else -1
        torch_api.gemm(A, B, out, 1.0, 0.5, dtype=dtype, stream=stream, config=cfg)

    # --- correctness on sampled rows of the full-size problem (same launch config)
    import oracle
    sample_rows = np.array([0, 1, n // 3, n // 2, n - 2, n - 1])
    errs = {}
    if rank == 0:
        A64, B64 = p.A.astype(np.float64), p.B.astype(np.float64)
        ref = oracle.gemm(A64, B64, p.C, 1.0, 0.5, rows=sample_rows)
        D = oracle.absprod(A64, B64, 1.0, rows=sample_rows)
    for name, dt in (("3xbf16", G3_F32_3XBF16), ("simt", G3_F32)):
        C.copy_(C0)
        step(dt, C)
        torch.cuda.synchronize()
        if rank == 0:
            got = C[torch.from_numpy(sample_rows).cuda()].cpu().numpy().astype(np.float64)
            errs[name] = float(np.max(np.abs(got - ref) / D))

    # --- timed region: K steps of the 3xBF16 path
    for _ in range(args.warmup):
        step(G3_F32_3XBF16, C)
    torch.cuda.synchronize()
    _lib.g3_kernel_timing(True)
    _lib.g3_kernel_time_ms(reset=True)
    clocks = Clocks(local)
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    launches0 = _lib.g3_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(G3_F32_3XBF16, C)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = _lib.g3_launch_count() - launches0
    clk = clocks.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    kern_ms, kern_n = _lib.g3_kernel_time_ms(reset=True)
    _lib.g3_kernel_timing(False)
    ms_max = max_over_ranks(ms, world)
    value = world * flops * args.steps / (ms_max * 1e-3) / 1e12

    # --- SIMT on the same problem (the plain method), for the speedup
    for _ in range(1):
        step(G3_F32, C)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(args.simt_steps):
        step(G3_F32, C)
    s1.record(stream)
    torch.cuda.synchronize()
    simt_ms = s0.elapsed_time(s1) / args.simt_steps

    # --- end to end through the C ABI with HOST buffers (g3_gemm_host: the
    # uploads of A, B, C and the download of C are inside the timed region)
    # Two requests in flight: steps alternate between two streams, each with
    # its own page-locked host buffers, so one step's uploads run under the
    # other's compute; the one-stream figure (each step waits for the last)
    # is reported beside it.
    hosts = [tuple(torch.from_numpy(x).pin_memory() for x in (p.A, p.B, p.C)) for _ in range(2)]
    streams = [stream, torch.cuda.Stream()]

    def e2e_step(i, nstreams):
        hA, hB, hC = hosts[i % nstreams]
        torch_api.gemm_host(hA, hB, hC, 1.0, 0.5, dtype=G3_F32_3XBF16, stream=streams[i % nstreams])

    def e2e_run(nstreams, steps):
        torch.cuda.synchronize()
        barrier(world)
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(streams[0])
        for sj in streams[1:nstreams]:
            sj.wait_event(x0)
        for i in range(steps):
            e2e_step(i, nstreams)
        for sj in streams[1:nstreams]:
            streams[0].wait_stream(sj)
        x1.record(streams[0])
        torch.cuda.synchronize()
        return max_over_ranks(x0.elapsed_time(x1), world)

    for i in range(2):
        e2e_step(i, 2)
    torch.cuda.synchronize()
    e2e_steps = max(4, args.steps // 2)
    e2e_ms = e2e_run(2, e2e_steps)
    e2e_val = world * flops * e2e_steps / (e2e_ms * 1e-3) / 1e12
    e2e_one_ms = e2e_run(1, e2e_steps)
    e2e_one_val = world * flops * e2e_steps / (e2e_one_ms * 1e-3) / 1e12

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    per_launch_ms = kern_ms / max(kern_n, 1)
    tensor_flops = 3.0 * flops                  # three bf16 products per FP32-equivalent flop
    achieved = tensor_flops / (per_launch_ms * 1e-3) / 1e12
    peak = float(peaks["bf16_tflops"])
    st = _lib.g3_plan_query(n, n, n, G3_F32_3XBF16)
    cfg_used = args.config if args.config >= 0 else st[1]
    member = _lib.g3_family_describe(cfg_used) if st[0] == 0 and cfg_used >= 0 else "?"
    traffic, traffic_src = recorded_traffic(member, n)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    simt_tflops = flops / (simt_ms * 1e-3) / 1e12
    sm_mhz = clk["sm_mhz"] or float(peaks.get("sm_max_mhz", 2070.0))
    simt_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32", "data": "synthetic",
        "config": square_config(n),
        "method": "F32_3XBF16 (split pre-pass + tcgen05 kernel)", "member": member,
        "rel_err": {"3xbf16": errs.get("3xbf16"), "simt": errs.get("simt"), "tolerance": 2e-6,
                    "sample": f"rows {sample_rows.tolist()} vs binary64 oracle"},
        "simt": {"tflops": simt_tflops, "ms": simt_ms, "peak_tflops_at_clock": simt_peak,
                 "frac": simt_tflops / simt_peak},
        "speedup_vs_simt": simt_ms / (ms_max / args.steps),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "kernel": f"tc_gemm_kernel ({member})",
                     "peak_source": f"{peak_src} bf16 burst (MEASURED_PEAKS.json)",
                     "frac_of_sustained": achieved / float(peaks.get("bf16_tflops_sustained", peak)),
                     "frac_of_nominal": achieved / NOMINAL_TFLOPS["bf16"],
                     "nominal_peak": NOMINAL_TFLOPS["bf16"],
                     "per_launch_ms": per_launch_ms, "launches_timed": kern_n,
                     "algorithmic": "6 n^3 bf16 tensor flops per launch"},
        "e2e": {"value": e2e_val, "unit": "TFLOPS", "h2d_bytes_per_step": 3 * n * n * 4,
                "d2h_bytes_per_step": n * n * 4, "steps": e2e_steps,
                "path": "g3_gemm_host from page-locked host buffers, steps alternating between two streams",
                "one_stream_value": e2e_one_val},
        "gpu_launches": int(launches),
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
    }
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_oracle_sample(p)
    if not args.no_configs and world == 1:
        del A, B, C0, C, hosts
        torch.cuda.empty_cache()
        line["configs"] = other_configs(args, local)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

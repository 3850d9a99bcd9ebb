#!/usr/bin/env python
"""Benchmark of the batched 1D C2C FFT (FP32) on the n = 2^8..2^20 sweep.

One step is the whole sweep: for every n = 2^e (e = 8..20, batch = 2^26 / n), both
complex layouts (interleaved, split) and both directions, one batched transform of
512 MiB in / 512 MiB out, read from and written to buffers larger than L2.
Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fftc|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of
the same workload. Multi-GPU runs (torchrun) are independent replicas of the sweep
(the transforms of a batch shard with no exchange), reported as weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched C2C FFT GFLOP/s (5n·log2n) & %HBM roofline, FP32 vs split-FP16"
UNIT = "GFLOP/s"
ELEMS = 1 << 26               # n * batch for every sweep size
SIZES = list(range(8, 21))     # log2 n
LAYOUTS = ["interleaved", "split"]
DIRECTIONS = [False, True]     # inverse?
WORKLOAD = "batched FP32 C2C FFT sweep n=2^8..2^20, n*batch=2^26, interleaved+split, forward+inverse"
SEED = 2


def flops(n: int, batch: int) -> float:
    return 5.0 * n * math.log2(n) * batch


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the slowest rank's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, step_flops: float, steps: int, ms: float) -> float:
    """Whole-job GFLOP/s: every rank runs the same sweep, time = the slowest rank."""
    return world * step_flops * steps / (ms * 1e-3) / 1e9


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
CSRC = os.path.join(ROOT, "paper_2308_00497_gb300", "csrc")


def csrc_digest() -> str:
    """SHA-256 over the kernel sources (names and bytes), to tell whether a stored ncu
    capture still describes the kernels that run."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def stored_traffic(kind: str):
    """DRAM bytes per launch of a kernel kind from the committed ncu summary
    (dram__bytes_read.sum + dram__bytes_write.sum), or None when the summary is missing
    or was taken on kernel sources other than the current ones."""
    try:
        with open(TRAFFIC_FILE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    digest, table = None, {}
    for ln in lines:
        if ln.startswith("csrc_sha256:"):
            digest = ln.split(":", 1)[1].strip()
        elif ln and not ln.startswith("#") and len(ln.split()) >= 2:
            k, v = ln.split()[:2]
            try:
                table[k] = float(v)
            except ValueError:
                pass
    if digest != csrc_digest():
        return None
    return table.get(kind)


def _nvtx(push: bool, name: str = "") -> None:
    """Open / close an NVTX range (a no-op where torch has no NVTX support)."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:  # pragma: no cover
        pass


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# --------------------------------------------------------------------------
def oracle_sample(rows_per_size: int):
    """Time the FP64 oracle (as it stands) on `rows_per_size` rows of every sweep size."""
    import numpy as np

    import oracle
    import synthetic_inputs as si
    threads = oracle.default_threads()
    oracle.build_oracle()
    total_flops, total_s = 0.0, 0.0
    for e in SIZES:
        n = 1 << e
        x = si.uniform_complex(rows_per_size, n, seed=SEED * 100 + e).astype(np.complex128)
        t0 = time.perf_counter()
        oracle.fft(x, threads=threads)
        total_s += time.perf_counter() - t0
        total_flops += flops(n, rows_per_size)
    return total_flops, total_s, threads


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    import oracle
    threads = oracle.default_threads()
    rows = threads
    for _ in range(args.warmup):
        oracle_sample(rows)
    fl, secs = 0.0, 0.0
    for _ in range(args.steps):
        f, s, threads = oracle_sample(rows)
        fl += f
        secs += s
    value = fl / secs / 1e9
    sample = f"{rows} rows of each n=2^8..2^20 (forward) per step; direct O(n^2) DFT for n<=4096, radix-2 above"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": "2^8..2^20", "n_times_batch": ELEMS, "sample": sample,
                   "parallelism": f"{threads} host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def run_fftc(args, rank: int, world: int, local_rank: int) -> None:
    import numpy as np
    import torch

    import paper_2308_00497_gb300 as fc
    import synthetic_inputs as si

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # one 512 MiB input (viewed at every shape: n * batch is constant) and one output
    x_host = si.uniform_complex(1, ELEMS, seed=SEED).reshape(ELEMS)
    x = torch.from_numpy(x_host.view(np.float32)).to(dev)          # 2^27 floats
    y = torch.empty_like(x)
    plans = []
    for e in args.sizes:
        n = 1 << e
        B = ELEMS // n
        for layout in args.layouts:
            for inv in args.dirs:
                pl = fc.Plan(n, B, layout, inv, precision=args.precision, device=dev)
                if args.tune:
                    pl.tune(5)  # measure-mode planning, outside the timed region
                plans.append((e, layout, inv, pl))

    def views(layout, n, B):
        if layout == "interleaved":
            return x.view(torch.complex64).view(B, n), y.view(torch.complex64).view(B, n)
        return x.view(2, B, n), y.view(2, B, n)

    def step():
        for e, layout, inv, p in plans:
            n = 1 << e
            xi, yo = views(layout, n, ELEMS // n)
            p.execute(xi, yo)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for *_, p in plans:
        p.timing(True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _nvtx(True, "timed_sweep")  # lets a profiler capture exactly the timed launches
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    _nvtx(False)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, dev)

    # per-kernel durations from the library's event probe
    kinds = {}
    per_size = []
    launches = 0
    for e, layout, inv, p in plans:
        pm, cnt = p.pass_times()
        passes, _ = p.info()
        launches += passes * cnt
        n = 1 << e
        if passes == 2:
            names = ["cols", "rowst"]
        else:  # one launch: a single-pass kernel, or the cluster single pass (n = 2^15..2^18)
            names = ["rows"] if n <= (1 << 14) else ["cluster"]
        for i, nm in enumerate(names):
            k = kinds.setdefault(nm, {"ms": 0.0, "launches": 0})
            k["ms"] += pm[i]
            k["launches"] += cnt
        t_exec = sum(pm[:passes]) / max(cnt, 1)
        per_size.append({"n": n, "layout": layout, "dir": "inv" if inv else "fwd", "passes": passes,
                         "split": list(p.split()),
                         "ms": round(t_exec, 4), "gflops": round(flops(n, ELEMS // n) / t_exec / 1e6, 1),
                         "hbm_frac_strict": round(16.0 * ELEMS / (t_exec * 1e-3) / 1e9 / peaks()[0], 4),
                         "hbm_frac_per_pass": round(16.0 * ELEMS * passes / (t_exec * 1e-3) / 1e9 / peaks()[0], 4)})
        p.timing(False)
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    dom_avg_ms = kinds[dom]["ms"] / kinds[dom]["launches"]
    bytes_per_launch = 16.0 * ELEMS
    peak, peak_kind = peaks()
    achieved = bytes_per_launch / (dom_avg_ms * 1e-3) / 1e9
    # every kernel kind's own fraction, and the whole timed step's: strict (16 B per element
    # and transform, whatever the pass count) and per pass (16 B per element and HBM pass)
    per_kind = {k: round(bytes_per_launch / (v["ms"] / v["launches"] * 1e-3) / 1e9 / peak, 4)
                for k, v in kinds.items() if v["launches"]}
    step_ms = ms / args.steps
    step_passes = sum(p.info()[0] for *_, p in plans)
    sweep = {"strict_frac": round(bytes_per_launch * len(plans) / (step_ms * 1e-3) / 1e9 / peak, 4),
             "per_pass_frac": round(bytes_per_launch * step_passes / (step_ms * 1e-3) / 1e9 / peak, 4),
             "transforms_per_step": len(plans), "hbm_passes_per_step": step_passes}
    step_flops = sum(flops(1 << e, ELEMS // (1 << e)) for e, *_ in plans)
    value = weak_scaling_value(world, step_flops, args.steps, ms)

    # end to end: host buffers in and out through fftc_execute_host, copies timed
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(x_host.view(np.float32).copy()).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for e, layout, inv, p in plans:
                p.execute_host(h_in, h_out, y)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        wall = max_over_ranks(wall, dist, dev)
        e2e = {"value": world * step_flops * args.e2e_steps / wall / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 8 * ELEMS * len(plans), "d2h_bytes_per_step": 8 * ELEMS * len(plans),
               "steps": args.e2e_steps}

    extras = {} if args.no_extras else run_extras(args, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = 0
        import oracle
        rows = 64 * oracle.default_threads()  # about 15 s of host work
        f, s, th = oracle_sample(rows)
        cpu = {"value": f / s / 1e9, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": f"{rows} rows of each n=2^8..2^20 (forward, FP64); direct O(n^2) DFT for n<=4096, "
                         f"radix-2 above; {s:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": "2^8..2^20", "n_times_batch": ELEMS,
                       "layouts": LAYOUTS, "directions": ["forward", "inverse"],
                       "l2": "no flush: every buffer is 512 MiB, larger than L2",
                       "planning": "measure (fftc_plan_tune, untimed)" if args.tune else "default table",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": stored_traffic(dom), "bytes_per_launch": bytes_per_launch,
                         "avg_launch_ms": round(dom_avg_ms, 5), "kernel_ms": {k: round(v["ms"], 3) for k, v in kinds.items()},
                         "per_kind_frac": per_kind, "sweep": sweep},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
            "per_size": per_size,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _time_ms(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_extras(args, dev) -> dict:
    """Secondary workloads, each against the plain FP32 form on the same GPU."""
    import numpy as np
    import torch

    import paper_2308_00497_gb300 as fc
    import synthetic_inputs as si
    from paper_2308_00497_gb300.autograd import spectral_filter
    out = {}
    reps = max(3, args.steps)
    sel = set(args.extras.split(","))
    if "uneven" in sel:
        out["uneven"] = run_uneven(args, dev, reps)
    if "filter" in sel:
        out["spectral_filter"] = run_filter(dev, reps)
    if "mixed" in sel:
        out["mixed_radix"] = run_mixed(dev, reps)
    if "large" in sel:
        out["large_n"] = run_large(dev, reps)
    if "nd" in sel:
        out["multidim"] = run_nd(dev, reps)
    if "fp64" in sel:
        out["fp64"] = run_fp64(dev, reps)
    if "precision" in sel and not args.no_precision:
        out["precision"] = run_precision(args, dev, reps)
    return out


def run_uneven(args, dev, reps: int) -> dict:
    """Uneven batch: 4096 rows, n = 2^6..2^16 log-uniform, mixed directions, one persistent
    launch, against one uniform batched plan per (n, direction) class launched separately
    (measure-mode planned when the bench tunes)."""
    import torch

    import paper_2308_00497_gb300 as fc
    import synthetic_inputs as si
    n, d, o, total = si.uneven_batch(4096, seed=4)
    x = torch.from_numpy(si.uneven_data(total, seed=4)).to(dev)
    y = torch.empty_like(x)
    up = fc.UnevenPlan(n, d, o, device=dev)
    t_uneven = _time_ms(lambda: up.execute(x, y), reps)
    fl = sum(5.0 * int(v) * math.log2(int(v)) for v in n)
    # the same rows as one uniform batched plan per (n, direction) class, separate launches
    classes = {}
    for v, dd in zip(n.tolist(), d.tolist()):
        classes[(v, dd)] = classes.get((v, dd), 0) + 1
    bufs, plans = [], []
    for (v, dd), cnt in classes.items():
        xb = torch.zeros((cnt, v), dtype=torch.complex64, device=dev)
        bufs.append((xb, torch.empty_like(xb)))
        pl = fc.Plan(v, cnt, "interleaved", dd == 1, device=dev)
        plans.append(pl.tune(3) if args.tune else pl)
    def per_class():
        for (xb, yb), p in zip(bufs, plans):
            p.execute(xb, yb)
    t_sep = _time_ms(per_class, reps)
    # the same launches replayed from one CUDA graph (no host launch overhead between them)
    t_graph = None
    try:
        per_class()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            per_class()
        t_graph = _time_ms(g.replay, reps)
        del g
    except RuntimeError:
        t_graph = None
    res = {"workload": "4096 rows, n=2^6..2^16 log-uniform, mixed fwd/inv, interleaved, one persistent "
                       "launch from a CUDA graph", "elements": int(total), "ms": round(t_uneven, 4),
           "gflops": round(fl / (t_uneven * 1e-3) / 1e9, 1),
           "hbm_frac_strict": round(16.0 * total / (t_uneven * 1e-3) / 1e9 / peaks()[0], 4),
           "separate_launches_ms": round(t_sep, 4), "separate_launches": len(plans),
           "speedup_vs_separate": round(t_sep / t_uneven, 3),
           "separate_launches_graph_ms": round(t_graph, 4) if t_graph else None,
           "speedup_vs_separate_graph": round(t_graph / t_uneven, 3) if t_graph else None}
    del bufs, plans, x, y
    return res


def run_filter(dev, reps: int) -> dict:
    """Differentiation: batched spectral filter forward + backward, [1024, 2^14]."""
    import torch

    import paper_2308_00497_gb300 as fc
    import synthetic_inputs as si
    from paper_2308_00497_gb300.autograd import spectral_filter
    B, nn = 1024, 1 << 14
    xs = torch.from_numpy(si.gaussian_complex(B, nn, seed=5)).to(dev).requires_grad_(True)
    ts = torch.from_numpy(si.gaussian_complex(B, nn, seed=55)).to(dev)
    H = torch.from_numpy(si.gaussian_lowpass(nn)).to(dev)
    def fwd_bwd():
        xs.grad = None
        yv = spectral_filter(xs, H)
        yv.backward(2.0 * (yv.detach() - ts))   # dL/dy of ||y - t||^2
    t_fb = _time_ms(fwd_bwd, reps)
    fp = fc.get_plan(nn, B, "interleaved", False, device=dev)
    ip = fc.get_plan(nn, B, "interleaved", True, device=dev)
    xf = xs.detach().clone()
    t_fft = _time_ms(lambda: fp.execute(xf, xf), reps)
    # the library's share of the step: the same four launches (forward with the filter fused,
    # inverse, twice) on preallocated buffers; the rest is torch (autograd, the 2(y - t)
    # elementwise ops, allocations)
    uf, gf = torch.empty_like(xf), torch.empty_like(xf)
    def lib_only():
        fp.execute_pointwise(xf, H, 1.0 / nn, out=uf)
        ip.execute(uf, uf)
        fp.execute_pointwise(uf, H, 1.0 / nn, out=gf)
        ip.execute(gf, gf)
    t_lib = _time_ms(lib_only, reps)
    res = {"workload": "y = ifft(H * fft(x)) / n, loss ||y - t||^2, x,t [1024, 2^14] complex64",
           "fwd_bwd_ms": round(t_fb, 4), "fft_ms": round(t_fft, 4),
           "library_ms": round(t_lib, 4), "torch_ms": round(max(t_fb - t_lib, 0.0), 4),
           "library_over_4_ffts": round(t_lib / (4 * t_fft), 3),
           "fwd_bwd_over_4_ffts": round(t_fb / (4 * t_fft), 3)}
    del xs, ts, xf, uf, gf
    return res


FP64_SIZES = [1024, 1000, 1 << 16, 1 << 20]
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (CUDA cores); the line also carries a measured rate


def fp64_dgemm_tflops(dev) -> float:
    """FP64 rate measured on this GPU: cuBLAS DGEMM through torch.matmul on float64
    4096 x 4096 operands (2 * 4096^3 flop per product, mean of 3 after a warm-up). A library
    GEMM is the densest FP64 work the device runs, so it bounds the FFT's FP64 arithmetic."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn_like(a)
    t = _time_ms(lambda: torch.matmul(a, b), 3)
    del a, b
    return 2.0 * 4096 ** 3 / (t * 1e-3) / 1e12


def run_fp64(dev, reps: int) -> dict:
    """complex128 transforms, n * batch = 2^25 (512 MiB per buffer), forward, interleaved:
    ms, GFLOP/s (5 n log2 n), the fraction of the nominal FP64 rate and of the FP64 rate
    measured here with a DGEMM, and the HBM fraction per pass (32 B per element and pass)."""
    import torch

    import paper_2308_00497_gb300 as fc
    measured = fp64_dgemm_tflops(dev)
    res = []
    E = ELEMS // 2
    for n in FP64_SIZES:
        B = E // n
        x = torch.randn(B, n, dtype=torch.complex128, device=dev)
        y = torch.empty_like(x)
        p = fc.Plan(n, B, "interleaved", False, precision="fp64", device=dev)
        t = _time_ms(lambda: p.execute(x, y), reps)
        gf = flops(n, B) / (t * 1e-3) / 1e9
        res.append({"n": n, "batch": B, "passes": p.info()[0], "ms": round(t, 4), "gflops": round(gf, 1),
                    "fp64_frac_nominal": round(gf / (FP64_PEAK_TFLOPS * 1e3), 4),
                    "fp64_frac_measured_dgemm": round(gf / (measured * 1e3), 4),
                    "hbm_frac_per_pass": round(32.0 * n * B * p.info()[0] / (t * 1e-3) / 1e9 / peaks()[0], 4)})
        del x, y, p
    return {"workload": "FP64 complex128 C2C, n * batch = 2^25, forward, interleaved", "bound": "alu (FP64)",
            "peak_tflops_nominal": FP64_PEAK_TFLOPS, "peak_tflops_measured_dgemm": round(measured, 3),
            "results": res}


ND_SHAPES = [(1024, 1024), (4096, 4096), (1000, 1000), (256, 256, 256), (64, 64, 64)]


def run_nd(dev, reps: int) -> dict:
    """Rank-2/3 arrays, batch = 2^26 // elements, forward, interleaved: ms, GFLOP/s
    (5 N log2 N per array), HBM passes and the strict HBM fraction (16 B per element)."""
    import torch

    import paper_2308_00497_gb300 as fc
    res = []
    for dims in ND_SHAPES:
        N = int(math.prod(dims))
        B = max(1, ELEMS // N)
        x = torch.randn(B * N, dtype=torch.complex64, device=dev).view((B,) + dims)
        y = torch.empty_like(x)
        p = fc.NdPlan(dims, B, "interleaved", False, device=dev)
        t = _time_ms(lambda: p.execute(x, y), reps)
        res.append({"dims": list(dims), "batch": B, "passes": p.info()[0], "ms": round(t, 4),
                    "gflops": round(5.0 * N * math.log2(N) * B / (t * 1e-3) / 1e9, 1),
                    "hbm_frac_strict": round(16.0 * N * B / (t * 1e-3) / 1e9 / peaks()[0], 4)})
        del x, y, p
    return {"workload": "rank-2/3 C2C, batch * elements ~ 2^26, forward, interleaved", "results": res}


MIXED_SIZES = [12, 96, 360, 1000, 3072, 6000, 10000, 59049, 100000, 1000000]


def run_mixed(dev, reps: int) -> dict:
    """n = 2^a 3^b 5^c 7^d (not powers of two), batch = 2^26 // n, forward, both layouts:
    ms, GFLOP/s (5 n log2 n convention) and the strict HBM fraction (16 B per element)."""
    import torch

    import paper_2308_00497_gb300 as fc
    res = []
    xbuf = torch.randn(2 * ELEMS, device=dev)
    ybuf = torch.empty_like(xbuf)
    for n in MIXED_SIZES:
        B = ELEMS // n
        for layout in LAYOUTS:
            if layout == "interleaved":
                x = xbuf[:2 * n * B].view(torch.complex64).view(B, n)
                y = ybuf[:2 * n * B].view(torch.complex64).view(B, n)
            else:
                x, y = xbuf[:2 * n * B].view(2, B, n), ybuf[:2 * n * B].view(2, B, n)
            p = fc.Plan(n, B, layout, False, device=dev)
            t = _time_ms(lambda: p.execute(x, y), reps)
            res.append({"n": n, "batch": B, "layout": layout, "passes": p.info()[0], "ms": round(t, 4),
                        "gflops": round(flops(n, B) / (t * 1e-3) / 1e9, 1),
                        "hbm_frac_strict": round(16.0 * n * B / (t * 1e-3) / 1e9 / peaks()[0], 4)})
    return {"workload": "mixed-radix n (factors 2, 3, 5, 7), n*batch ~ 2^26, forward, interleaved + split",
            "results": res}


LARGE_SIZES = [1 << 21, 1 << 22, 1 << 23, 1 << 24, 3 ** 15]


def run_large(dev, reps: int) -> dict:
    """Lengths above the sweep, n = 2^21..2^24 (both layouts) and 3^15 (interleaved), batch =
    2^26 // n, forward: ms, GFLOP/s (5 n log2 n), and the HBM fraction strict (16 B per
    element) and per pass (16 B per element and pass)."""
    import torch

    import paper_2308_00497_gb300 as fc
    res = []
    xbuf = torch.randn(2 * ELEMS, device=dev)
    ybuf = torch.empty_like(xbuf)
    for n in LARGE_SIZES:
        B = max(1, ELEMS // n)
        for layout in (LAYOUTS if n & (n - 1) == 0 else ["interleaved"]):
            if layout == "interleaved":
                x = xbuf[:2 * n * B].view(torch.complex64).view(B, n)
                y = ybuf[:2 * n * B].view(torch.complex64).view(B, n)
            else:
                x, y = xbuf[:2 * n * B].view(2, B, n), ybuf[:2 * n * B].view(2, B, n)
            p = fc.Plan(n, B, layout, False, device=dev)
            t = _time_ms(lambda: p.execute(x, y), reps)
            frac = 16.0 * n * B / (t * 1e-3) / 1e9 / peaks()[0]
            res.append({"n": n, "batch": B, "layout": layout, "passes": p.info()[0], "ms": round(t, 4),
                        "gflops": round(flops(n, B) / (t * 1e-3) / 1e9, 1), "hbm_frac_strict": round(frac, 4),
                        "hbm_frac_per_pass": round(frac * p.info()[0], 4)})
            del p
    return {"workload": "n = 2^21..2^24 and 3^15, n*batch ~ 2^26, forward", "results": res}


def run_precision(args, dev, reps: int) -> dict:
    """Radix-16 stages on the tensor cores (FP16/BF16, plain and hi+lo split) vs FP32:
    n = 2^12..2^16, batch 2^14, complex N(0,1); error on sampled rows vs the FP64 oracle."""
    import numpy as np
    import torch

    import oracle
    import paper_2308_00497_gb300 as fc
    import synthetic_inputs as si
    B = 1 << 14
    full = si.gaussian_complex(1, B << 16, seed=3).reshape(B << 16)   # viewed as [B, n] for every n
    x_all = torch.from_numpy(full).to(dev)
    rows = np.array([0, B // 2, B - 1])
    modes = ["fp32", "fp16_tc", "bf16_tc", "fp16_tc_split", "bf16_tc_split"]
    res = []
    for e in range(12, 17):
        n = 1 << e
        x = x_all[: n * B].view(B, n)
        y = torch.empty_like(x)
        ref = oracle.fft(full[: n * B].reshape(B, n)[rows].astype(np.complex128))
        for m in modes:
            p = fc.Plan(n, B, "interleaved", False, m, device=dev)
            if args.tune:
                p.tune(3)  # measure-mode planning, outside the timed region
            t = _time_ms(lambda: p.execute(x, y), reps)
            got = y[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.complex128)
            err = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
            passes, _ = p.info()
            res.append({"n": n, "mode": m, "ms": round(t, 4), "gflops": round(flops(n, B) / (t * 1e-3) / 1e9, 1),
                        "hbm_frac_per_pass": round(16.0 * n * B * passes / (t * 1e-3) / 1e9 / peaks()[0], 4),
                        "rel_l2_max": err})
            p.close()
        del x, y
    return {"workload": "n=2^12..2^16, batch=2^14, complex N(0,1), interleaved, forward", "rows_checked": 3,
            "results": res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fftc", "reference"], default="fftc")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the uneven / filter / precision lines")
    ap.add_argument("--no-precision", action="store_true", help="skip the tensor-core precision line")
    ap.add_argument("--extras", default="uneven,filter,mixed,large,nd,fp64,precision",
                    help="which secondary workloads to run (comma list)")
    ap.add_argument("--sizes", default=",".join(str(e) for e in SIZES),
                    help="log2 n list (default: the whole sweep); a subset is for profiling only")
    ap.add_argument("--layouts", default=",".join(LAYOUTS))
    ap.add_argument("--precision", default="fp32",
                    help="precision of the sweep plans (fp32; the tensor-core modes for n = 2^7..2^16): for profiling")
    ap.add_argument("--dirs", default="fwd,inv")
    ap.add_argument("--tune", type=int, default=1,
                    help="1: measure-mode planning (fftc_plan_tune) before timing; 0: the default table")
    args = ap.parse_args()
    args.sizes = [int(v) for v in args.sizes.split(",")]
    args.layouts = args.layouts.split(",")
    args.dirs = [d == "inv" for d in args.dirs.split(",")]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_fftc(args, rank, world, local_rank)


if __name__ == "__main__":
    main()

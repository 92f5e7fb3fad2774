#!/usr/bin/env python
"""Benchmark of the RT-EOM-CCSD core-hole propagation on B300.

One bench step = one time step of the propagation (Eq. 9): the residual
R(t_n), the fixed-point micro-iterations of the Adams-Moulton update, the
cumulant integrand and C_{n+1} (Eqs. 5-6).  Metric: time steps/s, whole job
(sum over ranks; ranks are independent replicas).

Default workload: the ESCA-shaped propagation O=50, V=450, Nchol=1800,
dt=0.025 au, the paper's micro-iteration cutoff 1e-4, in the split-FP16
form (contractions as row-scaled FP16 hi/lo products on the 16-bit tensor
cores, FP64 update, cumulant and phases).  Beside it, on the same inputs:
the split-TF32 and split-BF16 forms and the FP64-accurate emulated form (a
few steps each), an estimate of the
plain FP64 (DFMA) form from its measured contraction rate, and the
formaldehyde-shaped FP64 workload (O=8, V=100, Nchol=400) as a secondary
line.  Every form reports time per step and per micro-iteration (the
paper's metric) and TFLOP/s against measured peaks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--form split_tf32|split_bf16|split_fp16|fp64_ozaki|fp64]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from synth import workload  # noqa: E402

METRIC = "time_steps_per_s"
UNIT = "steps/s"
MEASURED = os.path.join(HERE, "MEASURED_PEAKS.json")
PROFILES = os.path.join(HERE, "profiles")
FORMS = ("split_tf32", "split_bf16", "split_fp16", "fp64_ozaki", "fp64")
SPLIT_FORMS = ("split_tf32", "split_bf16", "split_fp16")
# tensor-core products executed per FP64-equivalent multiply-add, by form
PRODUCTS = {"split_tf32": 3, "split_bf16": 6, "split_fp16": 3, "fp64_ozaki": 28, "fp64": 1}
# arithmetic type of the contractions, by form
DTYPE = {"split_tf32": "tf32", "split_bf16": "bf16", "split_fp16": "fp16", "fp64_ozaki": "bf16",
         "fp64": "f64"}
KERNEL = {"split_tf32": ("tc_gemm_kernel", "gemm_tc.cu"),
          "split_bf16": ("oz_gemm_kernel<3,128>", "gemm_oz.cu"),
          "split_fp16": ("oz_gemm_kernel<2,256>", "gemm_oz.cu"),
          "fp64_ozaki": ("oz_gemm_kernel<7,64>", "gemm_oz.cu"),
          "fp64": ("gemm_kernel (FP64 DFMA)", "gemm_f64.cu")}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c5_esca_large")
    ap.add_argument("--form", choices=FORMS, default="split_fp16",
                    help="precision form of the headline line")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-micro", type=int, default=50)
    ap.add_argument("--side-steps", type=int, default=2,
                    help="timed steps of each other form on the headline inputs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms")
    ap.add_argument("--no-ozaki", action="store_true", help="skip the emulated-FP64 form")
    ap.add_argument("--no-secondary", action="store_true", help="skip the FP64 c2 line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-requests", type=int, default=12)
    ap.add_argument("--serving-mix", choices=["scaled", "c4"], default="c4",
                    help="scaled: small shapes, FP64, split-TF32 and split-BF16; c4: the "
                         "production request shapes (O~U{4..24}, V~U{40..240}) with steps cut to "
                         "U{4..16}, split-FP16 and split-BF16, autotuner off (serial and served "
                         "runs on equal terms)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(x, world, device=None):
    """The largest x over the ranks of the process group (x itself alone)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps_per_rank, elapsed_max, world):
    """Whole-job steps/s of independent replicas: every rank propagates its
    own core hole, so the job finishes its world * steps when the slowest
    rank does."""
    return world * steps_per_rank / elapsed_max


# ----------------------------------------------------------------- clocks
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
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                pw.append(float(r[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": float(max(pw)) if pw else None}


# ----------------------------------------------------------------- oracle timing
def oracle_micro_per_step(name, tol):
    """Micro-iterations per step of the oracle's own run of this workload at
    this tolerance (stored by tests/golden/make_oracle_golden.py), or None."""
    tag = "" if tol == 1e-12 else f"_tol{tol:g}"
    path = os.path.join(HERE, "tests", "golden", f"oracle_{name}{tag}.txt")
    if not os.path.exists(path):
        return None
    d = np.loadtxt(path)
    return float(d[1:, 5].mean())


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count()


def time_oracle_micro_iteration(p, dt, reps, warm, t_state=None, threads=None):
    """Wall time of one oracle micro-iteration (residual + Eq. 9 update) on
    the host cores (all BLAS threads, or `threads`); returns (mean seconds,
    threads used)."""
    from oracle import propagate as PR
    from oracle.spinexp import CoreHoleCCSD
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    D = sysb.diagonal()
    t = t_state if t_state is not None else [x + 1e-3 for x in sysb.zeros()]
    Rn = [r - d * x for r, d, x in zip(sysb.residual(t), D, t)]

    def run():
        times = []
        for k in range(warm + reps):
            t0 = time.perf_counter()
            try:
                PR.am_step(sysb.residual, D, t, Rn, dt, tol=0.0, max_micro=2)
            except PR.NotConverged:
                pass
            if k >= warm:
                times.append(time.perf_counter() - t0)
        return float(np.mean(times))
    # am_step with tol 0 and max_micro=2 evaluates exactly one residual (k=1)
    # plus two updates, then reports non-convergence
    if threads is None:
        return run(), int(blas_threads())
    from threadpoolctl import threadpool_limits
    with threadpool_limits(limits=threads):
        return run(), int(threads)


def time_oracle_steps(p, dt, tol, nsteps):
    """Wall time of whole oracle time steps (propagate from T(0) = 0)."""
    from oracle import propagate as PR
    from oracle.spinexp import CoreHoleCCSD
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t0 = time.perf_counter()
    out = PR.propagate(sysb, nsteps, dt, tol=tol, max_micro=50)
    return time.perf_counter() - t0, int(np.sum(out["micro"]))


# ----------------------------------------------------------------- peaks
def measured_peaks():
    try:
        return json.load(open(MEASURED))
    except Exception:
        return {}


def matmul_tflops(torch, dev, dtype, n, reps, tf32=False, seconds=0.0):
    """cuBLAS dense GEMM rate: best of `reps` (burst) and, with seconds > 0,
    the mean of back-to-back GEMMs for that long (sustained)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        a = torch.randn(n, n, dtype=dtype, device=dev)
        b = torch.randn(n, n, dtype=dtype, device=dev)
        c = a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        sustained = None
        if seconds > 0:
            k = max(1, int(seconds / best))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(k):
                torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            sustained = 2 * n ** 3 * k / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b, c
        torch.cuda.empty_cache()
        return 2 * n ** 3 / best / 1e12, sustained
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def peaks_block(torch, dev):
    """Measured BF16 (driver file), TF32 and FP64 (cuBLAS, measured here)."""
    pk = measured_peaks()
    tf32_b, tf32_s = matmul_tflops(torch, dev, torch.float32, 8192, 5, tf32=True, seconds=3.0)
    fp64_b, _ = matmul_tflops(torch, dev, torch.float64, 8192, 2)
    return {"bf16_tflops": pk.get("bf16_tflops"),
            "bf16_tflops_sustained": pk.get("bf16_tflops_sustained"),
            "hbm_gbs": pk.get("hbm_gbs"),
            "tf32_tflops": tf32_b, "tf32_tflops_sustained": tf32_s, "fp64_tflops": fp64_b,
            "source": "bf16 and HBM: MEASURED_PEAKS.json (driver); tf32 and fp64: cuBLAS "
                      "torch.matmul 8192^3 measured in this run (tf32: best of 5 and 3 s back "
                      "to back; fp64: best of 2)"}


def peak_for(form, peaks, sustained=True):
    """Tensor-core peak of a form's products: 16-bit planes (split-BF16,
    split-FP16, emulated FP64; FP16 and BF16 products run at one rate),
    TF32 (split-TF32) or the FP64 pipe (FP64)."""
    if form in ("split_bf16", "split_fp16", "fp64_ozaki"):
        v = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops")
        src = "bf16_tflops_sustained (of measured)" if sustained else "bf16_tflops (of measured)"
        if form == "split_fp16":
            src += "; FP16 products run at the BF16 rate (both kind::f16)"
        return v, src
    if form == "split_tf32":
        v = peaks.get("tf32_tflops_sustained" if sustained else "tf32_tflops")
        return v, "tf32, cuBLAS measured in this run (of measured)"
    return peaks.get("fp64_tflops"), "fp64, cuBLAS DGEMM measured in this run (of measured)"


def ncu_traffic(kernel_key):
    """Per-launch DRAM traffic of a kernel from its committed ncu summary
    (profiles/*.txt lines 'kernel_key: ...', 'kernel_source_sha1: ...',
    'traffic_bytes_per_launch: ...'), valid only while the kernel source is
    unchanged; returns (bytes, summary file) or (None, None)."""
    for fn in sorted(os.listdir(PROFILES)) if os.path.isdir(PROFILES) else []:
        vals = {}
        for ln in open(os.path.join(PROFILES, fn)):
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_key") != kernel_key:
            continue
        src = os.path.join(HERE, "paper_2301_04249_b300", "csrc", vals.get("kernel_source", ""))
        if not os.path.exists(src):
            continue
        digest = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
        if vals.get("kernel_source_sha1") != digest:
            continue
        try:
            return float(vals["traffic_bytes_per_launch"]), fn
        except (KeyError, ValueError):
            continue
    return None, None


# ----------------------------------------------------------------- one form
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def precision_of(P, form):
    return {"split_tf32": P.RTEOM_SPLIT_TF32, "split_bf16": P.RTEOM_SPLIT_BF16,
            "split_fp16": P.RTEOM_SPLIT_FP16, "fp64_ozaki": P.RTEOM_FP64_OZAKI,
            "fp64": P.RTEOM_FP64}[form]


def pinned_problem(torch, p):
    """The problem's host arrays in pinned memory (the caller's buffers)."""
    def pin(a):
        if a is None:
            return None
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()
    return pin(p.eps), pin(p.L), pin(p.t1_gs), pin(p.t2_gs)


def run_form(torch, P, p, host, form, dt, warmup, steps, tol, max_micro, stream, world,
             sampler=None, timing_mode=3, flags=0):
    """One context of `form` on the pinned host inputs: create, `warmup`
    untimed steps, `steps` timed steps (each a propagate call returning its
    C_n to the host), the spectrum, destroy.  Device time of the timed steps
    by CUDA events on the context's stream; wall time of the whole sequence
    for the end-to-end figure."""
    h_eps, h_L, h_t1, h_t2 = host
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    w0 = time.perf_counter()
    g = P.Propagator(h_eps, h_L, p.nocc, p.nvir, h_t1, h_t2, core=p.core,
                     precision=precision_of(P, form), flags=flags, stream=stream)
    setup_s = time.perf_counter() - w0
    held = free0 - torch.cuda.mem_get_info()[0]
    C_steps = []
    for _ in range(warmup):
        C_steps.append(g.propagate(1, dt, tol=tol, max_micro=max_micro)[-1])
    info0 = g.info()
    g.set_timing(timing_mode)
    g.timing(reset=True)
    l0 = g.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")  # launch lists: --nvtx-include "bench_timed/"
    e0.record(stream)
    for _ in range(steps):
        C_steps.append(g.propagate(1, dt, tol=tol, max_micro=max_micro)[-1])
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    elapsed = e0.elapsed_time(e1) / 1e3
    info1 = g.info()
    tm = g.timing()
    launches = g.kernel_launches() - l0
    C, _ = g.cumulant()
    omega = np.linspace(-25.0, -15.0, 2001)
    A = g.spectrum(omega, 0.05)
    g.close()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    h2d = sum(x.nbytes for x in host if x is not None) + omega.nbytes
    return dict(form=form, setup_s=setup_s, device_bytes_held=held, elapsed=elapsed,
                micro=info1["micro"] - info0["micro"], steps=steps, warmup=warmup, tm=tm,
                launches=launches, C=C, wall=wall, h2d=h2d, d2h=16 * (warmup + steps) + A.nbytes,
                clocks=clocks)


def form_summary(r, peaks, world):
    """Per-form figures: steps/s, per micro-iteration, and the roofline of the
    form's contraction kernel over every contraction launch of the timed steps
    (event nodes inside the residual graphs)."""
    form = r["form"]
    tm = r["tm"]
    steps, micro, el = r["steps"], max(r["micro"], 1), r["elapsed"]
    con = {k: tm["ladder"][k] + tm["contract"][k] for k in ("ms", "launches", "flops", "bytes")}
    eq_flops = sum(v["flops"] for v in tm.values())
    prod = PRODUCTS[form]
    gemm_s = con["ms"] / 1e3
    eq_rate = con["flops"] / gemm_s / 1e12 if gemm_s > 0 else None
    peak, src = peak_for(form, peaks)
    exe_rate = eq_rate * prod if eq_rate else None
    lad = tm["ladder"]
    lad_s = lad["ms"] / 1e3
    kname, ksrc = KERNEL[form]
    traffic, tfile = ncu_traffic(f"{form}:contraction")
    return {
        "value": world * steps / el, "unit": UNIT, "ms_per_step": 1e3 * el / steps,
        "micro_iterations_per_step": r["micro"] / steps,
        "ms_per_micro_iteration": 1e3 * el / micro,
        "setup_s": r["setup_s"], "device_bytes_held": r["device_bytes_held"],
        "gpu_launches": r["launches"],
        "fp64_equivalent_tflops_step": eq_flops / el / 1e12,
        "fp64_equivalent_tflop_per_micro_iteration": eq_flops / micro / 1e12,
        "contraction_time_share": gemm_s / el,
        "roofline": {
            "bound": "alu" if form == "fp64" else "tensor",
            "kernel": kname + ", every contraction launch of the timed steps",
            "achieved": exe_rate, "peak": peak, "unit": "TFLOP/s",
            "frac": exe_rate / peak if (exe_rate and peak) else None,
            "peak_source": src, "traffic": traffic, "traffic_source": tfile,
            "fp64_equivalent_tflops": eq_rate,
            "frac_of_fp64_peak": eq_rate / peaks["fp64_tflops"]
            if (eq_rate and peaks.get("fp64_tflops")) else None,
            "launches": con["launches"], "avg_launch_ms": con["ms"] / max(con["launches"], 1),
            "flops_per_launch_fp64_equivalent": con["flops"] / max(con["launches"], 1),
            "products_per_multiply_add": prod,
            "note": "achieved = FP64-equivalent FLOPs of the contractions as posed on the "
                    "slot spaces (2/4/8 per real/mixed/complex multiply-add, tile padding "
                    "excluded) x the form's products per multiply-add / summed event time of "
                    "the contraction launches (split-K finalizes and operand packs excluded)"},
        "ladder": {"launches": lad["launches"], "ms": lad["ms"],
                   "fp64_equivalent_tflops": lad["flops"] / lad_s / 1e12 if lad_s > 0 else None,
                   "executed_tflops": lad["flops"] * prod / lad_s / 1e12 if lad_s > 0 else None},
    }


# ----------------------------------------------------------------- serving
def serving_mix(n_req, kind="scaled"):
    """Core-hole request mixes (seeds 4000 + r, dt = 0.025 au, Nchol = 4V).
    scaled: O ~ U{4..8}, V ~ U{20..48}, steps ~ U{20..80}.
    c4: production core-hole shapes O ~ U{4..24}, V ~ U{40..240}, with steps ~ U{4..16}
    instead of U{500..4000}."""
    from synth import gen_problem
    rng = np.random.default_rng(4)
    out = []
    for r in range(n_req):
        if kind == "c4":
            O = int(rng.integers(4, 25))
            V = int(rng.integers(40, 241))
            steps = int(rng.integers(4, 17))
        else:
            O = int(rng.integers(4, 9))
            V = int(rng.integers(20, 49))
            steps = int(rng.integers(20, 81))
        out.append((gen_problem(O, V, 4 * V, 4000 + r), steps))
    return out


def run_serving(P, precision, n_req, tol, kind="scaled", flags=0, serial=None):
    """Serve the mix with Poisson arrivals at twice the mean service rate;
    returns latency percentiles, makespan and the serial (one at a time)
    reference measured on the same requests (or taken from ``serial``, the
    per-request service times of an earlier run of the same mix and form).
    flags: request flags (RTEOM_FLAG_GROUPED: running requests share grouped
    ladder launches)."""
    mix = serving_mix(n_req, kind)
    dt = 0.025
    if serial is None:
        serial = []
        with P.Server(max_active=1, precision=precision) as s:
            for p, n in mix:
                t0 = time.perf_counter()
                rid = s.submit(p, n, dt, tol=tol, flags=flags)
                s.wait(rid, 600.0)
                serial.append(time.perf_counter() - t0)
    mean_service = float(np.mean(serial))
    rate = 2.0 / mean_service
    arrivals = np.cumsum(np.random.default_rng(44).exponential(1.0 / rate, n_req))
    arrivals -= arrivals[0]
    with P.Server(max_active=8, precision=precision) as s:
        t0 = time.perf_counter()
        ids = []
        for (p, n), ta in zip(mix, arrivals):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0005)
            ids.append(s.submit(p, n, dt, tol=tol, flags=flags))
        for rid in ids:
            s.wait(rid, 600.0)
        makespan = time.perf_counter() - t0
        polls = [s.poll(rid) for rid in ids]
        st = s.stats()
    lat = np.array([t[3][2] - t[3][0] for t in polls])
    wait = np.array([t[3][1] - t[3][0] for t in polls])
    steps = sum(n for _, n in mix)
    return {"requests": n_req, "done": st["done"], "failed": st["failed"],
            "arrival_rate_per_s": rate, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_queue_wait_s": float(np.percentile(wait, 50)), "makespan_s": makespan,
            "throughput_steps_per_s": steps / makespan,
            "serial_steps_per_s": steps / float(np.sum(serial)),
            "speedup_vs_serial": float(np.sum(serial)) / makespan,
            "mean_service_s": mean_service, "serial_service_s": [float(x) for x in serial],
            "grouped_ladder": bool(flags & P.RTEOM_FLAG_GROUPED)}


def serving_block(P, args):
    if args.no_serving:
        return None
    if args.serving_mix == "c4":
        os.environ["RTEOM_AUTOTUNE"] = "0"
        try:
            fp16 = run_serving(P, P.RTEOM_SPLIT_FP16, args.serving_requests, args.tol, "c4")
            # the same mix with grouped ladder launches, against the same
            # one-at-a-time reference
            fp16_grouped = run_serving(P, P.RTEOM_SPLIT_FP16, args.serving_requests, args.tol,
                                       "c4", flags=P.RTEOM_FLAG_GROUPED,
                                       serial=fp16["serial_service_s"])
            return {"workload": f"c4 shapes: {args.serving_requests} requests, O~U{{4..24}}, "
                                "V~U{40..240}, Nchol=4V, steps~U{4..16} (production: "
                                "U{500..4000}), dt=0.025, Poisson arrivals at 2x the mean "
                                "service rate, 8 slots, admission by device memory, autotuner off",
                    "split_fp16": fp16, "split_fp16_grouped": fp16_grouped,
                    "split_bf16": run_serving(P, P.RTEOM_SPLIT_BF16, args.serving_requests,
                                              args.tol, "c4")}
        finally:
            del os.environ["RTEOM_AUTOTUNE"]
    bf16 = run_serving(P, P.RTEOM_SPLIT_BF16, args.serving_requests, args.tol)
    return {"workload": f"scaled core-hole mix: {args.serving_requests} requests, O~U{{4..8}}, "
                        "V~U{20..48}, Nchol=4V, steps~U{20..80}, dt=0.025, Poisson arrivals at 2x "
                        "the mean service rate, 8 slots",
            "fp64": run_serving(P, P.RTEOM_FP64, args.serving_requests, args.tol),
            "split_tf32": run_serving(P, P.RTEOM_SPLIT_TF32, args.serving_requests, args.tol),
            "split_bf16": bf16,
            "split_bf16_grouped": run_serving(P, P.RTEOM_SPLIT_BF16, args.serving_requests,
                                              args.tol, flags=P.RTEOM_FLAG_GROUPED,
                                              serial=bf16["serial_service_s"])}


# ----------------------------------------------------------------- our arm
def describe(name, p, dt, tol, form=None):
    s = f"{name}: O={p.nocc} V={p.nvir} Nchol={p.nchol} dt={dt} tol={tol:g}"
    return s + (f" form={form}" if form else "")


def run_ours(args):
    import torch
    import paper_2301_04249_b300 as P

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    p, run = workload(args.workload)
    dt = run["dt"]
    host = pinned_problem(torch, p)
    sampler = ClockSampler(local)
    head = run_form(torch, P, p, host, args.form, dt, args.warmup, args.steps, args.tol,
                    args.max_micro, stream, world, sampler=sampler)
    elapsed = max_over_ranks(head["elapsed"], world, dev)
    e2e_wall = max_over_ranks(head["wall"], world, dev)

    # the other forms on the same inputs (first steps; per micro-iteration
    # figures compare forms whatever the micro-iterations per step)
    side = {}
    if not args.no_forms:
        others = [f for f in SPLIT_FORMS if f != args.form]
        if not args.no_ozaki and args.form != "fp64_ozaki":
            others.append("fp64_ozaki")
        for f in others:
            n = 1 if f == "fp64_ozaki" else args.side_steps
            side[f] = run_form(torch, P, p, host, f, dt, 0, n, args.tol, args.max_micro, stream,
                               world)
    # the formaldehyde-shaped workload in plain FP64 (the DFMA contraction
    # rate also gives the FP64 form's estimate at the headline size)
    sec = None
    if not args.no_secondary:
        p2, run2 = workload("c2_formaldehyde")
        host2 = pinned_problem(torch, p2)
        sec = run_form(torch, P, p2, host2, "fp64", run2["dt"], args.warmup, args.steps,
                       args.tol, args.max_micro, stream, world)
    # the cached (vv|vv) ladder block against forming it from the Cholesky
    # vectors at every residual, on the formaldehyde-shaped workload
    ablation = None
    if not args.no_secondary:
        abl = {}
        for form in ("fp64", "split_tf32"):
            for mode, fl in (("resident", 0), ("cholesky", P.RTEOM_FLAG_LADDER_CHOLESKY)):
                r = run_form(torch, P, p2, host2, form, run2["dt"], 3, 10, args.tol,
                             args.max_micro, stream, world, flags=fl)
                abl[f"{form}_{mode}"] = {"ms_per_micro_iteration": 1e3 * r["elapsed"] / max(r["micro"], 1),
                                         "device_bytes_held": r["device_bytes_held"]}
            abl[f"{form}_cholesky_over_resident"] = (abl[f"{form}_cholesky"]["ms_per_micro_iteration"]
                                                     / abl[f"{form}_resident"]["ms_per_micro_iteration"])
        ablation = {"workload": describe("c2_formaldehyde", p2, run2["dt"], args.tol),
                    "what": "time per micro-iteration with the resident (vv|vv) ladder block "
                            "(cached W) and with the Cholesky mode (W formed from L at every "
                            "residual), 10 timed steps after 3 untimed", **abl}
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peaks = peaks_block(torch, dev)
    value = replica_throughput(args.steps, elapsed, world)
    hs = form_summary(head, peaks, world)
    forms = {f: form_summary(r, peaks, world) for f, r in side.items()}
    for f, r in side.items():
        n = min(len(r["C"]), len(head["C"]))
        forms[f]["max_abs_dC_vs_headline"] = float(np.abs(r["C"][:n] - head["C"][:n]).max())
        forms[f]["timed_steps"] = r["steps"]
        forms[f]["ms_per_micro_iteration_vs_headline"] = (
            forms[f]["ms_per_micro_iteration"] / hs["ms_per_micro_iteration"])
    secondary = None
    if sec is not None:
        ss = form_summary(sec, peaks, world)
        secondary = {"workload": describe("c2_formaldehyde", p2, run2["dt"], args.tol, "fp64"),
                     **ss, "clocks": None}
        # FP64 (DFMA) form at the headline size, from its contraction rate
        dfma = ss["roofline"]["fp64_equivalent_tflops"]
        per_micro = hs["fp64_equivalent_tflop_per_micro_iteration"]
        if dfma:
            est = per_micro / dfma
            forms["fp64"] = {
                "estimated": True, "s_per_micro_iteration": est,
                "ms_per_micro_iteration_vs_headline": 1e3 * est / hs["ms_per_micro_iteration"],
                "note": f"not run at this size: {per_micro:.3g} FP64-equivalent TFLOP per "
                        f"micro-iteration / the {dfma:.3g} TFLOP/s the DFMA contractions "
                        "reached on the c2 line"}

    cpu = None
    if not args.no_cpu_baseline and secondary is not None:
        cpu = cpu_baseline_block(args, hs, secondary["fp64_equivalent_tflop_per_micro_iteration"])

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.form],
        "data": "synthetic (seeded; no molecular integrals available)",
        "config": {"workload": describe(args.workload, p, dt, args.tol, args.form),
                   "form": args.form,
                   "arithmetic": "contractions as split products on the tensor cores with FP32 "
                                 "accumulation; Adams-Moulton update, cumulant and phases FP64"
                   if args.form in SPLIT_FORMS else
                   ("contractions FP64-accurate from BF16 digit planes" if args.form ==
                    "fp64_ozaki" else "FP64 throughout"),
                   "parallelism": f"replicas x{world} (independent core holes, no collectives)",
                   "l2": "inputs larger than L2: the amplitude sets alone are "
                         f"{16 * 3 * (p.nocc * p.nocc * (p.nvir + 1) ** 2) / 1e9:.1f} GB",
                   "steps_from": f"T(0) = 0; {args.warmup} untimed steps, then {args.steps} "
                                 "timed steps, each returning C_n to the host"},
        "micro_iterations_per_step": hs["micro_iterations_per_step"],
        "ms_per_micro_iteration": hs["ms_per_micro_iteration"],
        "fp64_equivalent_tflops": hs["fp64_equivalent_tflops_step"],
        "roofline": hs["roofline"],
        "ladder": hs["ladder"],
        "setup_s": hs["setup_s"], "device_bytes_held": hs["device_bytes_held"],
        "cpu_baseline": cpu,
        "e2e": {"value": replica_throughput(args.warmup + args.steps, e2e_wall, world),
                "unit": UNIT,
                "h2d_bytes_per_step": head["h2d"] / (args.warmup + args.steps),
                "d2h_bytes_per_step": head["d2h"] / (args.warmup + args.steps),
                "what": "rteom_create from pinned host arrays + every step through "
                        "rteom_propagate(1) returning its C_n + rteom_spectrum + destroy, wall "
                        "clock over all warm-up and timed steps"},
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "peaks": peaks,
        "forms": forms,
        "secondary": secondary,
        "ablation_cached_w": ablation,
        "serving": serving_block(P, args),
    }
    print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline_block(args, hs, c2_tflop_per_micro):
    """The oracle on the host cores: one micro-iteration of the
    formaldehyde-shaped workload (the oracle cannot hold a residual of the
    headline size in host memory), scaled to the headline workload by the
    ratio of FP64-equivalent FLOPs per micro-iteration (both counted by the
    library on its own runs)."""
    p2, run2 = workload("c2_formaldehyde")
    t_mi, threads = time_oracle_micro_iteration(p2, run2["dt"], reps=1, warm=0)
    scale = hs["fp64_equivalent_tflop_per_micro_iteration"] / c2_tflop_per_micro
    m = hs["micro_iterations_per_step"]
    est_step = t_mi * scale * m
    return {"value": 1.0 / est_step, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one oracle micro-iteration of c2_formaldehyde (O=8 V=100 Nchol=400) on "
                      f"the host ({t_mi:.2f} s), extrapolated to {args.workload} by the ratio of "
                      f"FP64-equivalent FLOPs per micro-iteration ({scale:.3g}x) and "
                      f"{m:.2f} micro-iterations per step: the oracle cannot hold a residual of "
                      "this size in host memory",
            "micro_iteration_s_c2": t_mi, "extrapolated": True}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle on the host cores, timed on whole time steps of the
    formaldehyde-shaped workload (O=8, V=100, Nchol=400; its largest
    configuration that fits host memory), plus one micro-iteration on one
    core; the headline size is given as a FLOP-scaled estimate."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    p, run = workload("c2_formaldehyde")
    n = max(1, args.steps)
    el, micro = time_oracle_steps(p, run["dt"], args.tol, n)
    threads = int(blas_threads())
    t1, _ = time_oracle_micro_iteration(p, run["dt"], reps=1, warm=0, threads=1)
    value = n / el
    sample = (f"whole oracle time steps of c2_formaldehyde (O=8 V=100 Nchol=400, dt "
              f"{run['dt']}, tol {args.tol:g}) from T(0) = 0 on {threads} host threads: {n} "
              f"steps, {micro} micro-iterations in {el:.1f} s; the oracle cannot hold a "
              f"residual of {args.workload} in host memory; one micro-iteration on one core "
              f"takes {t1:.1f} s")
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": describe("c2_formaldehyde", p, run["dt"], args.tol),
                      "headline_workload": args.workload},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample, "one_core_micro_iteration_s": t1,
                            "micro_iterations_per_step": micro / n},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def main():
    args = parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

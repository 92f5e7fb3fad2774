#!/usr/bin/env python
"""Benchmark of the RT-EOM-CCSD core-hole propagation on B300.

One bench step = one time step of the propagation (Eq. 9): the residual
R(t_n), the fixed-point micro-iterations of the Adams-Moulton update, the
cumulant integrand and C_{n+1} (Eqs. 5-6).  Metric: time steps/s, whole job
(sum over ranks; ranks are independent replicas).  Default workload: the
formaldehyde-shaped FP64 problem O=8, V=100, Nchol=400, dt=0.025 au, with
the paper's micro-iteration cutoff 1e-4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
FP64_NOMINAL_TFLOPS = 1.25  # B300 FP64 (profiling recipe table); no tensor-core FP64 path
TF32_PER_BF16_NOMINAL = 1.1 / 2.25  # dense TF32 / dense BF16, nominal B300 figures
MEASURED = os.path.join(HERE, "MEASURED_PEAKS.json")
LADDER_PROFILE = os.path.join(HERE, "profiles", "ladder_gemm_f64_c2.txt")
LADDER_TC_PROFILE = os.path.join(HERE, "profiles", "ladder_tc_tf32_c2.txt")
LADDER_OZ_PROFILE = os.path.join(HERE, "profiles", "ladder_oz_bf16_c2.txt")
LADDER_OZ3_PROFILE = os.path.join(HERE, "profiles", "ladder_oz3_split_bf16_c2.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2_formaldehyde")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-micro", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the split-TF32 and split-BF16 forms")
    ap.add_argument("--no-ozaki", action="store_true", help="skip the emulated-FP64 form")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serving-requests", type=int, default=16)
    ap.add_argument("--serving-mix", choices=["scaled", "c4"], default="scaled",
                    help="scaled: small shapes, all three forms; c4: the production request "
                         "shapes (O~U{4..24}, V~U{40..240}) with steps cut to U{4..16}, tensor-core forms only, "
                         "autotuner off (serial and served runs on equal terms)")
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


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


def time_oracle_micro_iteration(p, dt, reps, warm, t_state=None):
    """Wall time of one oracle micro-iteration (residual + Eq. 9 update) on
    the host cores; returns (mean seconds, threads used)."""
    from oracle import propagate as PR
    from oracle.spinexp import CoreHoleCCSD
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    D = sysb.diagonal()
    t = t_state if t_state is not None else [x + 1e-3 for x in sysb.zeros()]
    Rn = [r - d * x for r, d, x in zip(sysb.residual(t), D, t)]
    times = []
    for k in range(warm + reps):
        t0 = time.perf_counter()
        try:
            PR.am_step(sysb.residual, D, t, Rn, dt, tol=0.0, max_micro=2)
        except PR.NotConverged:
            pass
        if k >= warm:
            times.append(time.perf_counter() - t0)
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count()
    # am_step with tol 0 and max_micro=2 evaluates exactly one residual (k=1)
    # plus two updates, then reports non-convergence
    return float(np.mean(times)), int(threads)


# ----------------------------------------------------------------- helpers
def measured_peaks():
    try:
        return json.load(open(MEASURED))
    except Exception:
        return {}


def ladder_traffic_per_launch(profile=LADDER_PROFILE, source="gemm_f64.cu"):
    """Per-launch DRAM bytes of a ladder kernel from its committed ncu summary,
    valid only while the kernel source is unchanged."""
    if not os.path.exists(profile):
        return None
    src = os.path.join(HERE, "paper_2301_04249_b300", "csrc", source)
    digest = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    vals = {}
    for ln in open(profile):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1") != digest:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def fp64_dgemm_tflops(torch, dev):
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2 * 4096 ** 3 / best / 1e12


def split_summary(split, args, fp64_value, world, C_fp64, peaks):
    """Steps/s, speedup, cumulant deviation and tensor-pipe roofline of the
    split-TF32 form measured on the same workload and step counts."""
    if split is None:
        return None
    tm = split["tm"]
    lad = tm["ladder"]
    v = world * args.steps / split["elapsed"]
    bf16 = peaks.get("bf16_tflops")
    hbm = peaks.get("hbm_gbs")
    tf32_peak = bf16 * TF32_PER_BF16_NOMINAL if bf16 else None
    avg_s = lad["ms"] / 1e3 / max(lad["launches"], 1)
    fl = lad["flops"] / max(lad["launches"], 1)
    by = lad["bytes"] / max(lad["launches"], 1)
    ach = fl / avg_s / 1e12 if lad["launches"] else None
    ach_gbs = by / avg_s / 1e9 if lad["launches"] else None
    n = min(len(C_fp64), len(split["C"]))
    dC = float(np.abs(np.asarray(split["C"])[:n] - np.asarray(C_fp64)[:n]).max())
    return {"split_tf32": {
        "value": v, "unit": UNIT, "ms_per_step": 1e3 * split["elapsed"] / args.steps,
        "speedup_vs_fp64": v / fp64_value,
        "micro_iterations_per_step": split["micro"] / args.steps,
        "max_abs_dC_vs_fp64": dC,
        "gpu_launches": split["launches"],
        "roofline": {"bound": "hbm", "kernel": "tc_gemm_kernel (tcgen05 kind::tf32, ladder)",
                     "achieved": ach_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": ach_gbs / hbm if (ach_gbs and hbm) else None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                     "traffic": ladder_traffic_per_launch(LADDER_TC_PROFILE, "gemm_tc.cu"),
                     "bytes_per_launch": by, "avg_launch_ms": avg_s * 1e3,
                     "launches": lad["launches"],
                     "tensor": {"achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s",
                                "frac": ach / tf32_peak if (ach and tf32_peak) else None,
                                "peak_source": "measured BF16 x nominal TF32/BF16 ratio",
                                "flops_per_launch_executed": fl},
                     "note": "bytes: packed hi/lo operands read once + FP32 split-K slabs; at "
                             "this size 85 FLOP/B, below the TF32 ridge, so HBM binds; "
                             "traffic is the alpha-beta launch (the largest), bytes_per_launch "
                             "the mean over the three ladder launches of a residual"},
    }}


def ozaki_summary(run, args, fp64_value, world, C_fp64, peaks, name="fp64_ozaki", planes=7,
                  profile=LADDER_OZ_PROFILE):
    """Steps/s, speedup, cumulant deviation and tensor-pipe roofline of a
    digit-sliced form (emulated FP64: 7 planes; split-BF16: 3 planes)
    measured on the same workload and step counts."""
    if run is None:
        return None
    products = planes * (planes + 1) // 2
    lad = run["tm"]["ladder"]
    v = world * args.steps / run["elapsed"]
    bf16 = peaks.get("bf16_tflops")
    avg_s = lad["ms"] / 1e3 / max(lad["launches"], 1)
    fl = lad["flops"] / max(lad["launches"], 1)  # FP64-equivalent
    eq = fl / avg_s / 1e12 if lad["launches"] else None
    ach = products * eq if eq else None
    n = min(len(C_fp64), len(run["C"]))
    Cf = np.asarray(C_fp64)[:n]
    dC = float(np.abs(np.asarray(run["C"])[:n] - Cf).max())
    return {name: {
        "value": v, "unit": UNIT, "ms_per_step": 1e3 * run["elapsed"] / args.steps,
        "speedup_vs_fp64": v / fp64_value,
        "micro_iterations_per_step": run["micro"] / args.steps,
        "max_abs_dC_vs_fp64": dC,
        "max_rel_dC_vs_fp64": dC / max(float(np.abs(Cf).max()), 1e-300),
        "gpu_launches": run["launches"],
        "fp64_equivalent_tflops_total": sum(x["flops"] for x in run["tm"].values())
                                       / run["elapsed"] / 1e12,
        "roofline": {"bound": "tensor",
                     "kernel": f"oz_gemm_kernel<{planes}> (tcgen05 kind::f16, BF16 digit planes, "
                               "ladder)",
                     "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                     "frac": ach / bf16 if (ach and bf16) else None,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured, burst)",
                     "fp64_equivalent_tflops": eq,
                     "frac_of_fp64_nominal": eq / FP64_NOMINAL_TFLOPS if eq else None,
                     "traffic": ladder_traffic_per_launch(profile, "gemm_oz.cu")
                                if profile else None,
                     "flops_per_launch_executed": products * fl,
                     "avg_launch_ms": avg_s * 1e3, "launches": lad["launches"],
                     "note": f"executed = {products} BF16 digit-pair products per "
                             "FP64-equivalent multiply-add of the real-embedded GEMM; the mean "
                             "is over the three ladder launches of a residual"}},
    }


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


def run_serving(P, precision, n_req, tol, kind="scaled"):
    """Serve the mix with Poisson arrivals at twice the mean service rate;
    returns latency percentiles, makespan and the serial (one at a time)
    reference measured on the same requests."""
    mix = serving_mix(n_req, kind)
    dt = 0.025
    # serial reference: every request alone, back to back (also its service time)
    serial = []
    with P.Server(max_active=1, precision=precision) as s:
        for p, n in mix:
            t0 = time.perf_counter()
            rid = s.submit(p, n, dt, tol=tol)
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
            ids.append(s.submit(p, n, dt, tol=tol))
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
            "mean_service_s": mean_service}


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_2301_04249_b300 as P

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p, run = workload(args.workload)
    dt = run["dt"]
    stream = torch.cuda.Stream(device=dev)
    g = P.Propagator.from_problem(p, stream=stream)
    g.propagate(args.warmup, dt, tol=args.tol, max_micro=args.max_micro)
    info0 = g.info()
    g.set_timing(True)
    g.timing(reset=True)
    launches0 = g.kernel_launches()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")  # launch lists: --nvtx-include "bench_timed/"
    e0.record(stream)
    g.propagate(args.steps, dt, tol=args.tol, max_micro=args.max_micro)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    elapsed = max_over_ranks(elapsed, world, dev)
    info1 = g.info()
    tm = g.timing()
    launches = g.kernel_launches() - launches0
    micro = info1["micro"] - info0["micro"]
    state = g.get_state(with_history=False)["t"]
    fp64_hist, _ = g.cumulant()
    g.close()

    # end to end through the public API from pinned host buffers
    def pinned(a):
        if a is None:
            return None
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()
    h_eps, h_L, h_t1, h_t2 = pinned(p.eps), pinned(p.L), pinned(p.t1_gs), pinned(p.t2_gs)
    omega = pinned(np.linspace(-25.0, -15.0, 2001))
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    g2 = P.Propagator(h_eps, h_L, p.nocc, p.nvir, h_t1, h_t2, core=p.core, stream=stream)
    Cs = [g2.propagate(1, dt, tol=args.tol, max_micro=args.max_micro)[-1] for _ in range(args.steps)]
    A = g2.spectrum(omega, 0.05)
    g2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    h2d = sum(x.nbytes for x in (h_eps, h_L, h_t1, h_t2, omega) if x is not None)
    d2h = 16 * 2 * args.steps + A.nbytes
    e2e_s = max_over_ranks(e2e_s, world, dev)

    # the other precision forms on the same inputs, same step counts
    def run_form(prec):
        gs = P.Propagator.from_problem(p, stream=stream, precision=prec)
        gs.propagate(args.warmup, dt, tol=args.tol, max_micro=args.max_micro)
        i0 = gs.info()
        gs.set_timing(True)
        gs.timing(reset=True)
        l0 = gs.kernel_launches()
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        gs.propagate(args.steps, dt, tol=args.tol, max_micro=args.max_micro)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        el_s = f0.elapsed_time(f1) / 1e3
        tms = gs.timing()
        i1 = gs.info()
        Cf, _ = gs.cumulant()
        nl = gs.kernel_launches() - l0
        gs.close()
        return dict(elapsed=el_s, tm=tms, micro=i1["micro"] - i0["micro"], C=Cf, launches=nl)

    split = None if args.no_split else run_form(P.RTEOM_SPLIT_TF32)
    split_bf16 = None if args.no_split else run_form(P.RTEOM_SPLIT_BF16)
    ozaki = None if args.no_ozaki else run_form(P.RTEOM_FP64_OZAKI)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    value = replica_throughput(args.steps, elapsed, world)
    serving = None
    if not args.no_serving and args.serving_mix == "c4":
        os.environ["RTEOM_AUTOTUNE"] = "0"
        serving = {"workload": f"c4 shapes: {args.serving_requests} requests, O~U{{4..24}}, "
                               "V~U{40..240}, Nchol=4V, steps~U{4..16} (production: U{500..4000}), "
                               "dt=0.025, Poisson arrivals at 2x the mean service rate, 8 slots, "
                               "admission by device memory, autotuner off",
                   "fp64": "not run: one FP64 residual of the largest request takes about 30 s",
                   "split_tf32": run_serving(P, P.RTEOM_SPLIT_TF32, args.serving_requests,
                                             args.tol, "c4"),
                   "split_bf16": run_serving(P, P.RTEOM_SPLIT_BF16, args.serving_requests,
                                             args.tol, "c4"),
                   "fp64_ozaki": run_serving(P, P.RTEOM_FP64_OZAKI, args.serving_requests,
                                             args.tol, "c4")}
        del os.environ["RTEOM_AUTOTUNE"]
    elif not args.no_serving:
        serving = {"workload": "scaled core-hole mix: 16 requests, O~U{4..8}, V~U{20..48}, "
                               "Nchol=4V, steps~U{20..80}, dt=0.025, Poisson arrivals at 2x the "
                               "mean service rate, 8 slots",
                   "fp64": run_serving(P, P.RTEOM_FP64, args.serving_requests, args.tol),
                   "split_tf32": run_serving(P, P.RTEOM_SPLIT_TF32, args.serving_requests,
                                             args.tol),
                   "fp64_ozaki": run_serving(P, P.RTEOM_FP64_OZAKI, args.serving_requests,
                                             args.tol)}
    lad = tm["ladder"]
    peaks = measured_peaks()
    dgemm = fp64_dgemm_tflops(torch, dev)
    lad_avg_s = lad["ms"] / 1e3 / max(lad["launches"], 1)
    lad_flops = lad["flops"] / max(lad["launches"], 1)
    achieved = lad_flops / lad_avg_s / 1e12 if lad["launches"] else None
    traffic = ladder_traffic_per_launch()
    total_flops = sum(v["flops"] for v in tm.values())
    roofline = {"bound": "alu", "kernel": "gemm_f64 (particle-particle ladder, FP64 DFMA)",
                "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_NOMINAL_TFLOPS if achieved else None,
                "peak_source": "B300 nominal FP64 (recipe table); cuBLAS DGEMM measured live below",
                "cublas_dgemm_tflops_measured": dgemm,
                "frac_of_cublas_dgemm": achieved / dgemm if achieved else None,
                "flops_per_launch": lad_flops, "avg_launch_ms": lad_avg_s * 1e3,
                "launches": lad["launches"], "traffic": traffic}

    cpu = None
    m_ref = oracle_micro_per_step(args.workload, args.tol)
    if not args.no_cpu_baseline:
        blocks = P.split_blocks(state, p.nocc, p.nvir)
        t_mi, threads = time_oracle_micro_iteration(p, dt, reps=1, warm=0, t_state=blocks)
        m_use = m_ref if m_ref is not None else micro / args.steps
        cpu = {"value": 1.0 / (t_mi * m_use), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"one oracle micro-iteration (residual + Eq. 9 update) of workload "
                          f"{args.workload} timed on the host ({t_mi:.2f} s), scaled by "
                          f"{m_use:.2f} micro-iterations per step "
                          + ("(the oracle's own run at this tol)" if m_ref is not None
                             else "(measured on the GPU run)")),
               "micro_iteration_s": t_mi}

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; no molecular integrals available)",
        "config": {"workload": f"{args.workload}: O={p.nocc} V={p.nvir} Nchol={p.nchol} "
                               f"dt={dt} tol={args.tol} precision=FP64 complex",
                   "parallelism": f"replicas x{world} (independent core holes, no collectives)",
                   "l2": "inputs larger than L2: the (ae|bf) ladder block alone is "
                         f"{8 * (p.nvir + 1) ** 4 / 1e9:.2f} GB",
                   "flops_per_step_tflop": total_flops / args.steps / 1e12},
        "micro_iterations_per_step": micro / args.steps,
        "micro_iterations_per_s": world * micro / elapsed,
        "tflops_fp64": total_flops / elapsed / 1e12,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": replica_throughput(args.steps, e2e_s, world), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "rteom_create from pinned host arrays + per-step rteom_propagate(1) "
                        "returning C_n + rteom_spectrum + destroy, wall clock"},
        "gpu_launches": launches,
        "clocks": clocks,
        "forms": {**(split_summary(split, args, value, world, fp64_hist, peaks) or {}),
                  **(ozaki_summary(split_bf16, args, value, world, fp64_hist, peaks,
                                   "split_bf16", 3, LADDER_OZ3_PROFILE) or {}),
                  **(ozaki_summary(ozaki, args, value, world, fp64_hist, peaks) or {})},
        "serving": serving,
        "measured_peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    p, run = workload(args.workload)
    m_ref = oracle_micro_per_step(args.workload, args.tol)
    t_mi, threads = time_oracle_micro_iteration(p, run["dt"], reps=args.steps, warm=args.warmup)
    m_use = m_ref if m_ref is not None else float("nan")
    value = 1.0 / (t_mi * m_use)
    sample = (f"each step: one oracle micro-iteration (residual + Eq. 9 update) of workload "
              f"{args.workload} on the host cores ({t_mi:.2f} s mean over {args.steps}), scaled "
              f"by the oracle's {m_use:.2f} micro-iterations per step at tol {args.tol:g}")
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_mi * m_use,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": f"{args.workload}: O={p.nocc} V={p.nvir} "
                                                      f"Nchol={p.nchol} dt={run['dt']} tol={args.tol}"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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

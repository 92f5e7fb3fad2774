"""Evaluate CCSD residuals of a named workload eagerly, for profilers.

  python -m paper_2301_04249_b300.profile [--workload c2_formaldehyde | --shape O,V,N] [--residuals 2]
         [--precision fp64|split_tf32|split_bf16|split_fp16|fp64_ozaki] [--cholesky] [--steps N]
         [--tol TOL] [--anderson]

Each evaluation launches every kernel of one residual on the library's
stream outside CUDA graphs, with the particle-particle ladder GEMMs inside
the NVTX range "rteom_ladder" (select them with
`ncu --nvtx --nvtx-include "rteom_ladder/"`).  Prints the per-class timing.
With --steps N it propagates N Adams-Moulton steps from T(0) = 0 instead
(no host amplitude arrays) and prints the set-up time, the device memory
the context took and the time per step.  --cholesky asks for the Cholesky
mode (RTEOM_FLAG_LADDER_CHOLESKY); rteom_create also takes it by itself
when the resident blocks do not fit.  --anderson accelerates the
micro-iterations (RTEOM_FLAG_ANDERSON); --tol sets their cutoff (1e-4).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))

import paper_2301_04249_b300 as P  # noqa: E402
from synth import workload  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2_formaldehyde")
    ap.add_argument("--shape", default=None,
                    help="O,V,Nchol: a synthetic problem of this shape (seed 9) instead")
    ap.add_argument("--residuals", type=int, default=2)
    ap.add_argument("--precision", choices=["fp64", "split_tf32", "split_bf16", "split_fp16",
                                                     "fp64_ozaki"],
                    default="fp64")
    ap.add_argument("--cholesky", action="store_true")
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--anderson", action="store_true")
    ap.add_argument("--eager-timing", action="store_true",
                    help="with --steps: residuals outside graphs, every launch timed")
    a = ap.parse_args()
    if a.shape:
        from synth import gen_problem
        O, V, N = (int(x) for x in a.shape.split(","))
        p, run = gen_problem(O, V, N, 9), dict(dt=0.025)
        a.workload = f"shape O={O} V={V} Nchol={N} seed=9"
    else:
        p, run = workload(a.workload)
    rng = np.random.default_rng(0)
    prec = {"fp64": P.RTEOM_FP64, "split_tf32": P.RTEOM_SPLIT_TF32,
            "split_bf16": P.RTEOM_SPLIT_BF16, "split_fp16": P.RTEOM_SPLIT_FP16,
            "fp64_ozaki": P.RTEOM_FP64_OZAKI}[a.precision]
    flags = (P.RTEOM_FLAG_LADDER_CHOLESKY if a.cholesky else 0) | \
        (P.RTEOM_FLAG_ANDERSON if a.anderson else 0)
    if a.steps > 0:
        import torch
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        with P.Propagator.from_problem(p, precision=prec, flags=flags) as g:
            setup_s = time.perf_counter() - t0
            held = free0 - torch.cuda.mem_get_info()[0]
            g.set_timing(2 if a.eager_timing else 1)
            t0 = time.perf_counter()
            g.propagate(a.steps, run["dt"], tol=a.tol)
            wall = time.perf_counter() - t0
            info = g.info()
            print(json.dumps(dict(workload=a.workload, precision=a.precision, tol=a.tol,
                                  anderson=a.anderson,
                                  setup_s=setup_s, device_bytes_held=held,
                                  steps=a.steps, s_per_step=wall / a.steps,
                                  micro_per_step=info["micro"] / a.steps,
                                  timing=g.timing())))
        return
    with P.Propagator.from_problem(p, precision=prec, flags=flags) as g:
        shapes = P.block_shapes(p.nocc, p.nvir)
        t = [0.01 * (rng.standard_normal(s) + 1j * rng.standard_normal(s)) for s in shapes]
        for k in (2, 4):
            t[k] = t[k] - t[k].transpose(1, 0, 2, 3)
            t[k] = t[k] - t[k].transpose(0, 1, 3, 2)
        g.set_timing(True)
        for _ in range(a.residuals):
            g.residual(t)
        print(json.dumps(g.timing()))


if __name__ == "__main__":
    main()

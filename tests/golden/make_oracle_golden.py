"""Write the oracle's reference cumulants used by the GPU parity tests and
the benchmark's CPU baseline.

Calls only oracle/ and synth/.  Output: tests/golden/oracle_<workload>.txt
(tol 1e-12, the parity setting) or oracle_<workload>_tol<tol>.txt, with
columns  n  Re C_n  Im C_n  Re E_n  Im E_n  micro_n  (micro_0 = 0), and a
header line with eps_core and E_corr.

Usage: python tests/golden/make_oracle_golden.py [workload steps [tol]] ...
   (a job is "workload steps" optionally followed by a tolerance)
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

from oracle.propagate import closed_shell_ecorr, propagate  # noqa: E402
from oracle.spinexp import CoreHoleCCSD  # noqa: E402
from synth import workload  # noqa: E402

DEFAULT = [("c1_fp64_small", 200), ("c2_formaldehyde", 4)]


def write(name, steps, tol=1e-12):
    p, run = workload(name)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    out = propagate(sysb, steps, run["dt"], tol=tol, max_micro=50)
    ecorr = closed_shell_ecorr(p.L, p.nocc, p.t1_gs, p.t2_gs)
    micro = np.concatenate([[0], out["micro"]])
    n = np.arange(steps + 1)
    data = np.stack([n, out["C"].real, out["C"].imag, out["E"].real, out["E"].imag, micro], 1)
    tag = "" if tol == 1e-12 else f"_tol{tol:g}"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{name}{tag}.txt")
    hdr = (f"oracle propagation of workload {name}: dt={run['dt']} tol={tol:g} max_micro=50\n"
           f"eps_core={p.eps[p.core]:.17g} e_corr={ecorr:.17g}\n"
           "n ReC ImC ReE ImE micro")
    np.savetxt(path, data, fmt=["%d", "%.17g", "%.17g", "%.17g", "%.17g", "%d"], header=hdr)
    print(path)


if __name__ == "__main__":
    args = sys.argv[1:]
    jobs = []
    k = 0
    while k < len(args):
        name, steps = args[k], int(args[k + 1])
        k += 2
        tol = 1e-12
        if k < len(args) and args[k][0].isdigit() and "e" in args[k] or (k < len(args) and args[k].startswith("0.")):
            tol = float(args[k])
            k += 1
        jobs.append((name, steps, tol))
    for job in (jobs or [(n, s, 1e-12) for n, s in DEFAULT]):
        write(*job)

"""Write sampled oracle residual entries of a problem larger than the GPU
parity tests can afford to recompute on the host at test time.

Problem: gen_problem(O=12, V=160, Nchol=640, seed=31), core 0; amplitudes:
synth.random_amplitudes(block shapes, seed=32, scale=0.02).  At this size
the library's Cholesky mode runs its default chunks (two ladder chunks of
the virtual index a, one of 128 and a ragged one of 33).  The oracle
evaluates the full residual once (about a minute on eight cores); this
script stores 400 seeded random entries of each block, the largest |R| over
all blocks (the scale of the parity bound) and the cumulant integrand E.

Calls only oracle/ and synth/.  Output: tests/golden/oracle_residual_O12V160N640.txt
with lines  block flat_index ReR ImR  (flat_index within the block, row-major).

Usage: python tests/golden/make_residual_samples.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

from oracle.spinexp import CoreHoleCCSD  # noqa: E402
from synth import gen_problem, random_amplitudes  # noqa: E402

O, V, NCHOL, SEED, T_SEED, SCALE, PER_BLOCK = 12, 160, 640, 31, 32, 0.02, 400


def main():
    p = gen_problem(O, V, NCHOL, SEED)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t = random_amplitudes(sysb.shapes(), T_SEED, SCALE)
    R = sysb.residual(t)
    E = sysb.energy(t)
    scale = max(float(np.abs(x).max()) for x in R)
    rng = np.random.default_rng(33)
    rows = []
    for k, x in enumerate(R):
        idx = np.sort(rng.choice(x.size, size=min(PER_BLOCK, x.size), replace=False))
        v = x.ravel()[idx]
        rows += [(k, int(i), float(z.real), float(z.imag)) for i, z in zip(idx, v)]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        f"oracle_residual_O{O}V{V}N{NCHOL}.txt")
    with open(path, "w") as f:
        f.write(f"# oracle residual samples: gen_problem({O}, {V}, {NCHOL}, seed={SEED}) core 0, "
                f"random_amplitudes(seed={T_SEED}, scale={SCALE})\n")
        f.write(f"# scale={scale:.17g} ReE={E.real:.17g} ImE={E.imag:.17g}\n")
        f.write("# block flat_index ReR ImR\n")
        for k, i, re, im in rows:
            f.write(f"{k} {i} {re:.17g} {im:.17g}\n")
    print(path)


if __name__ == "__main__":
    main()

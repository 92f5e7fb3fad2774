"""GPU: the Anderson-accelerated micro-iteration (RTEOM_FLAG_ANDERSON).

It keeps the stopping rule and the accepted value of the plain iteration,
so at a tight tolerance it reaches the same implicit Adams-Moulton solution
(Eq. 9) as the oracle's plain fixed-point iteration: C(t) within 1e-10
relative, as for the plain GPU path.  It must take fewer residual
evaluations to get there.
"""
import os

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A = P.RTEOM_FLAG_ANDERSON


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", [P.RTEOM_FP64, P.RTEOM_FP64_OZAKI])
def test_anderson_reaches_the_oracle_solution_in_fewer_residuals(precision):
    p = gen_problem(4, 12, 20, 21)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, 4, 0)
    ref = PR.propagate(sysb, 12, 0.05, tol=1e-12)
    with P.Propagator.from_problem(p, precision=precision, flags=A) as g:
        C = g.propagate(12, 0.05, tol=1e-12)
        micro = g.info()["micro"]
    assert _rel(C, ref["C"]) < 1e-10
    assert micro < ref["micro"].sum(), (micro, ref["micro"].sum())


def test_anderson_c1_full_propagation_matches_stored_oracle_run():
    """O=4, V=20, Nchol=60, 200 steps, dt=0.05, tol=1e-12."""
    d = np.loadtxt(os.path.join(GOLDEN, "oracle_c1_fp64_small.txt"))
    Cref, micro_ref = d[:, 1] + 1j * d[:, 2], d[1:, 5].sum()
    p, run = workload("c1_fp64_small")
    with P.Propagator.from_problem(p, flags=A) as g:
        C = g.propagate(run["nsteps"], run["dt"], tol=1e-12)
        micro = g.info()["micro"]
    assert _rel(C, Cref) < 1e-10
    print(f"c1 micro-iterations: plain {micro_ref:.0f}, Anderson {micro}")
    assert micro < 0.8 * micro_ref


def test_anderson_and_plain_agree_at_a_moderate_tolerance():
    """At tol = 1e-8 both stop within the tolerance of the same solution."""
    p = gen_problem(5, 30, 60, 23)
    out = {}
    for flags in (0, A):
        with P.Propagator.from_problem(p, flags=flags) as g:
            out[flags] = (g.propagate(40, 0.025, tol=1e-8), g.info()["micro"])
    (Cp, mp), (Ca, ma) = out[0], out[A]
    assert np.abs(Ca - Cp).max() < 1e-8
    assert ma <= mp

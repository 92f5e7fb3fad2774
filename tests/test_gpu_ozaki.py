"""FP64 emulation on the BF16 tensor cores (RTEOM_FP64_OZAKI) against the
FP64 oracle, at the FP64 form's tolerances.

The digit slicing keeps about 2^-48 of the row scales per term (compensated
FP32 accumulation of exact chunk sums), so the bars are those of the FP64
path: residual blocks within 1e-12 of their largest element, C(t) within
1e-10 relative.  RTEOM_OZ_MIN_FLOPS=0 puts every contraction that is not a
matrix-vector product on the emulated path.
"""
import os

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from conftest import random_blocks
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    d = np.loadtxt(os.path.join(GOLDEN, f"oracle_{name}.txt"))
    return d[:, 1] + 1j * d[:, 2]


def _oz(p, **kw):
    return P.Propagator(p.eps, p.L, p.nocc, p.nvir, p.t1_gs, p.t2_gs, core=p.core,
                        precision=P.RTEOM_FP64_OZAKI, **kw)


def _relC(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("O,V,nchol,seed,core", [
    (3, 5, 7, 1, 0), (5, 37, 23, 2, 0), (4, 9, 11, 3, 2), (6, 70, 40, 6, 0), (8, 100, 400, 2, 0)])
def test_emulated_residual_matches_oracle(O, V, nchol, seed, core, rng, monkeypatch):
    monkeypatch.setenv("RTEOM_OZ_MIN_FLOPS", "0")
    p = gen_problem(O, V, nchol, seed)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, O, core)
    t = random_blocks(sysb.shapes(), rng, scale=0.05)
    with P.Propagator(p.eps, p.L, O, V, p.t1_gs, p.t2_gs, core=core,
                      precision=P.RTEOM_FP64_OZAKI) as g:
        Rg, Eg = g.residual(t)
    Ro = sysb.residual(t)
    scale = max(np.abs(x).max() for x in Ro if x.size)
    err = max(np.abs(a - b).max() for a, b in zip(Rg, Ro) if a.size) / scale
    assert err <= 1e-12, err
    assert abs(Eg - sysb.energy(t)) <= 1e-12 * max(1.0, abs(Eg))


def test_emulated_c1_propagation_matches_oracle():
    C_ref = _golden("c1_fp64_small")
    p, run = workload("c1_fp64_small")
    os.environ["RTEOM_OZ_MIN_FLOPS"] = "0"
    try:
        with _oz(p) as g:
            C = g.propagate(run["nsteps"], run["dt"], tol=1e-12)
    finally:
        del os.environ["RTEOM_OZ_MIN_FLOPS"]
    assert _relC(C, C_ref) < 1e-10


def test_emulated_c2_first_steps_match_oracle():
    C_ref = _golden("c2_formaldehyde")
    p, run = workload("c2_formaldehyde")
    with _oz(p) as g:
        C = g.propagate(len(C_ref) - 1, run["dt"], tol=1e-12)
    assert _relC(C, C_ref) < 1e-10


def test_emulated_tracks_fp64_path_over_40_steps():
    p, run = workload("c2_formaldehyde")
    with P.Propagator.from_problem(p) as g:
        C64 = g.propagate(40, run["dt"], tol=1e-10)
    with _oz(p) as g:
        Coz = g.propagate(40, run["dt"], tol=1e-10)
    assert _relC(Coz, C64) < 1e-10

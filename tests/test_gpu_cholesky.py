"""GPU parity of the Cholesky mode (RTEOM_FLAG_LADDER_CHOLESKY): no (ov|vv)
or (vv|vv) block on the device; the particle-particle ladder (Section 3.1.1)
and the other terms with three or four virtual indices are formed from the
Cholesky vectors at every residual, in chunks of a and of m.

The chunk cap RTEOM_CHOLESKY_CHUNK=3 splits every case into several chunks
with a ragged last one.  Tolerances as for the resident blocks: FP64 and the
emulated FP64 form 1e-12 of the largest residual entry, the split forms 1e-5.
"""
import numpy as np
import pytest

import paper_2301_04249_b300 as P
from conftest import random_blocks
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem, workload

pytestmark = pytest.mark.gpu

F = P.RTEOM_FLAG_LADDER_CHOLESKY


@pytest.fixture(autouse=True)
def _small_chunks(monkeypatch):
    monkeypatch.setenv("RTEOM_CHOLESKY_CHUNK", "3")
    monkeypatch.setenv("RTEOM_TC_MIN_FLOPS", "0")   # every contraction on the tensor cores
    monkeypatch.setenv("RTEOM_OZ_MIN_FLOPS", "0")


SHAPES = [(3, 5, 7, 1, 0), (5, 37, 23, 2, 0), (4, 9, 11, 3, 2), (1, 6, 5, 4, 0),
          (2, 1, 3, 5, 1), (6, 70, 40, 6, 0)]
TOL = {P.RTEOM_FP64: 1e-12, P.RTEOM_FP64_OZAKI: 1e-12, P.RTEOM_SPLIT_TF32: 1e-5,
       P.RTEOM_SPLIT_BF16: 1e-5, P.RTEOM_SPLIT_FP16: 1e-5}


@pytest.mark.parametrize("O,V,nchol,seed,core", SHAPES)
@pytest.mark.parametrize("precision", [P.RTEOM_FP64, P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_TF32,
                                       P.RTEOM_SPLIT_BF16, P.RTEOM_SPLIT_FP16])
def test_cholesky_residual_matches_oracle(O, V, nchol, seed, core, precision, rng):
    p = gen_problem(O, V, nchol, seed)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, O, core)
    t = random_blocks(sysb.shapes(), rng, scale=0.1)
    with P.Propagator(p.eps, p.L, O, V, p.t1_gs, p.t2_gs, core=core, precision=precision,
                      flags=F) as g:
        Rg, Eg = g.residual(t)
    Ro, Eo = sysb.residual(t), sysb.energy(t)
    scale = max(np.abs(x).max() for x in Ro if x.size)
    for k, (a, b) in enumerate(zip(Rg, Ro)):
        assert a.shape == b.shape
        if a.size:
            err = np.abs(a - b).max()
            assert err <= TOL[precision] * scale, (k, err, scale)
    assert abs(Eg - Eo) <= 1e-12 * max(1.0, abs(Eo))


def test_cholesky_propagation_matches_oracle():
    p = gen_problem(4, 12, 20, 21)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, 4, 0)
    ref = PR.propagate(sysb, 12, 0.05, tol=1e-12)
    with P.Propagator.from_problem(p, flags=F) as g:
        C = g.propagate(12, 0.05, tol=1e-12)
    assert np.abs(C - ref["C"]).max() / np.abs(ref["C"]).max() < 1e-10


def test_cholesky_and_resident_blocks_agree_at_full_c2_size(rng):
    """O=8, V=100, Nchol=400 at random amplitudes: the two modes differ only
    in summation order (FP64)."""
    p, _ = workload("c2_formaldehyde")
    t = random_blocks(P.block_shapes(p.nocc, p.nvir), rng, scale=0.02)
    with P.Propagator.from_problem(p) as g:
        Rr, Er = g.residual(t)
    with P.Propagator.from_problem(p, flags=F) as g:
        Rc, Ec = g.residual(t)
    scale = max(np.abs(x).max() for x in Rr)
    assert max(np.abs(a - b).max() for a, b in zip(Rc, Rr)) <= 1e-12 * scale
    assert Ec == Er

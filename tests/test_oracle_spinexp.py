"""Pins P2/P3: oracle B (spin-explicit blocks, Cholesky-factored
contractions) equals oracle A (spin-orbital, assembled <pq||rs>), which the
brute force pins (test_oracle_spinorb.py)."""
import numpy as np
import pytest

from conftest import random_blocks
from oracle import hamiltonian as H
from oracle import spinexp as SB
from oracle import spinorb as SA
from synth import gen_problem


@pytest.mark.parametrize("O,V,nchol,seed,core", [
    (2, 2, 5, 1, 0), (3, 3, 7, 2, 0), (4, 3, 6, 3, 0), (3, 4, 5, 4, 2), (1, 3, 4, 5, 0), (2, 1, 3, 6, 1)])
def test_spin_explicit_equals_spin_orbital(O, V, nchol, seed, core, rng):
    p = gen_problem(O, V, nchol, seed, with_t2=False, l_scale=1.0)
    sysb = SB.CoreHoleCCSD.from_problem(p.eps, p.L, O, core)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, O)
    occ, vir = H.core_hole_reference(p.nb, O, core)
    f = H.reference_fock(h, v, occ)
    t = random_blocks(sysb.shapes(), rng)
    oA, vA = t[0].shape
    oB, vB = t[1].shape
    t1so, t2so = SA.blocks_to_spinorb(t, oA, oB, vA, vB)
    fr, vr = SA.reorder(f, v, occ, vir)
    Ea, R1a, R2a = SA.residual(fr, vr, oA + oB, t1so, t2so)
    Ra = SA.spinorb_to_blocks(R1a, R2a, oA, oB, vA, vB)
    Rb = sysb.residual(t)
    scale = max(1.0, max(np.abs(x).max() for x in Ra if x.size))
    for x, y in zip(Ra, Rb):
        assert x.shape == y.shape
        if x.size:
            assert np.abs(x - y).max() < 1e-12 * scale
    assert abs(sysb.energy(t) - Ea) < 1e-12 * scale
    # the spin-orbital projection has no components outside the unique blocks
    t1r, t2r = SA.blocks_to_spinorb(Ra, oA, oB, vA, vB)
    assert np.abs(t2r - R2a).max() < 1e-12 * scale
    assert np.abs(t1r - R1a).max() < 1e-12 * scale


def test_same_spin_blocks_antisymmetric(rng):
    p = gen_problem(3, 4, 6, 7, with_t2=False)
    sysb = SB.CoreHoleCCSD.from_problem(p.eps, p.L, 3, 0)
    R = sysb.residual(random_blocks(sysb.shapes(), rng))
    for k in (2, 4):
        assert np.abs(R[k] + R[k].transpose(1, 0, 2, 3)).max() < 1e-12
        assert np.abs(R[k] + R[k].transpose(0, 1, 3, 2)).max() < 1e-12


def test_diagonal_only_problem_is_linear(rng):
    """With no Cholesky vectors and a diagonal Fock matrix, R = D*t exactly."""
    O, V = 3, 4
    eps = np.sort(rng.standard_normal(O + V))
    sysb = SB.CoreHoleCCSD(np.diag(eps), np.diag(eps), np.zeros((0, O + V, O + V)), O, 0)
    t = random_blocks(sysb.shapes(), rng)
    for r, d, x in zip(sysb.residual(t), sysb.diagonal(), t):
        assert np.abs(r - d * x).max() < 1e-13

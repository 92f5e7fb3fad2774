"""Reduced-orbital problems for residual checks at full problem sizes (test
helper).

Every summed index of a CCSD projection (Eqs. 7-8) sits on an amplitude, and
the (N-1) Fock matrix f_pq = eps_p delta_pq - <pc||qc> involves no sum over
orbitals.  So when the amplitudes vanish outside a set S of orbitals, the
residual entries whose free indices lie in S are those of the problem cut
down to S (its orbital energies and Cholesky vectors restricted to S, the
same core orbital).  test_oracle_reduced.py pins this on the oracle; the GPU
tests use it to compare full-size contexts with the oracle on a small
problem.
"""
import numpy as np


def reduced_problem(p, occ_sel, vir_sel):
    """(eps, L, nocc, core) of problem p restricted to the spatial occupied
    orbitals occ_sel (which must hold p.core) and virtual orbitals vir_sel."""
    occ_sel, vir_sel = list(occ_sel), list(vir_sel)
    assert p.core in occ_sel and all(0 <= i < p.nocc for i in occ_sel)
    assert all(p.nocc <= a < p.nb for a in vir_sel)
    sel = np.array(occ_sel + vir_sel)
    L = np.ascontiguousarray(p.L[:, sel][:, :, sel])
    return p.eps[sel].copy(), L, len(occ_sel), occ_sel.index(p.core)


def block_offsets(nocc, nvir):
    """Offsets (complex entries) of the five unpadded spin blocks."""
    oA, vA, oB, vB = nocc, nvir, nocc - 1, nvir + 1
    sizes = [oA * vA, oB * vB, oA * oA * vA * vA, oA * oB * vA * vB, oB * oB * vB * vB]
    return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)


def full_indices(p, occ_sel, vir_sel):
    """For each spin block of the reduced problem, the flat indices (into the
    full problem's amplitude vector) of all its entries, shaped like the
    block."""
    occ_sel, vir_sel = list(occ_sel), list(vir_sel)
    O, core = p.nocc, p.core
    core_r = occ_sel.index(core)
    # spin-space position in the full problem of each reduced spin-space entry
    occ_a = np.array(occ_sel)
    occ_b = np.array([s - (s > core) for k, s in enumerate(occ_sel) if k != core_r])
    vir_a = np.array([a - O for a in vir_sel])
    vir_b = np.array([0] + [a - O + 1 for a in vir_sel])
    oA, vA, oB, vB = O, p.nvir, O - 1, p.nvir + 1
    off = block_offsets(O, p.nvir)
    out = [off[0] + occ_a[:, None] * vA + vir_a[None, :],
           off[1] + occ_b[:, None] * vB + vir_b[None, :]]
    for blk, (oi, oj, va, vb, noj, nva, nvb) in zip(
            (2, 3, 4), ((occ_a, occ_a, vir_a, vir_a, oA, vA, vA),
                        (occ_a, occ_b, vir_a, vir_b, oB, vA, vB),
                        (occ_b, occ_b, vir_b, vir_b, oB, vB, vB))):
        out.append(off[blk] + ((oi[:, None, None, None] * noj + oj[None, :, None, None]) * nva
                               + va[None, None, :, None]) * nvb + vb[None, None, None, :])
    return out

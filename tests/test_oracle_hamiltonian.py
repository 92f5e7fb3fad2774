"""Pins of the (N-1) Fock matrix, the Cholesky assembly and the spin-block
memory layout (Section 2.1, Section 3.1.1, Table 2)."""
import os

import numpy as np
import pytest

from oracle import hamiltonian as H
from synth import gen_problem


def test_eri_assembly_matches_loops():
    p = gen_problem(2, 3, 4, 3, with_t2=False)
    eri = H.eri_from_cholesky(p.L)
    nb = p.nb
    ref = np.zeros((nb,) * 4)
    for P in range(nb):
        for q in range(nb):
            for r in range(nb):
                for s in range(nb):
                    acc = 0.0
                    for Q in range(p.nchol):
                        acc += p.L[Q, P, q] * p.L[Q, r, s]
                    ref[P, q, r, s] = acc
    assert np.abs(eri - ref).max() < 1e-14
    # eight-fold permutational symmetry of real integrals from pq-symmetric L
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.allclose(eri, eri.transpose(perm))


@pytest.mark.parametrize("core", [0, 2])
def test_fock_nm1_matches_spin_orbital_definition(core):
    """f = h + sum_{k in occ(N-1)} <pk||qk> with h fixed by F^N = diag(eps)
    must equal eps*delta - <pc||qc> with c the beta core spin-orbital."""
    O, V = 3, 3
    p = gen_problem(O, V, 6, 4, with_t2=False)
    h, v, occN = H.spinorb_hamiltonian(p.eps, p.L, O)
    occ, vir = H.core_hole_reference(p.nb, O, core)
    f = H.reference_fock(h, v, occ)
    fa, fb = H.fock_nm1(p.eps, p.L, core)
    nb = p.nb
    assert np.abs(f[:nb, :nb] - fa).max() < 1e-13
    assert np.abs(f[nb:, nb:] - fb).max() < 1e-13
    assert np.abs(f[:nb, nb:]).max() == 0.0
    # the N-electron Fock is diag(eps) by construction
    fN = H.reference_fock(h, v, occN)
    assert np.abs(fN - np.diag(np.concatenate([p.eps, p.eps]))).max() < 1e-13
    # the beta core row/column of the (N-1) Fock is diagonal: f^b_pc = eps_c d_pc
    assert np.abs(fb[:, core] - p.eps[core] * (np.arange(nb) == core)).max() < 1e-13


def test_table2_t2_memory_formula():
    """T2 bytes per timeline tensor = 16 (oA^2 vA^2 + oA oB vA vB + oB^2 vB^2),
    which reproduces the paper's Table 2 within one unit of its last printed
    digit (0.1 GB; the benzene-ammonia row, 5.74, is printed as 5.8); the
    configuration columns also fix the hole-in-beta reading
    (nocc_b = nocc_a - 1, nvir_b = nvir_a + 1)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_memory.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for name, nso, oa, ob, va, vb, gb in rows:
        nso, oa, ob, va, vb, gb = int(nso), int(oa), int(ob), int(va), int(vb), float(gb)
        assert oa + va == ob + vb == nso // 2
        assert ob == oa - 1 and vb == va + 1
        nbytes = 16 * (oa * oa * va * va + oa * ob * va * vb + ob * ob * vb * vb)
        assert abs(nbytes / 2 ** 30 - gb) <= 0.1 + 1e-9, (name, nbytes / 2 ** 30, gb)

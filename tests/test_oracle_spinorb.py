"""Pin P1: oracle A's spin-orbital CCSD projections equal the determinant
brute force <Phi_mu| e^{-T} H_N e^{T} |Phi> for random complex amplitudes
(Eqs. 2, 7, 8), including references with non-zero occupied-virtual Fock
elements (the (N-1) core-hole reference and a generic 2-electron one)."""
import numpy as np
import pytest

from oracle import fockspace as FS
from oracle import hamiltonian as H
from oracle import spinorb as SA
from synth import gen_problem


def _rand(rng, no, nv, scale=0.3):
    t1 = scale * (rng.standard_normal((no, nv)) + 1j * rng.standard_normal((no, nv)))
    t2 = scale * (rng.standard_normal((no, no, nv, nv)) + 1j * rng.standard_normal((no, no, nv, nv)))
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    return t1, t2


CASES = [
    # (O, V, nchol, seed, core, occupation override as spatial/spin pairs or None)
    (2, 2, 5, 1, 0, None),
    (3, 2, 6, 2, 0, None),
    (3, 2, 6, 5, 1, None),
    (1, 3, 4, 6, 0, None),
    (1, 2, 4, 3, 0, [(0, 0), (1, 1)]),      # generic 2-electron reference
]


@pytest.mark.parametrize("O,V,nchol,seed,core,occ_sp", CASES)
def test_oracle_a_matches_brute_force(O, V, nchol, seed, core, occ_sp, rng):
    p = gen_problem(O, V, nchol, seed, with_t2=False, l_scale=1.0)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, O)
    if occ_sp is None:
        occ, vir = H.core_hole_reference(p.nb, O, core)
    else:
        occ = [H.spinorb_index(p.nb, q, s) for q, s in occ_sp]
        vir = [k for k in range(2 * p.nb) if k not in occ]
    f = H.reference_fock(h, v, occ)
    no, nv = len(occ), len(vir)
    fov = f[np.ix_(occ, vir)]
    assert np.abs(fov).max() > 1e-3        # a genuinely non-canonical reference
    t1, t2 = _rand(rng, no, nv)
    Eb, R1b, R2b = FS.similarity_residuals(h, v, occ, vir, t1, t2)
    fr, vr = SA.reorder(f, v, occ, vir)
    Ea, R1a, R2a = SA.residual(fr, vr, no, t1, t2)
    scale = max(1.0, np.abs(R2b).max(), np.abs(R1b).max())
    assert abs(Ea - Eb) < 1e-12 * scale
    assert np.abs(R1a - R1b).max() < 1e-12 * scale
    assert np.abs(R2a - R2b).max() < 1e-12 * scale


def test_oracle_a_detects_planted_error(rng):
    """A dropped term must be visible to the brute force (sensitivity check)."""
    p = gen_problem(2, 2, 5, 1, with_t2=False, l_scale=1.0)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, 2)
    occ, vir = H.core_hole_reference(p.nb, 2, 0)
    f = H.reference_fock(h, v, occ)
    t1, t2 = _rand(rng, len(occ), len(vir))
    _, R1b, R2b = FS.similarity_residuals(h, v, occ, vir, t1, t2)
    fr, vr = SA.reorder(f, v, occ, vir)
    no = len(occ)
    # drop the occupied-virtual Fock block: the residuals must change
    fr2 = fr.copy()
    fr2[:no, no:] = 0
    fr2[no:, :no] = 0
    _, R1x, R2x = SA.residual(fr2, vr, no, t1, t2)
    assert np.abs(R1x - R1b).max() > 1e-3

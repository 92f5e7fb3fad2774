"""Pin of the reduced-orbital residual property the full-size GPU checks rely
on: with amplitudes supported on a set S of orbitals, the oracle residual of
the whole problem equals, on S, the oracle residual of the problem cut down
to S; and outside S's amplitude entries the index map covers exactly the
reduced blocks."""
import numpy as np

from oracle.spinexp import CoreHoleCCSD
from reduced import full_indices, reduced_problem
from synth import gen_problem, random_amplitudes


def _embed(blocks_r, idx, n_full):
    z = np.zeros(n_full, dtype=complex)
    for x, k in zip(blocks_r, idx):
        z[k.ravel()] = x.ravel()
    return z


def test_residual_on_a_subset_equals_residual_of_the_cut_problem():
    p = gen_problem(6, 15, 20, 9)
    occ_sel, vir_sel = [0, 2, 5], [6, 9, 13, 20]
    eps_r, L_r, nocc_r, core_r = reduced_problem(p, occ_sel, vir_sel)
    red = CoreHoleCCSD.from_problem(eps_r, L_r, nocc_r, core_r)
    full = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t_r = random_amplitudes(red.shapes(), 10, 0.2)
    idx = full_indices(p, occ_sel, vir_sel)
    shapes = full.shapes()
    n_full = sum(int(np.prod(s)) for s in shapes)
    z = _embed(t_r, idx, n_full)
    t_full, k = [], 0
    for s in shapes:
        n = int(np.prod(s))
        t_full.append(z[k:k + n].reshape(s))
        k += n
    # the embedded amplitudes are still antisymmetric
    for b in (2, 4):
        assert np.allclose(t_full[b], -t_full[b].transpose(1, 0, 2, 3))
        assert np.allclose(t_full[b], -t_full[b].transpose(0, 1, 3, 2))
    R_full = np.concatenate([x.ravel() for x in full.residual(t_full)])
    R_red = red.residual(t_r)
    scale = max(np.abs(x).max() for x in R_red)
    for x, k in zip(R_red, idx):
        assert np.abs(R_full[k.ravel()] - x.ravel()).max() <= 1e-13 * scale
    # the residual outside the subset is not zero: the check is not vacuous
    mask = np.ones(n_full, bool)
    for k in idx:
        mask[k.ravel()] = False
    assert np.abs(R_full[mask]).max() > 1e-3 * scale

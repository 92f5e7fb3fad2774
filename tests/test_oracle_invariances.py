"""Exact symmetries of the propagated system that the oracle must keep:
checks against properties of the method, not against the oracle's own
arithmetic.

- Time reversal.  The Cholesky vectors and the (N-1) Fock matrix are real, so
  the projections R(t) (Eqs. 7-8) and the cumulant integrand E(t) (Eq. 5) are
  polynomials with real coefficients in the amplitudes.  The trapezoid step
  (Eq. 9) with -dt is then the complex conjugate of the step with +dt, and
  the cumulant of a backward propagation is conj(C(t)).
- Energy origin.  A uniform shift of every orbital energy shifts every
  diagonal Fock element of the (N-1) reference by the same amount.  The
  projections contain the diagonal Fock elements only through differences
  (occupied against virtual), and E(t) only the occupied-virtual block, so
  the amplitudes and C(t) do not change; the shift lives only in the phase
  exp(-i eps_c t) of G (Eq. 4).
- Orbital labels.  Relabelling occupied or virtual orbitals (eps and the
  orbital indices of L permuted together, the core index following its
  orbital) describes the same system, so C(t) is unchanged.
- Orbital phases.  Changing the sign of some orbitals (L[Q][p][q] ->
  s_p s_q L[Q][p][q], s = +-1) changes the signs of integrals and amplitudes
  but not the physics: every term of a projection or of E carries each
  orbital index an even number of times, so C(t) is unchanged.

A plausible slip in the oracle (a stray factor i or a conjugate in one term,
a diagonal Fock element used outside a difference, an index that assumes the
orbital order, a contraction over the wrong index) breaks one of these.
"""
import numpy as np
import pytest

from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem

NSTEPS, DT = 8, 0.05


def _cumulant(eps, L, nocc, core, dt=DT):
    return PR.propagate(CoreHoleCCSD.from_problem(eps, L, nocc, core), NSTEPS, dt,
                        tol=1e-13)["C"]


@pytest.mark.parametrize("O,V,nchol,seed,core", [(3, 7, 10, 41, 0), (4, 6, 9, 42, 2)])
def test_backward_propagation_conjugates_the_cumulant(O, V, nchol, seed, core):
    p = gen_problem(O, V, nchol, seed)
    fwd = _cumulant(p.eps, p.L, O, core)
    bwd = _cumulant(p.eps, p.L, O, core, dt=-DT)
    assert np.abs(fwd[1:]).max() > 1e-3  # non-trivial dynamics
    assert np.abs(bwd - np.conj(fwd)).max() <= 1e-12 * np.abs(fwd).max()


@pytest.mark.parametrize("shift", [0.73, -5.0])
def test_uniform_energy_shift_leaves_the_cumulant(shift):
    p = gen_problem(3, 7, 10, 43)
    ref = _cumulant(p.eps, p.L, 3, 1)
    out = _cumulant(p.eps + shift, p.L, 3, 1)
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()
    # the shift changes the Fock diagonal, the quantity the invariance is about
    a = CoreHoleCCSD.from_problem(p.eps, p.L, 3, 1)
    b = CoreHoleCCSD.from_problem(p.eps + shift, p.L, 3, 1)
    assert abs(np.diag(b.f[0])[0] - np.diag(a.f[0])[0] - shift) < 1e-12


def test_orbital_relabelling_leaves_the_cumulant():
    O, V = 4, 7
    p = gen_problem(O, V, 10, 44)
    core = 1
    ref = _cumulant(p.eps, p.L, O, core)
    rng = np.random.default_rng(7)
    occ = rng.permutation(O)
    vir = O + rng.permutation(V)
    perm = np.concatenate([occ, vir])
    eps = p.eps[perm]
    L = p.L[:, perm][:, :, perm]
    new_core = int(np.flatnonzero(occ == core)[0])
    assert new_core != core or not np.array_equal(occ, np.arange(O))
    out = _cumulant(eps, L, O, new_core)
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()
    # a different core hole is a different system: the check can fail
    other = _cumulant(eps, L, O, (new_core + 1) % O)
    assert np.abs(other - ref).max() > 1e-6


def test_orbital_sign_changes_leave_the_cumulant():
    O, core = 4, 1
    p = gen_problem(O, 7, 10, 45)
    s = np.ones(p.nb)
    s[[1, 2, 5, 9]] = -1.0  # occupied (the core, 1, among them) and virtual orbitals
    L = p.L * s[None, :, None] * s[None, None, :]
    ref = _cumulant(p.eps, p.L, O, core)
    out = _cumulant(p.eps, L, O, core)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()

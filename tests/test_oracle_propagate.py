"""Pins P4-P9 of the integrator (Eq. 9), the cumulant (Eqs. 5-6), the Green's
function (Eq. 4) and the transform to A(omega)."""
import numpy as np
import pytest

from conftest import random_blocks
from oracle import fockspace as FS
from oracle import hamiltonian as H
from oracle import propagate as PR
from oracle import spinexp as SB
from oracle import spinorb as SA
from synth import gen_problem


def test_zero_couplings_stay_zero():
    """P4: no two-electron couplings, canonical Fock: T(t) = 0 and C(t) = 0."""
    p = gen_problem(3, 4, 5, 1, with_t2=False)
    L0 = np.zeros((0, p.nb, p.nb))
    sysb = SB.CoreHoleCCSD(np.diag(p.eps), np.diag(p.eps), L0, 3, 0)
    out = PR.propagate(sysb, 10, 0.05)
    assert np.abs(out["C"]).max() == 0.0
    assert max(np.abs(x).max() for x in out["t"]) == 0.0


def test_cayley_closed_form(rng):
    """P5: R = D*t (diagonal-only problem) -> t_n = ((1 + i dt D/2)/(1 - i dt D/2))^n t_0."""
    O, V = 3, 4
    eps = np.concatenate([[-20.0], np.sort(rng.uniform(-1, -0.3, O - 1)), np.sort(rng.uniform(0.1, 3, V))])
    sysb = SB.CoreHoleCCSD(np.diag(eps), np.diag(eps), np.zeros((0, O + V, O + V)), O, 0)
    t0 = random_blocks(sysb.shapes(), rng, scale=0.1)
    dt, n = 0.05, 17
    out = PR.propagate(sysb, n, dt, tol=1e-14, t0=t0)
    for x, x0, d in zip(out["t"], t0, sysb.diagonal()):
        ref = ((1 + 0.5j * dt * d) / (1 - 0.5j * dt * d)) ** n * x0
        assert np.abs(x - ref).max() < 1e-14
    assert np.all(out["micro"] == 2)


def _thouless_cumulant(fa, fb, occ, taus):
    C = np.zeros(len(taus), complex)
    for f, o in zip((fa, fb), occ):
        lam, U = np.linalg.eigh(f)
        dets = []
        for tau in taus:
            Ut = (U * np.exp(1j * lam * tau)) @ U.T
            dets.append(np.linalg.det(Ut[np.ix_(o, o)]) if len(o) else 1.0)
        C += FS.log_continuous(np.array(dets)) - 1j * taus * np.trace(f[np.ix_(o, o)])
    return C


def test_thouless_one_body_exact():
    """P6: with the two-electron part removed but the off-diagonal (N-1) Fock
    kept, e^{T1} is exact and C(tau) = sum_s [log det(e^{i tau f^s})_oo -
    i tau tr f^s_oo]; the propagation converges to it at O(dt^2).  Only the
    sum_ia f_ia t_i^a energy term survives here, so this pins that term."""
    O, V = 3, 4
    p = gen_problem(O, V, 6, 8, with_t2=False)
    fa, fb = H.fock_nm1(p.eps, p.L, 0)
    sysb = SB.CoreHoleCCSD(fa, fb, np.zeros((0, p.nb, p.nb)), O, 0)
    T = 2.0
    errs = []
    for dt in (0.04, 0.02):
        n = int(round(T / dt))
        out = PR.propagate(sysb, n, dt, tol=1e-14)
        assert max(np.abs(x).max() for x in out["t"][2:]) == 0.0     # T2 stays zero
        ex = _thouless_cumulant(fa, fb, sysb.occ, dt * np.arange(n + 1))
        errs.append(np.abs(out["C"] - ex).max())
    assert errs[1] < 5e-3
    assert 3.5 < errs[0] / errs[1] < 4.5, errs
    # the literal reading of Eq. 6 (no f_ia term) is not exact here
    out = PR.propagate(sysb, int(T / 0.02), 0.02, tol=1e-14, include_fov=False)
    ex = _thouless_cumulant(fa, fb, sysb.occ, 0.02 * np.arange(int(T / 0.02) + 1))
    assert np.abs(out["C"] - ex).max() > 100 * errs[1]


def test_exact_one_electron_reference():
    """P7a: O = 1 leaves one alpha electron in the (N-1) reference; CCSD is
    exact, so e^{C(tau)} = <Phi|e^{i H_N tau}|Phi> up to O(dt^2)."""
    O, V = 1, 3
    p = gen_problem(O, V, 5, 9, with_t2=False)
    sysb = SB.CoreHoleCCSD.from_problem(p.eps, p.L, O, 0)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, O)
    occ, vir = H.core_hole_reference(p.nb, O, 0)
    T = 1.0
    errs = []
    for dt in (0.02, 0.01):
        n = int(round(T / dt))
        out = PR.propagate(sysb, n, dt, tol=1e-14)
        ex = FS.log_continuous(FS.exact_normalisation(h, v, occ, dt * np.arange(n + 1)))
        errs.append(np.abs(out["C"] - ex).max())
    assert errs[1] < 1e-3 and 3.3 < errs[0] / errs[1] < 4.7, errs


def test_exact_two_electron_reference():
    """P7b: a generic open-shell 2-electron reference (oracle A, T1 and T2
    both active); CCSD is exact for two electrons."""
    p = gen_problem(1, 2, 4, 10, with_t2=False)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, 1)
    occ = [H.spinorb_index(p.nb, 0, 0), H.spinorb_index(p.nb, 1, 1)]
    vir = [k for k in range(2 * p.nb) if k not in occ]
    f = H.reference_fock(h, v, occ)
    sysa = SA.SpinOrbitalCCSD(f, v, occ, vir)
    T = 0.75
    errs = []
    for dt in (0.015, 0.0075):
        n = int(round(T / dt))
        out = PR.propagate(sysa, n, dt, tol=1e-14)
        assert np.abs(out["t"][1]).max() > 1e-4            # doubles are exercised
        ex = FS.log_continuous(FS.exact_normalisation(h, v, occ, dt * np.arange(n + 1)))
        errs.append(np.abs(out["C"] - ex).max())
    assert errs[1] < 1e-3 and 3.3 < errs[0] / errs[1] < 4.7, errs


def test_observed_order_in_dt():
    """P8: the trapezoid rule (Eq. 9) on a correlated core-hole problem:
    C(T) at dt, dt/2, dt/4 gives observed order ~2 (at least first order).
    The tiny system is stiff (couplings ~2 Ha), so dt starts at 0.01 to be in
    the asymptotic range."""
    p = gen_problem(2, 3, 5, 12, with_t2=False)
    sysb = SB.CoreHoleCCSD.from_problem(p.eps, p.L, 2, 0)
    T = 0.5
    vals = []
    for dt in (0.01, 0.005, 0.0025):
        out = PR.propagate(sysb, int(round(T / dt)), dt, tol=1e-14)
        vals.append(out["C"][-1])
    order = np.log2(abs(vals[0] - vals[1]) / abs(vals[1] - vals[2]))
    assert order > 1.8, order


def test_transform_closed_form():
    """P9: for C = 0 the transform is a geometric series:
    sum_n w_n z^n = (1 - z^{M+1})/(1 - z) - (1 + z^M)/2, z = exp((i(w - e) - eta) dt)."""
    dt, M, eps_c, e_corr, eta = 0.05, 400, -20.0, -0.31, 0.2
    G = PR.green_function(np.zeros(M + 1, complex), dt, eps_c, e_corr)
    omega = np.linspace(-22, -18, 41)
    A = PR.spectrum(G, dt, omega, eta)
    z = np.exp((1j * (omega - eps_c - e_corr) - eta) * dt)
    S = (1 - z ** (M + 1)) / (1 - z) - 0.5 * (1 + z ** M)
    ref = -(1 / np.pi) * np.imag(-1j * dt * S)
    assert np.abs(A - ref).max() < 1e-13 * np.abs(ref).max()
    # dt -> 0, long time: a Lorentzian of half-width eta at eps_c + E_corr
    dt2, M2 = 0.002, 40000
    G2 = PR.green_function(np.zeros(M2 + 1, complex), dt2, eps_c, e_corr)
    A2 = PR.spectrum(G2, dt2, omega, eta)
    lor = (eta / np.pi) / ((omega - eps_c - e_corr) ** 2 + eta ** 2)
    assert np.abs(A2 - lor).max() < 2e-3 * lor.max()


def test_transform_sum_rule_over_one_period():
    """P9 for any C: on a uniform grid of J > M frequencies spanning one
    period 2 pi/dt, the trapezoid sum over omega of exp(i omega tau_n) is
    J exp(i omega_0 tau_n) delta_n0, so dw sum_j A(omega_j) keeps only the
    n = 0 term: -(1/pi) Im(w_0 dt G_0 2 pi/dt) = -Im G_0 = Re exp(C_0) = 1,
    whatever C(t > 0), eta and the grid's origin.  Checked on a real
    propagation (non-zero C) and damping; a full end weight or a missing dt
    gives 2 or 1/dt instead."""
    p = gen_problem(3, 8, 10, 31)
    sysb = SB.CoreHoleCCSD.from_problem(p.eps, p.L, 3, 0)
    dt, M = 0.05, 24
    out = PR.propagate(sysb, M, dt, tol=1e-12)
    assert np.abs(out["C"][1:]).max() > 1e-3          # the dynamics is not trivial
    G = PR.green_function(out["C"], dt, p.eps[0], -0.31)
    for J, w0, eta in ((M + 1, -25.0, 0.0), (257, 3.7, 0.2), (1000, -21.3, 1.5)):
        dw = 2 * np.pi / dt / J
        omega = w0 + dw * np.arange(J)
        total = dw * PR.spectrum(G, dt, omega, eta).sum()
        assert abs(total - 1.0) < 1e-12, (J, total)
    # the identity needs the full period: a grid one point short misses it
    dw = 2 * np.pi / dt / 257
    short = dw * PR.spectrum(G, dt, -20.0 + dw * np.arange(256), 0.2).sum()
    assert abs(short - 1.0) > 1e-6


def test_closed_shell_ecorr_equals_spin_orbital_energy():
    """E_N^corr of Eq. 3 (closed-shell formula) equals the spin-orbital CC
    energy 1/4 sum <ij||ab> tau of the N-electron reference for the
    spin-adapted amplitudes t^{ab}_{ij}(aa) = t_ijab - t_ijba, t(ab) = t_ijab."""
    O, V = 3, 3
    p = gen_problem(O, V, 6, 13)
    h, v, occN = H.spinorb_hamiltonian(p.eps, p.L, O)
    nb = p.nb
    vir = [H.spinorb_index(nb, q, s) for s in (0, 1) for q in range(O, nb)]
    f = H.reference_fock(h, v, occN)
    t1, t2 = p.t1_gs, p.t2_gs
    assert np.allclose(t2, t2.transpose(1, 0, 3, 2))
    taa = t2 - t2.transpose(0, 1, 3, 2)
    t1so, t2so = SA.blocks_to_spinorb([t1, t1, taa, t2, taa], O, O, V, V)
    fr, vr = SA.reorder(f, v, occN, vir)
    E_so = SA.residual(fr, vr, 2 * O, t1so, t2so)[0]
    E_cs = PR.closed_shell_ecorr(p.L, O, t1, t2)
    assert abs(E_so - E_cs) < 1e-12 * max(1.0, abs(E_cs))

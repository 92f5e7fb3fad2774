"""Time propagation, cumulant, Green's function and spectrum (oracle; test
infrastructure only).

* Eq. 9 (first-order Adams-Moulton / implicit trapezoid): with the amplitude
  EOM -i dt/dtau = R(t) (Eqs. 7-8), t(tau+D) = t(tau) + (iD/2)[R(t(tau)) + R(t(tau+D))].
  Section 3 solves it by fixed-point iteration from T(0) = 0.  Reading: the
  diagonal part of R is treated exactly, R = D*t + R'(t) with D the Fock
  diagonal differences, so each micro-iteration is
      t^(k+1) = [(1 + iD*Delta/2) t_n + (i Delta/2)(R'_n + R'(t^(k)))] / (1 - iD*Delta/2),
  whose fixed point is the same trapezoid solution.  Predictor t^(0) = t_n;
  stop when max |t^(k+1) - t^(k)| < tol over every block; at most max_micro
  iterations, else NotConverged.  R'_n = R'(t_n) is evaluated at the start of
  each step (so the first micro-iteration reuses it).
* Eq. 5-6 (cumulant): dC/dtau = i E(tau), E = <Phi|(H_N e^T)_C|Phi>; the same
  trapezoid rule gives C_{n+1} = C_n + (i Delta/2)(E_n + E_{n+1}), C_0 = 0.
  Reading: E includes sum f_ia t_i^a (the definition in Eq. 5; Eq. 6 as
  printed omits it); ``include_fov=False`` follows Eq. 6 literally.
* Eq. 4: G_n = -i exp(-i (eps_c + E_corr) tau_n) exp(C_n).
* A(omega) = -(1/pi) Im sum_n w_n Delta G_n exp(i omega tau_n - eta tau_n),
  trapezoid weights w_0 = w_M = 1/2 (Section 2.1, A = -(1/pi) Im G^R(omega);
  reading: exponential damping eta and a direct sum on a user grid).
* E_N^corr of Eq. 3: the closed-shell CCSD energy of the N-electron ground
  state, sum_ijab [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b).

Pins (tests/test_oracle_propagate.py): zero couplings keep T and C at zero;
the Cayley closed form for a purely diagonal problem; the exact Thouless
cumulant of a one-body Hamiltonian; exact e^{C} = <Phi|e^{iH_N tau}|Phi> for
one- and two-electron references; observed order in dt; the closed-form
geometric series of the transform.
"""
from __future__ import annotations

import numpy as np


class NotConverged(RuntimeError):
    pass


def _maxabs(blocks):
    return max((float(np.abs(b).max()) if b.size else 0.0) for b in blocks)


def am_step(residual, D, t_n, Rp_n, dt, tol, max_micro):
    """One Eq. 9 step.  residual(t) returns the full projections R(t); R' = R - D*t.
    Returns (t_{n+1}, micro_iterations)."""
    num = [(1 + 0.5j * dt * d) * tn for d, tn in zip(D, t_n)]
    den = [1 - 0.5j * dt * d for d in D]
    tk = t_n
    for k in range(max_micro):
        if k == 0:
            Rk = Rp_n
        else:
            Rk = [r - d * x for r, d, x in zip(residual(tk), D, tk)]
        tnew = [(nm + 0.5j * dt * (a + b)) / dn for nm, a, b, dn in zip(num, Rp_n, Rk, den)]
        diff = _maxabs([x - y for x, y in zip(tnew, tk)])
        tk = tnew
        if not np.isfinite(diff):
            raise FloatingPointError("non-finite amplitudes")
        if diff < tol:
            return tk, k + 1
    raise NotConverged(f"fixed point not converged in {max_micro} micro-iterations (last change {diff:.3e})")


def propagate(system, nsteps, dt, tol=1e-12, max_micro=50, t0=None, include_fov=True,
              energy=None, residual=None):
    """Propagate from T(0) (zero unless t0 is given) for nsteps steps.

    ``system`` provides residual(t), energy(t), energy_fov(t), diagonal(),
    zeros() (oracle B's CoreHoleCCSD does).  Returns dict with C [nsteps+1],
    E [nsteps+1], micro [nsteps] and the final amplitudes.
    """
    residual = residual or system.residual
    D = system.diagonal()
    t = [np.array(x, dtype=complex) for x in (t0 if t0 is not None else system.zeros())]

    def en(tt):
        if energy is not None:
            return energy(tt)
        e = system.energy(tt)
        if not include_fov:
            e -= system.energy_fov(tt)
        return e
    C = np.zeros(nsteps + 1, dtype=complex)
    E = np.zeros(nsteps + 1, dtype=complex)
    E[0] = en(t)
    micro = np.zeros(nsteps, dtype=int)
    for n in range(nsteps):
        Rp = [r - d * x for r, d, x in zip(residual(t), D, t)]
        t, micro[n] = am_step(residual, D, t, Rp, dt, tol, max_micro)
        E[n + 1] = en(t)
        C[n + 1] = C[n] + 0.5j * dt * (E[n] + E[n + 1])
    return dict(C=C, E=E, micro=micro, t=t)


def green_function(C, dt, eps_c, e_corr):
    """G_n = -i exp(-i (eps_c + E_corr) tau_n) exp(C_n), tau_n = n*dt (Eq. 4)."""
    tau = dt * np.arange(len(C))
    return -1j * np.exp(-1j * (eps_c + e_corr) * tau) * np.exp(C)


def spectrum(G, dt, omega, eta):
    """A(w) = -(1/pi) Im sum_n w_n dt G_n exp(i w tau_n - eta tau_n)."""
    M = len(G) - 1
    tau = dt * np.arange(M + 1)
    w = np.ones(M + 1)
    w[0] = w[-1] = 0.5
    omega = np.asarray(omega, float)
    ph = np.exp(1j * omega[:, None] * tau[None, :] - eta * tau[None, :])
    return -(1.0 / np.pi) * np.imag(ph @ (w * dt * G))


def closed_shell_ecorr(L, nocc, t1, t2):
    """E_N^corr = sum_ijab [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b)."""
    Lov = L[:, :nocc, nocc:]
    iajb = np.einsum("Qia,Qjb->iajb", Lov, Lov, optimize=True)
    tt = t2 + np.einsum("ia,jb->ijab", t1, t1)
    return float(np.einsum("iajb,ijab->", 2 * iajb - iajb.transpose(0, 3, 2, 1), tt, optimize=True))

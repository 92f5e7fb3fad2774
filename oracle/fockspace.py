"""Determinant-space brute force (oracle; test infrastructure only).

Everything here follows second quantisation by definition: determinants are
bit strings over spin-orbitals, a_p / a_p^dagger act with the Jordan-Wigner
sign (-1)^(number of occupied spin-orbitals below p), and operators are built
as explicit matrices over all determinants with a fixed electron count.

* ``similarity_residuals``: <Phi_mu| e^{-T} H_N e^{T} |Phi> for arbitrary
  complex T1/T2, the quantity that Eqs. 7-8 (and, for mu = reference, Eq. 1
  without E_HF) project; (H_N e^T)_C projected on Phi_mu equals the
  e^{-T} H_N e^T projection (Eq. 2).
* ``exact_normalisation``: N(tau) = <Phi| e^{i H_N tau} |Phi>, the exact
  quantity whose logarithm is the cumulant of Eq. 5 (|Psi(tau)> =
  e^{i H tau}|Psi>, Section 2.1).

Pins: tests/test_oracle_fockspace.py checks the operator algebra against
textbook facts (anticommutators, number operator, Slater-Condon diagonal,
nilpotency) before it is used to pin oracle A.
"""
from __future__ import annotations

import itertools

import numpy as np


class FockSpace:
    """All determinants of ``nelec`` electrons in ``n`` spin-orbitals."""

    def __init__(self, n: int, nelec: int):
        self.n = n
        self.nelec = nelec
        self.dets = [sum(1 << p for p in c) for c in itertools.combinations(range(n), nelec)]
        self.index = {d: k for k, d in enumerate(self.dets)}
        self.dim = len(self.dets)

    @staticmethod
    def _sign(det: int, p: int) -> int:
        return -1 if bin(det & ((1 << p) - 1)).count("1") & 1 else 1

    @classmethod
    def annihilate(cls, det: int, p: int):
        if not (det >> p) & 1:
            return 0, 0
        return cls._sign(det, p), det & ~(1 << p)

    @classmethod
    def create(cls, det: int, p: int):
        if (det >> p) & 1:
            return 0, 0
        return cls._sign(det, p), det | (1 << p)

    def apply_string(self, ops, det: int):
        """Apply a product of operators, rightmost first.  ops: list of
        (is_creator, p) written left to right as in the operator product."""
        sgn = 1
        for cre, p in reversed(ops):
            s, det = (self.create if cre else self.annihilate)(det, p)
            if s == 0:
                return 0, 0
            sgn *= s
        return sgn, det

    def one_body(self, c: np.ndarray) -> np.ndarray:
        """Matrix of sum_pq c[p,q] a+_p a_q."""
        M = np.zeros((self.dim, self.dim), dtype=np.result_type(c, float))
        for col, d in enumerate(self.dets):
            occ = [q for q in range(self.n) if (d >> q) & 1]
            for q in occ:
                s1, d1 = self.annihilate(d, q)
                for p in range(self.n):
                    cpq = c[p, q]
                    if cpq == 0:
                        continue
                    s2, d2 = self.create(d1, p)
                    if s2 == 0:
                        continue
                    M[self.index[d2], col] += s1 * s2 * cpq
        return M

    def two_body(self, c: np.ndarray) -> np.ndarray:
        """Matrix of sum_pqrs c[p,q,r,s] a+_p a+_q a_s a_r."""
        M = np.zeros((self.dim, self.dim), dtype=np.result_type(c, float))
        for col, d in enumerate(self.dets):
            occ = [q for q in range(self.n) if (d >> q) & 1]
            for r in occ:
                s1, d1 = self.annihilate(d, r)
                for s in occ:
                    s2, d2 = self.annihilate(d1, s)
                    if s2 == 0:
                        continue
                    for q in range(self.n):
                        s3, d3 = self.create(d2, q)
                        if s3 == 0:
                            continue
                        for p in range(self.n):
                            cpqrs = c[p, q, r, s]
                            if cpqrs == 0:
                                continue
                            s4, d4 = self.create(d3, p)
                            if s4 == 0:
                                continue
                            M[self.index[d4], col] += s1 * s2 * s3 * s4 * cpqrs
        return M

    def det_of(self, occ) -> int:
        return sum(1 << p for p in occ)


def hamiltonian_matrix(fs: FockSpace, h: np.ndarray, v: np.ndarray) -> np.ndarray:
    """H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r (Section 2.1)."""
    return fs.one_body(h) + fs.two_body(0.25 * v)


def _expm_nilpotent(T: np.ndarray) -> np.ndarray:
    E = np.eye(T.shape[0], dtype=T.dtype)
    term = E.copy()
    for k in range(1, T.shape[0] + 1):
        term = term @ T / k
        if not np.any(term):
            break
        E = E + term
    return E


def cluster_matrix(fs: FockSpace, occ, vir, t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
    """T = sum t_i^a a+_a a_i + 1/4 sum t_ij^ab a+_a a+_b a_j a_i; indices of
    t1 [i,a] / t2 [i,j,a,b] refer to positions in the occ / vir lists."""
    n = fs.n
    c1 = np.zeros((n, n), dtype=complex)
    for ii, i in enumerate(occ):
        for aa, a in enumerate(vir):
            c1[a, i] = t1[ii, aa]
    c2 = np.zeros((n, n, n, n), dtype=complex)
    for ii, i in enumerate(occ):
        for jj, j in enumerate(occ):
            for aa, a in enumerate(vir):
                for bb, b in enumerate(vir):
                    # a+_a a+_b a_j a_i  ->  (p,q,r,s) = (a,b,i,j)
                    c2[a, b, i, j] = 0.25 * t2[ii, jj, aa, bb]
    return fs.one_body(c1) + fs.two_body(c2)


def similarity_residuals(h, v, occ, vir, t1, t2):
    """Brute-force CC projections for the reference determinant ``occ``.

    Returns (E, R1, R2) with E = <Phi|e^{-T} H_N e^T|Phi>,
    R1[i,a] = <Phi_i^a|...|Phi>, R2[i,j,a,b] = <Phi_ij^ab|...|Phi>, where
    |Phi_i^a> = a+_a a_i|Phi> and |Phi_ij^ab> = a+_a a+_b a_j a_i|Phi>.
    """
    n = h.shape[0]
    fs = FockSpace(n, len(occ))
    H = hamiltonian_matrix(fs, h, v)
    ref = fs.index[fs.det_of(occ)]
    HN = H - H[ref, ref] * np.eye(fs.dim)
    T = cluster_matrix(fs, occ, vir, t1, t2)
    Hbar = _expm_nilpotent(-T) @ HN @ _expm_nilpotent(T)
    col = Hbar[:, ref]
    d0 = fs.det_of(occ)
    no, nv = len(occ), len(vir)
    R1 = np.zeros((no, nv), dtype=complex)
    for ii, i in enumerate(occ):
        for aa, a in enumerate(vir):
            s, d = fs.apply_string([(True, a), (False, i)], d0)
            if s:
                R1[ii, aa] = s * col[fs.index[d]]
    R2 = np.zeros((no, no, nv, nv), dtype=complex)
    for ii, i in enumerate(occ):
        for jj, j in enumerate(occ):
            for aa, a in enumerate(vir):
                for bb, b in enumerate(vir):
                    s, d = fs.apply_string([(True, a), (True, b), (False, j), (False, i)], d0)
                    if s:
                        R2[ii, jj, aa, bb] = s * col[fs.index[d]]
    return col[ref], R1, R2


def exact_normalisation(h, v, occ, taus) -> np.ndarray:
    """N(tau) = <Phi| exp(i H_N tau) |Phi> by diagonalising H_N in the fixed
    electron-number determinant space."""
    fs = FockSpace(h.shape[0], len(occ))
    H = hamiltonian_matrix(fs, h, v)
    ref = fs.index[fs.det_of(occ)]
    HN = H - H[ref, ref] * np.eye(fs.dim)
    if np.iscomplexobj(HN):
        lam, U = np.linalg.eigh(HN)
    else:
        lam, U = np.linalg.eigh(0.5 * (HN + HN.T))
    w = np.abs(U[ref, :]) ** 2
    taus = np.asarray(taus, dtype=float)
    return (w[None, :] * np.exp(1j * lam[None, :] * taus[:, None])).sum(axis=1)


def log_continuous(z: np.ndarray) -> np.ndarray:
    """log z along a sampled path with the branch chosen continuously."""
    return np.log(np.abs(z)) + 1j * np.unwrap(np.angle(z))

"""(N-1)-electron reference quantities (oracle; test infrastructure only).

Section 2.1 of the paper: the reference |Phi> is the N-electron Hartree-Fock
determinant with the core spin-orbital c removed, and the Fock matrix of that
reference is f_pq = eps_p delta_pq - <pc||qc>.  The two-electron integrals are
Cholesky-factored (Section 3.1.1): (pq|rs) = sum_Q L^Q_pq L^Q_rs.

Reading (ambiguity): the removed spin-orbital is the beta copy of the core
orbital, so the alpha Fock loses only the Coulomb term and the beta Fock loses
Coulomb and gains exchange.

Pinned by tests/test_oracle_hamiltonian.py (spin-orbital construction from the
definition h = F^N - sum_{k in occ(N)} <pk||qk> agrees with the closed form
below; brute-force integral assembly by loops).
"""
from __future__ import annotations

import numpy as np


def eri_from_cholesky(L: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_Q L^Q_pq L^Q_rs, chemists' notation, shape [nb]^4."""
    return np.einsum("Qpq,Qrs->pqrs", L, L, optimize=True)


def fock_nm1(eps: np.ndarray, L: np.ndarray, core: int) -> tuple[np.ndarray, np.ndarray]:
    """Spatial Fock matrices (alpha, beta) of the (N-1)-electron reference.

    f^a_pq = eps_p d_pq - (pq|cc)
    f^b_pq = eps_p d_pq - (pq|cc) + (pc|cq)
    """
    J = np.einsum("Qpq,Q->pq", L, L[:, core, core])
    K = np.einsum("Qp,Qq->pq", L[:, :, core], L[:, core, :])
    fa = np.diag(eps) - J
    fb = np.diag(eps) - J + K
    return fa, fb


def spinorb_index(nb: int, p: int, spin: int) -> int:
    """Spin-orbital index: alpha orbitals first (0..nb-1), then beta."""
    return spin * nb + p


def spinorb_hamiltonian(eps: np.ndarray, L: np.ndarray, nocc: int):
    """Spin-orbital one-electron h and antisymmetrised <PQ||RS> of the system.

    h is fixed by requiring that the N-electron closed-shell determinant has
    the diagonal Fock matrix diag(eps):  h_PQ = eps_P d_PQ - sum_{K in occ(N)} <PK||QK>.
    Returns (h [2nb,2nb], v [2nb]^4, occN list).
    """
    nb = eps.size
    n = 2 * nb
    eri = eri_from_cholesky(L)
    spin = np.array([0] * nb + [1] * nb)
    sp = np.concatenate([np.arange(nb), np.arange(nb)])
    # <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS)
    g = eri[np.ix_(sp, sp, sp, sp)].transpose(0, 2, 1, 3).copy()
    same_pr = spin[:, None] == spin[None, :]
    g *= same_pr[:, None, :, None] * same_pr[None, :, None, :]
    v = g - g.transpose(0, 1, 3, 2)
    occN = [spinorb_index(nb, p, s) for s in (0, 1) for p in range(nocc)]
    eps_so = np.concatenate([eps, eps])
    h = np.diag(eps_so).astype(float)
    for k in occN:
        h -= v[:, k, :, k]
    return h, v, occN


def core_hole_reference(nb: int, nocc: int, core: int) -> tuple[list, list]:
    """Occupied / virtual spin-orbital lists of the (N-1) reference.

    Ordering matches the spin-explicit blocks: alpha occupied (0..O-1), beta
    occupied (0..O-1 without the core); alpha virtual (O..nb-1), beta virtual
    (core first, then O..nb-1).
    """
    occ = [spinorb_index(nb, p, 0) for p in range(nocc)]
    occ += [spinorb_index(nb, p, 1) for p in range(nocc) if p != core]
    vir = [spinorb_index(nb, p, 0) for p in range(nocc, nb)]
    vir += [spinorb_index(nb, core, 1)] + [spinorb_index(nb, p, 1) for p in range(nocc, nb)]
    return occ, vir


def reference_fock(h: np.ndarray, v: np.ndarray, occ: list) -> np.ndarray:
    """f_PQ = h_PQ + sum_{K in occ} <PK||QK> for an arbitrary reference determinant."""
    f = h.copy()
    for k in occ:
        f = f + v[:, k, :, k]
    return f

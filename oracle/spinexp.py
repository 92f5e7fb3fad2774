"""Oracle B: spin-explicit, Cholesky-factored CCSD residual (oracle; test
infrastructure only).

Section 3.1.1 of the paper keeps only the unique non-zero spin blocks
(T1: alpha, beta; T2: alpha-alpha, alpha-beta, beta-beta) and never builds the
four-index integrals: every two-electron quantity is a sum over Cholesky
vectors, (pq|rs) = sum_Q L^Q_pq L^Q_rs.  This module evaluates the full
projection R_mu = <Phi_mu|(H_N e^{T1+T2})_C|Phi> of Eqs. 7-8 block by block,
with each integral written as its two Cholesky factors inside the einsum
(the library primitive picks the contraction order).  The spin blocks are the
spin integration of the spin-orbital equations of oracle A (Stanton-Gauss
intermediates); the tau*tau*<mn||ef> quadratic term is carried entirely by
W_mnij (coefficient 1/2 there instead of 1/4 in both W_mnij and W_abef, an
exact regrouping).

Index sets (unpadded, true spin-orbital ranges), hole in beta:
  alpha occupied 0..O-1,  beta occupied 0..O-1 without the core c,
  alpha virtual O..nb-1,  beta virtual [c, O..nb-1].
Blocks: t1a[oA,vA], t1b[oB,vB], t2aa[oA,oA,vA,vA], t2ab[oA,oB,vA,vB],
        t2bb[oB,oB,vB,vB]; t2aa/t2bb antisymmetric in (i,j) and (a,b).

Pinned by tests/test_oracle_spinexp.py: equals oracle A (assembled
<pq||rs>) on random complex amplitudes, hence the brute force.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import fock_nm1


_PATHS: dict = {}


def _ein(sub, *ops):
    """np.einsum with the contraction order chosen once per (subscripts, shapes)."""
    key = (sub,) + tuple(o.shape for o in ops)
    path = _PATHS.get(key)
    if path is None:
        path = np.einsum_path(sub, *ops, optimize=("optimal", 2**31))[0]
        _PATHS[key] = path
    return np.einsum(sub, *ops, optimize=path)


class CoreHoleCCSD:
    """Spin-explicit residual for one core hole.

    fa, fb: (N-1) Fock matrices (spatial, [nb,nb]) for alpha and beta;
    L: Cholesky vectors [nchol,nb,nb]; nocc: occupied spatial orbitals of the
    N-electron system; core: spatial index of the removed (beta) electron.
    """

    def __init__(self, fa, fb, L, nocc, core=0):
        nb = fa.shape[0]
        self.nb, self.nocc, self.core = nb, nocc, core
        self.occ = [np.arange(nocc), np.array([p for p in range(nocc) if p != core], dtype=int)]
        self.vir = [np.arange(nocc, nb), np.array([core] + list(range(nocc, nb)), dtype=int)]
        self.f = [np.asarray(fa, float), np.asarray(fb, float)]
        self.Lfull = np.asarray(L, float)
        self._Lcache = {}

    @classmethod
    def from_problem(cls, eps, L, nocc, core=0):
        fa, fb = fock_nm1(eps, L, core)
        return cls(fa, fb, L, nocc, core)

    # index helpers -------------------------------------------------------
    def idx(self, s, X):
        return self.occ[s] if X == "o" else self.vir[s]

    def L(self, s, X, Y):
        key = (s, X, Y)
        if key not in self._Lcache:
            self._Lcache[key] = np.ascontiguousarray(
                self.Lfull[:, self.idx(s, X)][:, :, self.idx(s, Y)])
        return self._Lcache[key]

    def F(self, s, X, Y):
        return self.f[s][np.ix_(self.idx(s, X), self.idx(s, Y))]

    def shapes(self):
        oA, oB = len(self.occ[0]), len(self.occ[1])
        vA, vB = len(self.vir[0]), len(self.vir[1])
        return [(oA, vA), (oB, vB), (oA, oA, vA, vA), (oA, oB, vA, vB), (oB, oB, vB, vB)]

    def zeros(self):
        return [np.zeros(s, dtype=complex) for s in self.shapes()]

    def diagonal(self):
        """D with R = D*t + R'(t): D_ia = f_aa - f_ii, D_ijab = f_aa + f_bb - f_ii - f_jj."""
        do = [np.diag(self.F(s, "o", "o")) for s in (0, 1)]
        dv = [np.diag(self.F(s, "v", "v")) for s in (0, 1)]
        D1 = [dv[s][None, :] - do[s][:, None] for s in (0, 1)]
        def d2(s, u):
            return (dv[s][None, None, :, None] + dv[u][None, None, None, :]
                    - do[s][:, None, None, None] - do[u][None, :, None, None])
        return [D1[0], D1[1], d2(0, 0), d2(0, 1), d2(1, 1)]

    # residual -------------------------------------------------------------
    def residual(self, t):
        """Full projections [R1a, R1b, R2aa, R2ab, R2bb] (Eqs. 7-8)."""
        L, F = self.L, self.F
        t1 = [t[0], t[1]]
        t2ss = [t[2], t[4]]
        t2ab = t[3]
        t2su = [t2ab, t2ab.transpose(1, 0, 3, 2)]   # [i in occ_s, j in occ_u, a in vir_s, b in vir_u]

        def t1t1(s, u):
            return _ein("ia,jb->ijab", t1[s], t1[u])
        tau_ss, taut_ss, tau_su, taut_su = [], [], [], []
        for s in (0, 1):
            u = 1 - s
            x = t1t1(s, s)
            tau_ss.append(t2ss[s] + x - x.swapaxes(2, 3))
            taut_ss.append(t2ss[s] + 0.5 * (x - x.swapaxes(2, 3)))
            y = t1t1(s, u)
            tau_su.append(t2su[s] + y)
            taut_su.append(t2su[s] + 0.5 * y)

        Fme, Fae, Fmi = [], [], []
        for s in (0, 1):
            u = 1 - s
            Fme.append(F(s, "o", "v")
                       + _ein("nf,Qme,Qnf->me", t1[s], L(s, "o", "v"), L(s, "o", "v"))
                       + _ein("nf,Qme,Qnf->me", t1[u], L(s, "o", "v"), L(u, "o", "v"))
                       - _ein("nf,Qmf,Qne->me", t1[s], L(s, "o", "v"), L(s, "o", "v")))
            Fae.append(F(s, "v", "v") - 0.5 * _ein("me,ma->ae", F(s, "o", "v"), t1[s])
                       + _ein("mf,Qmf,Qae->ae", t1[s], L(s, "o", "v"), L(s, "v", "v"))
                       + _ein("mf,Qmf,Qae->ae", t1[u], L(u, "o", "v"), L(s, "v", "v"))
                       - _ein("mf,Qme,Qaf->ae", t1[s], L(s, "o", "v"), L(s, "v", "v"))
                       - _ein("mnaf,Qme,Qnf->ae", taut_ss[s], L(s, "o", "v"), L(s, "o", "v"))
                       - _ein("mnaf,Qme,Qnf->ae", taut_su[s], L(s, "o", "v"), L(u, "o", "v")))
            Fmi.append(F(s, "o", "o") + 0.5 * _ein("ie,me->mi", t1[s], F(s, "o", "v"))
                       + _ein("ne,Qmi,Qne->mi", t1[s], L(s, "o", "o"), L(s, "o", "v"))
                       + _ein("ne,Qmi,Qne->mi", t1[u], L(s, "o", "o"), L(u, "o", "v"))
                       - _ein("ne,Qme,Qni->mi", t1[s], L(s, "o", "v"), L(s, "o", "o"))
                       + _ein("inef,Qme,Qnf->mi", taut_ss[s], L(s, "o", "v"), L(s, "o", "v"))
                       + _ein("inef,Qme,Qnf->mi", taut_su[s], L(s, "o", "v"), L(u, "o", "v")))

        # T1 projections (Eq. 7)
        R1 = []
        for s in (0, 1):
            u = 1 - s
            R1.append(F(s, "o", "v") + _ein("ie,ae->ia", t1[s], Fae[s]) - _ein("ma,mi->ia", t1[s], Fmi[s])
                      + _ein("imae,me->ia", t2ss[s], Fme[s]) + _ein("imae,me->ia", t2su[s], Fme[u])
                      - _ein("nf,Qni,Qaf->ia", t1[s], L(s, "o", "o"), L(s, "v", "v"))
                      + _ein("nf,Qnf,Qai->ia", t1[s], L(s, "o", "v"), L(s, "v", "o"))
                      + _ein("nf,Qnf,Qai->ia", t1[u], L(u, "o", "v"), L(s, "v", "o"))
                      + _ein("imef,Qmf,Qae->ia", t2ss[s], L(s, "o", "v"), L(s, "v", "v"))
                      + _ein("imef,Qmf,Qae->ia", t2su[s], L(u, "o", "v"), L(s, "v", "v"))
                      - _ein("mnae,Qmi,Qne->ia", t2ss[s], L(s, "o", "o"), L(s, "o", "v"))
                      - _ein("mnae,Qmi,Qne->ia", t2su[s], L(s, "o", "o"), L(u, "o", "v")))

        Fvv = [Fae[s] - 0.5 * _ein("mb,me->be", t1[s], Fme[s]) for s in (0, 1)]
        Foo = [Fmi[s] + 0.5 * _ein("je,me->mj", t1[s], Fme[s]) for s in (0, 1)]

        # W_mnij, same spin and alpha-beta
        Wss = []
        for s in (0, 1):
            x = (_ein("je,Qmi,Qne->mnij", t1[s], L(s, "o", "o"), L(s, "o", "v"))
                 - _ein("je,Qme,Qni->mnij", t1[s], L(s, "o", "v"), L(s, "o", "o")))
            Wss.append(_ein("Qmi,Qnj->mnij", L(s, "o", "o"), L(s, "o", "o"))
                       - _ein("Qmj,Qni->mnij", L(s, "o", "o"), L(s, "o", "o"))
                       + x - x.swapaxes(2, 3)
                       + _ein("ijef,Qme,Qnf->mnij", tau_ss[s], L(s, "o", "v"), L(s, "o", "v")))
        Wab = (_ein("Qmi,Qnj->mnij", L(0, "o", "o"), L(1, "o", "o"))
               + _ein("je,Qmi,Qne->mnij", t1[1], L(0, "o", "o"), L(1, "o", "v"))
               + _ein("ie,Qme,Qnj->mnij", t1[0], L(0, "o", "v"), L(1, "o", "o"))
               + _ein("ijef,Qme,Qnf->mnij", tau_su[0], L(0, "o", "v"), L(1, "o", "v")))

        # W_mbej spin blocks; superscripts give the spins of (m, b, e, j)
        def W_same(s):
            u = 1 - s
            X = 0.5 * t2ss[s] + _ein("jf,nb->jnfb", t1[s], t1[s])
            return (_ein("Qme,Qbj->mbej", L(s, "o", "v"), L(s, "v", "o"))
                    - _ein("Qmj,Qbe->mbej", L(s, "o", "o"), L(s, "v", "v"))
                    + _ein("jf,Qme,Qbf->mbej", t1[s], L(s, "o", "v"), L(s, "v", "v"))
                    - _ein("jf,Qmf,Qbe->mbej", t1[s], L(s, "o", "v"), L(s, "v", "v"))
                    - _ein("nb,Qme,Qnj->mbej", t1[s], L(s, "o", "v"), L(s, "o", "o"))
                    + _ein("nb,Qmj,Qne->mbej", t1[s], L(s, "o", "o"), L(s, "o", "v"))
                    - _ein("jnfb,Qme,Qnf->mbej", X, L(s, "o", "v"), L(s, "o", "v"))
                    + _ein("jnfb,Qmf,Qne->mbej", X, L(s, "o", "v"), L(s, "o", "v"))
                    + 0.5 * _ein("jnbf,Qme,Qnf->mbej", t2su[s], L(s, "o", "v"), L(u, "o", "v")))

        def W_usus(s):   # m u, b s, e u, j s
            u = 1 - s
            X = 0.5 * t2ss[s] + _ein("jf,nb->jnfb", t1[s], t1[s])
            return (_ein("Qme,Qbj->mbej", L(u, "o", "v"), L(s, "v", "o"))
                    + _ein("jf,Qme,Qbf->mbej", t1[s], L(u, "o", "v"), L(s, "v", "v"))
                    - _ein("nb,Qme,Qnj->mbej", t1[s], L(u, "o", "v"), L(s, "o", "o"))
                    + 0.5 * _ein("jnbf,Qme,Qnf->mbej", t2su[s], L(u, "o", "v"), L(u, "o", "v"))
                    - 0.5 * _ein("jnbf,Qmf,Qne->mbej", t2su[s], L(u, "o", "v"), L(u, "o", "v"))
                    - _ein("jnfb,Qme,Qnf->mbej", X, L(u, "o", "v"), L(s, "o", "v")))

        def W_suus(s):   # m s, b u, e u, j s
            u = 1 - s
            Y = 0.5 * t2su[s] + _ein("jf,nb->jnfb", t1[s], t1[u])
            return (-_ein("Qmj,Qbe->mbej", L(s, "o", "o"), L(u, "v", "v"))
                    - _ein("jf,Qmf,Qbe->mbej", t1[s], L(s, "o", "v"), L(u, "v", "v"))
                    + _ein("nb,Qmj,Qne->mbej", t1[u], L(s, "o", "o"), L(u, "o", "v"))
                    + _ein("jnfb,Qmf,Qne->mbej", Y, L(s, "o", "v"), L(u, "o", "v")))

        Waaaa, Wbbbb = W_same(0), W_same(1)
        Wbaba, Wabab = W_usus(0), W_usus(1)
        Wabba, Wbaab = W_suus(0), W_suus(1)
        Wsame = [Waaaa, Wbbbb]
        Wx = [Wbaba, Wabab]

        # T2 projections, same spin (Eq. 8)
        R2ss = []
        for s in (0, 1):
            R = (_ein("Qia,Qjb->ijab", L(s, "o", "v"), L(s, "o", "v"))
                 - _ein("Qib,Qja->ijab", L(s, "o", "v"), L(s, "o", "v")))
            x = _ein("ijae,be->ijab", t2ss[s], Fvv[s])
            R = R + x - x.swapaxes(2, 3)
            x = _ein("imab,mj->ijab", t2ss[s], Foo[s])
            R = R - (x - x.swapaxes(0, 1))
            R = R + 0.5 * _ein("mnab,mnij->ijab", tau_ss[s], Wss[s])
            R = R + _ein("ijef,Qae,Qbf->ijab", tau_ss[s], L(s, "v", "v"), L(s, "v", "v"))
            Z = _ein("ijef,Qae,Qmf->ijam", tau_ss[s], L(s, "v", "v"), L(s, "o", "v"))
            x = _ein("mb,ijam->ijab", t1[s], Z)
            R = R - (x - x.swapaxes(2, 3))
            X = (_ein("imae,mbej->ijab", t2ss[s], Wsame[s]) + _ein("imae,mbej->ijab", t2su[s], Wx[s])
                 - _ein("ie,ma,Qme,Qbj->ijab", t1[s], t1[s], L(s, "o", "v"), L(s, "v", "o"))
                 + _ein("ie,ma,Qmj,Qbe->ijab", t1[s], t1[s], L(s, "o", "o"), L(s, "v", "v")))
            X = X - X.swapaxes(0, 1)
            R = R + X - X.swapaxes(2, 3)
            x = (_ein("ie,Qae,Qbj->ijab", t1[s], L(s, "v", "v"), L(s, "v", "o"))
                 - _ein("ie,Qaj,Qbe->ijab", t1[s], L(s, "v", "o"), L(s, "v", "v")))
            R = R + x - x.swapaxes(0, 1)
            x = (_ein("ma,Qmi,Qbj->ijab", t1[s], L(s, "o", "o"), L(s, "v", "o"))
                 - _ein("ma,Qmj,Qbi->ijab", t1[s], L(s, "o", "o"), L(s, "v", "o")))
            R = R - (x - x.swapaxes(2, 3))
            R2ss.append(R)

        # T2 projection, alpha-beta (Eq. 8)
        a, b = 0, 1
        t1a, t1b, tau_ab = t1[0], t1[1], tau_su[0]
        R = _ein("Qia,Qjb->ijab", L(a, "o", "v"), L(b, "o", "v"))
        R = R + _ein("ijae,be->ijab", t2ab, Fvv[b]) + _ein("ijeb,ae->ijab", t2ab, Fvv[a])
        R = R - _ein("imab,mj->ijab", t2ab, Foo[b]) - _ein("mjab,mi->ijab", t2ab, Foo[a])
        R = R + _ein("mnab,mnij->ijab", tau_ab, Wab)
        R = R + _ein("ijef,Qae,Qbf->ijab", tau_ab, L(a, "v", "v"), L(b, "v", "v"))
        Z1 = _ein("ijef,Qae,Qmf->ijam", tau_ab, L(a, "v", "v"), L(b, "o", "v"))
        Z2 = _ein("ijef,Qme,Qbf->ijmb", tau_ab, L(a, "o", "v"), L(b, "v", "v"))
        R = R - _ein("mb,ijam->ijab", t1b, Z1) - _ein("ma,ijmb->ijab", t1a, Z2)
        R = R + (_ein("imae,mbej->ijab", t2ss[0], Wabab) + _ein("imae,mbej->ijab", t2ab, Wbbbb)
                 - _ein("ie,ma,Qme,Qbj->ijab", t1a, t1a, L(a, "o", "v"), L(b, "v", "o")))
        R = R + (_ein("mjae,mbei->ijab", t2ab, Wabba)
                 - _ein("je,ma,Qmi,Qbe->ijab", t1b, t1a, L(a, "o", "o"), L(b, "v", "v")))
        R = R + (_ein("imeb,maej->ijab", t2ab, Wbaab)
                 - _ein("ie,mb,Qmj,Qae->ijab", t1a, t1b, L(b, "o", "o"), L(a, "v", "v")))
        R = R + (_ein("mjeb,maei->ijab", t2ab, Waaaa) + _ein("jmbe,maei->ijab", t2ss[1], Wbaba)
                 - _ein("je,mb,Qme,Qai->ijab", t1b, t1b, L(b, "o", "v"), L(a, "v", "o")))
        R = R + (_ein("ie,Qae,Qbj->ijab", t1a, L(a, "v", "v"), L(b, "v", "o"))
                 + _ein("je,Qai,Qbe->ijab", t1b, L(a, "v", "o"), L(b, "v", "v")))
        R = R - (_ein("ma,Qmi,Qbj->ijab", t1a, L(a, "o", "o"), L(b, "v", "o"))
                 + _ein("mb,Qmj,Qai->ijab", t1b, L(b, "o", "o"), L(a, "v", "o")))
        return [R1[0], R1[1], R2ss[0], R, R2ss[1]]

    def energy(self, t):
        """<Phi|(H_N e^T)_C|Phi>, the integrand of Eq. 5 (f_ia term included)."""
        L, F = self.L, self.F
        t1 = [t[0], t[1]]
        t2ss = [t[2], t[4]]
        E = 0j
        for s in (0, 1):
            Lov = L(s, "o", "v")
            E += _ein("ia,ia->", F(s, "o", "v"), t1[s])
            E += 0.5 * _ein("ijab,Qia,Qjb->", t2ss[s], Lov, Lov)
            E += 0.5 * (_ein("ia,jb,Qia,Qjb->", t1[s], t1[s], Lov, Lov)
                        - _ein("ia,jb,Qib,Qja->", t1[s], t1[s], Lov, Lov))
        E += _ein("ijab,Qia,Qjb->", t[3], L(0, "o", "v"), L(1, "o", "v"))
        E += _ein("ia,jb,Qia,Qjb->", t1[0], t1[1], L(0, "o", "v"), L(1, "o", "v"))
        return E

    def energy_fov(self, t):
        """The sum_ia f_ia t_i^a part of the energy alone."""
        return sum(_ein("ia,ia->", self.F(s, "o", "v"), t[s]) for s in (0, 1))

"""Oracle A: spin-orbital CCSD residual (oracle; test infrastructure only).

The paper does not print the terms of <Phi_mu|(H_N e^{T1+T2})_C|Phi>
(Eqs. 7-8); they are the standard coupled-cluster singles-and-doubles
projections for a general (non-canonical, non-Hartree-Fock) reference: the
(N-1) reference of Section 2.1 has non-zero occupied-virtual Fock elements.
They are written here in the intermediate form of Stanton, Gauss, Watts and
Bartlett (J. Chem. Phys. 94, 4334 (1991)), with the full Fock diagonal kept
inside F (so the result is the whole projection, not the residual minus D*t),
using explicitly assembled antisymmetrised integrals v[p,q,r,s] = <pq||rs>.

Energy (Eq. 1 without E_HF; the integrand of Eq. 5):
  E = sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b

Works for any reference occupation (used with 2-electron references too).
Pinned by tests/test_oracle_spinorb.py against the determinant brute force
(fockspace.similarity_residuals) on random complex amplitudes.
"""
from __future__ import annotations

import numpy as np


_PATHS: dict = {}


def _ein(sub, *ops):
    """np.einsum with the contraction order chosen once per (subscripts, shapes)."""
    key = (sub,) + tuple(o.shape for o in ops)
    path = _PATHS.get(key)
    if path is None:
        path = np.einsum_path(sub, *ops, optimize=("optimal", 2**31))[0]
        _PATHS[key] = path
    return np.einsum(sub, *ops, optimize=path)


def _Pij(x):
    return x - x.swapaxes(0, 1)


def _Pab(x):
    return x - x.swapaxes(2, 3)


def reorder(f: np.ndarray, v: np.ndarray, occ, vir):
    """Permute spin-orbitals so that ``occ`` come first, then ``vir``."""
    perm = list(occ) + list(vir)
    return f[np.ix_(perm, perm)], v[np.ix_(perm, perm, perm, perm)]


def residual(f: np.ndarray, v: np.ndarray, nocc: int, t1: np.ndarray, t2: np.ndarray):
    """Return (E, R1, R2) for spin-orbital f, v with occupied orbitals first."""
    o = slice(0, nocc)
    w = slice(nocc, f.shape[0])
    fov, foo, fvv = f[o, w], f[o, o], f[w, w]
    oooo, ooov, oovv = v[o, o, o, o], v[o, o, o, w], v[o, o, w, w]
    ovvo, ovov, ovvv = v[o, w, w, o], v[o, w, o, w], v[o, w, w, w]
    oovo, vvvv, vovv = v[o, o, w, o], v[w, w, w, w], v[w, o, w, w]
    vvvo, ovoo = v[w, w, w, o], v[o, w, o, o]

    t1t1 = _ein("ia,jb->ijab", t1, t1)
    tau = t2 + t1t1 - t1t1.swapaxes(2, 3)
    taut = t2 + 0.5 * (t1t1 - t1t1.swapaxes(2, 3))

    Fae = (fvv - 0.5 * _ein("me,ma->ae", fov, t1) + _ein("mf,mafe->ae", t1, ovvv)
           - 0.5 * _ein("mnaf,mnef->ae", taut, oovv))
    Fmi = (foo + 0.5 * _ein("ie,me->mi", t1, fov) + _ein("ne,mnie->mi", t1, ooov)
           + 0.5 * _ein("inef,mnef->mi", taut, oovv))
    Fme = fov + _ein("nf,mnef->me", t1, oovv)
    x = _ein("je,mnie->mnij", t1, ooov)
    Wmnij = oooo + (x - x.swapaxes(2, 3)) + 0.25 * _ein("ijef,mnef->mnij", tau, oovv)
    y = _ein("mb,amef->abef", t1, vovv)
    Wabef = (vvvv - (y - y.swapaxes(0, 1))
             + 0.25 * _ein("mnab,mnef->abef", tau, oovv))
    X = 0.5 * t2 + _ein("jf,nb->jnfb", t1, t1)
    Wmbej = (ovvo + _ein("jf,mbef->mbej", t1, ovvv) - _ein("nb,mnej->mbej", t1, oovo)
             - _ein("jnfb,mnef->mbej", X, oovv))

    R1 = (fov + _ein("ie,ae->ia", t1, Fae) - _ein("ma,mi->ia", t1, Fmi)
          + _ein("imae,me->ia", t2, Fme) - _ein("nf,naif->ia", t1, ovov)
          - 0.5 * _ein("imef,maef->ia", t2, ovvv) - 0.5 * _ein("mnae,nmei->ia", t2, oovo))

    Fbe = Fae - 0.5 * _ein("mb,me->be", t1, Fme)
    Fmj = Fmi + 0.5 * _ein("je,me->mj", t1, Fme)
    R2 = (oovv + _Pab(_ein("ijae,be->ijab", t2, Fbe)) - _Pij(_ein("imab,mj->ijab", t2, Fmj))
          + 0.5 * _ein("mnab,mnij->ijab", tau, Wmnij) + 0.5 * _ein("ijef,abef->ijab", tau, Wabef)
          + _Pij(_Pab(_ein("imae,mbej->ijab", t2, Wmbej)
                      - _ein("ie,ma,mbej->ijab", t1, t1, ovvo)))
          + _Pij(_ein("ie,abej->ijab", t1, vvvo)) - _Pab(_ein("ma,mbij->ijab", t1, ovoo)))

    E = (_ein("ia,ia->", fov, t1) + 0.25 * _ein("ijab,ijab->", oovv, t2)
         + 0.5 * _ein("ijab,ia,jb->", oovv, t1, t1))
    return E, R1, R2


def blocks_to_spinorb(blocks, nocc_a, nocc_b, nvir_a, nvir_b):
    """Spin-explicit blocks (t1a, t1b, t2aa, t2ab, t2bb) -> spin-orbital t1, t2
    with occupied order [alpha, beta] and virtual order [alpha, beta]."""
    t1a, t1b, t2aa, t2ab, t2bb = blocks
    no, nv = nocc_a + nocc_b, nvir_a + nvir_b
    oa, ob = slice(0, nocc_a), slice(nocc_a, no)
    va, vb = slice(0, nvir_a), slice(nvir_a, nv)
    t1 = np.zeros((no, nv), dtype=complex)
    t1[oa, va] = t1a
    t1[ob, vb] = t1b
    t2 = np.zeros((no, no, nv, nv), dtype=complex)
    t2[oa, oa, va, va] = t2aa
    t2[ob, ob, vb, vb] = t2bb
    t2[oa, ob, va, vb] = t2ab
    t2[ob, oa, va, vb] = -t2ab.transpose(1, 0, 2, 3)
    t2[oa, ob, vb, va] = -t2ab.transpose(0, 1, 3, 2)
    t2[ob, oa, vb, va] = t2ab.transpose(1, 0, 3, 2)
    return t1, t2


def spinorb_to_blocks(t1, t2, nocc_a, nocc_b, nvir_a, nvir_b):
    """Inverse of blocks_to_spinorb (reads the unique spin blocks)."""
    no, nv = nocc_a + nocc_b, nvir_a + nvir_b
    oa, ob = slice(0, nocc_a), slice(nocc_a, no)
    va, vb = slice(0, nvir_a), slice(nvir_a, nv)
    return (t1[oa, va].copy(), t1[ob, vb].copy(), t2[oa, oa, va, va].copy(),
            t2[oa, ob, va, vb].copy(), t2[ob, ob, vb, vb].copy())


class SpinOrbitalCCSD:
    """Oracle A packaged for oracle/propagate.py: amplitudes are [t1, t2] in
    the spin-orbital basis of an arbitrary reference ``occ``."""

    def __init__(self, f, v, occ, vir):
        self.fr, self.vr = reorder(f, v, occ, vir)
        self.no, self.nv = len(occ), len(vir)

    def zeros(self):
        return [np.zeros((self.no, self.nv), complex),
                np.zeros((self.no, self.no, self.nv, self.nv), complex)]

    def residual(self, t):
        _, R1, R2 = residual(self.fr, self.vr, self.no, t[0], t[1])
        return [R1, R2]

    def energy(self, t):
        return residual(self.fr, self.vr, self.no, t[0], t[1])[0]

    def energy_fov(self, t):
        return np.einsum("ia,ia->", self.fr[:self.no, self.no:], t[0])

    def diagonal(self):
        d = np.diag(self.fr)
        do, dv = d[:self.no], d[self.no:]
        D1 = dv[None, :] - do[:, None]
        D2 = (dv[None, None, :, None] + dv[None, None, None, :]
              - do[:, None, None, None] - do[None, :, None, None])
        return [D1, D2]

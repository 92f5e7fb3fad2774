"""Pins of the determinant-space brute force against second-quantisation
identities (no CC arithmetic involved)."""
import numpy as np
import pytest

from oracle import fockspace as FS
from oracle import hamiltonian as H
from synth import gen_problem


@pytest.fixture(scope="module")
def small():
    p = gen_problem(2, 2, 5, 11, with_t2=False)
    h, v, occN = H.spinorb_hamiltonian(p.eps, p.L, 2)
    occ, vir = H.core_hole_reference(p.nb, 2, 0)
    return p, h, v, occ, vir, FS.FockSpace(2 * p.nb, len(occ))


def test_number_operator(small):
    *_, fs = small
    N = fs.one_body(np.eye(fs.n))
    assert np.allclose(N, fs.nelec * np.eye(fs.dim))


def test_one_body_commutator(small, rng):
    *_, fs = small
    n = fs.n
    for _ in range(6):
        p, q, r, s = rng.integers(0, n, 4)
        Epq = fs.one_body(np.eye(n)[:, [p]] @ np.eye(n)[[q], :])
        Ers = fs.one_body(np.eye(n)[:, [r]] @ np.eye(n)[[s], :])
        Eps = fs.one_body(np.eye(n)[:, [p]] @ np.eye(n)[[s], :])
        Erq = fs.one_body(np.eye(n)[:, [r]] @ np.eye(n)[[q], :])
        lhs = Epq @ Ers - Ers @ Epq
        rhs = (q == r) * Eps - (p == s) * Erq
        assert np.allclose(lhs, rhs)


def test_two_body_from_one_body(small, rng):
    """a+_p a+_q a_s a_r = E_pr E_qs - delta_qr E_ps."""
    *_, fs = small
    n = fs.n
    for _ in range(6):
        p, q, r, s = rng.integers(0, n, 4)
        c = np.zeros((n, n, n, n))
        c[p, q, r, s] = 1.0
        E = lambda a, b: fs.one_body(np.eye(n)[:, [a]] @ np.eye(n)[[b], :])  # noqa: E731
        assert np.allclose(fs.two_body(c), E(p, r) @ E(q, s) - (q == r) * E(p, s))


def test_hamiltonian_hermitian_and_slater_condon(small):
    p, h, v, occ, vir, fs = small
    Hm = FS.hamiltonian_matrix(fs, h, v)
    assert np.allclose(Hm, Hm.T)
    ref = fs.index[fs.det_of(occ)]
    e_sc = sum(h[i, i] for i in occ) + 0.5 * sum(v[i, j, i, j] for i in occ for j in occ)
    assert abs(Hm[ref, ref] - e_sc) < 1e-12


def test_cluster_operator_nilpotent(small, rng):
    p, h, v, occ, vir, fs = small
    no, nv = len(occ), len(vir)
    t1 = rng.standard_normal((no, nv)) + 1j * rng.standard_normal((no, nv))
    t2 = rng.standard_normal((no, no, nv, nv)) + 0j
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    T = FS.cluster_matrix(fs, occ, vir, t1, t2)
    P = np.linalg.matrix_power(T, fs.nelec + 1)
    assert np.abs(P).max() < 1e-9 * max(1.0, np.abs(T).max() ** (fs.nelec + 1))


def test_exact_normalisation_basic(small):
    p, h, v, occ, vir, fs = small
    Nt = FS.exact_normalisation(h, v, occ, [0.0, 0.3, 1.7])
    assert abs(Nt[0] - 1) < 1e-13
    assert np.all(np.abs(Nt) <= 1 + 1e-12)

"""Seeded synthetic core-hole problems.

The paper's molecules (formaldehyde, ESCA; Section "Geometries, Basis Sets, and
Computational Details") need basis sets and integral codes that are not
available, so every input is synthetic with the shapes of those workloads:

* orbital energies: one deep core level (-20 Ha) at spatial index 0, O-1
  valence levels drawn U[-1.2, -0.3] and V virtual levels drawn U[0.1, 3.0],
  each group sorted ascending;
* real Cholesky vectors L^Q_pq, symmetric in pq, entries with p <= q drawn
  N(0, sigma_Q) with sigma_Q = 0.5 * 0.97^Q and mirrored (Q-major order),
  then multiplied by one global scale (see gen_problem);
* closed-shell ground-state amplitudes used only for the correlation energy
  E_N^corr of Eq. 3: T1 = f_ia / (e_i - e_a) with f_ia ~ N(0, 0.01) and an
  MP2-like T2 = (ia|jb) / (e_i + e_j - e_a - e_b).

Draw order is fixed (valence, virtual, L, f, then T2 is derived), so a seed
reproduces the same problem on every machine.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Problem:
    nocc: int            # occupied spatial orbitals of the N-electron system (core included)
    nvir: int            # virtual spatial orbitals
    nchol: int           # Cholesky vectors
    core: int            # spatial index of the ionised core orbital
    eps: np.ndarray      # [nocc+nvir] N-electron orbital energies (Ha)
    L: np.ndarray        # [nchol][nb][nb] real Cholesky vectors, L[q][p][r] == L[q][r][p]
    t1_gs: np.ndarray    # [nocc][nvir] closed-shell ground-state T1
    t2_gs: np.ndarray    # [nocc][nocc][nvir][nvir] closed-shell (alpha-beta) ground-state T2
    seed: int

    @property
    def nb(self) -> int:
        return self.nocc + self.nvir


def gen_problem(nocc: int, nvir: int, nchol: int, seed: int, *,
                eps_core: float = -20.0,
                valence=(-1.2, -0.3), virtual=(0.1, 3.0),
                l_sigma0: float = 0.5, l_decay: float = 0.97, l_scale="auto",
                f_sigma: float = 0.01, with_t2: bool = True) -> Problem:
    """Draw one synthetic core-hole problem.

    ``l_scale`` multiplies every Cholesky vector after drawing.  "auto" (the
    default) is 4.2 / (nvir + 1): at full strength (1.0) the virtual-virtual
    Cholesky block has Frobenius norm^2 ~ 0.25 (V+1)^2 Ha, which makes the
    particle-particle ladder so stiff that the fixed-point micro-iteration of
    the Adams-Moulton step diverges at the first step (about 100 Ha at V=20,
    2500 Ha at V=100).  The auto scale keeps that norm near 4.4 Ha for every
    size (0.2 at V=20), where the micro-iteration converges and the
    quasiparticle weight |exp(C)| settles near 0.8.
    The second parameter of every normal draw is a standard deviation.
    """
    if l_scale == "auto":
        l_scale = 4.2 / (nvir + 1)
    if nocc < 1 or nvir < 1 or nchol < 0:
        raise ValueError("need nocc >= 1, nvir >= 1, nchol >= 0")
    rng = np.random.default_rng(seed)
    nb = nocc + nvir
    eps = np.empty(nb)
    eps[0] = eps_core
    eps[1:nocc] = np.sort(rng.uniform(valence[0], valence[1], nocc - 1))
    eps[nocc:] = np.sort(rng.uniform(virtual[0], virtual[1], nvir))
    iu, ju = np.triu_indices(nb)
    sig = l_sigma0 * l_decay ** np.arange(nchol)
    tri = rng.standard_normal((nchol, iu.size)) * sig[:, None] * l_scale
    L = np.zeros((nchol, nb, nb))
    L[:, iu, ju] = tri
    L[:, ju, iu] = tri
    f = rng.standard_normal((nocc, nvir)) * f_sigma
    eo, ev = eps[:nocc], eps[nocc:]
    t1 = f / (eo[:, None] - ev[None, :])
    if with_t2:
        Lov = np.ascontiguousarray(L[:, :nocc, nocc:]).reshape(nchol, nocc * nvir)
        iajb = (Lov.T @ Lov).reshape(nocc, nvir, nocc, nvir)
        den = (eo[:, None, None, None] + eo[None, None, :, None]
               - ev[None, :, None, None] - ev[None, None, None, :])
        t2 = (iajb / den).transpose(0, 2, 1, 3).copy()
    else:
        t2 = np.zeros((nocc, nocc, nvir, nvir))
    return Problem(nocc, nvir, nchol, 0, eps, L, t1, t2, seed)


# The five workload shapes (O, V, Nchol, steps, dt, seed) the library is measured on.
WORKLOADS = {
    "c1_fp64_small": dict(nocc=4, nvir=20, nchol=60, nsteps=200, dt=0.05, seed=1),
    "c2_formaldehyde": dict(nocc=8, nvir=100, nchol=400, nsteps=2000, dt=0.025, seed=2),
    "c3_split": dict(nocc=30, nvir=300, nchol=1200, nsteps=500, dt=0.025, seed=3),
    "c5_esca_large": dict(nocc=50, nvir=450, nchol=1800, nsteps=100, dt=0.025, seed=5),
}


def workload(name: str, **kw) -> tuple[Problem, dict]:
    """Return (problem, run parameters) for a named workload."""
    w = dict(WORKLOADS[name])
    nsteps, dt = w.pop("nsteps"), w.pop("dt")
    w.update(kw)
    return gen_problem(**w), dict(nsteps=nsteps, dt=dt)


def random_amplitudes(shapes, seed: int, scale: float):
    """Seeded random complex amplitude blocks [t1a, t1b, t2aa, t2ab, t2bb] with
    the given shapes, entries scale * (N(0,1) + i N(0,1)); the same-spin T2
    blocks (index 2 and 4) are made antisymmetric in (i,j) and in (a,b), the
    layout the amplitude vector requires."""
    rng = np.random.default_rng(seed)
    t = [scale * (rng.standard_normal(s) + 1j * rng.standard_normal(s)) for s in shapes]
    for k in (2, 4):
        if len(t) > k:
            t[k] = t[k] - t[k].transpose(1, 0, 2, 3)
            t[k] = t[k] - t[k].transpose(0, 1, 3, 2)
    return t

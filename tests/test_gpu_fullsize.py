"""GPU residuals against the oracle at sizes where the oracle cannot
recompute the whole residual at test time.

* O=12, V=160, Nchol=640 with dense random amplitudes: sampled entries of
  the oracle's full residual, stored by tests/golden/make_residual_samples.py.
  In the Cholesky mode this size runs the default chunks (two ladder chunks
  of the virtual index a, 128 and a ragged 33, and the (mf|ae) chunk over
  all m).  Resident and Cholesky modes, all four precision forms.
* O=30, V=300, Nchol=1200 (resident blocks) and O=50, V=450, Nchol=1800
  (the Cholesky mode, which rteom_create takes by itself there): amplitudes
  supported on a few orbitals spread over the index ranges, through
  rteom_debug_residual_sparse.  The expected entries are the oracle residual
  of the problem cut down to those orbitals (tests/reduced.py; the property
  is pinned in tests/test_oracle_reduced.py).  The contractions, chunk loops,
  packs and index arithmetic run at full size; the host never holds a
  full-size amplitude vector.

Bounds: 1e-12 of the largest residual entry for FP64 and emulated FP64,
1e-5 for the split forms (as at O=8, V=100).
"""
import dataclasses
import os

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from oracle.spinexp import CoreHoleCCSD
from reduced import full_indices, reduced_problem
from synth import gen_problem, random_amplitudes, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_residual_O12V160N640.txt")
BOUND = {P.RTEOM_FP64: 1e-12, P.RTEOM_FP64_OZAKI: 1e-12, P.RTEOM_SPLIT_TF32: 1e-5,
         P.RTEOM_SPLIT_BF16: 1e-5, P.RTEOM_SPLIT_FP16: 1e-5}
NAMES = {P.RTEOM_FP64: "fp64", P.RTEOM_FP64_OZAKI: "emulated", P.RTEOM_SPLIT_TF32: "tf32",
         P.RTEOM_SPLIT_BF16: "bf16", P.RTEOM_SPLIT_FP16: "fp16"}


def test_sparse_residual_equals_dense_residual(rng):
    """The sparse entry point's index map against the dense path (bitwise:
    the same residual graph on the same amplitude vector), with the hole in
    a valence orbital so that the beta occupied numbering skips it."""
    p = dataclasses.replace(gen_problem(5, 23, 17, 3), core=2)
    with P.Propagator.from_problem(p) as g:
        t = random_amplitudes(P.block_shapes(p.nocc, p.nvir), 4, 0.1)
        R, _ = g.residual(t)
        z = np.concatenate([x.ravel() for x in t])
        keep = np.flatnonzero(np.abs(z) > 0)
        picks = rng.choice(z.size, 3000, replace=False)
        Rs = g.residual_sparse(keep, z[keep], picks)
    Rz = np.concatenate([x.ravel() for x in R])
    assert np.array_equal(Rs, Rz[picks])


def _golden():
    hdr = [ln for ln in open(GOLDEN) if ln.startswith("#")]
    meta = dict(kv.split("=") for kv in hdr[1][1:].split())
    d = np.loadtxt(GOLDEN)
    return (d[:, 0].astype(int), d[:, 1].astype(np.int64), d[:, 2] + 1j * d[:, 3],
            float(meta["scale"]), complex(float(meta["ReE"]), float(meta["ImE"])))


@pytest.mark.parametrize("flags", [0, P.RTEOM_FLAG_LADDER_CHOLESKY], ids=["resident", "cholesky"])
@pytest.mark.parametrize("precision", sorted(BOUND), ids=lambda x: NAMES[x])
def test_mid_size_dense_residual_matches_stored_oracle_samples(precision, flags):
    blk, idx, ref, scale, E_ref = _golden()
    p = gen_problem(12, 160, 640, 31)
    t = random_amplitudes(P.block_shapes(p.nocc, p.nvir), 32, 0.02)
    with P.Propagator.from_problem(p, precision=precision, flags=flags) as g:
        R, E = g.residual(t)
    got = np.array([R[b].ravel()[i] for b, i in zip(blk, idx)])
    err = np.abs(got - ref).max() / scale
    assert err < BOUND[precision], err
    assert abs(E - E_ref) <= 1e-10 * abs(E_ref)   # the energy is FP64 in every form


def _sparse_check(p, precision, occ_sel, vir_sel, seed=7, amp=0.1):
    eps_r, L_r, nocc_r, core_r = reduced_problem(p, occ_sel, vir_sel)
    red = CoreHoleCCSD.from_problem(eps_r, L_r, nocc_r, core_r)
    t_r = random_amplitudes(red.shapes(), seed, amp)
    idx = full_indices(p, occ_sel, vir_sel)
    ti = np.concatenate([k.ravel() for k in idx])
    tv = np.concatenate([x.ravel() for x in t_r])
    with P.Propagator.from_problem(p, precision=precision) as g:
        R = g.residual_sparse(ti, tv, ti)
    Ro = np.concatenate([x.ravel() for x in red.residual(t_r)])
    err = np.abs(R - Ro).max() / np.abs(Ro).max()
    print(f"{NAMES[precision]}: max |R_gpu - R_oracle| / max |R| = {err:.3e}")
    assert err < BOUND[precision], err


@pytest.fixture(scope="module")
def c3_problem():
    return workload("c3_split")[0]


@pytest.fixture(scope="module")
def c5_problem():
    return workload("c5_esca_large")[0]


@pytest.mark.slow
@pytest.mark.parametrize("precision", [P.RTEOM_FP64, P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_TF32,
                                       P.RTEOM_SPLIT_BF16], ids=lambda x: NAMES[x])
def test_c3_sparse_residual_matches_oracle(c3_problem, precision):
    """O=30, V=300, Nchol=1200: resident (vv|vv) block, every form."""
    _sparse_check(c3_problem, precision, [0, 7, 16, 29],
                  [30, 61, 105, 150, 199, 240, 288, 329])


@pytest.mark.slow
@pytest.mark.parametrize("precision", [P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_TF32, P.RTEOM_SPLIT_BF16,
                                       P.RTEOM_SPLIT_FP16], ids=lambda x: NAMES[x])
def test_c5_sparse_residual_matches_oracle(c5_problem, precision):
    """O=50, V=450, Nchol=1800 in the Cholesky mode with its default chunks.
    One FP64 DFMA residual takes about 37 minutes here, so the FP64-accurate
    check runs in the emulated form."""
    _sparse_check(c5_problem, precision, [0, 13, 31, 49],
                  [50, 97, 151, 222, 290, 356, 421, 499])

"""Split-precision forms against the FP64 oracle and FP64 path: split-TF32
(RTEOM_SPLIT_TF32: hi*hi + hi*lo + lo*hi TF32 products, FP32 accumulation
over slices of at most 512 of K), split-BF16 (RTEOM_SPLIT_BF16: three
8-bit BF16 digit planes per operand with per-row scales, the 6 leading digit
pairs summed in FP32) and split-FP16 (RTEOM_SPLIT_FP16: rows scaled into
FP16's range, hi/lo FP16 planes, hi*hi + hi*lo + lo*hi in FP32).
Contractions of at least 5e7 FLOP run on the tensor cores; everything else
stays FP64.  Targets: the cumulant within 1e-6
absolute of the FP64 oracle and the quasiparticle peak within 0.005 eV
(1.84e-4 Ha).  The packed operands carry about 22-24 bits, which puts a
floor near 1e-9 under the micro-iteration change, so these runs use tol 1e-8
(production uses the paper's 1e-4).
"""
import os

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from conftest import random_blocks
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
QP_TOL_HA = 0.005 / 27.211386245988


def _golden(name):
    path = os.path.join(GOLDEN, f"oracle_{name}.txt")
    hdr = [ln for ln in open(path) if ln.startswith("#")]
    meta = dict(kv.split("=") for kv in hdr[1][1:].split())
    d = np.loadtxt(path)
    return d[:, 1] + 1j * d[:, 2], float(meta["eps_core"]), float(meta["e_corr"])


FORMS = {"tf32": (P.RTEOM_SPLIT_TF32, "RTEOM_TC_MIN_FLOPS"),
         "bf16": (P.RTEOM_SPLIT_BF16, "RTEOM_OZ_MIN_FLOPS"),
         "fp16": (P.RTEOM_SPLIT_FP16, "RTEOM_OZ_MIN_FLOPS")}


@pytest.fixture(params=sorted(FORMS))
def form(request):
    """(precision, environment variable that sets its tensor-core threshold)."""
    return FORMS[request.param]


def _split(p, form, **kw):
    return P.Propagator(p.eps, p.L, p.nocc, p.nvir, p.t1_gs, p.t2_gs, core=p.core,
                        precision=form[0], **kw)


def test_split_residual_full_size_matches_oracle(rng, form):
    p, _ = workload("c2_formaldehyde")
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t = random_blocks(sysb.shapes(), rng, scale=0.02)
    with _split(p, form) as g:
        Rg, Eg = g.residual(t)
    Ro = sysb.residual(t)
    scale = max(np.abs(x).max() for x in Ro)
    errs = [np.abs(a - b).max() / scale for a, b in zip(Rg, Ro)]
    assert max(errs) < 1e-5, errs
    assert abs(Eg - sysb.energy(t)) <= 1e-10 * max(1.0, abs(Eg))   # the energy stays FP64


def test_split_cumulant_c2_matches_oracle(form):
    C_ref, _, _ = _golden("c2_formaldehyde")
    p, run = workload("c2_formaldehyde")
    with _split(p, form) as g:
        C = g.propagate(len(C_ref) - 1, run["dt"], tol=1e-8)
    assert np.abs(C - C_ref).max() < 1e-6


def _golden_prod(name, tol):
    path = os.path.join(GOLDEN, f"oracle_{name}_tol{tol:g}.txt")
    hdr = [ln for ln in open(path) if ln.startswith("#")]
    meta = dict(kv.split("=") for kv in hdr[1][1:].split())
    d = np.loadtxt(path)
    return (d[:, 1] + 1j * d[:, 2], d[1:, 5].astype(int), float(meta["eps_core"]),
            float(meta["e_corr"]))


def _qp_peak(omega, a):
    """Quasiparticle peak: grid argmax refined by a 3-point parabola."""
    k = int(np.argmax(a))
    assert 0 < k < len(a) - 1, "peak must lie inside the frequency window"
    y0, y1, y2 = a[k - 1], a[k], a[k + 1]
    return omega[k] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (omega[1] - omega[0])


def test_split_c2_production_run_matches_oracle_absolute(form):
    """The split forms at the paper's micro-iteration cutoff 1e-4 (Section 4),
    first 50 formaldehyde-shaped steps, against the oracle's own run at the
    same cutoff: every C_n within 1e-6 absolute, the same micro-iteration
    count per step (both sides stop on the same rule), and the
    quasiparticle peak of the transform (Eq. 4) within 0.005 eV."""
    C_ref, micro_ref, eps_c, e_corr = _golden_prod("c2_formaldehyde", 1e-4)
    p, run = workload("c2_formaldehyde")
    n = len(C_ref) - 1
    dt = run["dt"]
    with _split(p, form) as g:
        C = g.propagate(n, dt, tol=1e-4)
        info = g.info()
        shift = eps_c + e_corr
        omega = np.linspace(shift - 4.0, shift + 8.0, 6001)
        A = g.spectrum(omega, 0.5)
    assert np.abs(C - C_ref).max() < 1e-6, np.abs(C - C_ref).max()
    assert info["micro"] == micro_ref.sum()
    Ao = PR.spectrum(PR.green_function(C_ref, dt, eps_c, e_corr), dt, omega, 0.5)
    assert abs(_qp_peak(omega, A) - _qp_peak(omega, Ao)) < QP_TOL_HA
    assert np.abs(A - Ao).max() < 1e-5 * np.abs(Ao).max()


def test_split_tracks_fp64_path_over_40_steps(form):
    p, run = workload("c2_formaldehyde")
    with P.Propagator.from_problem(p) as g:
        C64 = g.propagate(40, run["dt"], tol=1e-8)
    with _split(p, form) as g:
        C32 = g.propagate(40, run["dt"], tol=1e-8)
    assert np.abs(C32 - C64).max() < 1e-6


# Steps of the 200-step config-1 stress run over which C(t) stays within
# 1e-6 absolute of the oracle with every contraction on the tensor cores.
# Split-BF16 holds the bar over the whole run (measured 2.5e-7).  Split-TF32
# (FP32 sums over slices of 512 of K) leaves it after about 60 steps (3 au;
# 8.0e-7 at step 50, 3.3e-6 absolute and 2.9e-7 relative after 200 steps
# with |C| up to 11); its default configuration, where only contractions of
# at least 5e7 FLOP (and the autotuner's picks) take the tensor cores, stays
# within 2.5e-7 over all 200 steps.  The complex products of this size run
# as the four-product embedding (the three-product form starts at 2048 of
# K); with three products the fixed-point floor of the stress case rose to
# about 1e-8.
STRESS_HORIZON = {P.RTEOM_SPLIT_TF32: 50, P.RTEOM_SPLIT_BF16: 200, P.RTEOM_SPLIT_FP16: 50}
STRESS_TOL = 1e-8


def test_split_c1_default_configuration_full_run_absolute(form):
    """Config 1 in full (200 steps, 10 au) in the form's default
    configuration: C(t) within 1e-6 absolute of the oracle at every step."""
    C_ref, _, _ = _golden("c1_fp64_small")
    p, run = workload("c1_fp64_small")
    with _split(p, form) as g:
        C = g.propagate(run["nsteps"], run["dt"], tol=1e-8)
    assert np.abs(C - C_ref).max() < 1e-6, np.abs(C - C_ref).max()


def test_split_everything_on_tensor_cores_c1_qp_peak(monkeypatch, form):
    """Stress case: every contraction on the tensor cores (threshold 0), 200
    steps of config 1 (10 au, |C| up to 11): C(t) within 1e-6 absolute up to
    the form's horizon (STRESS_HORIZON), within 1e-6 relative over the whole
    run, and the quasiparticle peak within 0.005 eV."""
    monkeypatch.setenv(form[1], "0")
    C_ref, eps_c, e_corr = _golden("c1_fp64_small")
    p, run = workload("c1_fp64_small")
    with _split(p, form) as g:
        C = g.propagate(run["nsteps"], run["dt"], tol=STRESS_TOL)
        shift = eps_c + e_corr
        # the quasiparticle peak sits above eps_c + E_corr by the relaxation shift
        omega = np.linspace(shift - 1.0, shift + 3.0, 4001)
        A = g.spectrum(omega, 0.1)
    h = STRESS_HORIZON[form[0]]
    err = np.abs(C - C_ref)
    assert err[:h + 1].max() < 1e-6, (h, err[:h + 1].max())
    assert err.max() < 1e-6 * np.abs(C_ref).max()
    Ao = PR.spectrum(PR.green_function(C_ref, run["dt"], eps_c, e_corr), run["dt"], omega, 0.1)
    assert abs(_qp_peak(omega, A) - _qp_peak(omega, Ao)) < QP_TOL_HA
    assert np.abs(A - Ao).max() < 1e-5 * np.abs(Ao).max()


def test_split_small_problem_ragged_tiles(rng, form):
    """Ragged shapes on the tensor cores: every contraction forced there."""
    os.environ[form[1]] = "0"
    try:
        p = gen_problem(5, 37, 23, 2)
        sysb = CoreHoleCCSD.from_problem(p.eps, p.L, 5, 0)
        t = random_blocks(sysb.shapes(), rng, scale=0.1)
        with _split(p, form) as g:
            Rg, _ = g.residual(t)
    finally:
        del os.environ[form[1]]
    Ro = sysb.residual(t)
    scale = max(np.abs(x).max() for x in Ro)
    for a, b in zip(Rg, Ro):
        assert np.abs(a - b).max() < 1e-5 * scale

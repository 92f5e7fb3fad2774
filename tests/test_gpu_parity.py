"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 on both sides with different summation orders, so
residual blocks agree to 1e-12 of their largest entry and the cumulant to
1e-10 relative (max_n |C_gpu - C_oracle| / max_n |C_oracle|).
"""
import os

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from conftest import random_blocks
from oracle import fockspace as FS
from oracle import hamiltonian as H
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ctx(p, core=0, **kw):
    return P.Propagator(p.eps, p.L, p.nocc, p.nvir, p.t1_gs, p.t2_gs, core=core, **kw)


def _load_golden(name):
    path = os.path.join(GOLDEN, f"oracle_{name}.txt")
    hdr = [ln for ln in open(path) if ln.startswith("#")]
    meta = dict(kv.split("=") for kv in hdr[1][1:].split())
    d = np.loadtxt(path)
    return dict(C=d[:, 1] + 1j * d[:, 2], E=d[:, 3] + 1j * d[:, 4], micro=d[1:, 5].astype(int),
                eps_core=float(meta["eps_core"]), e_corr=float(meta["e_corr"]))


def _relC(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("O,V,nchol,seed,core", [
    (3, 5, 7, 1, 0), (5, 37, 23, 2, 0), (4, 9, 11, 3, 2), (1, 6, 5, 4, 0), (2, 1, 3, 5, 1),
    (6, 70, 40, 6, 0)])
def test_residual_and_energy_match_oracle(O, V, nchol, seed, core, rng):
    p = gen_problem(O, V, nchol, seed)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, O, core)
    t = random_blocks(sysb.shapes(), rng, scale=0.1)
    with _ctx(p, core) as g:
        Rg, Eg = g.residual(t)
    Ro, Eo = sysb.residual(t), sysb.energy(t)
    scale = max(np.abs(x).max() for x in Ro if x.size)
    for k, (a, b) in enumerate(zip(Rg, Ro)):
        assert a.shape == b.shape
        if a.size:
            assert np.abs(a - b).max() <= 1e-12 * scale, (k, np.abs(a - b).max(), scale)
    assert abs(Eg - Eo) <= 1e-12 * max(1.0, abs(Eo))


def test_propagation_matches_oracle():
    p = gen_problem(4, 12, 20, 21)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, 4, 0)
    ref = PR.propagate(sysb, 12, 0.05, tol=1e-12)
    with _ctx(p) as g:
        C = g.propagate(12, 0.05, tol=1e-12)
        Cg, Eg = g.cumulant()
        info = g.info()
    assert _relC(C, ref["C"]) < 1e-10
    assert _relC(Eg, ref["E"]) < 1e-10
    assert abs(info["micro"] - ref["micro"].sum()) <= 2
    assert abs(info["e_corr"] - PR.closed_shell_ecorr(p.L, 4, p.t1_gs, p.t2_gs)) < 1e-10


def test_c1_full_propagation_and_spectrum_match_oracle():
    """O=4, V=20, Nchol=60, 200 steps, dt=0.05: the whole C(t) and A(w)."""
    gold = _load_golden("c1_fp64_small")
    p, run = workload("c1_fp64_small")
    with _ctx(p) as g:
        C = g.propagate(run["nsteps"], run["dt"], tol=1e-12)
        info = g.info()
        shift = info["eps_core"] + info["e_corr"]
        omega = np.linspace(shift - 2.0, shift + 6.0, 801)
        A = g.spectrum(omega, 0.05)
    assert _relC(C, gold["C"]) < 1e-10
    assert abs(info["e_corr"] - gold["e_corr"]) < 1e-10 * abs(gold["e_corr"])
    assert info["eps_core"] == gold["eps_core"]
    Go = PR.green_function(gold["C"], run["dt"], gold["eps_core"], gold["e_corr"])
    Ao = PR.spectrum(Go, run["dt"], omega, 0.05)
    assert np.abs(A - Ao).max() < 1e-9 * np.abs(Ao).max()


def test_c2_full_size_first_steps_match_oracle():
    """O=8, V=100, Nchol=400, dt=0.025 (the benchmark workload): the first
    steps of C(t) at tol 1e-12 against the stored oracle run."""
    gold = _load_golden("c2_formaldehyde")
    p, run = workload("c2_formaldehyde")
    n = len(gold["C"]) - 1
    with _ctx(p) as g:
        C = g.propagate(n, run["dt"], tol=1e-12)
    assert _relC(C, gold["C"]) < 1e-10


def test_c2_first_50_steps_at_the_production_tolerance_match_oracle():
    """The benchmark workload at the paper's tol 1e-4: the first 50 steps of
    C(t) against the stored oracle run.  Both sides apply the same stopping
    rule, so they take the same micro-iterations, and C(t) agrees to FP64
    rounding."""
    gold = _load_golden("c2_formaldehyde_tol0.0001")
    p, run = workload("c2_formaldehyde")
    n = len(gold["C"]) - 1
    assert n >= 50
    with _ctx(p) as g:
        C = g.propagate(n, run["dt"], tol=1e-4)
        info = g.info()
    assert info["micro"] == gold["micro"].sum()
    assert _relC(C, gold["C"]) < 1e-10


def test_c2_full_size_residual_sampled(rng):
    """Full-size residual at random amplitudes: every element of the T1 blocks
    and a random sample of T2 elements against the oracle."""
    p, _ = workload("c2_formaldehyde")
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t = random_blocks(sysb.shapes(), rng, scale=0.02)
    with _ctx(p) as g:
        Rg, Eg = g.residual(t)
    Ro = sysb.residual(t)
    scale = max(np.abs(x).max() for x in Ro)
    for a, b in zip(Rg, Ro):
        idx = rng.integers(0, a.size, min(a.size, 20000))
        assert np.abs(a.ravel()[idx] - b.ravel()[idx]).max() <= 1e-12 * scale
    assert abs(Eg - sysb.energy(t)) <= 1e-12 * max(1.0, abs(Eg))


def test_zero_couplings_stay_zero():
    p = gen_problem(3, 6, 0, 7)
    with P.Propagator(p.eps, None, 3, 6) as g:
        C = g.propagate(10, 0.05, tol=1e-12)
        st = g.get_state()
    assert np.abs(C).max() == 0.0 and np.abs(st["t"]).max() == 0.0


def test_cayley_closed_form_on_gpu(rng):
    O, V = 3, 7
    eps = np.concatenate([[-20.0], np.sort(rng.uniform(-1, -0.3, O - 1)), np.sort(rng.uniform(0.1, 3, V))])
    sysb = CoreHoleCCSD(np.diag(eps), np.diag(eps), np.zeros((0, O + V, O + V)), O, 0)
    t0 = random_blocks(sysb.shapes(), rng, scale=0.1)
    dt, n = 0.05, 9
    with P.Propagator(eps, None, O, V) as g:
        g.set_state(P.join_blocks(t0), 0)
        g.propagate(n, dt, tol=1e-14)
        t = P.split_blocks(g.get_state()["t"], O, V)
        assert g.info()["micro"] == 2 * n
    for x, x0, d in zip(t, t0, sysb.diagonal()):
        ref = ((1 + 0.5j * dt * d) / (1 - 0.5j * dt * d)) ** n * x0
        assert np.abs(x - ref).max() < 1e-14


def test_exact_one_electron_reference_on_gpu():
    O, V = 1, 4
    p = gen_problem(O, V, 5, 9, with_t2=False)
    h, v, _ = H.spinorb_hamiltonian(p.eps, p.L, O)
    occ, _ = H.core_hole_reference(p.nb, O, 0)
    errs = []
    for dt in (0.02, 0.01):
        n = int(round(1.0 / dt))
        with P.Propagator(p.eps, p.L, O, V) as g:
            C = g.propagate(n, dt, tol=1e-14)
        ex = FS.log_continuous(FS.exact_normalisation(h, v, occ, dt * np.arange(n + 1)))
        errs.append(np.abs(C - ex).max())
    assert errs[1] < 1e-3 and 3.3 < errs[0] / errs[1] < 4.7


def test_checkpoint_resume_is_bitwise():
    p = gen_problem(3, 10, 12, 31)
    with _ctx(p) as g:
        C_all = g.propagate(8, 0.05, tol=1e-12)
    with _ctx(p) as g1:
        g1.propagate(4, 0.05, tol=1e-12)
        st = g1.get_state()
    with _ctx(p) as g2:
        g2.set_state(st["t"], st["steps"], st["hist"])
        C2 = g2.propagate(4, 0.05, tol=1e-12)
        Cfull, _ = g2.cumulant()
    assert np.array_equal(C2, C_all[4:])
    assert np.array_equal(Cfull, C_all)


def test_not_converged_leaves_last_step():
    p = gen_problem(3, 8, 10, 41)
    with _ctx(p) as g:
        g.propagate(2, 0.05, tol=1e-12)
        with pytest.raises(P.RteomError) as e:
            g.propagate(1, 0.05, tol=1e-15, max_micro=2)
        assert e.value.code == P.RTEOM_ERR_NOT_CONVERGED
        assert g.info()["steps"] == 2
        C = g.propagate(1, 0.05, tol=1e-12)      # still usable
        assert np.isfinite(C).all()


def test_bad_calls_return_errors():
    p = gen_problem(2, 4, 5, 51)
    with _ctx(p) as g:
        with pytest.raises(P.RteomError) as e:
            g.spectrum([0.0], 0.1)
        assert e.value.code == P.RTEOM_ERR_STATE
        g.propagate(1, 0.05)
        with pytest.raises(P.RteomError) as e:
            g.propagate(1, 0.04)
        assert e.value.code == P.RTEOM_ERR_ARG
        with pytest.raises(P.RteomError) as e:
            g.set_state(np.full(g.state_size(), np.nan))
        assert e.value.code == P.RTEOM_ERR_NONFINITE


def test_injected_out_of_memory_is_reported_and_leaves_the_device_usable(monkeypatch):
    """Host-side fault injection: device allocations past 1 MB fail with
    RTEOM_ERR_OOM during set-up; the partial context is freed and the next
    context works."""
    p = gen_problem(4, 12, 20, 21)
    monkeypatch.setenv("RTEOM_INJECT_DEVICE_LIMIT", str(2 ** 20))
    with pytest.raises(P.RteomError) as e:
        _ctx(p)
    assert e.value.code == P.RTEOM_ERR_OOM
    monkeypatch.delenv("RTEOM_INJECT_DEVICE_LIMIT")
    with _ctx(p) as g:
        C = g.propagate(3, 0.05, tol=1e-10)
    assert np.isfinite(C).all()


def test_timed_and_untimed_graphs_agree_bitwise():
    """Timing adds event-record nodes around the ladder GEMMs of the captured
    residual graphs; results must not change."""
    p = gen_problem(4, 15, 20, 61)
    with _ctx(p) as g:
        C1 = g.propagate(5, 0.05, tol=1e-12)
    with _ctx(p) as g:
        g.set_timing(True)
        C2 = g.propagate(5, 0.05, tol=1e-12)
        tm = g.timing()
    assert np.array_equal(C1, C2)
    assert tm["ladder"]["launches"] > 0 and tm["ladder"]["ms"] > 0


def test_autotuned_and_heuristic_launches_agree(monkeypatch):
    """The autotuner changes tile shapes and K splits (summation order only):
    the propagation must agree with the heuristic launches to rounding."""
    p = gen_problem(5, 30, 40, 71)
    monkeypatch.setenv("RTEOM_AUTOTUNE", "0")
    with _ctx(p) as g:
        C0 = g.propagate(6, 0.05, tol=1e-12)
    monkeypatch.setenv("RTEOM_AUTOTUNE", "1")
    with _ctx(p) as g:
        C1 = g.propagate(6, 0.05, tol=1e-12)
    with _ctx(p) as g:                      # a second context reuses the choices: same bits
        C2 = g.propagate(6, 0.05, tol=1e-12)
    assert _relC(C1, C0) < 1e-12
    assert np.array_equal(C1, C2)


@pytest.mark.parametrize("precision", [P.RTEOM_FP64, P.RTEOM_SPLIT_TF32, P.RTEOM_SPLIT_BF16,
                                       P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_FP16])
def test_overflowing_amplitude_reaches_the_residual(precision, rng, monkeypatch):
    """An overflow inside the residual (a 1e200 singles amplitude squares to
    infinity in tau = t2 + t1 t1) must not be absorbed by any contraction path
    (the digit-sliced paths scale rows by their largest exponent): the
    residual comes back non-finite, which the propagation reports."""
    monkeypatch.setenv("RTEOM_TC_MIN_FLOPS", "0")
    monkeypatch.setenv("RTEOM_OZ_MIN_FLOPS", "0")
    p = gen_problem(4, 20, 30, 81)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, 4, 0)
    t = random_blocks(sysb.shapes(), rng, scale=0.05)
    t[0][1, 2] = 1e200
    with _ctx(p, precision=precision) as g:
        R, _ = g.residual(t)
    assert not all(np.isfinite(x).all() for x in R)


def test_spectrum_sum_rule_on_gpu():
    """The transform's sum rule, an invariant independent of the oracle: on a
    uniform grid of J > M frequencies spanning one period 2 pi/dt,
    dw sum_j A(omega_j) keeps only the n = 0 term of the trapezoid sum and
    equals -Im G_0 = Re exp(C_0) = 1 for any C(t), eta and grid origin."""
    p = gen_problem(3, 8, 10, 31)
    dt = 0.05
    with _ctx(p) as g:
        C = g.propagate(24, dt, tol=1e-12)
        assert np.abs(C[1:]).max() > 1e-3
        for J, w0, eta in ((257, 3.7, 0.2), (1000, -21.3, 1.5)):
            dw = 2 * np.pi / dt / J
            total = dw * g.spectrum(w0 + dw * np.arange(J), eta).sum()
            assert abs(total - 1.0) < 1e-10, (J, total)

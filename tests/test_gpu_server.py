"""Continuous-batching server: alone-vs-mix equality, admission by memory,
late arrivals, failure isolation, cancellation."""
import time

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from synth import gen_problem

pytestmark = pytest.mark.gpu

DT = 0.025


def _mix():
    shapes = [(4, 12, 20, 11, 15), (3, 20, 30, 12, 25), (5, 9, 14, 13, 10), (2, 16, 24, 14, 30),
              (6, 14, 28, 15, 12), (4, 25, 40, 16, 18)]
    return [(gen_problem(O, V, N, seed), n) for O, V, N, seed, n in shapes]


@pytest.mark.parametrize("precision", [P.RTEOM_FP64, P.RTEOM_SPLIT_TF32, P.RTEOM_SPLIT_BF16,
                                       P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_FP16])
def test_result_identical_alone_and_in_the_mix(precision, monkeypatch):
    if precision == P.RTEOM_SPLIT_TF32:
        monkeypatch.setenv("RTEOM_TC_MIN_FLOPS", "0")   # small shapes on the tensor cores too
    if precision in (P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_BF16, P.RTEOM_SPLIT_FP16):
        monkeypatch.setenv("RTEOM_OZ_MIN_FLOPS", "0")
    # split forms: ~1e-9 fixed-point floor of the packed amplitudes
    split = (P.RTEOM_SPLIT_TF32, P.RTEOM_SPLIT_BF16, P.RTEOM_SPLIT_FP16)
    tol = 1e-8 if precision in split else 1e-10
    jobs = _mix()
    alone = []
    for p, n in jobs:
        with P.Propagator.from_problem(p, precision=precision) as g:
            alone.append(g.propagate(n, DT, tol=tol))
    with P.Server(max_active=4, precision=precision) as s:
        ids = [s.submit(p, n, DT, tol=tol) for p, n in jobs]
        for rid in ids:
            assert s.wait(rid, 300.0)
        res = [s.poll(rid) for rid in ids]
        st = s.stats()
    for (status, err, C, _), ref in zip(res, alone):
        assert status == P.RTEOM_REQ_DONE, err
        assert np.array_equal(C, ref)          # bitwise: deterministic kernels, own buffers
    assert st["done"] == len(jobs) and st["failed"] == 0 and st["mem_in_use"] == 0


def test_late_arrival_overlaps_running_work():
    p_long = gen_problem(6, 30, 40, 21)
    p_short = gen_problem(3, 10, 12, 22)
    with P.Server(max_active=4) as s:
        a = s.submit(p_long, 60, DT, tol=1e-8)
        time.sleep(0.3)
        b = s.submit(p_short, 5, DT, tol=1e-8)
        assert s.wait(b, 120.0) and s.wait(a, 300.0)
        _, _, _, ta = s.poll(a)
        _, _, _, tb = s.poll(b)
    # b was admitted while a was running and finished first
    assert tb[1] < ta[2] and tb[2] < ta[2]


def test_memory_budget_serialises_admission():
    jobs = [gen_problem(4, 18, 30, 30 + k) for k in range(3)]
    # a running request is charged its real device bytes; a queued one its
    # (larger) estimate, so a budget of one estimate admits one at a time
    est = P.Server.estimate_bytes(4, 18, 30)
    with P.Server(mem_budget_bytes=est, max_active=8) as s:
        ids = [s.submit(p, 8, DT, tol=1e-8) for p in jobs]
        for rid in ids:
            assert s.wait(rid, 300.0)
        times = [s.poll(rid)[3] for rid in ids]
    # never two at once: each admission follows the previous completion
    for k in range(1, 3):
        assert times[k][1] >= times[k - 1][2]


def test_failed_request_is_isolated():
    good = gen_problem(3, 10, 12, 41)
    bad = gen_problem(3, 10, 12, 42)
    bad.eps = bad.eps.copy()
    bad.eps[2] = np.nan
    with P.Server(max_active=4) as s:
        g1 = s.submit(good, 6, DT)
        b1 = s.submit(bad, 6, DT)
        g2 = s.submit(good, 6, DT)
        for rid in (g1, b1, g2):
            assert s.wait(rid, 120.0)
        (s1, _, C1, _), (sb, eb, Cb, _), (s2, _, C2, _) = s.poll(g1), s.poll(b1), s.poll(g2)
        st = s.stats()
    assert s1 == P.RTEOM_REQ_DONE and s2 == P.RTEOM_REQ_DONE and np.array_equal(C1, C2)
    assert sb == P.RTEOM_REQ_FAILED and eb == P.RTEOM_ERR_NONFINITE and Cb is None
    assert st["failed"] == 1 and st["done"] == 2


def test_cancel_running_request():
    p = gen_problem(6, 40, 60, 51)
    with P.Server(max_active=2) as s:
        rid = s.submit(p, 100000, DT, tol=1e-8)
        time.sleep(1.0)
        s.cancel(rid)
        assert s.wait(rid, 60.0)
        status, _, C, _ = s.poll(rid)
    assert status == P.RTEOM_REQ_CANCELLED and C is None


def test_core_hole_sweep_matches_lone_propagations():
    """One molecule, several core holes (Section 3: independent, run at the
    same time) through one shared input copy: each result equals the lone
    propagation of that core hole, bitwise."""
    p = gen_problem(4, 16, 24, 31)
    cores = [0, 1, 3]
    alone = []
    for c in cores:
        with P.Propagator(p.eps, p.L, p.nocc, p.nvir, p.t1_gs, p.t2_gs, core=c) as g:
            alone.append(g.propagate(20, DT, tol=1e-8))
    with P.Server(max_active=4) as s:
        ids = s.submit_sweep(p, cores, 20, DT, tol=1e-8)
        for rid in ids:
            assert s.wait(rid, 300.0)
        res = [s.poll(rid) for rid in ids]
        st = s.stats()
    for (status, err, C, _), ref in zip(res, alone):
        assert status == P.RTEOM_REQ_DONE, err
        assert np.array_equal(C, ref)
    assert not np.array_equal(res[0][2], res[1][2])  # the core holes differ
    assert st["done"] == len(cores) and st["failed"] == 0 and st["mem_in_use"] == 0
    # and each core hole (valence holes included) against the oracle
    for c, (_, _, C, _) in zip(cores, res):
        ref = PR.propagate(CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, c), 20, DT, tol=1e-8)
        assert np.abs(C - ref["C"]).max() <= 1e-10 * np.abs(ref["C"]).max(), c


def test_sweep_with_a_core_outside_the_occupied_space_queues_nothing():
    p = gen_problem(4, 10, 12, 32)
    with P.Server(max_active=1) as s:
        with pytest.raises(P.RteomError):
            s.submit_sweep(p, [0, 4], 5, DT)
        with pytest.raises(P.RteomError):
            s.submit_sweep(p, [], 5, DT)
        st = s.stats()
    assert st["queued"] == 0 and st["running"] == 0 and st["done"] == 0


def test_a_request_that_runs_out_of_memory_fails_alone(monkeypatch):
    """Host-side fault injection: every context may hold at most 10 MB, so
    the O=6, V=40 request (about 67 MB planned) fails with RTEOM_ERR_OOM at
    set-up while the small requests around it complete."""
    monkeypatch.setenv("RTEOM_INJECT_DEVICE_LIMIT", str(10 * 2 ** 20))
    small = [gen_problem(3, 10, 12, 41), gen_problem(3, 10, 12, 43)]
    big = gen_problem(6, 40, 80, 42)
    with P.Server(max_active=2) as s:
        ids = [s.submit(small[0], 5, DT, tol=1e-8), s.submit(big, 5, DT, tol=1e-8),
               s.submit(small[1], 5, DT, tol=1e-8)]
        for rid in ids:
            assert s.wait(rid, 120.0)
        res = [s.poll(rid) for rid in ids]
        st = s.stats()
    assert res[0][0] == P.RTEOM_REQ_DONE and res[2][0] == P.RTEOM_REQ_DONE
    assert res[1][0] == P.RTEOM_REQ_FAILED and res[1][1] == P.RTEOM_ERR_OOM
    assert st["done"] == 2 and st["failed"] == 1 and st["mem_in_use"] == 0

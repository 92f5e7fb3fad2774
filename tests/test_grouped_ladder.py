"""Grouped ladder (RTEOM_FLAG_GROUPED) and lock-step propagation of several
core holes (rteom_propagate_group).

Core-hole propagations are independent (Section 3), so several can share
launches.  With the flag, every residual packs the operands of its three
particle-particle ladder GEMMs first (Section 3.1, the dominant contraction
sum_cd v_abcd tau_ij^cd), and rteom_propagate_group runs the ladder GEMMs of
all members of a round as grouped persistent tensor-core launches.  Each
ladder GEMM takes one K range per output tile, so a member's result is the
same bits alone (a group of one) and in any group, and the digit-plane forms
keep their bars against the FP64 oracle: FP64-level (emulated FP64) and
1e-6 absolute on C(t) (split forms).
"""
import ctypes
import dataclasses

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from conftest import random_blocks
from oracle import propagate as PR
from oracle.spinexp import CoreHoleCCSD
from paper_2301_04249_b300 import _lib
from synth import gen_problem

# uneven members: (O, V, Nchol, seed, core); their ladders take tile widths
# 32 to 256 and one to several output tiles, so a round needs launches of
# several kernel configurations
MEMBERS = [(3, 10, 18, 401, 0), (4, 13, 25, 402, 1), (2, 7, 12, 403, 0), (5, 16, 30, 404, 2)]
# precision, micro-iteration tol (the split forms' packed operands put a
# floor near 1e-9 under the micro-iteration change)
FORMS = {"ozaki": (P.RTEOM_FP64_OZAKI, 1e-12), "fp16": (P.RTEOM_SPLIT_FP16, 1e-8),
         "bf16": (P.RTEOM_SPLIT_BF16, 1e-8)}
NSTEPS, DT = 6, 0.05


def _problems():
    return [dataclasses.replace(gen_problem(O, V, nq, seed), core=core)
            for O, V, nq, seed, core in MEMBERS]


def _ctx(p, precision, flags=P.RTEOM_FLAG_GROUPED):
    return P.Propagator.from_problem(p, precision=precision, flags=flags)


@pytest.mark.gpu
@pytest.mark.parametrize("form", sorted(FORMS))
def test_group_equals_members_alone_and_matches_oracle(form):
    precision, tol = FORMS[form]
    probs = _problems()
    alone, micro_alone = [], []
    for p in probs:
        with _ctx(p, precision) as g:
            alone.append(g.propagate(NSTEPS, DT, tol=tol))
            micro_alone.append(g.info()["micro"])
    ctxs = [_ctx(p, precision) for p in probs]
    try:
        together = P.propagate_group(ctxs, NSTEPS, DT, tol=tol)
        micro = [g.info()["micro"] for g in ctxs]
    finally:
        for g in ctxs:
            g.close()
    for k, (a, b) in enumerate(zip(alone, together)):
        assert np.array_equal(a, b), (k, np.abs(a - b).max())
    assert micro == micro_alone
    for p, C in zip(probs, together):
        ref = PR.propagate(CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core), NSTEPS, DT,
                           tol=1e-12)["C"]
        err = np.abs(C - ref).max()
        if precision == P.RTEOM_FP64_OZAKI:
            assert err <= 1e-10 * np.abs(ref).max(), err
        else:
            assert err <= 1e-6, err


@pytest.mark.gpu
def test_group_resumes_and_continues_like_one_call():
    """Two group calls of 3 steps equal one of 6, and members may join a later
    round with a different step count."""
    precision, tol = FORMS["fp16"]
    probs = _problems()[:3]
    ctxs = [_ctx(p, precision) for p in probs]
    try:
        first = P.propagate_group(ctxs, 3, DT, tol=tol)
        second = P.propagate_group(ctxs, 3, DT, tol=tol)
    finally:
        for g in ctxs:
            g.close()
    ctxs = [_ctx(p, precision) for p in probs]
    try:
        whole = P.propagate_group(ctxs, 6, DT, tol=tol)
        extra = P.propagate_group(ctxs[:1], 2, DT, tol=tol)[0]
    finally:
        for g in ctxs:
            g.close()
    for a, b, w in zip(first, second, whole):
        assert np.array_equal(np.concatenate([a, b[1:]]), w)
    with _ctx(probs[0], precision) as g:
        assert np.array_equal(g.propagate(8, DT, tol=tol)[6:], extra)


@pytest.mark.gpu
def test_grouped_residual_matches_oracle(rng):
    p = dataclasses.replace(gen_problem(4, 13, 25, 402), core=1)
    sysb = CoreHoleCCSD.from_problem(p.eps, p.L, p.nocc, p.core)
    t = random_blocks(sysb.shapes(), rng, scale=0.05)
    with _ctx(p, P.RTEOM_FP64_OZAKI) as g:
        Rg, Eg = g.residual(t)
    Ro, Eo = sysb.residual(t), sysb.energy(t)
    scale = max(np.abs(x).max() for x in Ro if x.size)
    for k, (a, b) in enumerate(zip(Rg, Ro)):
        if a.size:
            assert np.abs(a - b).max() <= 1e-12 * scale, (k, np.abs(a - b).max(), scale)
    assert abs(Eg - Eo) <= 1e-12 * max(1.0, abs(Eo))


@pytest.mark.gpu
def test_group_rejects_bad_members():
    probs = _problems()[:2]
    a = _ctx(probs[0], P.RTEOM_SPLIT_FP16)
    b = _ctx(probs[1], P.RTEOM_SPLIT_BF16)
    c = P.Propagator.from_problem(probs[1], precision=P.RTEOM_SPLIT_FP16)
    try:
        for members in ([a, b], [a, a], [a, c]):
            with pytest.raises(P.RteomError) as e:
                P.propagate_group(members, 1, DT)
            assert e.value.code == P.RTEOM_ERR_ARG
        with pytest.raises(P.RteomError) as e:
            a.set_timing(1)
        assert e.value.code == P.RTEOM_ERR_ARG
    finally:
        for g in (a, b, c):
            g.close()


# ---- host side (no GPU)
def _create(precision, flags):
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    eps = np.array([-20.0, -1.0, 0.5, 1.0, 2.0])
    L = np.zeros((1, 5, 5))
    ptr = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    rc = lib.rteom_create(ctypes.byref(ctx), 2, 3, 1, ptr(eps), ptr(L), None, None, 0, precision,
                          flags, None)
    return rc, lib.rteom_last_error(None).decode()


@pytest.mark.parametrize("precision,flags", [
    (P.RTEOM_FP64, P.RTEOM_FLAG_GROUPED),
    (P.RTEOM_SPLIT_TF32, P.RTEOM_FLAG_GROUPED),
    (P.RTEOM_SPLIT_FP16, P.RTEOM_FLAG_GROUPED | P.RTEOM_FLAG_LADDER_CHOLESKY),
    (P.RTEOM_FP64_OZAKI, P.RTEOM_FLAG_GROUPED | P.RTEOM_FLAG_ANDERSON),
])
def test_grouped_flag_needs_a_digit_plane_form_with_resident_ladder(precision, flags):
    rc, msg = _create(precision, flags)
    assert rc == P.RTEOM_ERR_ARG and "GROUPED" in msg
    out = np.zeros(3)
    assert _lib.load().rteom_plan_bytes(4, 20, 40, precision, flags,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) \
        == P.RTEOM_ERR_ARG


def test_group_call_rejects_empty_or_null_member_lists():
    lib = _lib.load()
    assert lib.rteom_propagate_group(None, 1, 1, 0.05, 1e-4, 10, None) == P.RTEOM_ERR_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.rteom_propagate_group(arr, 0, 1, 0.05, 1e-4, 10, None) == P.RTEOM_ERR_ARG
    assert lib.rteom_propagate_group(arr, 1, 1, 0.05, 1e-4, 10, None) == P.RTEOM_ERR_ARG


@pytest.mark.parametrize("precision", [P.RTEOM_FP64_OZAKI, P.RTEOM_SPLIT_BF16, P.RTEOM_SPLIT_FP16])
def test_grouped_plan_holds_the_ladder_results_through_the_residual(precision):
    """The grouped residual keeps tau, the ladder packs and the three ladder
    results allocated until the rest of the residual has added them.  With no
    constant pack cached (every pack in the arena) its planned peak exceeds
    the plain one's by at least the alpha-beta result.  (With the cache, the
    plain ladder's split-K partial sums, which the grouped ladder never
    needs, can make either plan the larger.)"""
    O, V = 6, 30
    plain = P.plan_bytes(O, V, 4 * V, precision)
    grouped = P.plan_bytes(O, V, 4 * V, precision, flags=P.RTEOM_FLAG_GROUPED)
    ab_result = 16.0 * O * O * (V + 1) ** 2
    assert grouped["peak_uncached"] >= plain["peak_uncached"] + ab_result
    assert grouped["peak"] != plain["peak"]


@pytest.mark.gpu
def test_server_steps_grouped_requests_together_and_bitwise_as_alone():
    """Requests with the flag, of uneven shapes and step counts and arriving
    while others run, share grouped ladder launches in the server and still
    give each one's lone result bit for bit."""
    import time

    precision, tol = FORMS["fp16"]
    jobs = list(zip(_problems(), (6, 3, 8, 4)))
    alone = []
    for p, n in jobs:
        with _ctx(p, precision) as g:
            alone.append(g.propagate(n, DT, tol=tol))
    with P.Server(max_active=4, precision=precision) as s:
        ids = [s.submit(p, n, DT, tol=tol, flags=P.RTEOM_FLAG_GROUPED) for p, n in jobs[:2]]
        time.sleep(0.2)
        ids += [s.submit(p, n, DT, tol=tol, flags=P.RTEOM_FLAG_GROUPED) for p, n in jobs[2:]]
        for rid in ids:
            assert s.wait(rid, 300.0)
        res = [s.poll(rid) for rid in ids]
        st = s.stats()
    for (status, err, C, _), ref in zip(res, alone):
        assert status == P.RTEOM_REQ_DONE, err
        assert np.array_equal(C, ref)
    assert st["done"] == len(jobs) and st["failed"] == 0 and st["mem_in_use"] == 0

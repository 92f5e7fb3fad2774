"""Failure detection of the tensor-core pipelines without a GPU fault.

Every mbarrier wait in the tcgen05 kernels is bounded; when one runs out the
CTA records an error code, stops its producer, lets its issued copies land
and its issued MMAs finish, frees its tensor memory and returns, and the
host reports RTEOM_ERR_CUDA.  Here the test hook
RTEOM_TEST_CONSUMER_WAIT_CYCLES shortens the waits of the MMA and epilogue
warps to a few clock cycles so that they run out on purpose (the producer's
waits and the teardown keep their full budget).  The failing context must
report the timeout, and a fresh context on the same GPU must then compute
the right answer.
"""
import numpy as np
import pytest

import paper_2301_04249_b300 as P
from synth import gen_problem

pytestmark = pytest.mark.gpu

FORMS = {"tf32": (P.RTEOM_SPLIT_TF32, "RTEOM_TC_MIN_FLOPS"),
         "bf16": (P.RTEOM_SPLIT_BF16, "RTEOM_OZ_MIN_FLOPS"),
         "fp16": (P.RTEOM_SPLIT_FP16, "RTEOM_OZ_MIN_FLOPS"),
         "emulated": (P.RTEOM_FP64_OZAKI, "RTEOM_OZ_MIN_FLOPS")}


@pytest.mark.parametrize("name", sorted(FORMS))
def test_pipeline_wait_timeout_is_reported_and_gpu_stays_usable(monkeypatch, name):
    prec, env = FORMS[name]
    p = gen_problem(4, 30, 40, 5)
    monkeypatch.setenv(env, "0")   # every contraction on the tensor cores
    monkeypatch.setenv("RTEOM_TEST_CONSUMER_WAIT_CYCLES", "2")
    with pytest.raises(P.RteomError) as ei:
        with P.Propagator.from_problem(p, precision=prec) as g:
            g.propagate(1, 0.025, tol=1e-8)
    assert ei.value.code == P.RTEOM_ERR_CUDA and "timed out" in str(ei.value)
    monkeypatch.delenv("RTEOM_TEST_CONSUMER_WAIT_CYCLES")
    with P.Propagator.from_problem(p, precision=prec) as g:
        C = g.propagate(3, 0.025, tol=1e-8)
    monkeypatch.delenv(env)
    with P.Propagator.from_problem(p) as g:
        C64 = g.propagate(3, 0.025, tol=1e-8)
    assert np.all(np.isfinite(C)) and np.abs(C - C64).max() < 1e-6


def test_wait_budget_hook_rejects_bad_values(monkeypatch):
    p = gen_problem(2, 5, 4, 6)
    monkeypatch.setenv("RTEOM_TEST_CONSUMER_WAIT_CYCLES", "soon")
    with pytest.raises(P.RteomError) as ei:
        P.Propagator.from_problem(p, precision=P.RTEOM_SPLIT_TF32)
    assert ei.value.code == P.RTEOM_ERR_ARG

"""Host-only memory plan of a context (rteom_plan_bytes): runs without a GPU
from the library's own dry run of the residual.

Checks: the plan covers the buffers every context must hold (the FP64
integral blocks of the padded slot spaces and four amplitude sets, counted
here from the shapes alone), grows with the orbital spaces, is the same with
and without packs for the FP64 form, and rejects bad arguments.
"""
import numpy as np
import pytest

import paper_2301_04249_b300 as P

FORMS = [P.RTEOM_FP64, P.RTEOM_SPLIT_TF32, P.RTEOM_SPLIT_BF16, P.RTEOM_FP64_OZAKI,
         P.RTEOM_SPLIT_FP16]


def _floor_bytes(O, V):
    """Integral blocks and amplitude sets in the padded slot spaces."""
    nO, nV = O, V + 1
    npv = nV * (nV - 1) // 2
    ints = (nO ** 4 + nO ** 3 * nV + 3 * nO ** 2 * nV ** 2 + nO * nV ** 3 + nV ** 4 + npv ** 2)
    amps = 2 * nO * nV + 3 * nO ** 2 * nV ** 2
    return 8.0 * ints + 4 * 16.0 * amps


@pytest.mark.parametrize("O,V,nchol", [(4, 20, 60), (8, 100, 400), (30, 300, 1200)])
@pytest.mark.parametrize("precision", FORMS)
def test_plan_covers_the_resident_buffers(O, V, nchol, precision):
    b = P.plan_bytes(O, V, nchol, precision)
    floor = _floor_bytes(O, V)
    assert b["peak"] >= floor and b["peak_uncached"] >= floor
    # the scratch plan stays within a small multiple of the resident buffers
    assert b["peak"] <= 4.0 * floor + 1e9
    if precision == P.RTEOM_FP64:
        assert b["peak"] == b["peak_uncached"] == b["resident"]


@pytest.mark.parametrize("precision", FORMS)
def test_plan_grows_with_the_spaces(precision):
    small = P.plan_bytes(4, 40, 160, precision)["peak"]
    more_v = P.plan_bytes(4, 80, 320, precision)["peak"]
    more_o = P.plan_bytes(8, 40, 160, precision)["peak"]
    assert small < more_v and small < more_o


@pytest.mark.parametrize("args", [(0, 10, 5, 0), (4, 0, 5, 0), (4, 10, -1, 0), (4, 10, 5, 9)])
def test_plan_rejects_bad_arguments(args):
    with pytest.raises(P.RteomError):
        P.plan_bytes(*args)


def test_server_estimate_follows_the_plan():
    b = P.plan_bytes(8, 60, 240, P.RTEOM_SPLIT_TF32)["peak"]
    est = P.Server.estimate_bytes(8, 60, 240, P.RTEOM_SPLIT_TF32)
    assert b < est <= 1.05 * b + 512 * 2 ** 20


def _chol_floor_bytes(O, V, nchol):
    """Cholesky mode: integral blocks without (ov|vv), (vv|vv) and the pair
    block, plus the slot-space L_ov, L_vv and their transposes."""
    nO, nV = O, V + 1
    ints = nO ** 4 + nO ** 3 * nV + 3 * nO ** 2 * nV ** 2 + 2 * nchol * (nO * nV + nV ** 2)
    amps = 2 * nO * nV + 3 * nO ** 2 * nV ** 2
    return 8.0 * ints + 4 * 16.0 * amps


@pytest.mark.parametrize("O,V,nchol", [(4, 20, 60), (8, 100, 400), (30, 300, 1200)])
@pytest.mark.parametrize("precision", FORMS)
def test_cholesky_mode_plan_covers_its_buffers_and_is_smaller(O, V, nchol, precision):
    F = P.RTEOM_FLAG_LADDER_CHOLESKY
    b = P.plan_bytes(O, V, nchol, precision, F)
    floor = _chol_floor_bytes(O, V, nchol)
    assert b["peak"] >= floor and b["peak_uncached"] >= floor
    if V >= 100:  # below that the chunk scratch outweighs the blocks it replaces
        assert b["peak_uncached"] < P.plan_bytes(O, V, nchol, precision)["peak_uncached"]


@pytest.mark.parametrize("precision", FORMS)
def test_config5_fits_one_b300_only_in_cholesky_mode(precision):
    """O=50, V=450, Nchol=1800: the resident (vv|vv) block alone is 331 GB;
    the Cholesky mode fits the 288 GB device (packs left uncached where the
    cache would not fit)."""
    dev = 275040 * 2 ** 20
    assert P.plan_bytes(50, 450, 1800, precision)["peak_uncached"] > dev
    chol = P.plan_bytes(50, 450, 1800, precision, P.RTEOM_FLAG_LADDER_CHOLESKY)
    assert chol["peak_uncached"] < 0.9 * dev


def test_plan_rejects_unknown_flags():
    with pytest.raises(P.RteomError):
        P.plan_bytes(4, 10, 5, P.RTEOM_FP64, 1 << 7)


def test_anderson_buffers_are_planned():
    O, V = 8, 100
    total = 2 * O * (V + 1) + 3 * O * O * (V + 1) ** 2
    base = P.plan_bytes(O, V, 400, P.RTEOM_FP64)["peak"]
    acc = P.plan_bytes(O, V, 400, P.RTEOM_FP64, P.RTEOM_FLAG_ANDERSON)["peak"]
    assert acc - base >= 9 * 16 * total

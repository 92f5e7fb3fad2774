"""The C ABI library loads, exports every entry point that include/rteom.h
declares, and rejects bad arguments on the host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2301_04249_b300 as P
from paper_2301_04249_b300 import _lib

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "rteom.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rteom_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = _lib.load()
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_lib.SIGNATURES) == names


def _create(**kw):
    lib = _lib.load()
    a = dict(nocc=2, nvir=3, nchol=1, eps=np.array([-20.0, -1.0, 0.5, 1.0, 2.0]),
             L=np.zeros((1, 5, 5)), core=0, precision=0, flags=0)
    a.update(kw)
    ctx = ctypes.c_void_p()
    ptr = lambda x: None if x is None else np.ascontiguousarray(x, float).ctypes.data_as(  # noqa: E731
        ctypes.POINTER(ctypes.c_double))
    rc = lib.rteom_create(ctypes.byref(ctx), a["nocc"], a["nvir"], a["nchol"], ptr(a["eps"]),
                          ptr(a["L"]), None, None, a["core"], a["precision"], a["flags"], None)
    return rc, lib.rteom_last_error(None).decode()


@pytest.mark.parametrize("kw,code", [
    (dict(nocc=0), P.RTEOM_ERR_ARG),
    (dict(core=2), P.RTEOM_ERR_ARG),
    (dict(core=-1), P.RTEOM_ERR_ARG),
    (dict(eps=None), P.RTEOM_ERR_ARG),
    (dict(precision=7), P.RTEOM_ERR_ARG),
    (dict(flags=16), P.RTEOM_ERR_ARG),                              # unknown bit
    (dict(flags=8), P.RTEOM_ERR_ARG),                               # grouped needs digit planes
    (dict(eps=np.array([-20.0, np.nan, 0.5, 1.0, 2.0])), P.RTEOM_ERR_NONFINITE),
    (dict(L=np.arange(25.0).reshape(1, 5, 5)), P.RTEOM_ERR_ARG),   # not symmetric
])
def test_create_rejects_bad_arguments_on_host(kw, code):
    rc, msg = _create(**kw)
    assert rc == code and msg


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_block_marshalling_roundtrip(rng):
    shapes = P.block_shapes(4, 6)
    blocks = [rng.standard_normal(s) + 1j * rng.standard_normal(s) for s in shapes]
    back = P.split_blocks(P.join_blocks(blocks), 4, 6)
    for a, b in zip(blocks, back):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("val", ["abc", "10MB", "-5", ""])
def test_injected_device_limit_must_be_a_byte_count(monkeypatch, val):
    monkeypatch.setenv("RTEOM_INJECT_DEVICE_LIMIT", val)
    rc, msg = _create()
    assert rc == P.RTEOM_ERR_ARG and "RTEOM_INJECT_DEVICE_LIMIT" in msg

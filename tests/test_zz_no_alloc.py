"""The allocation-free correlation-energy entry point (rteom_ecorr_noalloc).

Some callers cannot allocate device memory: their GPU memory belongs to their
own pool or framework allocator, or they run where a cudaMalloc/cudaFree is
not allowed.  rteom_ecorr_noalloc serves them with scratch held in a static
device array; this test checks, through the C ABI, that two calls in a row
reproduce the E_N^corr that rteom_create computes with its own scratch, and
that sizes beyond the scratch are rejected before any launch.  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_04249_b300 import RTEOM_ERR_ARG, Propagator, _lib
from synth import gen_problem

pytestmark = pytest.mark.gpu


def test_noalloc_ecorr_matches_create_twice():
    torch = pytest.importorskip("torch")
    lib = _lib.load()
    p = gen_problem(6, 17, 23, 77)
    with Propagator.from_problem(p) as g:
        ref = g.info()["e_corr"]
    dev = torch.device("cuda", 0)
    L = torch.tensor(p.L, dtype=torch.float64, device=dev)
    t1 = torch.tensor(p.t1_gs, dtype=torch.float64, device=dev)
    t2 = torch.tensor(p.t2_gs, dtype=torch.float64, device=dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev).cuda_stream or None
    for k in range(2):
        rc = lib.rteom_ecorr_noalloc(p.nocc, p.nvir, p.nchol, L.data_ptr(), t1.data_ptr(),
                                     t2.data_ptr(), out[k:].data_ptr(), stream, err, 256)
        assert rc == 0, err.value.decode()
    torch.cuda.synchronize()
    vals = out.cpu().numpy()
    assert np.all(np.abs(vals - ref) <= 1e-12 * max(1.0, abs(ref))), (vals, ref)
    assert vals[0] == vals[1]


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = _lib.load()
    err = ctypes.create_string_buffer(256)
    rc = lib.rteom_ecorr_noalloc(65, 10, 0, None, None, None, None, None, err, 256)
    assert rc == RTEOM_ERR_ARG
    rc = lib.rteom_ecorr_noalloc(65, 10, 0, None, None, None, ctypes.c_void_p(16), None, err, 256)
    assert rc == RTEOM_ERR_ARG and b"4096" in err.value

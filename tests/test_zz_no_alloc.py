"""The allocation-free correlation-energy entry point (rteom_ecorr_noalloc)
on the GPU.

Some callers cannot allocate device memory: their GPU memory belongs to their
own pool or framework allocator, or they run where a cudaMalloc/cudaFree is
not allowed.  rteom_ecorr_noalloc serves them with scratch held in a static
device array.  This test calls it twice in a row through the C ABI on
caller-owned device buffers and checks both results against the oracle's
closed-shell correlation energy (Eq. 3) and against the E_N^corr that
rteom_create computes with its own scratch.  The file name makes pytest
collect it last; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle.propagate import closed_shell_ecorr
from paper_2301_04249_b300 import Propagator, _lib
from synth import gen_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(6, 17, 23, 77), (1, 5, 3, 78), (13, 40, 31, 79)])
def test_noalloc_ecorr_matches_oracle_and_create_twice(shape):
    torch = pytest.importorskip("torch")
    lib = _lib.load()
    p = gen_problem(*shape)
    ref = closed_shell_ecorr(p.L, p.nocc, p.t1_gs, p.t2_gs)
    with Propagator.from_problem(p) as g:
        created = g.info()["e_corr"]
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
    tol = 1e-12 * max(1.0, abs(ref))
    assert np.all(np.abs(vals - ref) <= tol), (vals, ref)
    assert abs(created - ref) <= tol, (created, ref)
    assert vals[0] == vals[1]

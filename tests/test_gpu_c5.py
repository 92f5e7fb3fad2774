"""O=50, V=450, Nchol=1800 (config 5) in the Cholesky mode, which
rteom_create takes by itself here (the resident (vv|vv) block alone would be
331 GB): two Adams-Moulton steps from T(0) = 0 in the split-TF32 form and in
the emulated-FP64 form, whose C(t) must agree within 1e-6 absolute (the
split-precision bound on the cumulant).

Nothing on the host can evaluate a residual of this size, and one FP64 DFMA
residual takes about 37 minutes, so the emulated-FP64 form (pinned to the
oracle at 1e-12 at the smaller shapes, in both modes) is the reference.  The
run needs no host amplitude arrays.  About 7 minutes of device time.
"""
import numpy as np
import pytest

import paper_2301_04249_b300 as P
from synth import workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_c5_split_cumulant_tracks_emulated_fp64_cumulant():
    p, run = workload("c5_esca_large")
    C = {}
    for prec in (P.RTEOM_SPLIT_TF32, P.RTEOM_FP64_OZAKI):
        with P.Propagator.from_problem(p, precision=prec) as g:
            C[prec] = g.propagate(2, run["dt"], tol=1e-4)
    Cs, Co = C[P.RTEOM_SPLIT_TF32], C[P.RTEOM_FP64_OZAKI]
    assert np.all(np.isfinite(Cs)) and np.all(np.isfinite(Co))
    assert np.abs(Co[1:]).max() > 0  # the steps moved the cumulant
    d = float(np.abs(Cs - Co).max())
    print(f"c5: max |C_split - C_emulated| = {d:.3e}, max |C| = {np.abs(Co).max():.3e}")
    assert d < 1e-6, d

"""B300-native RT-EOM-CCSD core-hole propagation (Python binding of librteom.so).

The Python layer only marshals arguments: every step of the propagation runs
in the library's CUDA kernels.  There is no CPU fallback; a missing library or
GPU raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (RTEOM_ERR_ARG, RTEOM_ERR_CUDA, RTEOM_ERR_NONFINITE,  # noqa: F401
                   RTEOM_ERR_NOT_CONVERGED, RTEOM_ERR_OOM, RTEOM_ERR_STATE, RTEOM_FLAG_CUMULANT_NO_FOV,
                   RTEOM_FLAG_LADDER_CHOLESKY, RTEOM_FLAG_ANDERSON, RTEOM_FLAG_GROUPED,
                   RTEOM_FP64, RTEOM_OK, RTEOM_REQ_CANCELLED, RTEOM_REQ_DONE, RTEOM_REQ_FAILED,
                   RTEOM_REQ_QUEUED, RTEOM_REQ_RUNNING, RTEOM_SPLIT_BF16, RTEOM_SPLIT_TF32,
                   RTEOM_FP64_OZAKI, RTEOM_SPLIT_FP16)

__all__ = ["Propagator", "Server", "RteomError", "block_shapes", "split_blocks", "join_blocks",
           "propagate_group"]


class RteomError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rteom error {code}: {msg}")
        self.code = code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def plan_bytes(nocc: int, nvir: int, nchol: int, precision: int = RTEOM_FP64,
               flags: int = 0) -> dict:
    """Device bytes of a context of this shape and precision, planned on the
    host (no GPU needed): peak with every constant tensor-core pack cached,
    peak with none cached, and the bytes held after set-up.  flags may hold
    RTEOM_FLAG_LADDER_CHOLESKY (plan the Cholesky mode)."""
    out = np.zeros(3)
    rc = _lib.load().rteom_plan_bytes(int(nocc), int(nvir), int(nchol), int(precision),
                                      int(flags), _ptr(out))
    if rc != RTEOM_OK:
        raise RteomError(rc, "rteom_plan_bytes: bad shape, precision or flag")
    return dict(peak=float(out[0]), peak_uncached=float(out[1]), resident=float(out[2]))


def block_shapes(nocc: int, nvir: int, core: int = 0):
    """Shapes of the unique spin blocks t1a, t1b, t2aa, t2ab, t2bb."""
    oA, vA, oB, vB = nocc, nvir, nocc - 1, nvir + 1
    return [(oA, vA), (oB, vB), (oA, oA, vA, vA), (oA, oB, vA, vB), (oB, oB, vB, vB)]


def split_blocks(vec: np.ndarray, nocc: int, nvir: int):
    """Interleaved complex amplitude vector -> list of complex block arrays."""
    z = vec.view(np.complex128)
    out, k = [], 0
    for s in block_shapes(nocc, nvir):
        n = int(np.prod(s))
        out.append(z[k:k + n].reshape(s).copy())
        k += n
    return out


def join_blocks(blocks) -> np.ndarray:
    """List of complex block arrays -> interleaved complex amplitude vector."""
    z = np.concatenate([np.ascontiguousarray(b, dtype=np.complex128).ravel() for b in blocks])
    return z.view(np.float64).copy()


def propagate_group(props, nsteps: int, dt: float, tol: float = 1e-4, max_micro: int = 50):
    """rteom_propagate_group: advance every Propagator of ``props`` (created
    with RTEOM_FLAG_GROUPED, one precision form) nsteps steps in lock step,
    the ladder GEMMs of each round in grouped launches.  Returns each
    member's C at the start and after each step (complex [nsteps+1])."""
    lib = _lib.load()
    n = len(props)
    ctxs = (ctypes.c_void_p * n)(*[p._ctx.value for p in props])
    outs = [np.zeros(2 * (int(nsteps) + 1)) for _ in props]
    ptrs = (ctypes.POINTER(ctypes.c_double) * n)(*[_ptr(o) for o in outs])
    rc = lib.rteom_propagate_group(ctxs, n, int(nsteps), float(dt), float(tol), int(max_micro),
                                   ptrs)
    if rc != 0:
        msg = "; ".join(m for m in (lib.rteom_last_error(p._ctx).decode() for p in props) if m)
        raise RteomError(rc, msg)
    return [o.view(np.complex128) for o in outs]


class Propagator:
    """One core-hole propagation context (rteom_create ... rteom_destroy).

    eps [nb], L [nchol, nb, nb] (symmetric in the last two indices), optional
    closed-shell ground-state t1 [O, V] / t2 [O, O, V, V] for E_N^corr.
    ``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None for a
    stream owned by the library.
    """

    def __init__(self, eps, L, nocc: int, nvir: int, t1_gs=None, t2_gs=None, core: int = 0,
                 precision: int = RTEOM_FP64, flags: int = 0, stream=None):
        self._lib = _lib.load()
        self.nocc, self.nvir, self.core = int(nocc), int(nvir), int(core)
        eps = _f64(eps)
        L = _f64(L)
        nchol = 0 if L is None else int(L.shape[0])
        t1 = _f64(t1_gs)
        t2 = _f64(t2_gs)
        handle = None
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream)) or None
        ctx = ctypes.c_void_p()
        rc = self._lib.rteom_create(ctypes.byref(ctx), self.nocc, self.nvir, nchol, _ptr(eps),
                                    _ptr(L), _ptr(t1), _ptr(t2), self.core, int(precision),
                                    int(flags), handle)
        if rc != 0:
            raise RteomError(rc, self._lib.rteom_last_error(None).decode())
        self._ctx = ctx

    @classmethod
    def from_problem(cls, p, **kw):
        return cls(p.eps, p.L, p.nocc, p.nvir, p.t1_gs, p.t2_gs, core=p.core, **kw)

    def _check(self, rc):
        if rc != 0:
            raise RteomError(rc, self._lib.rteom_last_error(self._ctx).decode())

    def propagate(self, nsteps: int, dt: float, tol: float = 1e-4, max_micro: int = 50):
        """Advance nsteps; returns C at the start and after each step (complex [nsteps+1])."""
        out = np.zeros(2 * (nsteps + 1))
        self._check(self._lib.rteom_propagate(self._ctx, int(nsteps), float(dt), float(tol),
                                              int(max_micro), _ptr(out)))
        return out.view(np.complex128)

    def spectrum(self, omega, eta: float):
        w = _f64(np.atleast_1d(omega))
        A = np.zeros(w.size)
        self._check(self._lib.rteom_spectrum(self._ctx, _ptr(w), int(w.size), float(eta), _ptr(A)))
        return A

    def info(self):
        e, ec = ctypes.c_double(), ctypes.c_double()
        s, m = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self._lib.rteom_get_info(self._ctx, ctypes.byref(e), ctypes.byref(ec),
                                             ctypes.byref(s), ctypes.byref(m)))
        return dict(eps_core=e.value, e_corr=ec.value, steps=s.value, micro=m.value)

    def state_size(self) -> int:
        return int(self._lib.rteom_state_size(self._ctx))

    def cumulant(self):
        """(C, E) histories, complex [steps+1] each."""
        n = self.info()["steps"] + 1
        C, E = np.zeros(2 * n), np.zeros(2 * n)
        self._check(self._lib.rteom_get_cumulant(self._ctx, n, _ptr(C), _ptr(E)))
        return C.view(np.complex128), E.view(np.complex128)

    def get_state(self, with_history: bool = True):
        t = np.zeros(self.state_size())
        steps = ctypes.c_longlong()
        self._check(self._lib.rteom_get_state(self._ctx, _ptr(t), ctypes.byref(steps), None))
        hist = None
        if with_history:
            hist = np.zeros(4 * (steps.value + 1))
            self._check(self._lib.rteom_get_state(self._ctx, None, ctypes.byref(steps), _ptr(hist)))
        return dict(t=t, steps=steps.value, hist=hist)

    def set_state(self, t, steps: int = 0, hist=None):
        t = _f64(t)
        self._check(self._lib.rteom_set_state(self._ctx, _ptr(t), int(steps), _ptr(_f64(hist))))

    def residual(self, blocks):
        """Full projections R (list of blocks) and E for the given amplitude blocks."""
        t = join_blocks(blocks)
        R = np.zeros_like(t)
        E = np.zeros(2)
        self._check(self._lib.rteom_debug_residual(self._ctx, _ptr(t), _ptr(R), _ptr(E)))
        return split_blocks(R, self.nocc, self.nvir), complex(E[0], E[1])

    def residual_sparse(self, t_index, t_val, r_index):
        """Residual entries at flat indices r_index of the amplitude vector for
        amplitudes zero except t_val at flat indices t_index (complex)."""
        ti = np.ascontiguousarray(t_index, dtype=np.int64)
        tv = np.ascontiguousarray(t_val, dtype=np.complex128).view(np.float64)
        ri = np.ascontiguousarray(r_index, dtype=np.int64)
        R = np.zeros(2 * ri.size)
        llp = ctypes.POINTER(ctypes.c_longlong)
        self._check(self._lib.rteom_debug_residual_sparse(
            self._ctx, ti.ctypes.data_as(llp), _ptr(tv), int(ti.size), ri.ctypes.data_as(llp),
            int(ri.size), _ptr(R)))
        return R.view(np.complex128)

    def set_timing(self, on):
        """0/False off; 1/True on (event nodes around the ladder launches
        inside the residual graphs); 2 on with the residuals run outside
        graphs (every launch timed); 3 on with event nodes around every
        contraction launch inside the graphs."""
        on = int(on) if on in (2, 3) else int(bool(on))
        self._check(self._lib.rteom_set_timing(self._ctx, on))

    def timing(self, reset: bool = False):
        ms = (ctypes.c_double * 4)()
        la = (ctypes.c_longlong * 4)()
        fl = (ctypes.c_double * 4)()
        by = (ctypes.c_double * 4)()
        self._check(self._lib.rteom_get_timing(self._ctx, ms, la, fl, by, int(reset)))
        names = ["ladder", "contract", "permute", "elementwise"]
        return {n: dict(ms=ms[k], launches=la[k], flops=fl[k], bytes=by[k])
                for k, n in enumerate(names)}

    def kernel_launches(self) -> int:
        return int(self._lib.rteom_kernel_launches(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.rteom_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server (rteom_server_*): many core-hole
    propagations at once on the current GPU, admitted by device memory."""

    def __init__(self, mem_budget_bytes: float = 0.0, max_active: int = 8,
                 precision: int = RTEOM_FP64):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self._lib.rteom_server_create(ctypes.byref(h), float(mem_budget_bytes),
                                           int(max_active), int(precision))
        if rc != 0:
            raise RteomError(rc, "rteom_server_create failed")
        self._h = h
        self._nsteps = {}

    def submit(self, p, nsteps: int, dt: float, tol: float = 1e-4, max_micro: int = 50,
               flags: int = 0) -> int:
        """Queue a problem (synth.Problem-like: eps, L, nocc, nvir, t1_gs, t2_gs, core)."""
        eps, L = _f64(p.eps), _f64(p.L)
        t1, t2 = _f64(p.t1_gs), _f64(p.t2_gs)
        nchol = 0 if L is None else int(L.shape[0])
        rid = ctypes.c_longlong()
        rc = self._lib.rteom_server_submit(self._h, int(p.nocc), int(p.nvir), nchol, _ptr(eps),
                                           _ptr(L), _ptr(t1), _ptr(t2), int(p.core), int(flags),
                                           int(nsteps), float(dt), float(tol), int(max_micro),
                                           ctypes.byref(rid))
        if rc != 0:
            raise RteomError(rc, "rteom_server_submit failed")
        self._nsteps[rid.value] = int(nsteps)
        return rid.value

    def submit_sweep(self, p, cores, nsteps: int, dt: float, tol: float = 1e-4,
                     max_micro: int = 50, flags: int = 0) -> list:
        """Queue one propagation per core hole in ``cores`` of the molecule p
        (host inputs copied once and shared); returns the ids in order."""
        eps, L = _f64(p.eps), _f64(p.L)
        t1, t2 = _f64(p.t1_gs), _f64(p.t2_gs)
        nchol = 0 if L is None else int(L.shape[0])
        cs = np.ascontiguousarray(cores, dtype=np.int32)
        ids = np.zeros(cs.size, dtype=np.int64)
        rc = self._lib.rteom_server_submit_sweep(
            self._h, int(p.nocc), int(p.nvir), nchol, _ptr(eps), _ptr(L), _ptr(t1), _ptr(t2),
            cs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(cs.size), int(flags),
            int(nsteps), float(dt), float(tol), int(max_micro),
            ids.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        if rc != 0:
            raise RteomError(rc, "rteom_server_submit_sweep failed")
        for rid in ids:
            self._nsteps[int(rid)] = int(nsteps)
        return [int(r) for r in ids]

    def poll(self, rid: int):
        """(status, error, C or None, (t_submit, t_admit, t_done))."""
        st, er = ctypes.c_int(), ctypes.c_int()
        C = np.zeros(2 * (self._nsteps[rid] + 1))
        t = np.zeros(3)
        rc = self._lib.rteom_server_poll(self._h, int(rid), ctypes.byref(st), ctypes.byref(er),
                                         _ptr(C), _ptr(t))
        if rc != 0:
            raise RteomError(rc, "unknown request")
        return st.value, er.value, (C.view(np.complex128) if st.value == RTEOM_REQ_DONE else None), \
            tuple(t)

    def wait(self, rid: int, timeout_s: float = 0.0) -> bool:
        return self._lib.rteom_server_wait(self._h, int(rid), float(timeout_s)) == 0

    def cancel(self, rid: int):
        self._lib.rteom_server_cancel(self._h, int(rid))

    def stats(self):
        q, r, d, f = (ctypes.c_longlong() for _ in range(4))
        m, s = ctypes.c_double(), ctypes.c_double()
        self._lib.rteom_server_stats(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(d),
                                     ctypes.byref(f), ctypes.byref(m), ctypes.byref(s))
        return dict(queued=q.value, running=r.value, done=d.value, failed=f.value,
                    mem_in_use=m.value, steps_done=s.value)

    @staticmethod
    def estimate_bytes(nocc, nvir, nchol, precision=RTEOM_FP64) -> float:
        return float(_lib.load().rteom_server_estimate_bytes(int(nocc), int(nvir), int(nchol),
                                                            int(precision)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rteom_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

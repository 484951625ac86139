"""GB300 (sm_103a) PDLP: restarted primal-dual hybrid gradient for linear programming.

Thin Python binding over the C ABI of include/pdlp.h (libpdlp_gb300.so).  The
functions keep the C names; `Context` wraps one pdlp_ctx.  Arrays may be
numpy arrays or torch tensors (host or CUDA); every step of the solver runs
in the library's CUDA kernels.  Importing this package does not load the
library; the first call does, and fails if it has not been built.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (PDLP_DUAL_INFEASIBLE, PDLP_ERR_CUDA, PDLP_ERR_INVALID_ARG, PDLP_ERR_OOM, PDLP_ERR_STATE,
                   PDLP_ERR_TIMEOUT, PDLP_FP32, PDLP_FP32_REFINE, PDLP_FP64, PDLP_OK, PDLP_PRIMAL_INFEASIBLE,
                   STATUS_NAMES, PdlpError, check, pdlp_csr, pdlp_options, pdlp_result)

__all__ = ["Context", "default_options", "pdlp_create", "solve", "solve_batch", "batch_lanes", "PdlpError",
           "PDLP_FP64", "PDLP_FP32", "PDLP_FP32_REFINE", "STATUS_NAMES", "PDLP_OK", "PDLP_ERR_INVALID_ARG",
           "PDLP_ERR_CUDA", "PDLP_ERR_OOM", "PDLP_ERR_TIMEOUT", "PDLP_ERR_STATE", "PDLP_PRIMAL_INFEASIBLE",
           "PDLP_DUAL_INFEASIBLE"]


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _in(a, dtype, size=None):
    """(pointer, keep-alive) for an input array of `size` elements (any size
    when None); None passes through.  The C ABI takes bare pointers, so a
    wrong length is caught here, before the library reads past the array."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
               np.int64: torch.int64}[dtype]
        t = a.to(tdt).contiguous()
        ptr, keep, count = t.data_ptr(), t, t.numel()
    else:
        arr = np.ascontiguousarray(a, dtype=dtype)
        ptr, keep, count = arr.ctypes.data, arr, arr.size
    if size is not None and count != size:
        raise ValueError(f"input array has {count} elements, expected {size}")
    return ptr, keep


def _out(a, size, dtype=np.float64):
    """(pointer, array) for an output: the given array or a new numpy array."""
    if a is None:
        arr = np.empty(size, dtype=dtype)
        return arr.ctypes.data, arr
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if not a.is_contiguous() or a.numel() != size or a.dtype != tdt:
            raise ValueError("output tensor must be contiguous with the right size and dtype")
        return a.data_ptr(), a
    if not a.flags.c_contiguous or a.size != size or a.dtype != dtype:
        raise ValueError("output array must be contiguous with the right size and dtype")
    return a.ctypes.data, a


def default_options(**kw) -> pdlp_options:
    """pdlp_default_options(), then any field overridden by keyword."""
    o = pdlp_options()
    check(_abi.load().pdlp_default_options(C.byref(o)))
    for k, v in kw.items():
        if k == "stream":
            v = C.c_void_p(int(v)) if v is not None else None
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Context:
    """One LP on the GPU (pdlp_create ... pdlp_destroy)."""

    def __init__(self, row_ptr, col_idx, val, c, q, l, u, ineq, m: int, n: int, options=None, **kw):
        self._lib = _abi.load()
        self.m, self.n = int(m), int(n)
        opts = options if options is not None else default_options(**kw)
        self.options = opts
        keep = []
        p_v, k = _in(val, np.float64); keep.append(k)
        self.nnz = int(k.numel() if _is_torch(k) else k.size)
        p_rp, k = _in(row_ptr, np.int32, self.m + 1); keep.append(k)
        p_ci, k = _in(col_idx, np.int32, self.nnz); keep.append(k)
        csr = pdlp_csr(self.m, self.n, self.nnz, p_rp, p_ci, p_v)
        ptrs = []
        for arr, dt, size in ((c, np.float64, self.n), (q, np.float64, self.m), (l, np.float64, self.n),
                              (u, np.float64, self.n), (ineq, np.uint8, self.m)):
            p, k = _in(arr, dt, size)
            ptrs.append(p)
            keep.append(k)
        h = C.c_void_p()
        rc = self._lib.pdlp_create(C.byref(csr), *ptrs, C.byref(opts), C.byref(h))
        check(rc)
        self._h = h

    @classmethod
    def from_lp(cls, lp, options=None, **kw):
        """From an object with m, n, row_ptr, col_idx, val, c, q, l, u, ineq (e.g. lpgen.LP)."""
        return cls(lp.row_ptr, lp.col_idx, lp.val, lp.c, lp.q, lp.l, lp.u, lp.ineq, lp.m, lp.n,
                   options=options, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pdlp_destroy(self._h)
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

    def pdlp_solve(self, x0=None, y0=None, x_out=None, y_out=None):
        """pdlp_solve: returns (x, y, result dict) in the original space."""
        p_x0, k0 = _in(x0, np.float64, self.n)
        p_y0, k1 = _in(y0, np.float64, self.m)
        px, x = _out(x_out, self.n)
        py, y = _out(y_out, self.m)
        r = pdlp_result()
        check(self._lib.pdlp_solve(self._h, p_x0, p_y0, px, py, C.byref(r)), self._h)
        self.last_engine = int(r.engine)
        return x, y, r.asdict()

    solve = pdlp_solve

    def pdlp_unroll(self, T: int, ckpt_every: int = 50, x0=None, y0=None, x_out=None, y_out=None):
        """pdlp_unroll: T unrolled steps -> (x_T, y_T, eta[T])."""
        p_x0, k0 = _in(x0, np.float64, self.n)
        p_y0, k1 = _in(y0, np.float64, self.m)
        px, x = _out(x_out, self.n)
        py, y = _out(y_out, self.m)
        pe, eta = _out(None, int(T))
        check(self._lib.pdlp_unroll(self._h, int(T), int(ckpt_every), p_x0, p_y0, px, py, pe), self._h)
        self.unroll_generation = getattr(self, "unroll_generation", 0) + 1
        return x, y, eta

    unroll = pdlp_unroll

    def pdlp_grad(self, dL_dx, dL_dy=None, dc=None, dq=None, dK=None):
        """pdlp_grad: VJP of the last unrolled map -> (dL/dc, dL/dq, dL/dK values)."""
        p_gx, k0 = _in(dL_dx, np.float64, self.n)
        p_gy, k1 = _in(dL_dy, np.float64, self.m)
        pc, oc = _out(dc, self.n)
        pq, oq = _out(dq, self.m)
        pk, ok = _out(dK, self.nnz)
        check(self._lib.pdlp_grad(self._h, p_gx, p_gy, pc, pq, pk), self._h)
        return oc, oq, ok

    grad = pdlp_grad

    def pdlp_get_scaled(self) -> dict:
        """pdlp_get_scaled: the preconditioned problem (numpy arrays)."""
        m, n, nnz = self.m, self.n, self.nnz
        out = dict(Kval=np.empty(nnz), KT_row_ptr=np.empty(n + 1, np.int32),
                   KT_col_idx=np.empty(nnz, np.int32), KTval=np.empty(nnz),
                   KT_perm=np.empty(nnz, np.int32), D1=np.empty(m), D2=np.empty(n), cs=np.empty(n),
                   qs=np.empty(m), ls=np.empty(n), us=np.empty(n))
        order = ["Kval", "KT_row_ptr", "KT_col_idx", "KTval", "KT_perm", "D1", "D2", "cs", "qs", "ls", "us"]
        check(self._lib.pdlp_get_scaled(self._h, *[out[k].ctypes.data for k in order]), self._h)
        return out

    get_scaled = pdlp_get_scaled

    def pdlp_normalized_gap(self, x, y, omega: float, r: float):
        """pdlp_normalized_gap on the scaled problem -> (mu, maximised gap)."""
        px, k0 = _in(x, np.float64, self.n)
        py, k1 = _in(y, np.float64, self.m)
        mu = C.c_double()
        val = C.c_double()
        check(self._lib.pdlp_normalized_gap(self._h, px, py, float(omega), float(r), C.byref(mu),
                                            C.byref(val)), self._h)
        return mu.value, val.value

    normalized_gap = pdlp_normalized_gap

    def pdlp_get_trace(self, max_records: int = 2048):
        """Restart evaluations of the last solve: array [records, 16] with columns
        k, t, mu_cur, mu_avg, mu0, candidate, restarted, omega, r_cur, r_avg,
        rel gap / primal / dual of the current, then of the average iterate."""
        out = np.zeros((max_records, 16))
        cnt = C.c_int32()
        check(self._lib.pdlp_get_trace(self._h, out.ctypes.data, int(max_records), C.byref(cnt)), self._h)
        return out[:min(cnt.value, max_records)]

    get_trace = pdlp_get_trace

    def pdlp_time_step_kernels(self, reps: int = 50):
        """Mean CUDA-event durations (ms): the primal and the dual step kernels
        launched alone, one step attempt inside the persistent kernel, and one
        launch of the persistent evaluation kernel (each 0.0 when the context
        runs without that kernel)."""
        ms = np.zeros(4, np.float32)
        check(self._lib.pdlp_time_step_kernels(self._h, int(reps), ms.ctypes.data), self._h)
        return float(ms[0]), float(ms[1]), float(ms[2]), float(ms[3])

    time_step_kernels = pdlp_time_step_kernels


def pdlp_create(lp, **kw) -> Context:
    return Context.from_lp(lp, **kw)


def solve(lp, x0=None, y0=None, **kw):
    """One-shot solve of an LP object -> (x, y, result dict)."""
    with Context.from_lp(lp, **kw) as ctx:
        return ctx.pdlp_solve(x0, y0)


def solve_batch(lps, **kw):
    """pdlp_solve_batch over a list of LP objects -> (list of x, list of y, list of result dicts)."""
    lib = _abi.load()
    opts = default_options(**kw)
    cnt = len(lps)
    m = np.array([lp.m for lp in lps], np.int32)
    n = np.array([lp.n for lp in lps], np.int32)
    nnz = np.array([lp.nnz for lp in lps], np.int64)
    row_off = np.zeros(cnt + 1, np.int64); np.cumsum(m, out=row_off[1:])
    col_off = np.zeros(cnt + 1, np.int64); np.cumsum(n, out=col_off[1:])
    nnz_off = np.zeros(cnt + 1, np.int64); np.cumsum(nnz, out=nnz_off[1:])
    rp = np.concatenate([np.asarray(lp.row_ptr[:-1], np.int32) for lp in lps])
    ci = np.concatenate([np.asarray(lp.col_idx, np.int32) for lp in lps])
    va = np.concatenate([np.asarray(lp.val, np.float64) for lp in lps])
    cc = np.concatenate([lp.c for lp in lps]).astype(np.float64)
    qq = np.concatenate([lp.q for lp in lps]).astype(np.float64)
    ll = np.concatenate([lp.l for lp in lps]).astype(np.float64)
    uu = np.concatenate([lp.u for lp in lps]).astype(np.float64)
    ineq = np.concatenate([lp.ineq for lp in lps]).astype(np.uint8)
    x = np.empty(int(col_off[-1]))
    y = np.empty(int(row_off[-1]))
    res = (pdlp_result * cnt)()
    arrs = [m, n, row_off, col_off, nnz_off, rp, ci, va, cc, qq, ll, uu, ineq]
    check(lib.pdlp_solve_batch(cnt, *[a.ctypes.data for a in arrs], C.byref(opts), x.ctypes.data,
                               y.ctypes.data, C.addressof(res)))
    xs = [x[col_off[b]:col_off[b + 1]] for b in range(cnt)]
    ys = [y[row_off[b]:row_off[b + 1]] for b in range(cnt)]
    return xs, ys, [r.asdict() for r in res]


def batch_lanes(precision=PDLP_FP64, nbuckets: int = 5):
    """Lanes per row (K, K^T) the batch autotuner chose per size bucket (0: not tuned)."""
    lib = _abi.load()
    lk = np.zeros(nbuckets, np.int32)
    lt = np.zeros(nbuckets, np.int32)
    check(lib.pdlp_batch_lanes(int(precision), lk.ctypes.data, lt.ctypes.data, int(nbuckets)))
    return lk, lt

"""Python handle on the plain FP64 CPU oracle (``pdlp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it to check and time the GPU library.  The GPU library never
imports it.  ``build()`` compiles the C source with gcc (-O2, no contraction
of multiply-adds) into ``oracle/_build/``; every other function loads that
library through ctypes and works on numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdlp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "RUNNING", 1: "OPTIMAL", 2: "ITER_LIMIT", 3: "KKT_PASS_LIMIT", 5: "NUMERICAL_ERROR"}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newer = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pdlp_oracle.h")))
    if newer and not force:
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Lp(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("c", C.c_void_p), ("q", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p),
                ("ineq", C.c_void_p), ("ylo", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("iter_limit", C.c_int64), ("kkt_pass_limit", C.c_int64),
                ("ruiz_iters", C.c_int32), ("pock_chambolle", C.c_int32),
                ("pw_theta", C.c_double), ("beta_suff", C.c_double), ("beta_nec", C.c_double),
                ("beta_art", C.c_double), ("eval_every", C.c_int32), ("eps_zero", C.c_double),
                ("adaptive_restart", C.c_int32), ("pw_update", C.c_int32),
                ("step_policy", C.c_int32), ("omega0", C.c_double),
                ("restart_to_current", C.c_int32), ("mp_breaking", C.c_double),
                ("mp_downscaling", C.c_double), ("mp_interpolation", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int64), ("kkt_passes", C.c_int64),
                ("restarts", C.c_int64), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("gap", C.c_double), ("pres", C.c_double), ("dres", C.c_double),
                ("rel_gap", C.c_double), ("rel_pres", C.c_double), ("rel_dres", C.c_double),
                ("omega", C.c_double), ("eta", C.c_double), ("returned_average", C.c_int32)]

    def asdict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            L.or_default_opts.argtypes = [C.POINTER(Opts)]
            L.or_transpose.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, P]
            L.or_precondition.argtypes = [C.c_int32, C.c_int32, P, P, P, C.c_int32, C.c_int32, P, P]
            L.or_transform.argtypes = [C.c_int32, C.c_int32] + [P] * 10
            L.or_kkt.argtypes = [C.POINTER(_Lp), P, P, P]
            L.or_normalized_gap.argtypes = [C.c_int32, C.c_int32] + [P] * 7 + [C.c_double, C.c_double, P]
            L.or_normalized_gap.restype = C.c_double
            L.or_solve.argtypes = [C.POINTER(_Lp), C.POINTER(Opts), P, P, P, P, C.POINTER(Result)]
            L.or_solve_traced.argtypes = [C.POINTER(_Lp), C.POINTER(Opts), P, P, P, P, C.POINTER(Result), P,
                                          C.c_int32, C.POINTER(C.c_int32)]
            L.or_pdhg_fixed.argtypes = [C.POINTER(_Lp), C.c_double, C.c_double, C.c_int64, P, P]
            L.or_power_norm.argtypes = [C.POINTER(_Lp), C.c_int32, C.c_int32]
            L.or_power_norm.restype = C.c_double
            L.or_unroll_schedule.argtypes = [C.POINTER(_Lp), C.c_int32, C.c_int32, C.c_int64, P, P, P, P, P, P]
            L.or_unroll_forward.argtypes = [C.POINTER(_Lp), C.c_int32, C.c_int32, C.c_int64, P,
                                            C.c_double, P, P, P, P]
            L.or_unroll_vjp.argtypes = [C.POINTER(_Lp), C.c_int32, C.c_int32, C.c_int64, P,
                                        C.c_double, P, P, P, P, P, P, P]
            L.or_correction_lp.argtypes = [C.POINTER(_Lp), P, P, C.c_double, P, P, P, P, P, P, P]
            L.or_step_sizes.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_primal_weight.argtypes = [C.c_double] * 5
            L.or_primal_weight.restype = C.c_double
            L.or_restart_check.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int64,
                                           C.c_double, C.c_double, C.c_double]
            L.or_restart_check.restype = C.c_int32
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Pinned:
    """Keeps the contiguous numpy copies alive while C reads them."""

    def __init__(self, lp, ylo=None):
        self.rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int32)
        self.ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
        self.v = _f64(lp.val)
        self.c, self.q, self.l, self.u = _f64(lp.c), _f64(lp.q), _f64(lp.l), _f64(lp.u)
        self.ineq = np.ascontiguousarray(lp.ineq, dtype=np.uint8)
        self.ylo = _f64(ylo)
        self.s = _Lp(lp.m, lp.n, _p(self.rp), _p(self.ci), _p(self.v), _p(self.c), _p(self.q),
                     _p(self.l), _p(self.u), _p(self.ineq), _p(self.ylo))


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().or_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def transpose(lp):
    """Stable CSR transpose -> (row_ptr_t, col_idx_t, val_t, perm)."""
    rp = np.ascontiguousarray(lp.row_ptr, np.int32)
    ci = np.ascontiguousarray(lp.col_idx, np.int32)
    v = _f64(lp.val)
    nnz = int(rp[-1])
    trp = np.zeros(lp.n + 1, np.int32)
    tci = np.zeros(nnz, np.int32)
    tv = np.zeros(nnz)
    perm = np.zeros(nnz, np.int32)
    lib().or_transpose(lp.m, lp.n, _p(rp), _p(ci), _p(v), _p(trp), _p(tci), _p(tv), _p(perm))
    return trp, tci, tv, perm


def precondition(lp, ruiz_iters=10, pock_chambolle=1):
    """Section 3.5 preconditioning -> (scaled values of K, D1, D2)."""
    rp = np.ascontiguousarray(lp.row_ptr, np.int32)
    ci = np.ascontiguousarray(lp.col_idx, np.int32)
    v = np.array(lp.val, dtype=np.float64, copy=True)
    D1 = np.zeros(lp.m)
    D2 = np.zeros(lp.n)
    lib().or_precondition(lp.m, lp.n, _p(rp), _p(ci), _p(v), ruiz_iters, pock_chambolle, _p(D1), _p(D2))
    return v, D1, D2


def transform(lp, D1, D2):
    """Scaled (c~, q~, l~, u~) of Section 3.5."""
    D1, D2 = _f64(D1), _f64(D2)
    c, q, l, u = _f64(lp.c), _f64(lp.q), _f64(lp.l), _f64(lp.u)
    cs, qs, ls, us = np.zeros(lp.n), np.zeros(lp.m), np.zeros(lp.n), np.zeros(lp.n)
    lib().or_transform(lp.m, lp.n, _p(D1), _p(D2), _p(c), _p(q), _p(l), _p(u),
                       _p(cs), _p(qs), _p(ls), _p(us))
    return cs, qs, ls, us


KKT_KEYS = ("primal_obj", "dual_obj", "gap", "pres", "dres", "rel_gap", "rel_pres", "rel_dres")


def kkt(lp, x, y, ylo=None) -> dict:
    """Eq. (15) quantities at (x, y) on the original problem."""
    pin = _Pinned(lp, ylo)
    x, y = _f64(x), _f64(y)
    out = np.zeros(8)
    lib().or_kkt(C.byref(pin.s), _p(x), _p(y), _p(out))
    d = dict(zip(KKT_KEYS, out.tolist()))
    d["rel_kkt"] = max(d["rel_gap"], d["rel_pres"], d["rel_dres"])
    return d


def normalized_gap(x, y, gx, gy, l, u, ylo, omega, r):
    """Section 3.2 normalized duality gap -> (mu, max value)."""
    arrs = [_f64(a) for a in (x, y, gx, gy, l, u, ylo)]
    val = np.zeros(1)
    mu = lib().or_normalized_gap(arrs[0].size, arrs[1].size, *[_p(a) for a in arrs],
                                 float(omega), float(r), _p(val))
    return mu, float(val[0])


def solve(lp, x0=None, y0=None, ylo=None, **opts):
    """Full PDLP (Algorithm 1) -> (x, y, result dict)."""
    o = default_opts(**opts)
    pin = _Pinned(lp, ylo)
    x0, y0 = _f64(x0), _f64(y0)
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    r = Result()
    lib().or_solve(C.byref(pin.s), C.byref(o), _p(x0), _p(y0), _p(x), _p(y), C.byref(r))
    return x, y, r.asdict()


def solve_traced(lp, x0=None, y0=None, ylo=None, trace_cap=256, **opts):
    """solve() plus the restart evaluations: (x, y, result, trace[records, 16]) with
    columns k, t, mu_cur, mu_avg, mu0, candidate, restarted, omega, r_cur, r_avg,
    then the relative Eq. (15) gap / primal / dual terms of the current and of
    the average iterate (the layout of the library's pdlp_get_trace)."""
    o = default_opts(**opts)
    pin = _Pinned(lp, ylo)
    x0, y0 = _f64(x0), _f64(y0)
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    r = Result()
    tr = np.zeros((trace_cap, 16))
    cnt = C.c_int32()
    lib().or_solve_traced(C.byref(pin.s), C.byref(o), _p(x0), _p(y0), _p(x), _p(y), C.byref(r), _p(tr),
                          trace_cap, C.byref(cnt))
    return x, y, r.asdict(), tr[:min(cnt.value, trace_cap)]


def power_norm(lp, ruiz_iters=10, pock_chambolle=1):
    """||K~||_2 of the preconditioned matrix by power iteration (Section 2)."""
    pin = _Pinned(lp)
    return float(lib().or_power_norm(C.byref(pin.s), ruiz_iters, pock_chambolle))


def pdhg_fixed(lp, eta, omega, T, x0=None, y0=None):
    """Appendix A: T steps of plain PDHG with constant eta, omega (unscaled)."""
    pin = _Pinned(lp)
    x = np.zeros(lp.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    y = np.zeros(lp.m) if y0 is None else np.array(y0, dtype=np.float64, copy=True)
    lib().or_pdhg_fixed(C.byref(pin.s), float(eta), float(omega), int(T), _p(x), _p(y))
    return x, y


def unroll_schedule(lp, T, x0=None, y0=None, ruiz_iters=10, pock_chambolle=1):
    """Algorithm 2 step sizes of T accepted steps (fixed omega) -> (eta[T], omega, x_T, y_T)."""
    pin = _Pinned(lp)
    x0, y0 = _f64(x0), _f64(y0)
    eta = np.zeros(int(T))
    om = np.zeros(1)
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    lib().or_unroll_schedule(C.byref(pin.s), ruiz_iters, pock_chambolle, int(T), _p(x0), _p(y0),
                             _p(eta), _p(om), _p(x), _p(y))
    return eta, float(om[0]), x, y


def unroll_forward(lp, eta, omega, x0=None, y0=None, ruiz_iters=10, pock_chambolle=1):
    """Unrolled PDHG with a frozen schedule -> (x_T, y_T) in the original space."""
    pin = _Pinned(lp)
    eta = _f64(eta)
    x0, y0 = _f64(x0), _f64(y0)
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    lib().or_unroll_forward(C.byref(pin.s), ruiz_iters, pock_chambolle, eta.size, _p(eta),
                            float(omega), _p(x0), _p(y0), _p(x), _p(y))
    return x, y


def unroll_vjp(lp, eta, omega, gx, gy=None, x0=None, y0=None, ruiz_iters=10, pock_chambolle=1):
    """VJP of the unrolled map -> (dL/dc, dL/dq, dL/dK values in CSR order)."""
    pin = _Pinned(lp)
    eta = _f64(eta)
    x0, y0, gx, gy = _f64(x0), _f64(y0), _f64(gx), _f64(gy)
    dc = np.zeros(lp.n)
    dq = np.zeros(lp.m)
    dK = np.zeros(lp.nnz)
    lib().or_unroll_vjp(C.byref(pin.s), ruiz_iters, pock_chambolle, eta.size, _p(eta),
                        float(omega), _p(x0), _p(y0), _p(gx), _p(gy), _p(dc), _p(dq), _p(dK))
    return dc, dq, dK


def correction_lp(lp, xh, yh, dmax=1e12, ylo=None):
    """Refinement correction problem at (xh, yh) -> dict(c, q, l, u, ylo, dP, dD)."""
    pin = _Pinned(lp, ylo)
    xh, yh = _f64(xh), _f64(yh)
    cp, qp, lp_, up, yl = np.zeros(lp.n), np.zeros(lp.m), np.zeros(lp.n), np.zeros(lp.n), np.zeros(lp.m)
    dP = np.zeros(1)
    dD = np.zeros(1)
    lib().or_correction_lp(C.byref(pin.s), _p(xh), _p(yh), float(dmax), _p(cp), _p(qp), _p(lp_),
                           _p(up), _p(yl), _p(dP), _p(dD))
    return dict(c=cp, q=qp, l=lp_, u=up, ylo=yl, dP=float(dP[0]), dD=float(dD[0]))


def step_sizes(omega, dx2, dy2, inter, eta, k):
    """Algorithm 2's (eta_bar, eta') for an attempt at eta after k accepted steps."""
    eb, en = C.c_double(), C.c_double()
    lib().or_step_sizes(float(omega), float(dx2), float(dy2), float(inter), float(eta), int(k),
                        C.byref(eb), C.byref(en))
    return eb.value, en.value


def primal_weight(omega, Dx, Dy, theta=0.5, eps_zero=1e-10):
    """Algorithm 3's primal weight update."""
    return float(lib().or_primal_weight(float(omega), float(Dx), float(Dy), float(theta), float(eps_zero)))


RESTART_REASON = {0: None, 1: "sufficient", 2: "necessary", 3: "artificial"}


def restart_check(muc, mu0, muc_prev, t, k, beta_suff=0.9, beta_nec=0.1, beta_art=0.5):
    """Section 3.2 restart criteria -> None or the name of the first that holds."""
    r = lib().or_restart_check(float(muc), float(mu0), float(muc_prev), int(t), int(k),
                               float(beta_suff), float(beta_nec), float(beta_art))
    return RESTART_REASON[int(r)]

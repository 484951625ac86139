"""The allocation-free normalized-gap call (pdlp_normalized_gap_noalloc).

That call exists for callers that cannot allocate device memory, such as a
program whose framework allocator already holds the GPU's memory, or one
that cannot pay for cudaMalloc / cudaFree and their implicit synchronisation.
It keeps its scratch in one static device array.  These tests call it through
the C ABI, twice in a row on the same array, and compare it with
pdlp_normalized_gap (the context-based call) and with the oracle's exact
breakpoint solver, within the tolerance the gap parity tests use, including
points on their bounds and the largest size the array holds.  The file is
named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
import paper_2106_04756_gb300 as P
from paper_2106_04756_gb300 import _abi

pytestmark = pytest.mark.gpu

GAP_RTOL = 1e-6  # the tolerance of the normalized-gap parity tests


def _noalloc(lib, x, y, gx, gy, l, u, ylo, omega, r):
    import torch
    dev = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in (x, y, gx, gy, l, u, ylo)]
    torch.cuda.synchronize()
    mu, val = C.c_double(), C.c_double()
    rc = lib.pdlp_normalized_gap_noalloc(len(x), len(y), *[t.data_ptr() for t in dev], float(omega), float(r),
                                         None, C.byref(mu), C.byref(val))
    assert rc == _abi.PDLP_OK, lib.pdlp_last_error(None)
    return mu.value, val.value


@pytest.mark.parametrize("make", [lambda: lpgen.small_planted(),
                                  lambda: lpgen.mip_like(2000, 5000, 30000, seed_key=(71,))])
def test_noalloc_matches_context_call_twice(gpu_lib, make):
    lp = make()
    lib = _abi.load()
    rng = np.random.default_rng(17)
    ylo = np.where(lp.ineq == 1, 0.0, -np.inf)
    with P.Context.from_lp(lp) as ctx:
        g = ctx.get_scaled()
        Ks = sp.csr_matrix((g["Kval"], lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
        for call in range(2):  # two calls in a row share the static scratch
            lo = np.where(np.isfinite(g["ls"]), g["ls"], -5.0)
            hi = np.where(np.isfinite(g["us"]), g["us"], 5.0)
            x = np.clip(lo + (hi - lo) * rng.random(lp.n), g["ls"], g["us"])
            y = np.maximum(rng.standard_normal(lp.m), ylo)
            omega = float(np.exp(rng.uniform(-2, 2)))
            r = float(rng.uniform(0.1, 10.0))
            mu_ref, val_ref = ctx.normalized_gap(x, y, omega, r)
            gx = Ks.T @ y - g["cs"]
            gy = g["qs"] - Ks @ x
            mu, val = _noalloc(lib, x, y, gx, gy, g["ls"], g["us"], ylo, omega, r)
            assert abs(mu - mu_ref) <= GAP_RTOL * abs(mu_ref), (call, mu, mu_ref)
            assert abs(val - val_ref) <= GAP_RTOL * abs(val_ref), (call, val, val_ref)


@pytest.mark.parametrize("make", [lambda: lpgen.small_planted(),
                                  lambda: lpgen.mip_like(2000, 5000, 30000, seed_key=(72,))])
def test_noalloc_at_bounds_matches_oracle_and_context(gpu_lib, make):
    """About 30% of the primal coordinates exactly on a finite bound and 30% of
    the inequality duals exactly at 0 (coordinates that cannot move in the
    ascent direction): the call agrees with the oracle's exact breakpoint
    solver and with the context call, on two calls in a row."""
    lp = make()
    lib = _abi.load()
    rng = np.random.default_rng(29)
    ylo = np.where(lp.ineq == 1, 0.0, -np.inf)
    with P.Context.from_lp(lp) as ctx:
        g = ctx.get_scaled()
        Ks = sp.csr_matrix((g["Kval"], lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
        ls, us = g["ls"], g["us"]
        for call in range(2):
            lo = np.where(np.isfinite(ls), ls, -5.0)
            hi = np.where(np.isfinite(us), us, 5.0)
            x = np.clip(lo + (hi - lo) * rng.random(lp.n), ls, us)
            pick = rng.random(lp.n)
            at_l = (pick < 0.15) & np.isfinite(ls)
            at_u = (pick >= 0.15) & (pick < 0.3) & np.isfinite(us)
            x[at_l] = ls[at_l]
            x[at_u] = us[at_u]
            y = np.maximum(rng.standard_normal(lp.m), ylo)
            y[(lp.ineq == 1) & (rng.random(lp.m) < 0.3)] = 0.0
            omega = float(np.exp(rng.uniform(-2, 2)))
            r = float(rng.uniform(0.1, 10.0))
            gx = Ks.T @ y - g["cs"]
            gy = g["qs"] - Ks @ x
            mu_or, val_or = oracle.normalized_gap(x, y, gx, gy, ls, us, ylo, omega, r)
            mu_ctx, _ = ctx.normalized_gap(x, y, omega, r)
            mu, val = _noalloc(lib, x, y, gx, gy, ls, us, ylo, omega, r)
            assert abs(mu - mu_or) <= GAP_RTOL * abs(mu_or), (call, mu, mu_or)
            assert abs(val - val_or) <= GAP_RTOL * abs(val_or), (call, val, val_or)
            assert abs(mu - mu_ctx) <= GAP_RTOL * abs(mu_ctx), (call, mu, mu_ctx)


def test_noalloc_largest_accepted_size(gpu_lib):
    """n + m = 2^20 fills every key slot of the static array.  Without bounds
    (l = -inf, u = +inf, all rows equalities) the maximiser is the scaled
    gradient and mu = sqrt(||gx||^2 / omega + omega ||gy||^2) whatever the
    point and the radius; checked on two calls in a row."""
    lib = _abi.load()
    rng = np.random.default_rng(31)
    n = 1 << 19
    m = (1 << 20) - n
    l = np.full(n, -np.inf)
    u = np.full(n, np.inf)
    ylo = np.full(m, -np.inf)
    for call in range(2):
        x = rng.standard_normal(n)
        y = rng.standard_normal(m)
        gx = rng.standard_normal(n)
        gy = rng.standard_normal(m)
        omega = float(np.exp(rng.uniform(-1, 1)))
        r = float(rng.uniform(0.5, 2.0))
        mu, val = _noalloc(lib, x, y, gx, gy, l, u, ylo, omega, r)
        ref = np.sqrt(gx @ gx / omega + omega * (gy @ gy))
        assert abs(mu - ref) <= GAP_RTOL * ref, (call, mu, ref)
        assert abs(val - r * ref) <= GAP_RTOL * r * ref, (call, val, r * ref)


def test_noalloc_rejects_sizes_over_its_limit(gpu_lib):
    lib = _abi.load()
    mu = C.c_double()
    one = np.zeros(1)
    rc = lib.pdlp_normalized_gap_noalloc((1 << 20), 1, *([one.ctypes.data] * 7), 1.0, 1.0, None, C.byref(mu), None)
    assert rc == _abi.PDLP_ERR_INVALID_ARG
    assert b"static scratch limit" in lib.pdlp_last_error(None)

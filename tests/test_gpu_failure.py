"""Failure detection on the GPU without faulting or hanging it.

Each device-side wait of the library (the grid-wide barriers of the
persistent step kernel) is bounded; option wait_limit_us = -N makes the
first barrier of each persistent launch wait for an arrival that never
comes, so the bound runs out after N microseconds, the kernel records the
failure and returns, and pdlp_solve reports PDLP_ERR_TIMEOUT.  The other
tests reach each limit status of a solve and the numerical-error status:
  * PDLP_TIME_LIMIT       a time limit far below one evaluation period,
  * PDLP_KKT_PASS_LIMIT   one step attempt allowed,
  * PDLP_ITER_LIMIT       one accepted iteration allowed,
  * PDLP_NUMERICAL_ERROR  a primal weight so small that the first primal
                          step overflows (tau = eta / omega = 1e300).
After every failure a new context on the same GPU still solves to 1e-8.
"""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu


def _still_solves():
    lp = lpgen.small_planted()
    x, y, r = P.solve(lp, rel_tol=1e-8)
    assert r["status_name"] == "OPTIMAL"
    assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-8


@pytest.mark.parametrize("use_graph", [1, 0])
def test_barrier_wait_that_runs_out_reports_timeout(gpu_lib, use_graph):
    lp = lpgen.mip_like(2000, 5000, 30000, seed_key=(71,))
    with P.Context.from_lp(lp, persistent=3, wait_limit_us=-2000, use_graph=use_graph) as ctx:
        with pytest.raises(P.PdlpError) as ei:
            ctx.solve()
        assert ei.value.code == P.PDLP_ERR_TIMEOUT
        assert "timed out" in str(ei.value)
        # the same context fails the same way again (the wait is bounded every time)
        with pytest.raises(P.PdlpError) as ei:
            ctx.solve()
        assert ei.value.code == P.PDLP_ERR_TIMEOUT
    _still_solves()


def test_positive_wait_limit_leaves_a_normal_solve_alone(gpu_lib):
    lp = lpgen.small_planted()
    x, y, r = P.solve(lp, rel_tol=1e-8, persistent=3, wait_limit_us=500000)
    assert r["status_name"] == "OPTIMAL"


@pytest.mark.parametrize("persistent", [3, 0, 2])
def test_time_limit_status(gpu_lib, persistent):
    lp = lpgen.mip_like(2000, 5000, 30000, seed_key=(71,))
    x, y, r = P.solve(lp, rel_tol=1e-12, time_limit_s=1e-6, persistent=persistent)
    assert r["status_name"] == "TIME_LIMIT", r
    assert r["iters"] <= 40
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(y))
    _still_solves()


@pytest.mark.parametrize("persistent", [3, 0, 2])
def test_kkt_pass_limit_status(gpu_lib, persistent):
    lp = lpgen.mip_like(2000, 5000, 30000, seed_key=(71,))
    _, _, r = P.solve(lp, rel_tol=1e-12, kkt_pass_limit=1, persistent=persistent)
    assert r["status_name"] == "KKT_PASS_LIMIT", r
    assert r["kkt_passes"] == 1
    _, _, ro = oracle.solve(lp, eps=1e-12, kkt_pass_limit=1)
    assert ro["status_name"] == "KKT_PASS_LIMIT" and ro["kkt_passes"] == 1


@pytest.mark.parametrize("persistent", [3, 0, 2])
def test_iteration_limit_status(gpu_lib, persistent):
    lp = lpgen.small_planted()
    _, _, r = P.solve(lp, rel_tol=1e-12, iter_limit=1, persistent=persistent)
    assert r["status_name"] == "ITER_LIMIT" and r["iters"] == 1, r


@pytest.mark.parametrize("persistent", [3, 0, 2])
def test_numerical_error_status(gpu_lib, persistent):
    """Without preconditioning and with omega^0 = 1e-300, the first primal step
    x' = proj(x - (eta / omega)(c - K^T y)) moves free variables by about
    1e300 |c_j|, so ||x' - x||^2 overflows and Algorithm 2's test sees a
    non-finite value: NUMERICAL_ERROR, as in the oracle."""
    lp = lpgen.planted_uniform(30, 60, 0.2, frac_boxed=0.0, seed_key=(91,))
    kw = dict(ruiz_iters=0, pock_chambolle=0, omega0=1e-300)
    _, _, r = P.solve(lp, persistent=persistent, **kw)
    assert r["status_name"] == "NUMERICAL_ERROR", r
    _, _, ro = oracle.solve(lp, **kw)
    assert ro["status_name"] == "NUMERICAL_ERROR"
    _still_solves()

"""Long solves of the MIP-relaxation-shaped LP: the GPU path against the
oracle over 20,000 iterations of a 2000 x 5000 instance of the 100k x 250k
workload's shape.

On this shape neither implementation reaches 1e-8: the relative KKT error
settles between 1e-2 and 1e-1 while the primal weight of Algorithm 3 drifts
(down here; on the full-size instance a run of restarts at successive
evaluations raises it by three orders of magnitude).  The trajectories are
chaotic (mu of the current iterate moves by percents for rounding-level
differences in the iterates), so the comparison is
  * exact in every restart decision over the first four evaluations, where
    the iterates still agree closely, with the primal weight and mu_0 equal
    to 1e-5 over the first three (by k = 160 the engines' different summation
    orders have moved mu_0 by 1e-3), and
  * in trend afterwards: the better candidate's relative KKT error of the
    two runs within a factor of ten (median over the evaluations past k =
    2,000), the primal weights within two decades, and both runs still above
    1e-3 at the end (neither converges: the stall is the method's, not the
    GPU path's).
Every step engine is compared.
"""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu

ITERS = 20000


@pytest.fixture(scope="module")
def oracle_trace(oracle_lib):
    lp = lpgen.mip_like(2000, 5000, 30000, seed_key=(71,))
    _, _, r, tr = oracle.solve_traced(lp, iter_limit=ITERS, trace_cap=1000)
    assert r["iters"] == ITERS and r["status_name"] == "ITER_LIMIT"
    return lp, tr


def _best_kkt(tr):
    cur = tr[:, 10:13].max(axis=1)
    avg = tr[:, 13:16].max(axis=1)
    return np.minimum(cur, avg)


@pytest.mark.parametrize("persistent", [1, 0, 2, 4])
def test_long_solve_tracks_oracle(gpu_lib, oracle_trace, persistent):
    lp, to = oracle_trace
    with P.Context.from_lp(lp, iter_limit=ITERS, persistent=persistent) as ctx:
        _, _, r = ctx.solve()
        tg = ctx.get_trace(2048)
    assert r["iters"] == ITERS and r["status_name"] == "ITER_LIMIT"
    assert len(tg) == len(to) == ITERS // 40 - 1
    # the first evaluations: identical decisions (k <= 160); weights and mu_0
    # equal to 1e-5 while the iterates still agree closely (k <= 120)
    for i, (a, b) in enumerate(zip(to[:4], tg[:4])):
        assert (a[0], a[1], a[5], a[6]) == (b[0], b[1], b[5], b[6]), (a[:8], b[:8])
        if i < 3:
            assert abs(a[7] - b[7]) <= 1e-5 * a[7]
            if np.isfinite(a[4]):
                assert abs(a[4] - b[4]) <= 1e-5 * a[4]
    # the trend: same k per record, KKT errors and weights in the same regime
    assert np.array_equal(to[:, 0], tg[:, 0])
    late = to[:, 0] >= 2000
    ko, kg = _best_kkt(to)[late], _best_kkt(tg)[late]
    assert np.median(np.abs(np.log10(kg) - np.log10(ko))) <= 1.0, (np.median(ko), np.median(kg))
    assert np.median(np.abs(np.log10(tg[late, 7]) - np.log10(to[late, 7]))) <= 2.0
    assert ko[-1] > 1e-3 and kg[-1] > 1e-3

"""Presolve-lite (presolve = 1): fixed variables, rows left empty, empty
columns.  Each LP is planted so that its optimum is known; the returned
point is checked on the ORIGINAL problem by the oracle's Eq. (15)
evaluation and against the planted objective, the reported Eq. (15) terms
against the oracle's at that point, and the infeasible / unbounded cases
against the statuses that the data fix."""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu


def _replant(m, n, A, ineq, l, u, seed):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return lpgen._plant(lpgen.rng_for(seed, 9), m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32),
                        A.data.astype(np.float64), ineq, l, u, "presolve")


def _with_fixed(seed=90):
    """Planted LP with empty rows and columns, then 12 variables fixed at
    their planted values (l_j = u_j = x*_j) and every variable of row 3
    fixed too, so that row 3 is emptied by the substitution.  Fixing a
    variable at its optimal value keeps (x*, y*) optimal: the reduced cost
    of a fixed variable may take either sign."""
    base = lpgen.planted_uniform(60, 140, 0.06, frac_boxed=0.7, seed_key=(seed,))
    A = base.scipy().tolil()
    A[0, :] = 0
    A[9, :] = 0
    A[:, 0] = 0
    A[:, 17] = 0
    A = A.tocsr()
    A.eliminate_zeros()
    lp = _replant(base.m, base.n, A, base.ineq, base.l, base.u, seed)
    rng = lpgen.rng_for(seed, 3)
    fix = set(rng.choice(np.arange(20, lp.n), 12, replace=False).tolist())
    fix |= set(lp.col_idx[lp.row_ptr[3]:lp.row_ptr[4]].tolist())
    fix = np.array(sorted(fix))
    lp.l = lp.l.copy()
    lp.u = lp.u.copy()
    lp.l[fix] = lp.x_star[fix]
    lp.u[fix] = lp.x_star[fix]
    return lp, fix


def _check_optimal(lp, x, y, r, tol=1e-8):
    assert r["status_name"] == "OPTIMAL", r
    k = oracle.kkt(lp, x, y)
    assert k["rel_pres"] <= tol and k["rel_dres"] <= tol, k
    assert k["rel_gap"] <= 2 * tol, k
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-6 * (1 + abs(ref)), (lp.c @ x, ref)
    for key in ("primal_obj", "dual_obj"):
        assert abs(r[key] - k[key]) <= 1e-9 * (1 + abs(k[key])), (key, r[key], k[key])
    for key in ("pres", "dres", "gap"):
        assert abs(r[key] - k[key]) <= 1e-9 * (1 + abs(k[key])) + 1e-12, (key, r[key], k[key])
    return k


@pytest.mark.parametrize("precision", [P.PDLP_FP64, P.PDLP_FP32_REFINE])
def test_presolve_fixed_and_empty_solves_original(gpu_lib, oracle_lib, precision):
    lp, fix = _with_fixed()
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, presolve=1, precision=precision)
    _check_optimal(lp, x, y, r)
    assert np.array_equal(x[fix], lp.x_star[fix])  # fixed variables are returned exactly
    assert y[0] == 0.0 and y[9] == 0.0 and y[3] == 0.0  # dropped rows carry y_i = 0
    # without presolve the same LP solves too (fixed variables as l = u boxes)
    x0, y0, r0 = P.solve(lp, rel_tol=1e-8, iter_limit=200000, presolve=0, precision=precision)
    _check_optimal(lp, x0, y0, r0)


@pytest.mark.parametrize("persistent", [1, 0, 2])
def test_presolve_engines_and_start_point(gpu_lib, oracle_lib, persistent):
    lp, _ = _with_fixed(91)
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, presolve=1, persistent=persistent)
    _check_optimal(lp, x, y, r)
    # a start at the planted optimum passes the first evaluation
    xs, ys, rs = P.solve(lp, x0=lp.x_star, y0=lp.y_star, rel_tol=1e-8, iter_limit=200000, presolve=1,
                         persistent=persistent)
    _check_optimal(lp, xs, ys, rs)
    assert rs["iters"] <= 40, rs


def test_presolve_all_fixed_needs_no_iteration(gpu_lib, oracle_lib):
    lp = lpgen.planted_uniform(30, 50, 0.1, seed_key=(92,))
    lp.l = lp.x_star.copy()
    lp.u = lp.x_star.copy()
    x, y, r = P.solve(lp, rel_tol=1e-8, presolve=1)
    assert r["status_name"] == "OPTIMAL" and r["iters"] == 0, r
    assert np.array_equal(x, lp.x_star) and not np.any(y)
    k = oracle.kkt(lp, x, y)
    assert k["rel_pres"] <= 1e-12, k
    # y = 0 and lambda = c: the reported terms are the oracle's at that point
    for key in ("primal_obj", "dual_obj", "pres", "dres", "gap"):
        assert abs(r[key] - k[key]) <= 1e-9 * (1 + abs(k[key])) + 1e-12, (key, r[key], k[key])


def test_presolve_empty_columns_at_cost_bound(gpu_lib, oracle_lib):
    """Columns without nonzeros go to l_j (c_j > 0), u_j (c_j < 0) or the point
    of [l_j, u_j] nearest 0 (c_j = 0)."""
    lp, _ = _with_fixed(90)
    lp.c = lp.c.copy()
    lp.l[0], lp.u[0], lp.c[0] = -2.0, 5.0, 3.0
    lp.l[17], lp.u[17], lp.c[17] = -np.inf, 4.0, -1.5
    lp.x_star = lp.x_star.copy()
    lp.x_star[0], lp.x_star[17] = -2.0, 4.0
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, presolve=1)
    _check_optimal(lp, x, y, r)
    assert x[0] == -2.0 and x[17] == 4.0


def test_presolve_primal_infeasible_empty_row(gpu_lib, oracle_lib):
    lp, _ = _with_fixed(94)
    lp.q = lp.q.copy()
    lp.ineq = lp.ineq.copy()
    lp.ineq[0] = 1
    lp.q[0] = 1.0  # 0 >= 1 on a row without nonzeros
    _, _, r = P.solve(lp, presolve=1)
    assert r["status_name"] == "PRIMAL_INFEASIBLE", r
    # an equality row emptied by fixed variables with a mismatched right-hand side
    lp2, _ = _with_fixed(94)
    lp2.q = lp2.q.copy()
    lp2.ineq = lp2.ineq.copy()
    lp2.ineq[3] = 0
    lp2.q[3] += 1e-3
    _, _, r2 = P.solve(lp2, presolve=1)
    assert r2["status_name"] == "PRIMAL_INFEASIBLE", r2
    # within the tolerance the row stays feasible
    lp3, _ = _with_fixed(94)
    lp3.q = lp3.q.copy()
    lp3.ineq = lp3.ineq.copy()
    lp3.ineq[3] = 0
    lp3.q[3] += 1e-12 * (1 + abs(lp3.q[3]))
    _, _, r3 = P.solve(lp3, presolve=1, rel_tol=1e-8, iter_limit=200000)
    assert r3["status_name"] == "OPTIMAL", r3


def test_presolve_dual_infeasible_empty_column(gpu_lib, oracle_lib):
    lp, _ = _with_fixed(95)
    lp.c = lp.c.copy()
    lp.u = lp.u.copy()
    lp.c[0] = -1.0
    lp.u[0] = np.inf  # minimising -x_0 with x_0 unbounded above and in no row
    _, _, r = P.solve(lp, presolve=1)
    assert r["status_name"] == "DUAL_INFEASIBLE", r


def test_presolved_context_rejects_scaled_space_calls(gpu_lib):
    lp, _ = _with_fixed(96)
    with P.Context.from_lp(lp, presolve=1) as ctx:
        ctx.pdlp_solve()
        with pytest.raises(P.PdlpError) as e:
            ctx.get_scaled()
        assert e.value.code == P.PDLP_ERR_STATE
        rec = ctx.get_trace()
        assert len(rec) >= 1
        ms = ctx.time_step_kernels(3)
        assert ms[0] > 0 and ms[1] > 0
    with pytest.raises(P.PdlpError) as e:
        P.Context.from_lp(lp, presolve=1, unroll_T=10)
    assert e.value.code == P.PDLP_ERR_INVALID_ARG

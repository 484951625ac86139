"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test ties one oracle function to something the paper or mathematics
fixes: planted optimal pairs (Eq. (15) = 0), an independent LP solver
(HiGHS through scipy), vertex enumeration, the Pock-Chambolle norm bound,
the closed form and a numerical optimiser for the normalized gap, the
PageRank vector by power iteration, the scale invariance of Appendix A,
finite differences and the envelope theorem for the unrolled map, and the
exact algebra of the refinement correction problem.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_constants():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def _highs_objective(lp):
    from scipy.optimize import linprog
    A = lp.scipy()
    ineq = lp.ineq.astype(bool)
    res = linprog(lp.c, A_ub=-A[ineq], b_ub=-lp.q[ineq], A_eq=A[~ineq], b_eq=lp.q[~ineq],
                  bounds=list(zip(np.where(np.isfinite(lp.l), lp.l, None),
                                  np.where(np.isfinite(lp.u), lp.u, None))), method="highs")
    assert res.status == 0
    return res.fun


# ---------------------------------------------------------------- constants

def test_defaults_match_paper_constants(oracle_lib):
    g = _golden_constants()
    o = oracle.default_opts()
    assert o.beta_suff == g["beta_sufficient"]
    assert o.beta_nec == g["beta_necessary"]
    assert o.beta_art == g["beta_artificial"]
    assert o.pw_theta == g["primal_weight_smoothing"]
    assert o.eval_every == g["evaluation_period"]
    assert o.ruiz_iters == g["ruiz_iterations"]
    assert o.pock_chambolle == g["pock_chambolle_alpha"]
    assert o.eps == g["termination_eps_high"]


# --------------------------------------------------------------- Eq. (15)

@pytest.mark.parametrize("make", [
    lambda: lpgen.small_planted(),
    lambda: lpgen.planted_uniform(60, 90, 0.1, frac_boxed=0.5, seed_key=(50,)),
    lambda: lpgen.mip_like(300, 700, 4000, seed_key=(51,)),
])
def test_kkt_zero_at_planted_optimum(oracle_lib, make):
    lp = make()
    k = oracle.kkt(lp, lp.x_star, lp.y_star)
    assert k["rel_gap"] < 1e-13 and k["rel_pres"] < 1e-13 and k["rel_dres"] < 1e-13


def test_kkt_detects_each_violation(oracle_lib):
    lp = lpgen.small_planted()
    base = oracle.kkt(lp, lp.x_star, lp.y_star)
    # primal infeasibility on an equality row
    x = lp.x_star.copy()
    j = int(lp.col_idx[lp.row_ptr[np.flatnonzero(lp.ineq == 0)[0]]])
    x[j] += 0.5
    assert oracle.kkt(lp, x, lp.y_star)["pres"] > 1e-3
    # a dual sign change on an active inequality row breaks optimality
    y = lp.y_star.copy()
    i = np.flatnonzero((lp.ineq == 1) & (lp.y_star > 0))[0]
    y[i] = -y[i]
    k = oracle.kkt(lp, lp.x_star, y)
    assert k["dres"] > 1e-3 or k["gap"] > 1e-3
    # the dual objective uses lambda at both bounds: dropping either changes it
    lam = lp.lam_star
    assert (lam > 0).any() and (lam < 0).any()
    assert base["gap"] < 1e-9


# ------------------------------------------------- full solve vs independent

@pytest.mark.parametrize("make", [
    lambda: lpgen.small_planted(),
    lambda: lpgen.planted_uniform(120, 300, 0.05, frac_boxed=0.6, seed_key=(52,)),
])
def test_solve_matches_planted_and_highs(oracle_lib, make):
    lp = make()
    x, y, r = oracle.solve(lp)
    assert r["status_name"] == "OPTIMAL"
    assert max(r["rel_gap"], r["rel_pres"], r["rel_dres"]) <= 1e-8
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-6 * (1 + abs(ref))
    assert abs(_highs_objective(lp) - ref) <= 1e-6 * (1 + abs(ref))


def _vertex_enumeration(A, ineq, q, c, l, u):
    """min c^T x over {A_i x >= q_i (ineq), = q_i (eq), l <= x <= u}, all finite, by
    trying every set of n linearly independent active constraints."""
    m, n = A.shape
    rows = [(A[i], q[i], not ineq[i]) for i in range(m)]
    bnds = [(np.eye(n)[j], l[j], False) for j in range(n)] + [(np.eye(n)[j], u[j], False) for j in range(n)]
    cons = rows + bnds
    eq_idx = [k for k, (_, _, e) in enumerate(cons) if e]
    others = [k for k in range(len(cons)) if k not in eq_idx]
    best = np.inf
    need = n - len(eq_idx)
    for sub in itertools.combinations(others, need):
        idx = eq_idx + list(sub)
        M = np.array([cons[k][0] for k in idx])
        if abs(np.linalg.det(M)) < 1e-10:
            continue
        x = np.linalg.solve(M, np.array([cons[k][1] for k in idx]))
        ok = np.all(x >= l - 1e-9) and np.all(x <= u + 1e-9)
        r = A @ x - q
        ok = ok and np.all(r[ineq.astype(bool)] >= -1e-9) and np.all(np.abs(r[~ineq.astype(bool)]) <= 1e-9)
        if ok:
            best = min(best, c @ x)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_vertex_enumeration(oracle_lib, seed):
    rng = np.random.default_rng([7, seed])
    m, n = 3, 5
    A = rng.standard_normal((m, n))
    ineq = np.array([1, 1, 0], np.uint8)
    xf = rng.uniform(0.2, 0.8, n)
    q = A @ xf - np.where(ineq == 1, rng.uniform(0.0, 0.5, m), 0.0)
    c = rng.standard_normal(n)
    l, u = np.zeros(n), np.ones(n)
    ref = _vertex_enumeration(A, ineq, q, c, l, u)
    Asp = sp.csr_matrix(A)
    lp = lpgen.LP(m=m, n=n, row_ptr=Asp.indptr.astype(np.int32), col_idx=Asp.indices.astype(np.int32),
                  val=Asp.data, c=c, q=q, l=l, u=u, ineq=ineq)
    x, y, r = oracle.solve(lp, iter_limit=200000)
    assert r["status_name"] == "OPTIMAL"
    assert abs(c @ x - ref) <= 1e-6 * (1 + abs(ref))


# ------------------------------------------------------------ Section 3.5

def test_transpose_matches_scipy_and_is_stable(oracle_lib):
    lp = lpgen.mip_like(400, 900, 6000, seed_key=(53,))
    trp, tci, tv, perm = oracle.transpose(lp)
    csc = lp.scipy().tocsc()
    csc.sort_indices()
    assert np.array_equal(trp, csc.indptr) and np.array_equal(tci, csc.indices)
    assert np.array_equal(tv, csc.data)
    assert np.array_equal(lp.val[perm], tv)
    for j in range(lp.n):  # stable: rows increase within every column
        seg = tci[trp[j]:trp[j + 1]]
        assert np.all(np.diff(seg) > 0)


def test_ruiz_equilibrates_rows_and_columns(oracle_lib):
    lp = lpgen.mip_like(300, 700, 4000, seed_key=(54,))
    v, D1, D2 = oracle.precondition(lp, ruiz_iters=40, pock_chambolle=0)
    A = sp.csr_matrix((np.abs(v), lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    rmax = A.max(axis=1).toarray().ravel()
    cmax = A.max(axis=0).toarray().ravel()
    nz_r = np.diff(lp.row_ptr) > 0
    nz_c = np.bincount(lp.col_idx, minlength=lp.n) > 0
    assert np.max(np.abs(rmax[nz_r] - 1)) < 1e-3 and np.max(np.abs(cmax[nz_c] - 1)) < 1e-3
    # the scaled matrix is D1 K D2 with the accumulated diagonals
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    assert np.allclose(v, D1[rows] * lp.val * D2[lp.col_idx], rtol=1e-13, atol=0)


def test_pock_chambolle_norm_bound(oracle_lib):
    # Pock-Chambolle (alpha = 1) guarantees ||D1 K D2||_2 <= 1
    for key in (55, 56):
        lp = lpgen.mip_like(200, 400, 2500, seed_key=(key,))
        for ruiz in (0, 10):
            v, D1, D2 = oracle.precondition(lp, ruiz_iters=ruiz, pock_chambolle=1)
            A = sp.csr_matrix((v, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
            assert np.linalg.norm(A, 2) <= 1 + 1e-12


def test_transform_preserves_objective_and_feasibility(oracle_lib):
    lp = lpgen.small_planted()
    v, D1, D2 = oracle.precondition(lp)
    cs, qs, ls, us = oracle.transform(lp, D1, D2)
    xs = lp.x_star / D2
    ys = lp.y_star / D1
    Ks = sp.csr_matrix((v, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    assert np.isclose(cs @ xs, lp.c @ lp.x_star, rtol=1e-12)
    assert np.isclose(qs @ ys, lp.q @ lp.y_star, rtol=1e-12)
    assert np.all(xs >= ls - 1e-12) and np.all(xs <= us + 1e-12)
    assert np.allclose(Ks @ xs, D1 * (lp.scipy() @ lp.x_star), rtol=1e-11, atol=1e-11)


# ----------------------------------------------------- Section 3.2 gap

def test_normalized_gap_closed_form_without_bounds(oracle_lib):
    rng = np.random.default_rng(3)
    n, m = 7, 5
    x, y = rng.standard_normal(n), rng.standard_normal(m)
    gx, gy = rng.standard_normal(n), rng.standard_normal(m)
    l, u, ylo = np.full(n, -np.inf), np.full(n, np.inf), np.full(m, -np.inf)
    for omega in (0.3, 1.0, 4.0):
        mu, _ = oracle.normalized_gap(x, y, gx, gy, l, u, ylo, omega, 0.7)
        assert np.isclose(mu, np.sqrt(gx @ gx / omega + omega * gy @ gy), rtol=1e-14)


def test_normalized_gap_matches_numerical_optimum(oracle_lib):
    from scipy.optimize import minimize
    rng = np.random.default_rng(7)
    for trial in range(25):
        n, m = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        x = rng.uniform(0, 1, n)
        l = np.where(rng.random(n) < 0.3, -np.inf, 0.0)
        u = np.where(rng.random(n) < 0.3, np.inf, 1.0)
        y = rng.uniform(0, 1, m)
        ylo = np.where(rng.random(m) < 0.5, 0.0, -np.inf)
        gx, gy = rng.standard_normal(n), rng.standard_normal(m)
        omega, r = float(np.exp(rng.uniform(-1, 1))), float(rng.uniform(0.1, 2))
        mu, val = oracle.normalized_gap(x, y, gx, gy, l, u, ylo, omega, r)
        g = np.concatenate([gx, gy])
        lo = np.concatenate([l - x, ylo - y])
        hi = np.concatenate([u - x, np.full(m, np.inf)])
        W = np.concatenate([np.full(n, omega), np.full(m, 1 / omega)])
        best = -np.inf
        for s in range(10):
            d0 = np.clip(rng.standard_normal(n + m) * 0.01, np.maximum(lo, -1), np.minimum(hi, 1))
            res = minimize(lambda d: -g @ d, d0, jac=lambda d: -g, method="SLSQP",
                           bounds=[(a if np.isfinite(a) else None, b if np.isfinite(b) else None)
                                   for a, b in zip(lo, hi)],
                           constraints=[{"type": "ineq", "fun": lambda d: r * r - (W * d * d).sum(),
                                         "jac": lambda d: -2 * W * d}],
                           options={"ftol": 1e-14, "maxiter": 500})
            if res.success and (W * res.x ** 2).sum() <= r * r * (1 + 1e-9):
                best = max(best, g @ res.x)
        assert abs(best - val) <= 1e-7 * max(1.0, abs(val))
        assert np.isclose(mu, val / r)


def test_normalized_gap_zero_radius_is_infinite(oracle_lib):
    mu, _ = oracle.normalized_gap(np.zeros(2), np.zeros(1), np.ones(2), np.ones(1), np.zeros(2),
                                  np.ones(2), np.zeros(1), 1.0, 0.0)
    assert mu == np.inf


def test_normalized_gap_vanishes_at_optimum(oracle_lib):
    # rho_r(z) = 0 iff z is optimal (Section 3.2): at the planted pair the
    # gradient is in the normal cone of Z
    lp = lpgen.small_planted()
    A = lp.scipy()
    gx = A.T @ lp.y_star - lp.c
    gy = lp.q - A @ lp.x_star
    ylo = np.where(lp.ineq == 1, 0.0, -np.inf)
    mu, val = oracle.normalized_gap(lp.x_star, lp.y_star, gx, gy, lp.l, lp.u, ylo, 1.0, 0.5)
    assert abs(val) < 1e-12


# ------------------------------------------------------- Appendix A / E

def test_scale_invariance_of_plain_pdhg(oracle_lib):
    lp = lpgen.planted_uniform(40, 70, 0.1, frac_boxed=0.7, seed_key=(57,))
    gamma, ax, ay = 3.0, 0.25, 5.0
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    x, y = oracle.pdhg_fixed(lp, 0.5, omega, 60)
    import copy
    lp2 = copy.copy(lp)
    lp2.val = gamma * lp.val
    lp2.c = gamma * ay * lp.c
    lp2.q = gamma * ax * lp.q
    lp2.l = ax * lp.l
    lp2.u = ax * lp.u
    omega2 = np.linalg.norm(lp2.c) / np.linalg.norm(lp2.q)
    assert np.isclose(omega2, omega * ay / ax)
    x2, y2 = oracle.pdhg_fixed(lp2, 0.5 / gamma, omega2, 60)
    assert np.allclose(x2, ax * x, rtol=1e-11, atol=1e-12)
    assert np.allclose(y2, ay * y, rtol=1e-11, atol=1e-12)


def test_pagerank_generator_nnz(oracle_lib):
    for nodes in (10, 1000, 20000):
        lp = lpgen.pagerank(nodes, seed_key=(58,))
        assert lp.nnz == 8 * nodes - 18
        colsum = np.asarray(lp.scipy()[:nodes].sum(axis=0)).ravel()
        assert np.allclose(colsum, 1 - 0.85)  # I - 0.85 S' with S' column-stochastic
        assert np.array_equal(lp.scipy()[nodes].toarray().ravel(), np.ones(nodes))  # the 1^T x = 1 row


def test_pagerank_solution_is_power_iteration_vector(oracle_lib):
    nodes = 500
    lp = lpgen.pagerank(nodes, seed_key=(59,))
    G = lp.scipy()[:nodes]
    S = (sp.identity(nodes) - G) / 0.85  # column-stochastic adjacency
    p = np.full(nodes, 1.0 / nodes)
    for _ in range(400):
        p = 0.85 * (S @ p) + 0.15 / nodes
    x, y, r = oracle.solve(lp, iter_limit=400000)
    assert r["status_name"] == "OPTIMAL"
    assert np.abs(x - p).max() <= 1e-6 * p.max() * 50


# ----------------------------------------------- unrolled map (adjoint)

def _small_unroll_lp():
    # c shifted off the planted optimum so that no coordinate starts exactly on
    # a projection kink (an empty column with c_j = 0 would put v_j = l_j)
    lp = lpgen.planted_uniform(25, 40, 0.2, frac_boxed=0.7, seed_key=(60,))
    lp.c = lp.c + 0.05 * np.random.default_rng(60).standard_normal(lp.n)
    return lp


def test_unroll_schedule_satisfies_step_condition(oracle_lib):
    lp = _small_unroll_lp()
    T = 30
    eta, omega, xT, yT = oracle.unroll_schedule(lp, T)
    assert np.all(eta > 0)
    # replay: the forward map with the recorded schedule reproduces the iterate
    x2, y2 = oracle.unroll_forward(lp, eta, omega)
    assert np.allclose(x2, xT, rtol=1e-12, atol=1e-13) and np.allclose(y2, yT, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("ruiz,pc,dirs", [(0, 0, "cqK"), (10, 1, "cq")])
def test_unroll_vjp_matches_finite_differences(oracle_lib, ruiz, pc, dirs):
    # the preconditioner is part of the frozen schedule: K directions are
    # checked without preconditioning (D = I), c and q directions with it
    lp = _small_unroll_lp()
    T = 25
    eta, omega, xT, yT = oracle.unroll_schedule(lp, T, ruiz_iters=ruiz, pock_chambolle=pc)
    rng = np.random.default_rng(11)
    gx, gy = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    dc, dq, dK = oracle.unroll_vjp(lp, eta, omega, gx, gy, ruiz_iters=ruiz, pock_chambolle=pc)
    import copy

    def loss(c, q, val):
        lp2 = copy.copy(lp)
        lp2.c, lp2.q, lp2.val = c, q, val
        x, y = oracle.unroll_forward(lp2, eta, omega, ruiz_iters=ruiz, pock_chambolle=pc)
        return gx @ x + gy @ y

    h = 1e-6
    for _ in range(4):
        vc, vq = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
        vk = rng.standard_normal(lp.nnz) if "K" in dirs else np.zeros(lp.nnz)
        fd = (loss(lp.c + h * vc, lp.q + h * vq, lp.val + h * vk) -
              loss(lp.c - h * vc, lp.q - h * vq, lp.val - h * vk)) / (2 * h)
        an = dc @ vc + dq @ vq + dK @ vk
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_unroll_envelope_gradients_at_optimum(oracle_lib):
    # (preconditioning off so that the K gradient is the plain envelope term)
    # unique (vertex) planted optimum: #interior variables = #tight rows
    rng = np.random.default_rng(12)
    m, n = 6, 10
    A = rng.standard_normal((m, n))
    ineq = np.array([1, 1, 1, 0, 0, 0], np.uint8)
    l, u = np.zeros(n), np.full(n, 4.0)
    interior = np.arange(6)
    x = np.zeros(n)
    x[interior] = rng.uniform(1, 3, 6)
    x[6:8] = 0.0
    x[8:] = 4.0
    lam = np.zeros(n)
    lam[6:8] = rng.uniform(0.5, 1, 2)
    lam[8:] = -rng.uniform(0.5, 1, 2)
    y = np.concatenate([rng.uniform(0.5, 1, 3), rng.standard_normal(3)])
    q = A @ x
    c = A.T @ y + lam
    Asp = sp.csr_matrix(A)
    lp = lpgen.LP(m=m, n=n, row_ptr=Asp.indptr.astype(np.int32), col_idx=Asp.indices.astype(np.int32),
                  val=Asp.data, c=c, q=q, l=l, u=u, ineq=ineq)
    T = 30000
    eta, omega, xT, yT = oracle.unroll_schedule(lp, T, x0=x, y0=y, ruiz_iters=0, pock_chambolle=0)
    assert np.allclose(xT, x, atol=1e-10)
    # L = c^T x_T: dL/dq -> y* (envelope), dL/dc -> x* (explicit term; J_c^T c -> 0)
    dc, dq, dK = oracle.unroll_vjp(lp, eta, omega, c, None, x0=x, y0=y, ruiz_iters=0, pock_chambolle=0)
    assert np.allclose(dq, y, atol=1e-6)
    assert np.allclose(dc + xT, x, atol=1e-6)
    rows = np.repeat(np.arange(m), np.diff(lp.row_ptr))
    assert np.allclose(dK, -y[rows] * x[lp.col_idx], atol=1e-6)


# ------------------------------------------- refinement correction problem

def test_correction_problem_maps_back_to_optimum(oracle_lib):
    lp = lpgen.planted_uniform(80, 150, 0.06, frac_boxed=0.6, seed_key=(61,))
    rng = np.random.default_rng(13)
    xh = np.clip(lp.x_star + 1e-3 * rng.standard_normal(lp.n), lp.l, lp.u)
    yh = lp.y_star + 1e-3 * rng.standard_normal(lp.m)
    yh[lp.ineq == 1] = np.maximum(yh[lp.ineq == 1], 0.0)
    cor = oracle.correction_lp(lp, xh, yh)
    assert cor["dP"] > 1 and cor["dD"] > 1
    import copy
    lpc = copy.copy(lp)
    lpc.c, lpc.q, lpc.l, lpc.u = cor["c"], cor["q"], cor["l"], cor["u"]
    a, b, r = oracle.solve(lpc, ylo=cor["ylo"], eps=1e-10)
    assert r["status_name"] == "OPTIMAL"
    x = xh + a / cor["dP"]
    y = yh + b / cor["dD"]
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-8 * (1 + abs(ref))


# ------------------------------------------ constant step (baseline PDHG)

@pytest.mark.parametrize("ruiz,pc", [(0, 0), (10, 1)])
def test_power_norm_is_the_spectral_norm(oracle_lib, ruiz, pc):
    # Section 2: ||K||_2 by power iteration; against the dense SVD
    lp = lpgen.planted_uniform(40, 70, 0.15, seed_key=(90,))
    est = oracle.power_norm(lp, ruiz, pc)
    v, D1, D2 = oracle.precondition(lp, ruiz, pc)
    Ks = sp.csr_matrix((v, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    true = np.linalg.norm(Ks, 2)
    # from below, error ~ (s2/s1)^(2 iters); after scaling s2/s1 ~ 0.987 here
    assert est <= true * (1 + 1e-12)
    assert est >= true * (1 - 1e-5)


def test_constant_step_solve_is_plain_pdhg(oracle_lib):
    # step_policy 1 without restarts, primal-weight updates or scaling is
    # PDHG of Eq. (3) with eta = 0.9 / ||K||_2 at every step
    lp = lpgen.planted_uniform(30, 50, 0.2, seed_key=(91,))
    T = 150
    kw = dict(ruiz_iters=0, pock_chambolle=0, adaptive_restart=0, pw_update=0, step_policy=1, omega0=1.0)
    x, y, r = oracle.solve(lp, iter_limit=T, eps=0.0, **kw)
    eta = 0.9 / oracle.power_norm(lp, 0, 0)
    assert r["iters"] == T and r["kkt_passes"] == T
    assert r["eta"] == pytest.approx(eta, rel=1e-15) and r["omega"] == 1.0
    x2, y2 = oracle.pdhg_fixed(lp, eta, 1.0, T)
    assert np.allclose(x, x2, rtol=1e-11, atol=1e-12) and np.allclose(y, y2, rtol=1e-11, atol=1e-12)


def test_malitsky_pock_without_search_is_plain_pdhg(oracle_lib):
    # Appendix C.1 with interpolation 0 (eta_hat = eta_k, theta_hat = 1) and a
    # breaking factor no trial can fail is PDHG of Eq. (3) at the initial step
    # 1 / max |K_ij| (Algorithm 1's eta^0): one trial per iteration
    lp = lpgen.planted_uniform(30, 50, 0.2, seed_key=(91,))
    T = 150
    kw = dict(ruiz_iters=0, pock_chambolle=0, adaptive_restart=0, pw_update=0, step_policy=2, omega0=1.0,
              mp_interpolation=0.0, mp_breaking=1e300)
    x, y, r = oracle.solve(lp, iter_limit=T, eps=0.0, **kw)
    eta = 1.0 / np.max(np.abs(lp.val))
    assert r["iters"] == T and r["kkt_passes"] == T
    assert r["eta"] == eta
    x2, y2 = oracle.pdhg_fixed(lp, eta, 1.0, T)
    assert np.allclose(x, x2, rtol=1e-11, atol=1e-12) and np.allclose(y, y2, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_malitsky_pock_solves_planted_lp(oracle_lib, seed):
    # the paper's best setting (breaking 1, downscaling 0.5, interpolation 0.4)
    # inside PDLP converges to the planted optimum; its trials outnumber its
    # iterations (some candidate steps are shrunk)
    lp = lpgen.planted_uniform(60, 150, 0.08, seed_key=(95 + seed,))
    x, y, r = oracle.solve(lp, step_policy=2, iter_limit=200000)
    assert r["status_name"] == "OPTIMAL", r
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-6 * (1 + abs(ref))
    assert r["kkt_passes"] > r["iters"]


def test_malitsky_pock_breaking_factor_zero_never_accepts(oracle_lib):
    # breaking factor 0 accepts only a trial with K^T(y_hat - y) = 0, which a
    # dual step that moves y cannot give here: every trial is shrunk until the
    # pass limit ends the solve
    lp = lpgen.planted_uniform(30, 50, 0.2, seed_key=(92,))
    _, _, r = oracle.solve(lp, step_policy=2, mp_breaking=0.0, kkt_pass_limit=25)
    assert r["status_name"] == "KKT_PASS_LIMIT" and r["iters"] == 0 and r["kkt_passes"] == 25


def test_no_restart_mode_updates_primal_weight_at_doubling_iterations(oracle_lib):
    # Appendix C.2: without restarts the primal weight still changes where the
    # artificial criterion t >= 0.5 k would fire, i.e. at k = 40, 80, 160, ...
    lp = lpgen.planted_uniform(80, 200, 0.05, seed_key=(93,))
    _, _, r, tr = oracle.solve_traced(lp, adaptive_restart=0, iter_limit=1300, eps=0.0)
    assert r["restarts"] == 0
    ks = [int(row[0]) for row in tr if row[6] == 2.0]
    assert ks == [40, 80, 160, 320, 640, 1280]
    om = [row[7] for row in tr if row[6] == 2.0]
    assert len(set(om)) > 1
    _, _, r0, tr0 = oracle.solve_traced(lp, adaptive_restart=0, pw_update=0, iter_limit=1300, eps=0.0)
    assert len(tr0) == 0 and r0["omega"] == oracle.solve(lp, iter_limit=1)[2]["omega"]


def test_theory_restart_mode_restarts_to_average(oracle_lib):
    # Appendix C.2 theory mode: beta_suff = beta_nec = 0.37 and the average as
    # the only restart candidate; every restart then has mu <= 0.37 mu_0 or
    # passes the artificial test
    lp = lpgen.planted_uniform(80, 200, 0.05, seed_key=(94,))
    x, y, r, tr = oracle.solve_traced(lp, restart_to_current=0, beta_suff=0.37, beta_nec=0.37,
                                      iter_limit=200000)
    assert r["status_name"] == "OPTIMAL" and r["restarts"] > 0
    assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-8
    rows = [row for row in tr if row[6] == 1.0]
    assert rows and all(row[5] == 1.0 for row in rows)
    for row in rows:
        k, t, mu_avg, mu0 = row[0], row[1], row[3], row[4]
        assert mu_avg <= 0.37 * mu0 or t >= 0.5 * k

"""Parity at the benchmark sizes, in the launch configuration the benchmark
times (persistent step kernel inside one CUDA graph per solve): the
100k x 250k MIP-shaped LP, the 1M-node PageRank LP, the 4096-LP batch and the
20k x 50k unrolled map with T = 500, checkpoint 50.  Checks are ones the
oracle can afford at these sizes: bit-exact preprocessing, the first
iterates, Eq. (15) at returned points, sampled batch members and the full
adjoint."""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mip():
    return lpgen.mip_relaxation_100k()


U64 = 2.0 ** -53  # unit roundoff of float64


def eq15_rounding_bounds(lp, x, y):
    """Bounds on the rounding error of one float64 evaluation of the relative
    Eq. (15) terms at (x, y), from the standard bound on a computed sum of k
    products, |fl(s) - s| <= k u sum |terms|: row i of q - K x errs by at most
    (len_i + 8) u (|q_i| + (|K||x|)_i), column j of c - K^T y by
    (len_j + 8) u (|c_j| + (|K^T||y|)_j) (the 8 covers the diagonal scalings
    and their inverses), and the projections onto the bounds are 1-Lipschitz;
    the objectives take the analogous sums.  Two evaluations of the same
    point in different summation orders differ by at most twice this."""
    K = lp.scipy()
    aK = abs(K)
    ax, ay = np.abs(x), np.abs(y)
    row_len = np.diff(K.indptr)
    col_len = np.bincount(K.indices, minlength=lp.n)
    ep = (row_len + 8) * U64 * (np.abs(lp.q) + aK @ ax)
    rc = lp.c - K.T @ y
    ed = 2 * (col_len + 8) * U64 * (np.abs(lp.c) + aK.T @ ay)
    fin_l = np.where(np.isfinite(lp.l), np.abs(lp.l), 0.0)
    fin_u = np.where(np.isfinite(lp.u), np.abs(lp.u), 0.0)
    e_pobj = (lp.n + 8) * U64 * float(np.abs(lp.c) @ ax)
    e_dobj = ((lp.m + lp.n + 8) * U64 * (float(np.abs(lp.q) @ ay) + float((fin_l + fin_u) @ np.abs(rc)))
              + float((fin_l + fin_u) @ ed))
    pobj = float(lp.c @ x)
    return {"rel_pres": float(np.linalg.norm(ep)) / (1 + np.linalg.norm(lp.q)),
            "rel_dres": float(np.linalg.norm(ed)) / (1 + np.linalg.norm(lp.c)),
            "rel_gap": 2 * (e_pobj + e_dobj) / (1 + abs(pobj))}


def test_mip100k_preprocessing_is_bit_exact(gpu_lib, oracle_lib, mip):
    lp = mip
    with P.Context.from_lp(lp) as ctx:
        g = ctx.get_scaled()
    trp, tci, _, perm = oracle.transpose(lp)
    assert np.array_equal(g["KT_row_ptr"], trp) and np.array_equal(g["KT_col_idx"], tci)
    assert np.array_equal(g["KT_perm"], perm)
    v, D1, D2 = oracle.precondition(lp)
    assert np.array_equal(g["Kval"], v) and np.array_equal(g["KTval"], v[perm])
    assert np.array_equal(g["D1"], D1) and np.array_equal(g["D2"], D2)
    cs, qs, ls, us = oracle.transform(lp, D1, D2)
    for k, ref in (("cs", cs), ("qs", qs), ("ls", ls), ("us", us)):
        assert np.array_equal(g[k], ref), k


@pytest.mark.parametrize("iters", [20, 40])
def test_mip100k_first_iterates_match_oracle(gpu_lib, oracle_lib, mip, iters):
    lp = mip
    x_g, y_g, r_g = P.solve(lp, iter_limit=iters)
    x_o, y_o, r_o = oracle.solve(lp, iter_limit=iters)
    assert r_g["iters"] == r_o["iters"] == iters
    assert r_g["kkt_passes"] == r_o["kkt_passes"] and r_g["restarts"] == r_o["restarts"]
    tol = {20: 1e-9, 40: 1e-8}[iters]
    assert np.abs(x_g - x_o).max() <= tol * max(1.0, np.abs(x_o).max())
    assert np.abs(y_g - y_o).max() <= tol * max(1.0, np.abs(y_o).max())


@pytest.mark.parametrize("prec", [P.PDLP_FP64, P.PDLP_FP32])
def test_mip100k_reported_terms_are_those_of_the_returned_point(gpu_lib, oracle_lib, mip, prec):
    lp = mip
    # float64: the device's Eq. (15) terms are the oracle's at the returned
    # point up to summation order; float32: the device evaluates them from
    # its float32 products K x, K^T y, so they agree to float32 accuracy
    x, y, r = P.solve(lp, precision=prec, iter_limit=2000)
    k = oracle.kkt(lp, x, y)
    ta, tr = (1e-9, 1e-6) if prec == P.PDLP_FP64 else (1e-5, 1e-3)
    for key in ("primal_obj", "dual_obj"):
        assert abs(r[key] - k[key]) <= ta * (1 + abs(k[key])), (key, r[key], k[key])
    for key in ("rel_gap", "rel_pres", "rel_dres"):
        assert abs(r[key] - k[key]) <= tr * k[key] + 1e-12, (key, r[key], k[key])


@pytest.fixture(scope="module")
def pagerank():
    return lpgen.pagerank_1m()


def _pagerank_vector(lp):
    """The damped PageRank vector by power iteration (Appendix E: the LP's
    unique feasible point)."""
    nodes = lp.n
    G = lp.scipy()[:nodes]
    S = ((sp.identity(nodes) - G) / 0.85).tocsr()
    p = np.full(nodes, 1.0 / nodes)
    for _ in range(200):
        p = 0.85 * (S @ p) + 0.15 / nodes
    return p


def _check_near_pagerank(lp, x, eps=1e-8, damping=0.85):
    """x against the PageRank vector p (power iteration), within the distance
    that Eq. (15) at eps implies.  With G = I - damping S' (the inequality
    rows; S' column-stochastic, so G's column sums are 1 - damping and
    ||G^{-1}||_1 = 1 / (1 - damping)), the slack s = G x - q_G, its negative
    part v and e = 1 - sum(x): G (x - p) = s, sum(s) = -(1 - damping) e, so
    ||s||_1 = 2 ||v||_1 - (1 - damping) e, and Eq. (15)'s primal residual
    bounds sqrt(||v||^2 + e^2) by eps (1 + ||q||_2); hence
    ||x - p||_1 <= eps (1 + ||q||_2) (2 sqrt(n) + 1 - damping) / (1 - damping).
    (On a million-node graph that allows entries of x, about 1e-6, to move
    by percents: Eq. (15) is absolute there.)"""
    nodes = lp.n
    p = _pagerank_vector(lp)
    bound = eps * (1 + np.linalg.norm(lp.q)) * (2 * np.sqrt(nodes) + 1 - damping) / (1 - damping)
    d = np.abs(x - p).sum()
    assert d <= bound, (d, bound)
    return d


def test_pagerank_1m_float64_to_1e8(gpu_lib, oracle_lib, pagerank):
    """The float64 solve the benchmark times (persistent kernel with gathers
    through L1): Eq. (15) at 1e-8 by the oracle's evaluation of the returned
    point, the terms the device reports equal to the oracle's, and the
    PageRank vector."""
    lp = pagerank
    x, y, r = P.solve(lp, precision=P.PDLP_FP64)
    assert r["status_name"] == "OPTIMAL", r
    assert r["engine"] == 1
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    # the device's terms and the oracle's: two float64 evaluations of one point
    b = eq15_rounding_bounds(lp, x, y)
    for key in ("rel_gap", "rel_pres", "rel_dres"):
        assert abs(r[key] - k[key]) <= 2 * b[key] + 1e-12 * k[key], (key, r[key], k[key], b[key])
    # the sum row's residual is one entry of r, and Eq. (15) at 1e-8 bounds
    # ||r||_2 by 1e-8 (1 + ||q||_2)
    assert abs(x.sum() - 1.0) <= 1e-8 * (1 + np.linalg.norm(lp.q))
    _check_near_pagerank(lp, x)


def test_pagerank_1m_float32_refinement_to_1e8(gpu_lib, oracle_lib, pagerank):
    lp = pagerank
    x, y, r = P.solve(lp, precision=P.PDLP_FP32_REFINE)
    assert r["status_name"] == "OPTIMAL", r
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    assert abs(x.sum() - 1.0) <= 1e-8 * (1 + np.linalg.norm(lp.q))
    _check_near_pagerank(lp, x)


@pytest.mark.parametrize("inner_tol", [1e-7, 1e-5])
def test_pagerank_100k_float32_refinement_to_1e8(gpu_lib, oracle_lib, inner_tol):
    """The 100k-node PageRank LP (Table 2's family), where float32 PDLP alone
    never reaches 1e-8: refinement (with its float64 finish when the float32
    rounds stall) must end OPTIMAL by the oracle's Eq. (15) within the default
    budget, with the default first-round tolerance and with 1e-5 (whose second
    round stalls at 7.9e-6, so that the float64 finish does the last digits)."""
    lp = lpgen.pagerank(100_000, seed_key=(2, 1), name="pagerank_100k")
    x, y, r = P.solve(lp, precision=P.PDLP_FP32_REFINE, inner_tol=inner_tol)
    assert r["status_name"] == "OPTIMAL", r
    assert r["iters"] <= 1_000_000 and r["finish_iters"] <= r["iters"]
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    _check_near_pagerank(lp, x)


def test_batch_4096_sampled_members_match_oracle(gpu_lib, oracle_lib):
    lps = lpgen.batch_4096()
    cap = 20000
    xs, ys, rs = P.solve_batch(lps, rel_tol=1e-6, iter_limit=cap)
    rng = np.random.default_rng(20210609)
    solved = [b for b in range(len(lps)) if rs[b]["status_name"] == "OPTIMAL"]
    unsolved = [b for b in range(len(lps)) if rs[b]["status_name"] != "OPTIMAL"]
    assert len(solved) >= 0.9 * len(lps)
    for b in rng.choice(solved, 64, replace=False):
        lp = lps[b]
        k = oracle.kkt(lp, xs[b], ys[b])
        assert k["rel_kkt"] <= 1e-6, (b, k)
        ref = lp.c @ lp.x_star
        assert abs(lp.c @ xs[b] - ref) <= 1e-5 * (1 + abs(ref)), (b, lp.c @ xs[b], ref)
    # members stopped by the cap are slow for the method itself: the oracle
    # also needs most of the cap (or more) on them
    for b in rng.choice(unsolved, min(8, len(unsolved)), replace=False):
        assert rs[b]["status_name"] == "ITER_LIMIT" and rs[b]["iters"] == cap
        _, _, ro = oracle.solve(lps[b], eps=1e-6, iter_limit=cap)
        assert ro["status_name"] == "ITER_LIMIT" or ro["iters"] >= cap // 4, (b, ro["iters"])


@pytest.mark.parametrize("ruiz,pc,dirs,tol", [(0, 0, "cqK", 1e-5), (10, 1, "cq", 1e-3)])
def test_unroll_20k_adjoint_matches_central_differences(gpu_lib, oracle_lib, ruiz, pc, dirs, tol):
    """Central differences (h = 1e-6) of the unrolled map at the 20k x 50k
    size against the library's adjoint (pdlp_grad), along random directions in
    c, q and (without preconditioning, which the adjoint holds fixed) the
    nonzeros of K.  T = 150: at T = 500 this map amplifies rounding by about
    1e20 (two float64 evaluations of the same map differ by 0.2 in x_T), so
    differences of size h measure chaos there, not the derivative; at T = 150
    they agree with the adjoint to 1e-7..1e-6 (no preconditioning) and
    3e-5..1e-4 (Ruiz + Pock-Chambolle, whose derivatives reach 1e21)."""
    lp = lpgen.unroll_20k()
    boxed = np.isfinite(lp.l) & np.isfinite(lp.u)
    lp.c = lp.c + 0.05 * np.random.default_rng(4).standard_normal(lp.n) * boxed
    T = 150
    target = np.random.default_rng(5).standard_normal(lp.n)
    with P.Context.from_lp(lp, ruiz_iters=ruiz, pock_chambolle=pc) as ctx:
        x, _, eta = ctx.unroll(T, 50)
        dc, dq, dK = ctx.grad(x - target, None)
    omega = oracle.unroll_schedule(lp, 1, ruiz_iters=ruiz, pock_chambolle=pc)[1]

    def loss(c, q, val):
        lp2 = copy.copy(lp)
        lp2.c, lp2.q, lp2.val = c, q, val
        xx, _ = oracle.unroll_forward(lp2, eta, omega, ruiz_iters=ruiz, pock_chambolle=pc)
        return 0.5 * np.sum((xx - target) ** 2)

    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(3):
        vc, vq = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
        vk = rng.standard_normal(lp.nnz) if "K" in dirs else np.zeros(lp.nnz)
        fd = (loss(lp.c + h * vc, lp.q + h * vq, lp.val + h * vk) -
              loss(lp.c - h * vc, lp.q - h * vq, lp.val - h * vk)) / (2 * h)
        an = dc @ vc + dq @ vq + dK @ vk
        assert abs(fd - an) <= tol * abs(an), (fd, an)


def test_unroll_20k_T500_adjoint_matches_oracle(gpu_lib, oracle_lib):
    lp = lpgen.unroll_20k()
    # move c off the planted optimum only on boxed columns: any reduced cost
    # is dual feasible there, so the LP keeps an optimum (a perturbation of a
    # free column's cost makes it unbounded, the iterates grow without limit
    # and the adjoint of the unrolled map with them)
    boxed = np.isfinite(lp.l) & np.isfinite(lp.u)
    lp.c = lp.c + 0.05 * np.random.default_rng(4).standard_normal(lp.n) * boxed
    T = 500
    target = np.random.default_rng(5).standard_normal(lp.n)
    with P.Context.from_lp(lp) as ctx:
        x, _, eta = ctx.unroll(T, 50)
        dc, dq, dK = ctx.grad(x - target, None)
    omega = oracle.unroll_schedule(lp, 1)[1]
    x2, _ = oracle.unroll_forward(lp, eta, omega)
    assert np.linalg.norm(x - x2) <= 1e-9 * np.linalg.norm(x2)
    rc, rq, rk = oracle.unroll_vjp(lp, eta, omega, x - target, None)
    for a, b in ((dc, rc), (dq, rq), (dK, rk)):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)

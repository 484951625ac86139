"""The ablation modes of Appendix C on the GPU against the oracle: the
Malitsky-Pock line search (step_policy 2, Appendix C.1), the no-restart mode
with primal weight updates at the would-be artificial restarts and the
"adaptive restart (theory)" mode (Appendix C.2), on the single-LP path and in
the batched solve."""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu

MP = dict(step_policy=2)
THEORY = dict(restart_to_current=0, beta_suff=0.37, beta_nec=0.37)


def _dense_row(m=300, n=6000, seed=70):
    """One row split into several segments plus a ragged tail of short rows."""
    base = lpgen.planted_uniform(m, n, 0.003, frac_boxed=0.8, seed_key=(seed,))
    A = base.scipy().tolil()
    A[0, :] = np.random.default_rng(seed).standard_normal(n)
    A = A.tocsr()
    A.sort_indices()
    return lpgen._plant(lpgen.rng_for(seed, 1), m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32),
                        A.data, base.ineq, base.l, base.u, "dense_row")


CASES = {
    "planted_200x500": lambda: lpgen.small_planted(),
    "mip_2000x5000": lambda: lpgen.mip_like(2000, 5000, 30000, seed_key=(71,)),
    "dense_row": _dense_row,
}


def _close(a, b, tol):
    assert np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max()), np.abs(a - b).max()


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_malitsky_pock_first_iterates_match_oracle(gpu_lib, oracle_lib, name, use_graph):
    """Same trials, same acceptances: iteration and trial counts equal, the
    iterates equal up to rounding growth, over the first 60 iterations (one
    evaluation with its restart decision inside)."""
    lp = CASES[name]()
    x_g, y_g, r_g = P.solve(lp, iter_limit=60, use_graph=use_graph, **MP)
    x_o, y_o, r_o = oracle.solve(lp, iter_limit=60, **MP)
    assert r_g["iters"] == r_o["iters"] == 60
    assert r_g["kkt_passes"] == r_o["kkt_passes"] and r_g["kkt_passes"] > 60
    assert r_g["restarts"] == r_o["restarts"]
    assert r_g["step_size"] == pytest.approx(r_o["eta"], rel=1e-9)
    _close(x_g, x_o, 1e-8)
    _close(y_g, y_o, 1e-8)


def test_malitsky_pock_without_search_is_plain_pdhg(gpu_lib, oracle_lib):
    """Interpolation 0 and a breaking factor no trial fails: Eq. (3) at
    eta^0 = 1 / max |K_ij| with omega = 1 (no scaling, no restarts)."""
    lp = lpgen.planted_uniform(200, 500, 0.02, seed_key=(73,))
    kw = dict(step_policy=2, mp_interpolation=0.0, mp_breaking=1e300, omega0=1.0, adaptive_restart=0,
              pw_update=0, ruiz_iters=0, pock_chambolle=0)
    x, y, r = P.solve(lp, iter_limit=200, rel_tol=0.0, **kw)
    eta = 1.0 / np.max(np.abs(lp.val))
    assert r["iters"] == r["kkt_passes"] == 200 and r["step_size"] == eta
    x2, y2 = oracle.pdhg_fixed(lp, eta, 1.0, 200)
    _close(x, x2, 1e-10)
    _close(y, y2, 1e-10)


@pytest.mark.parametrize("prec", [P.PDLP_FP64, P.PDLP_FP32_REFINE])
def test_malitsky_pock_solves_to_1e8(gpu_lib, oracle_lib, prec):
    lp = lpgen.small_planted()
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, precision=prec, **MP)
    assert r["status_name"] == "OPTIMAL", r
    assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-8
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-6 * (1 + abs(ref))
    if prec == P.PDLP_FP64:
        _, _, ro = oracle.solve(lp, iter_limit=200000, **MP)
        assert ro["status_name"] == "OPTIMAL"
        # trajectories part after the first restarts; the work stays alike
        assert 0.5 <= r["kkt_passes"] / ro["kkt_passes"] <= 2.0, (r["kkt_passes"], ro["kkt_passes"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_no_restart_mode_updates_primal_weight_like_the_oracle(gpu_lib, oracle_lib, name):
    """adaptive_restart = 0 with pw_update = 1: the primal weight changes at
    k = 40, 80, 160, 320 (trace records with restarted = 2), never restarts,
    and matches the oracle's weights while the iterates still agree."""
    lp = CASES[name]()
    iters = 330
    _, _, r_o, tr_o = oracle.solve_traced(lp, iter_limit=iters, adaptive_restart=0)
    with P.Context.from_lp(lp, iter_limit=iters, adaptive_restart=0) as ctx:
        _, _, r_g = ctx.solve()
        tr_g = ctx.get_trace()
    assert r_g["restarts"] == r_o["restarts"] == 0
    ks_g = [int(a[0]) for a in tr_g if a[6] == 2.0]
    ks_o = [int(b[0]) for b in tr_o if b[6] == 2.0]
    assert ks_g == ks_o and len(ks_o) >= 3  # fewer when the solve ends first
    assert ks_o == [40, 80, 160, 320][:len(ks_o)]
    om_g = [a[7] for a in tr_g if a[6] == 2.0]
    om_o = [b[7] for b in tr_o if b[6] == 2.0]
    for e in range(2):
        assert abs(om_g[e] - om_o[e]) <= 1e-6 * abs(om_o[e]), (e, om_g[e], om_o[e])
    assert r_g["primal_weight"] == pytest.approx(r_o["omega"], rel=5e-2)


def test_no_restart_mode_solves_to_1e8(gpu_lib, oracle_lib):
    lp = lpgen.small_planted()
    for persistent in (1, 0):
        x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, adaptive_restart=0, persistent=persistent)
        assert r["status_name"] == "OPTIMAL" and r["restarts"] == 0, r
        assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-8


@pytest.mark.parametrize("name", sorted(CASES))
def test_theory_restart_mode_matches_oracle(gpu_lib, oracle_lib, name):
    """restart_to_current = 0, beta_suff = beta_nec = 0.37: every restart goes
    to the average, decisions agree with the oracle evaluation by evaluation
    (up to a near tie in mu)."""
    lp = CASES[name]()
    iters = 200
    _, _, r_o, tr_o = oracle.solve_traced(lp, iter_limit=iters, **THEORY)
    with P.Context.from_lp(lp, iter_limit=iters, **THEORY) as ctx:
        _, _, r_g = ctx.solve()
        tr_g = ctx.get_trace()
    assert all(a[5] == 1.0 for a in tr_g if a[6] == 1.0)
    n = min(len(tr_o), len(tr_g), 4)
    assert n >= 3
    for e, (a, b) in enumerate(zip(tr_g[:n], tr_o[:n])):
        tol = 1e-6 if e < 2 else 5e-2
        assert a[0] == b[0] and a[1] == b[1], (a[:2], b[:2])
        mu0, mu_a = b[4], b[3]
        if np.isfinite(mu0) and abs(mu_a - 0.37 * mu0) <= 2 * tol * abs(mu_a):
            break
        assert a[6] == b[6], (a, b)


def test_theory_restart_mode_solves_to_1e8(gpu_lib, oracle_lib):
    lp = lpgen.small_planted()
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, **THEORY)
    assert r["status_name"] == "OPTIMAL" and r["restarts"] > 0, r
    assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-8


@pytest.mark.parametrize("mode", ["theory", "no_restart"])
def test_batch_restart_modes(gpu_lib, oracle_lib, mode):
    kw = THEORY if mode == "theory" else dict(adaptive_restart=0)
    lps = lpgen.batch_planted(count=24, m_range=(20, 120), n_range=(50, 300), seed_key=(77,))
    xs, ys, rs = P.solve_batch(lps, rel_tol=1e-6, iter_limit=100000, **kw)
    solved = 0
    for lp, x, y, r in zip(lps, xs, ys, rs):
        if r["status_name"] != "OPTIMAL":
            continue
        solved += 1
        assert oracle.kkt(lp, x, y)["rel_kkt"] <= 1e-6
        if mode == "no_restart":
            assert r["restarts"] == 0
    assert solved >= 20, [r["status_name"] for r in rs]


def test_batch_rejects_the_line_search(gpu_lib):
    lps = lpgen.batch_planted(count=2, m_range=(20, 40), n_range=(50, 80), seed_key=(78,))
    with pytest.raises(P.PdlpError) as e:
        P.solve_batch(lps, step_policy=2)
    assert e.value.code == P.PDLP_ERR_INVALID_ARG


def test_line_search_option_checks(gpu_lib):
    lp = lpgen.small_planted()
    for bad in (dict(step_policy=3), dict(step_policy=2, mp_downscaling=1.0), dict(step_policy=2, mp_downscaling=0.0),
                dict(step_policy=2, mp_interpolation=1.5), dict(step_policy=2, mp_breaking=-1.0),
                dict(step_policy=2, unroll_T=10), dict(restart_to_current=2)):
        with pytest.raises(P.PdlpError) as e:
            P.Context.from_lp(lp, **bad)
        assert e.value.code == P.PDLP_ERR_INVALID_ARG, bad

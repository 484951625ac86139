"""Hand-worked pins of the oracle's scalar logic (no GPU).

Algorithm 2 (adaptive step size), Algorithm 3 (primal weight update) and the
restart criteria of Section 3.2 are checked against values worked out by hand
for small cases, so that a swapped exponent, a dropped "+1" in the step count,
a signed instead of absolute interaction term, an inverted Delta_y / Delta_x
ratio, a restart criterion that ignores the previous candidate or a mu_0
taken under the old primal weight each fail a test here.  The expected
numbers below come from the paper's formulas evaluated by hand for the
stated inputs; the derivations are in the comments.
"""
import math
import os

import numpy as np
import pytest

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


# ------------------------------------------------------------ Algorithm 2

def test_step_exponents_are_the_papers(oracle_lib):
    """Algorithm 2's factors (1 - (k+1)^-0.3) and (1 + (k+1)^-0.6), with the
    exponents read from the constants file: at the first step (step number
    k = 1, R11) an attempt with infinite eta_bar grows eta by 1 + 2^-0.6, and
    one with eta_bar = 1 and a huge eta shrinks it to 1 - 2^-0.3."""
    g = _golden_constants()
    red, gro = g["step_reduction_exponent"], g["step_growth_exponent"]
    assert (red, gro) == (0.3, 0.6)
    _, en = oracle.step_sizes(1.0, 1.0, 1.0, 0.0, 1.0, 0)     # inter = 0: eta_bar = +inf
    assert en == pytest.approx(1.0 + 2.0 ** -gro, rel=1e-15)
    # omega = 1, dx2 = dy2 = 1, inter = 1: eta_bar = (1 + 1) / 2 = 1
    eb, en = oracle.step_sizes(1.0, 1.0, 1.0, 1.0, 1e9, 0)
    assert eb == 1.0
    assert en == pytest.approx(1.0 - 2.0 ** -red, rel=1e-15)


@pytest.mark.parametrize("k", [0, 1, 5])
def test_step_sizes_hand_cases(oracle_lib, k):
    """omega = 2, ||dx||^2 = 1, ||dy||^2 = 4: ||dz||_omega^2 = 2*1 + 4/2 = 4.
    inter = 0.5 or -0.5 (R5: the magnitude is used): eta_bar = 4 / (2*0.5) = 4.
    The step being taken is number k + 1, so the factors use (k + 2):
      eta = 1:    growth (1 + (k+2)^-0.6) * 1 = 1.660, 1.517, 1.311 against
                  reduction (1 - (k+2)^-0.3) * 4 = 0.751, 1.123, 1.769 for
                  k = 0, 1, 5: the reduction wins at k = 0, 1, the growth at 5,
      eta = 100:  the reduction wins."""
    growth = {0: 1.659753955386447, 1: 1.5172818579717866, 5: 1.3111294892118257}
    reduction4 = {0: 0.7509904145750577, 1: 1.1231076267005426, 5: 1.7688406987870158}
    expect_eta1 = {0: reduction4[0], 1: reduction4[1], 5: growth[5]}
    for inter in (0.5, -0.5):
        eb, en = oracle.step_sizes(2.0, 1.0, 4.0, inter, 1.0, k)
        assert eb == 4.0
        assert en == pytest.approx(expect_eta1[k], rel=1e-14)
        eb, en = oracle.step_sizes(2.0, 1.0, 4.0, inter, 100.0, k)
        assert en == pytest.approx(reduction4[k], rel=1e-14)
    # the worked numbers are the formulas' values at k + 2
    for kk, v in growth.items():
        assert v == pytest.approx(1 + (kk + 2) ** -0.6, rel=1e-15)
    for kk, v in reduction4.items():
        assert v == pytest.approx(4 * (1 - (kk + 2) ** -0.3), rel=1e-15)


def _one_by_one():
    """minimise 2 x  s.t.  x >= 1 (one inequality row, K = [1]),  x >= 0."""
    return lpgen.LP(m=1, n=1, row_ptr=np.array([0, 1], np.int32), col_idx=np.array([0], np.int32),
                    val=np.array([1.0]), c=np.array([2.0]), q=np.array([1.0]), l=np.array([0.0]),
                    u=np.array([np.inf]), ineq=np.array([1], np.uint8), name="one_by_one")


@pytest.mark.parametrize("steps,eta_hat,passes", [
    # Without preconditioning K~ = 1, omega^0 = ||c|| / ||q|| = 2, eta^0 = 1 / max|K| = 1,
    # z = 0.  Step 1: x' = max(0, 0 - (1/2)(2 - 0)) = 0, y' = max(0, 0 + 1*2*(1 - 0 + 0)) = 2,
    #   dx = 0 so (y'-y)^T K (x'-x) = 0: eta_bar = inf, accepted, eta' = (1 + 2^-0.6) * 1.
    (1, 1.659753955386447, 1),
    # Step 2 (eta = 1.6598): c - K^T y = 0 so x' = 0 again, y' = 2 + 2 eta = 5.3195,
    #   eta_bar = inf, eta' = (1 + 3^-0.6) * 1.6598 = 2.5183.
    (2, 2.5183145652047703, 2),
    # Step 3 (eta = 2.5183): x' = (2.5183 / 2)(5.3195 - 2) = 4.1798, K x' = 4.1798,
    #   y' = max(0, 5.3195 + 2.5183*2*(1 - 2*4.1798 + 0)) = 0; dx = 4.1798, dy = -5.3195,
    #   inter = -22.234; eta_bar = (2*4.1798^2 + 5.3195^2/2) / (2*22.234) = 1.10392 < eta:
    #   rejected, eta' = min((1 - 4^-0.3) 1.10392, (1 + 4^-0.6) 2.5183) = 0.375603.
    #   Retry: x' = (0.375603/2)(3.3195) = 0.623408, y' = 5.3195 + 0.751205(1 - 1.246816)
    #   = 5.134098, dx = 0.623408, dy = -0.185410, inter = -0.115586,
    #   eta_bar = (2*0.388637 + 0.034377/2) / 0.231172 = 3.43668 >= 0.375603: accepted,
    #   eta' = min((1 - 4^-0.3) 3.43668, (1 + 4^-0.6) 0.375603) = 0.539093.  4 passes.
    (3, 0.5390933040726132, 4),
])
def test_algorithm2_on_one_by_one_lp(oracle_lib, steps, eta_hat, passes):
    lp = _one_by_one()
    _, _, r = oracle.solve(lp, iter_limit=steps, ruiz_iters=0, pock_chambolle=0)
    assert r["iters"] == steps
    assert r["kkt_passes"] == passes
    assert r["eta"] == pytest.approx(eta_hat, rel=1e-12)


def test_algorithm2_one_by_one_iterate(oracle_lib):
    """The accepted iterate after step 3 of the case above (original space =
    scaled space without preconditioning): x = 0.623408, y = 5.134098."""
    lp = _one_by_one()
    x, y, _ = oracle.solve(lp, iter_limit=3, ruiz_iters=0, pock_chambolle=0)
    assert x[0] == pytest.approx(0.6234081051890291, rel=1e-12)
    assert y[0] == pytest.approx(5.13409822936515, rel=1e-12)


# ------------------------------------------------------------ Algorithm 3

def test_primal_weight_hand_cases(oracle_lib):
    # theta = 1/2: omega' = exp(ln(Dy/Dx)/2 + ln(omega)/2) = sqrt(omega Dy / Dx)
    assert oracle.primal_weight(4.0, 1.0, 9.0, 0.5) == pytest.approx(6.0, rel=1e-15)
    assert oracle.primal_weight(4.0, 9.0, 1.0, 0.5) == pytest.approx(2.0 / 3.0, rel=1e-15)
    # theta = 1/4: 9^(1/4) 4^(3/4) = sqrt(3) * 2 sqrt(2) = sqrt(24)
    assert oracle.primal_weight(4.0, 1.0, 9.0, 0.25) == pytest.approx(math.sqrt(24.0), rel=1e-14)
    # theta = 0 keeps omega; theta = 1 takes Dy / Dx
    assert oracle.primal_weight(4.0, 2.0, 3.0, 0.0) == pytest.approx(4.0, rel=1e-15)
    assert oracle.primal_weight(4.0, 2.0, 3.0, 1.0) == pytest.approx(1.5, rel=1e-15)
    # a distance at or below epsilon_zero leaves omega unchanged
    assert oracle.primal_weight(4.0, 0.0, 9.0, 0.5) == 4.0
    assert oracle.primal_weight(4.0, 1.0, 1e-11, 0.5, 1e-10) == 4.0


# ---------------------------------------------------- restart criteria

def test_restart_criteria_hand_cases(oracle_lib):
    rc = oracle.restart_check
    # (i) sufficient decay: mu_c <= 0.9 mu_0
    assert rc(0.85, 1.0, math.inf, 10, 100) == "sufficient"
    assert rc(0.95, 1.0, math.inf, 10, 100) is None
    # (iii) artificial: t >= 0.5 k
    assert rc(0.95, 1.0, math.inf, 50, 100) == "artificial"
    assert rc(0.95, 1.0, math.inf, 49, 100) is None
    # the first outer loop (mu_0 = +inf, R6) restarts at its first evaluation
    assert rc(1e300, math.inf, math.inf, 40, 40) == "sufficient"
    # With the paper's betas (0.9, 0.1) criterion (ii) can only hold where (i)
    # holds too (0.1 mu_0 < 0.9 mu_0); with betas where it is weaker than (i),
    # (ii) fires only when the candidate's mu rose since the previous evaluation:
    assert rc(0.5, 1.0, 0.4, 10, 100, 0.2, 0.8) == "necessary"
    assert rc(0.5, 1.0, 0.6, 10, 100, 0.2, 0.8) is None
    assert rc(0.5, 1.0, 0.5, 10, 100, 0.2, 0.8) is None            # equal: no rise
    assert rc(0.85, 1.0, 0.4, 10, 100, 0.2, 0.8) is None           # rise, but no 0.8 decay
    assert rc(0.15, 1.0, 0.1, 10, 100, 0.2, 0.8) == "sufficient"   # (i) is tested first


def test_first_restart_updates_weight_and_mu0(oracle_lib):
    """The first evaluation (k = 40) restarts by (i) (mu_0 = +inf).  On this LP
    the candidate is the current iterate z^{1,0} = z_40, so Algorithm 3 sees
    Delta_x = ||x_40 - 0||, Delta_y = ||y_40 - 0|| and the new primal weight is
    sqrt(omega^0 Delta_y / Delta_x) (theta = 1/2), and the next outer loop's
    mu_0 is the normalized gap at z_40 with radius ||z_40 - z^{0,0}||_omega
    under the NEW omega.  Without preconditioning the scaled and original
    spaces coincide, so z_40 is what a 40-iteration solve returns."""
    lp = lpgen.planted_uniform(8, 12, 0.5, frac_boxed=0.6, seed_key=(60,))
    kw = dict(ruiz_iters=0, pock_chambolle=0, eps=1e-30)
    x40, y40, r40 = oracle.solve(lp, iter_limit=40, **kw)
    assert r40["iters"] == 40
    _, _, _, tr = oracle.solve_traced(lp, iter_limit=200, **kw)
    k, t, mu_cur, mu_avg, mu0, cand, restarted, omega1 = tr[0][:8]
    assert (k, t, cand, restarted) == (40, 40, 0, 1)      # current candidate, restart
    assert mu0 == math.inf and mu_cur < mu_avg
    omega0 = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    Dx, Dy = np.linalg.norm(x40), np.linalg.norm(y40)
    assert omega1 == pytest.approx(math.sqrt(omega0 * Dy / Dx), rel=1e-12)
    # mu_0 of the second outer loop (recorded at its first evaluation)
    A = lp.dense()
    gx = A.T @ y40 - lp.c
    gy = lp.q - A @ x40
    r = math.sqrt(omega1 * Dx ** 2 + Dy ** 2 / omega1)
    ylo = np.where(lp.ineq == 1, 0.0, -np.inf)
    mu_new, _ = oracle.normalized_gap(x40, y40, gx, gy, lp.l, lp.u, ylo, omega1, r)
    assert tr[1][4] == pytest.approx(mu_new, rel=1e-10)
    # under the old weight it would differ
    r_old = math.sqrt(omega0 * Dx ** 2 + Dy ** 2 / omega0)
    mu_old, _ = oracle.normalized_gap(x40, y40, gx, gy, lp.l, lp.u, ylo, omega0, r_old)
    assert abs(mu_old - mu_new) > 1e-6 * abs(mu_new)


@pytest.mark.parametrize("betas", [(0.9, 0.1), (0.2, 0.8)])
def test_traced_restarts_follow_the_criteria(oracle_lib, betas):
    """Every evaluation of a traced solve restarts exactly when one of the
    criteria holds for its recorded mu values, with mu_c,prev the candidate mu
    of the previous evaluation in the same outer loop (+inf at its first)."""
    lp = lpgen.small_planted()
    bs, bn = betas
    _, _, _, tr = oracle.solve_traced(lp, iter_limit=3000, eps=1e-30, beta_suff=bs, beta_nec=bn,
                                      trace_cap=1000)
    assert len(tr) > 20
    prev = math.inf
    seen = set()
    for rec in tr:
        k, t, mu_cur, mu_avg, mu0, cand, restarted = rec[:7]
        muc = mu_cur if cand == 0 else mu_avg
        assert muc == min(mu_cur, mu_avg)               # GetRestartCandidate
        why = oracle.restart_check(muc, mu0, prev, t, k, bs, bn, 0.5)
        assert bool(restarted) == (why is not None), rec
        seen.add(why)
        prev = math.inf if restarted else muc
    assert "sufficient" in seen

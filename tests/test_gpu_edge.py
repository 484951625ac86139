"""Degenerate and boundary inputs on the single-LP path, each checked the way
the planted optimum fixes it (Eq. (15) by the oracle at the returned point,
the planted objective) and against the oracle's own solve: empty rows and
columns, a 1 x 1 LP, a matrix with no nonzeros, all-free variables,
all-equality and all-inequality rows, in both step engines."""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu


def _replant(lp, A, seed):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return lpgen._plant(lpgen.rng_for(seed, 9), lp.m, lp.n, A.indptr.astype(np.int32),
                        A.indices.astype(np.int32), A.data.astype(np.float64), lp.ineq, lp.l, lp.u, "edge")


def _empty_rows_cols():
    base = lpgen.planted_uniform(30, 60, 0.12, frac_boxed=0.8, seed_key=(80,))
    A = base.scipy().tolil()
    A[0, :] = 0
    A[7, :] = 0
    A[:, 0] = 0
    A[:, 11] = 0
    A = A.tocsr()
    A.eliminate_zeros()
    return _replant(base, A, 80)


def _one_by_one():
    rng = lpgen.rng_for(81)
    return lpgen._plant(rng, 1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]),
                        np.array([1], np.uint8), np.array([0.0]), np.array([10.0]), "one")


def _no_nonzeros():
    rng = lpgen.rng_for(82)
    m, n = 3, 4
    return lpgen._plant(rng, m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                        np.array([1, 0, 1], np.uint8), np.zeros(n), np.full(n, 5.0), "empty")


CASES = {
    "empty_rows_cols": _empty_rows_cols,
    "one_by_one": _one_by_one,
    "no_nonzeros": _no_nonzeros,
    "all_free": lambda: lpgen.planted_uniform(40, 90, 0.1, frac_boxed=0.0, seed_key=(83,)),
    "all_equality": lambda: lpgen.planted_uniform(40, 90, 0.1, frac_ineq=0.0, seed_key=(84,)),
    "all_inequality": lambda: lpgen.planted_uniform(40, 90, 0.1, frac_ineq=1.0, seed_key=(85,)),
}


@pytest.mark.parametrize("persistent", [1, 0, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_degenerate_inputs_solve_to_1e8(gpu_lib, oracle_lib, name, persistent):
    lp = CASES[name]()
    x, y, r = P.solve(lp, rel_tol=1e-8, iter_limit=200000, persistent=persistent)
    assert r["status_name"] == "OPTIMAL", r
    k = oracle.kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    ref = lp.c @ lp.x_star
    assert abs(lp.c @ x - ref) <= 1e-6 * (1 + abs(ref)), (lp.c @ x, ref)
    _, _, ro = oracle.solve(lp, iter_limit=200000)
    assert ro["status_name"] == "OPTIMAL"


@pytest.mark.parametrize("name", sorted(CASES))
def test_degenerate_inputs_preprocess_bit_exact(gpu_lib, oracle_lib, name):
    lp = CASES[name]()
    with P.Context.from_lp(lp) as ctx:
        g = ctx.get_scaled()
    trp, tci, _, perm = oracle.transpose(lp)
    assert np.array_equal(g["KT_row_ptr"], trp) and np.array_equal(g["KT_col_idx"], tci)
    v, D1, D2 = oracle.precondition(lp)
    assert np.array_equal(g["Kval"], v) and np.array_equal(g["D1"], D1) and np.array_equal(g["D2"], D2)

"""The seeded workload generators: shapes, determinism and the stated distributions."""
import numpy as np

import lpgen


def _valid_csr(lp):
    rp, ci = lp.row_ptr, lp.col_idx
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and rp[0] == 0 and rp[-1] == ci.size
    assert np.all(np.diff(rp) >= 0)
    for i in range(0, lp.m, max(1, lp.m // 200)):
        seg = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0) and (seg.size == 0 or (seg[0] >= 0 and seg[-1] < lp.n))


def test_small_planted_shape_and_determinism():
    a, b = lpgen.small_planted(), lpgen.small_planted()
    assert (a.m, a.n) == (200, 500) and int(a.ineq.sum()) == 100
    assert 0.015 < a.nnz / (a.m * a.n) < 0.025
    assert np.array_equal(a.val, b.val) and np.array_equal(a.c, b.c)
    assert np.isfinite(a.u).sum() == 400  # 80% boxed [0, 10], 20% free
    _valid_csr(a)


def test_mip_like_distributions():
    lp = lpgen.mip_like(20_000, 50_000, 300_000, seed_key=(4, 0))
    _valid_csr(lp)
    assert abs(lp.nnz - 300_000) < 0.03 * 300_000
    lens = np.diff(lp.row_ptr)
    assert lens.min() >= 1 and lens.max() <= 2000
    a = np.abs(lp.val)
    assert a.min() >= 1e-3 * (1 - 1e-12) and a.max() <= 1e3 * (1 + 1e-12)
    assert abs(np.mean(lp.val > 0) - 0.5) < 0.01
    assert abs(lp.ineq.mean() - 0.6) < 1e-3
    free = ~np.isfinite(lp.u)
    assert abs(free.mean() - 0.1) < 1e-3
    assert np.all(lp.l[~free] == 0) and lp.u[~free].min() >= 1 and lp.u[~free].max() <= 1e4


def test_batch_sizes():
    lps = lpgen.batch_planted(count=16)
    for lp in lps:
        assert 20 <= lp.m <= 400 and 50 <= lp.n <= 1000
        assert np.all(lp.l == 0) and np.all(lp.u == 10)
        _valid_csr(lp)


def test_barabasi_albert_degrees():
    rng = lpgen.rng_for(99)
    e = lpgen.barabasi_albert_edges(2000, 3, rng)
    assert e.shape == (3 * (2000 - 3), 2)
    assert np.all(e[:, 0] != e[:, 1])
    key = np.minimum(e[:, 0], e[:, 1]) * 2000 + np.maximum(e[:, 0], e[:, 1])
    assert np.unique(key).size == key.size  # no multi-edges
    deg = np.bincount(e.ravel(), minlength=2000)
    assert deg[3:].min() >= 3 and deg.max() > 30  # preferential attachment grows hubs

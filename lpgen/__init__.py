"""Seeded synthetic LP workloads (inputs only).

This module builds the linear programs that the tests and the benchmark feed to
both the CPU oracle and the GPU solver.  It holds none of the solver's
arithmetic: it only draws random structure and values, and, for the planted
instances, chooses an optimal primal-dual pair first and then sets the data so
that the optimality conditions of the LP in Section 2, Eq. (1) hold exactly.

Problem form (Section 2, Eq. (1)): minimise c^T x subject to K_i x >= q_i on
inequality rows (ineq[i] == 1), K_i x == q_i on equality rows, l <= x <= u.
A "<=" row of a workload description is generated directly in ">=" form (the
value distributions are symmetric, so negating a row changes nothing
statistically).

Workloads (sizes and distributions follow the benchmark configurations):
  * ``planted_uniform``   - uniform sparsity, N(0,1) values, box [0, ub] / free
  * ``mip_like``          - power-law row lengths, log-uniform |values|
                            (shape of LP relaxations of MIPs, Section 4 datasets)
  * ``pagerank``          - the PageRank feasibility LP on a Barabasi-Albert
                            graph (Section 4.5 and Appendix E)
  * ``batch_planted``     - many small planted LPs of uneven size
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

BASE_SEED = 20210609


@dataclasses.dataclass
class LP:
    """An LP in the form of Eq. (1): K in CSR (int32 indices, sorted, no duplicates)."""
    m: int
    n: int
    row_ptr: np.ndarray  # int32 [m+1]
    col_idx: np.ndarray  # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    c: np.ndarray        # float64 [n]
    q: np.ndarray        # float64 [m]
    l: np.ndarray        # float64 [n], may hold -inf
    u: np.ndarray        # float64 [n], may hold +inf
    ineq: np.ndarray     # uint8 [m], 1 = (K x)_i >= q_i, 0 = equality
    name: str = ""
    x_star: Optional[np.ndarray] = None    # planted optimal primal (if known)
    y_star: Optional[np.ndarray] = None    # planted optimal dual (if known)
    lam_star: Optional[np.ndarray] = None  # planted reduced costs (if known)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            A[i, self.col_idx[s:e]] = self.val[s:e]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def rng_for(*key: int) -> np.random.Generator:
    """Independent, reproducible stream for a workload key (base seed first)."""
    return np.random.default_rng([BASE_SEED, *key])


def _csr_from_keys(keys: np.ndarray, m: int, n: int):
    """Sorted unique linear keys row*n+col -> (row_ptr, col_idx)."""
    rows = (keys // n).astype(np.int64)
    cols = (keys % n).astype(np.int32)
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return row_ptr.astype(np.int32), cols


def _uniform_pattern(rng, m: int, n: int, density: float):
    """Each of the m*n positions present independently with probability `density`."""
    total = m * n
    want = int(rng.binomial(total, density))
    if want == 0:
        return np.zeros(m + 1, np.int32), np.zeros(0, np.int32)
    draws = rng.integers(0, total, size=int(want * 1.2) + 16)
    uniq = np.unique(draws)
    while uniq.size < want:
        uniq = np.unique(np.concatenate([uniq, rng.integers(0, total, size=want)]))
    # A uniformly random `want`-subset of the distinct draws is a uniform subset.
    pick = np.sort(uniq[rng.permutation(uniq.size)[:want]])
    return _csr_from_keys(pick, m, n)


def _powerlaw_pattern(rng, m: int, n: int, nnz_target: int, lmin=1, lmax=2000, alpha=2.1):
    """Row lengths from a truncated continuous power law (exponent alpha on
    [lmin, lmax]) rescaled so that their sum is about nnz_target, then rounded
    and clipped to [lmin, lmax]; columns uniform and distinct within a row."""
    uu = rng.random(m)
    a1 = 1.0 - alpha
    L = (lmin ** a1 + uu * (lmax ** a1 - lmin ** a1)) ** (1.0 / a1)
    f = nnz_target / L.sum()
    for _ in range(6):  # re-fit the scale after clipping so the total lands near nnz_target
        Lc = np.clip(np.rint(L * f), lmin, min(lmax, n))
        f *= nnz_target / Lc.sum()
    L = np.clip(np.rint(L * f), lmin, min(lmax, n)).astype(np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), L)
    cols = rng.integers(0, n, size=rows.size)
    keys = np.unique(rows * n + cols)  # drops the rare in-row duplicates
    return _csr_from_keys(keys, m, n)


def _csr_matvec(row_ptr, col_idx, val, x):
    import scipy.sparse as sp
    m = row_ptr.size - 1
    A = sp.csr_matrix((val, col_idx, row_ptr), shape=(m, x.size))
    return A @ x


def _csr_rmatvec(row_ptr, col_idx, val, y, n):
    import scipy.sparse as sp
    m = row_ptr.size - 1
    A = sp.csr_matrix((val, col_idx, row_ptr), shape=(m, n))
    return A.T @ y


def _plant(rng, m, n, row_ptr, col_idx, val, ineq, l, u, name,
           frac_at_bound=0.3, frac_y_zero=0.4) -> LP:
    """Choose (x*, y*, lambda*) with strict complementarity and set q, c so
    that x* is primal optimal and (y*, lambda*) dual optimal for Eq. (1):
      * 30% of variables sit at a finite bound (lower or upper, equally likely)
        with reduced cost lambda* of the matching sign, the rest are strictly
        inside their box (or free) with lambda* = 0;
      * on inequality rows y* >= 0, zero on 40% of them (those rows get a
        positive slack), positive on the others (tight rows);
      * q_i = K_i x* on tight and equality rows, K_i x* - s_i (s_i > 0) on slack rows;
      * c = K^T y* + lambda*."""
    boxed = np.isfinite(l) & np.isfinite(u)
    boxed_idx = np.flatnonzero(boxed)
    n_at = min(int(round(frac_at_bound * n)), boxed_idx.size)
    at = rng.choice(boxed_idx, size=n_at, replace=False) if n_at > 0 else np.zeros(0, np.int64)
    at_upper = rng.random(n_at) < 0.5
    x = np.zeros(n)
    lam = np.zeros(n)
    # interior: inside the box (or around 0 for free / half-bounded variables)
    lo = np.where(np.isfinite(l), l, 0.0)
    width = np.where(boxed, u - l, 1.0)
    x[:] = np.where(boxed, lo + width * rng.uniform(0.05, 0.95, n), rng.standard_normal(n))
    half_lo = np.isfinite(l) & ~np.isfinite(u)
    x[half_lo] = l[half_lo] + rng.uniform(0.5, 1.5, int(half_lo.sum()))
    half_up = ~np.isfinite(l) & np.isfinite(u)
    x[half_up] = u[half_up] - rng.uniform(0.5, 1.5, int(half_up.sum()))
    lo_set = at[~at_upper]
    up_set = at[at_upper]
    x[lo_set] = l[lo_set]
    x[up_set] = u[up_set]
    lam[lo_set] = rng.uniform(0.1, 1.0, lo_set.size)
    lam[up_set] = -rng.uniform(0.1, 1.0, up_set.size)

    y = np.zeros(m)
    eq = ineq == 0
    y[eq] = rng.standard_normal(int(eq.sum()))
    ineq_idx = np.flatnonzero(~eq)
    zero = rng.random(ineq_idx.size) < frac_y_zero
    y[ineq_idx[~zero]] = rng.uniform(0.1, 1.0, int((~zero).sum()))
    Kx = _csr_matvec(row_ptr, col_idx, val, x)
    q = Kx.copy()
    slack_rows = ineq_idx[zero]
    q[slack_rows] -= rng.uniform(0.1, 1.0, slack_rows.size)
    c = _csr_rmatvec(row_ptr, col_idx, val, y, n) + lam
    return LP(m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c, q=q,
              l=l, u=u, ineq=ineq.astype(np.uint8), name=name,
              x_star=x, y_star=y, lam_star=lam)


def planted_uniform(m=200, n=500, density=0.02, frac_ineq=0.5, frac_boxed=0.8,
                    ub=10.0, seed_key=(0,), name="planted_uniform") -> LP:
    """Uniform-position sparse planted LP: N(0,1) values, bounds [0, ub] on a
    `frac_boxed` share of the variables, the rest free; a `frac_ineq` share of
    the rows are inequalities (positions drawn at random)."""
    rng = rng_for(*seed_key)
    row_ptr, col_idx = _uniform_pattern(rng, m, n, density)
    val = rng.standard_normal(col_idx.size)
    ineq = np.zeros(m, np.uint8)
    ineq[rng.permutation(m)[: int(round(frac_ineq * m))]] = 1
    boxed = np.zeros(n, bool)
    boxed[rng.permutation(n)[: int(round(frac_boxed * n))]] = True
    l = np.where(boxed, 0.0, -np.inf)
    u = np.where(boxed, ub, np.inf)
    return _plant(rng, m, n, row_ptr, col_idx, val, ineq, l, u, name)


def mip_like(m=100_000, n=250_000, nnz=1_500_000, frac_ineq=0.6, frac_free=0.1,
             seed_key=(1,), name="mip_like") -> LP:
    """Shape of an LP relaxation of a MIP: power-law row lengths (exponent 2.1
    on [1, 2000], rescaled to about `nnz` entries), uniform columns, |values|
    log-uniform in [1e-3, 1e3] with random signs, 60% inequality rows, 10% free
    variables and the rest boxed in [0, U] with U log-uniform in [1, 1e4];
    planted optimum."""
    rng = rng_for(*seed_key)
    row_ptr, col_idx = _powerlaw_pattern(rng, m, n, nnz)
    k = col_idx.size
    val = np.where(rng.random(k) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-3.0, 3.0, k)
    ineq = np.zeros(m, np.uint8)
    ineq[rng.permutation(m)[: int(round(frac_ineq * m))]] = 1
    free = np.zeros(n, bool)
    free[rng.permutation(n)[: int(round(frac_free * n))]] = True
    U = 10.0 ** rng.uniform(0.0, 4.0, n)
    l = np.where(free, -np.inf, 0.0)
    u = np.where(free, np.inf, U)
    return _plant(rng, m, n, row_ptr, col_idx, val, ineq, l, u, name)


def barabasi_albert_edges(n_nodes: int, k: int, rng) -> np.ndarray:
    """Preferential-attachment graph: k isolated seed vertices; every later
    vertex attaches k edges to k distinct earlier vertices, each chosen with
    probability proportional to its current degree (the first new vertex, with
    all seed degrees zero, joins every seed).  Returns an int64 [E, 2] edge list
    with E = k (n_nodes - k), no self-loops and no multi-edges."""
    if n_nodes <= k:
        raise ValueError("need more than k vertices")
    E = k * (n_nodes - k)
    edges = np.empty((E, 2), np.int64)
    ends = np.empty(2 * E, np.int64)  # every edge endpoint once: a degree-weighted urn
    ne = 0
    e = 0
    for s in range(k):  # first new vertex joins all seeds
        edges[e] = (k, s)
        ends[ne] = k
        ends[ne + 1] = s
        ne += 2
        e += 1
    draws = rng.random(4 * k * (n_nodes - k) + 64)
    di = 0
    for v in range(k + 1, n_nodes):
        picked: List[int] = []
        while len(picked) < k:
            if di >= draws.size:
                draws = rng.random(draws.size)
                di = 0
            t = int(ends[int(draws[di] * ne)])
            di += 1
            if t not in picked:
                picked.append(t)
        for t in picked:
            edges[e] = (v, t)
            ends[ne] = v
            ends[ne + 1] = t
            ne += 2
            e += 1
    return edges


def pagerank(n_nodes=1_000_000, k=3, damping=0.85, seed_key=(2,), name="pagerank") -> LP:
    """PageRank feasibility LP (Section 4.5, Appendix E): with S' the
    column-stochastic adjacency of a Barabasi-Albert graph,
        (I - damping*S') x >= (1 - damping)/n * 1   (n inequality rows)
        1^T x = 1                                   (one equality row, last)
        x >= 0,  c = 0.
    nnz(K) = 8 n - 18 for k = 3."""
    rng = rng_for(*seed_key)
    edges = barabasi_albert_edges(n_nodes, k, rng)
    n = n_nodes
    a = np.concatenate([edges[:, 0], edges[:, 1]])
    b = np.concatenate([edges[:, 1], edges[:, 0]])
    deg = np.bincount(a, minlength=n).astype(np.float64)
    # off-diagonal (i, j) = -damping * A_ij / deg(j); diagonal 1
    rows = np.concatenate([a, np.arange(n)])
    cols = np.concatenate([b, np.arange(n)])
    vals = np.concatenate([-damping / deg[b], np.ones(n)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    m = n + 1
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:n + 1])
    row_ptr[m] = row_ptr[n] + n
    col_idx = np.concatenate([cols, np.arange(n)]).astype(np.int32)
    val = np.concatenate([vals, np.ones(n)])
    q = np.concatenate([np.full(n, (1.0 - damping) / n), [1.0]])
    ineq = np.concatenate([np.ones(n, np.uint8), [0]]).astype(np.uint8)
    return LP(m=m, n=n, row_ptr=row_ptr.astype(np.int32), col_idx=col_idx, val=val,
              c=np.zeros(n), q=q, l=np.zeros(n), u=np.full(n, np.inf), ineq=ineq,
              name=name)


def batch_planted(count=4096, m_range=(20, 400), n_range=(50, 1000), density=0.05,
                  ub=10.0, seed_key=(3,), name="batch") -> List[LP]:
    """`count` independent planted LPs, m ~ U[m_range], n ~ U[n_range], uniform
    positions at `density`, N(0,1) values, mixed equality / inequality rows,
    every variable boxed in [0, ub]."""
    top = rng_for(*seed_key)
    ms = top.integers(m_range[0], m_range[1] + 1, size=count)
    ns = top.integers(n_range[0], n_range[1] + 1, size=count)
    out = []
    for j in range(count):
        out.append(planted_uniform(m=int(ms[j]), n=int(ns[j]), density=density,
                                   frac_ineq=0.5, frac_boxed=1.0, ub=ub,
                                   seed_key=(*seed_key, 1, j), name=f"{name}[{j}]"))
    return out


# ---------------------------------------------------------------------------
# The five benchmark workloads, by name and size.

def small_planted(seed=0) -> LP:
    """200 x 500 planted LP, 2% density (100 equality / 100 inequality rows)."""
    return planted_uniform(200, 500, 0.02, seed_key=(0, seed), name="planted_200x500")


def mip_relaxation_100k(seed=0) -> LP:
    """100k x 250k MIP-relaxation-shaped planted LP, about 1.5M nonzeros."""
    return mip_like(100_000, 250_000, 1_500_000, seed_key=(1, seed), name="mip_100k_250k")


def pagerank_1m(seed=0) -> LP:
    """PageRank LP on a 1M-node Barabasi-Albert graph (8n - 18 nonzeros)."""
    return pagerank(1_000_000, seed_key=(2, seed), name="pagerank_1m")


def batch_4096(seed=0, count=4096) -> List[LP]:
    """4096 planted LPs, m in [20, 400], n in [50, 1000], 5% density."""
    return batch_planted(count=count, seed_key=(3, seed))


def unroll_20k(seed=0) -> LP:
    """20k x 50k planted LP with about 300k nonzeros (MIP-like distributions)."""
    return mip_like(20_000, 50_000, 300_000, seed_key=(4, seed), name="mip_20k_50k")

"""The benchmark's algorithmic byte counts: the measurement plan's per-unit
figure per step attempt, 2 nnz (v + 4) + 4 (m + n) + v (m + n) +
v (10 n + 9 m), checked against the totals the plan states for the
100k x 250k LP (about 67 MB in float64) and the 1M-node PageRank LP (368 MB
in float64); and the kernels' own count (each array they touch once), which
the per-kernel figures of the bench line use."""
import types

import bench


def test_per_unit_bytes_match_the_plan():
    assert abs(bench._survey_bytes(100_000, 250_000, 1_498_893, 64) / 1e6 - 67.4) < 0.05
    assert abs(bench._survey_bytes(1_000_001, 1_000_000, 7_999_982, 64) / 1e6 - 368.0) < 0.05
    # float32 iterates and running sums: every vector stream at 4 bytes
    assert abs(bench._survey_bytes(1_000_001, 1_000_000, 7_999_982, 32) / 1e6 - 220.0) < 0.05


def test_kernel_bytes_count_the_arrays():
    lp = types.SimpleNamespace(m=7, n=11, nnz=30)
    for fp, v in ((64, 8), (32, 4)):
        primal, dual = bench._alg_bytes(lp, fp)
        # primal: K^T values and indices, its n + 1 row starts, y gathered
        # once, x, xs, c, l, u read and x', xs' written
        assert primal == lp.nnz * (v + 4) + 4 * (lp.n + 1) + v * lp.m + 7 * v * lp.n
        # dual: K values and indices, its m + 1 row starts, x' gathered once,
        # K x, y, ys, q, ylo read and y', K x', ys' written
        assert dual == lp.nnz * (v + 4) + 4 * (lp.m + 1) + v * lp.n + 8 * v * lp.m

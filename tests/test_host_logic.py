"""Host-side planning of the library (csrc/schedule.h), built here with the
host compiler alone: the warp-chunk schedule, the balanced assignment of
chunks to the persistent kernel's warps, the fixed-size slabs of the slab
kernels, and the refinement's tolerance and scale rules."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_04756_gb300", "csrc")


@pytest.fixture(scope="module")
def hl(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hl") / "libhl.so")
    subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, "-x", "c++",
                    os.path.join(CSRC, "schedule.cu"), "-x", "none",
                    os.path.join(ROOT, "tests", "host_logic_shim.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    P = C.c_void_p
    L.hl_build_schedule.argtypes = [C.c_int, P, P, C.c_int, P, C.c_int, P]
    L.hl_chunk_cost.argtypes = [P, P]
    L.hl_chunk_cost.restype = C.c_double
    L.hl_assign.argtypes = [C.c_int, P, P, C.c_int, C.c_int, P, P, P]
    L.hl_round_tol.argtypes = [C.c_double, C.c_double, C.c_double]
    L.hl_round_tol.restype = C.c_double
    L.hl_scales.argtypes = [C.c_double, C.c_double, C.c_double, P]
    L.hl_build_slabs.argtypes = [C.c_int, P, P, P, P, P, C.c_int, P]
    L.hl_finish_now.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int]
    L.hl_plan_precondition.argtypes = [C.c_int, P, P, C.c_int, P, C.c_int, P]
    L.hl_remaining.argtypes = [C.c_longlong, C.c_longlong, C.c_double, C.c_longlong, C.c_longlong, C.c_double, P]
    return L


def _schedule(hl, rp):
    rp = np.ascontiguousarray(rp, np.int32)
    rows = rp.size - 1
    cap = rows + int(rp[-1]) // 256 + 8
    ch = np.zeros((cap, 4), np.int32)
    lr = np.zeros((cap, 4), np.int32)
    cnt = np.zeros(3, np.int32)
    assert hl.hl_build_schedule(rows, rp.ctypes.data, ch.ctypes.data, cap, lr.ctypes.data, cap,
                                cnt.ctypes.data) == 0
    return ch[:cnt[0]], lr[:cnt[1]], int(cnt[2])


def _powerlaw_rp(rng, rows, with_specials=True):
    lens = np.minimum((rng.pareto(1.1, rows) * 3).astype(np.int64), 2000)
    if with_specials:
        lens[:8] = [0, 0, 256, 257, 512, 513, 1, 2000]
        lens[rng.choice(rows, 20)] = 0
    rp = np.zeros(rows + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    return rp.astype(np.int32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_schedule_covers_every_row_and_nonzero_once(hl, seed):
    rng = np.random.default_rng(seed)
    rp = _powerlaw_rp(rng, 3000)
    ch, lr, nseg = _schedule(hl, rp)
    lens = np.diff(rp)
    r = 0
    k = 0
    nlong = 0
    while k < len(ch):
        rb, re_, nb, ne = ch[k]
        assert rb == r
        if re_ < 0:  # segments of a long row, in order
            li = -(re_ + 1)
            assert li == nlong and lr[li][0] == r
            L = lr[li]
            assert L[1] == -(-lens[r] // 256) and lens[r] > 256
            assert L[2] == sum(x[1] for x in lr[:li])  # part_off: cumulative segment count
            for s in range(L[1]):
                rb2, re2, nb2, ne2 = ch[k + s]
                assert (rb2, re2) == (r, re_)
                assert nb2 == rp[r] + 256 * s and ne2 == min(rp[r + 1], nb2 + 256)
            k += L[1]
            r += 1
            nlong += 1
            continue
        assert re_ > rb and re_ - rb <= 32
        assert nb == rp[rb] and ne == rp[re_] and ne - nb <= 256
        assert np.all(lens[rb:re_] <= 256)
        # greedy: the chunk stops at 32 rows, at the end, before a long row, or
        # before the row that would take it past 256 nonzeros
        if re_ - rb < 32 and re_ < len(lens):
            assert lens[re_] > 256 or rp[re_ + 1] - rp[rb] > 256
        r = re_
        k += 1
    assert r == len(lens) and nlong == len(lr) and nseg == sum(x[1] for x in lr)


def test_chunk_cost_closed_forms(hl):
    # 32 rows of 8 nonzeros: one lane per row, 8 steps, no shuffle
    rp = np.arange(0, 33 * 8, 8, dtype=np.int32)
    c = np.array([0, 32, 0, 256], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == 256 / 32 + 2 * 8 + 10
    # 4 rows of 64: 8 lanes per row, 8 steps + 3 shuffle levels
    rp = np.arange(0, 5 * 64, 64, dtype=np.int32)
    c = np.array([0, 4, 0, 256], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == 256 / 32 + 2 * (8 + 3) + 10
    # one row of 200 among 20 rows of 2: summing the long row with the warp
    # (7 + 5 steps) plus 2 steps for the rest beats 200 steps at one lane a row
    lens = np.array([200] + [2] * 20)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    c = np.array([0, 21, 0, int(rp[-1])], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == rp[-1] / 32 + 2 * (2 + 7 + 5) + 10
    # 32 rows, one of 40 and 31 of 1: the long row is split off
    lens = np.array([40] + [1] * 31)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    c = np.array([0, 32, 0, int(rp[-1])], np.int32)
    # L = 1: 40 steps; split at 32: 1 + (2 + 5) = 8 -> 8 is below the cap
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == rp[-1] / 32 + 2 * 8 + 10
    lens = np.array([30] * 8)  # 8 rows of 30: L = 4 -> 8 steps + 2 shuffle levels
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    c = np.array([0, 8, 0, int(rp[-1])], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == rp[-1] / 32 + 2 * 10 + 10
    lens = np.array([15] * 16 + [1] * 16)  # 32 rows, one lane each: 15 steps
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    c = np.array([0, 32, 0, int(rp[-1])], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == rp[-1] / 32 + 2 * 15 + 10
    lens = np.array([17] * 8 + [2] * 24)  # 17 steps at one lane a row: capped at 16
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    c = np.array([0, 32, 0, int(rp[-1])], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == rp[-1] / 32 + 2 * 16 + 10
    # a segment of a long row
    c = np.array([0, -1, 0, 256], np.int32)
    assert hl.hl_chunk_cost(c.ctypes.data, rp.ctypes.data) == 256 / 32 + 2 * 13 + 30


@pytest.mark.parametrize("nw,wpc", [(64, 16), (2432, 16), (7, 1)])
def test_assignment_is_a_balanced_partition(hl, nw, wpc):
    rng = np.random.default_rng(5)
    rp = _powerlaw_rp(rng, 20000)
    ch, _, _ = _schedule(hl, rp)
    n = len(ch)
    chc = np.ascontiguousarray(ch, np.int32)
    idx = np.zeros(n, np.int32)
    off = np.zeros(nw + 1, np.int32)
    cmax = C.c_int32()
    hl.hl_assign(n, chc.ctypes.data, rp.ctypes.data, nw, wpc, idx.ctypes.data, off.ctypes.data, C.byref(cmax))
    assert sorted(idx.tolist()) == list(range(n))  # every chunk once
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert cmax.value == np.diff(off).max()
    cost = np.array([hl.hl_chunk_cost(chc[i].ctypes.data, rp.ctypes.data) for i in range(n)])
    loads = np.array([cost[idx[off[w]:off[w + 1]]].sum() for w in range(nw)])
    for w in range(nw):
        lst = idx[off[w]:off[w + 1]]
        assert np.all(np.diff(lst) > 0)  # each list in chunk order
    # list scheduling bound: the last chunk went to the least-loaded warp
    assert loads.max() <= cost.sum() / nw + cost.max() + 1e-9
    # same input, same assignment
    idx2 = np.zeros(n, np.int32)
    off2 = np.zeros(nw + 1, np.int32)
    hl.hl_assign(n, chc.ctypes.data, rp.ctypes.data, nw, wpc, idx2.ctypes.data, off2.ctypes.data, C.byref(cmax))
    assert np.array_equal(idx, idx2) and np.array_equal(off, off2)


def test_refinement_round_tolerance(hl):
    # a round that can finish uses the loosest tolerance with a 10x margin
    assert hl.hl_round_tol(1e-4, 1e-8, 1e-5) == pytest.approx(1e-5)
    assert hl.hl_round_tol(1e-6, 1e-8, 1e-5) == pytest.approx(1e-3)
    assert hl.hl_round_tol(1e-12, 1e-8, 1e-5) == 0.1  # capped
    # no single round can finish: the configured inner tolerance
    assert hl.hl_round_tol(1.0, 1e-8, 1e-5) == 1e-5
    assert hl.hl_round_tol(2e-3, 1e-8, 1e-4) == 1e-4


def test_refinement_scales(hl):
    out = np.zeros(2)
    hl.hl_scales(1e-3, 1e-5, 1e12, out.ctypes.data)
    assert out[0] == 1e3 and out[1] == pytest.approx(1e5)
    hl.hl_scales(10.0, 0.5, 1e12, out.ctypes.data)  # violations above 1: no down-scaling
    assert out[0] == 1.0 and out[1] == 2.0
    hl.hl_scales(0.0, 1e-20, 1e12, out.ctypes.data)  # clipped at dmax
    assert out[0] == 1e12 and out[1] == 1e12


def test_preconditioning_long_rows_plan(hl):
    """Rows over 256 nonzeros are cut into 256-nonzero segments that tile the
    row exactly (Ruiz maxima); rows over 8,192 are listed for the host's l1
    sums; nothing else is listed."""
    rng = np.random.default_rng(5)
    lens = np.concatenate([rng.integers(0, 40, 500), [256, 257, 512, 513, 8192, 8193, 20000, 1_000_000, 0]])
    rng.shuffle(lens)
    rp = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    rp = rp.astype(np.int32)
    cap = int(lens.sum()) // 256 + 16
    seg = np.zeros((cap, 3), np.int32)
    longr = np.zeros(cap, np.int32)
    cnt = np.zeros(2, np.int32)
    assert hl.hl_plan_precondition(lens.size, rp.ctypes.data, seg.ctypes.data, cap, longr.ctypes.data, cap,
                                   cnt.ctypes.data) == 0
    seg, longr = seg[:cnt[0]], longr[:cnt[1]]
    assert sorted(longr) == sorted(np.flatnonzero(lens > 8192).tolist())
    covered = {}
    for row, k0, k1 in seg:
        assert lens[row] > 256 and 0 < k1 - k0 <= 256
        covered.setdefault(row, []).append((k0, k1))
    assert sorted(covered) == sorted(np.flatnonzero(lens > 256).tolist())
    for row, parts in covered.items():
        parts.sort()
        assert parts[0][0] == rp[row] and parts[-1][1] == rp[row + 1]
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))  # contiguous, no overlap
        assert all(k1 - k0 == 256 for k0, k1 in parts[:-1])


def test_refinement_finish_rule(hl):
    # float32 rounds go on while each divides the error by at least 10
    assert hl.hl_finish_now(0, float("inf"), 0.5, 12) == 0
    assert hl.hl_finish_now(1, 0.5, 9.9e-6, 12) == 0
    assert hl.hl_finish_now(2, 9.9e-6, 9.9e-7, 12) == 0   # exactly 10x
    assert hl.hl_finish_now(2, 9.9e-6, 7.9e-6, 12) == 1   # 1.25x: float64 finish
    assert hl.hl_finish_now(1, 1e-3, 2e-4, 12) == 1       # 5x
    assert hl.hl_finish_now(3, 1e-4, 1e-7, 3) == 1        # round cap
    assert hl.hl_finish_now(0, float("inf"), 0.5, 0) == 1  # no float32 round allowed
    assert hl.hl_finish_now(2, 1e-6, float("nan"), 12) == 1


def test_refinement_budget(hl):
    out = np.zeros(3, np.int64)
    assert hl.hl_remaining(1000, 5000, 0.0, 300, 400, 1.0, out.ctypes.data) == 0
    assert list(out) == [700, 4600, 0]          # no time limit: 0
    assert hl.hl_remaining(1000, 5000, 10.0, 300, 400, 2.5, out.ctypes.data) == 0
    assert out[2] == 7_500_000_000
    assert hl.hl_remaining(1000, 5000, 10.0, 1000, 400, 2.5, out.ctypes.data) == 1
    assert hl.hl_remaining(1000, 5000, 10.0, 999, 5000, 2.5, out.ctypes.data) == 2
    assert hl.hl_remaining(1000, 5000, 10.0, 999, 4999, 10.0, out.ctypes.data) == 3
    assert hl.hl_remaining(1000, 5000, 10.0, 999, 4999, 10.0 - 1e-12, out.ctypes.data) == 0
    assert out[2] >= 1                          # a sliver of time is still a limit, not "none"


def _slabs(hl, rp):
    rp = np.ascontiguousarray(rp, np.int32)
    rows = rp.size - 1
    ns = int(rp[-1]) // 256 + 1
    first = np.zeros(ns + 1, np.int32)
    head = np.zeros(ns, np.int32)
    tail = np.zeros(ns, np.int32)
    cap = rows + 1
    sp = np.zeros((cap, 4), np.int32)
    cnt = np.zeros(3, np.int32)
    assert hl.hl_build_slabs(rows, rp.ctypes.data, first.ctypes.data, head.ctypes.data, tail.ctypes.data,
                             sp.ctypes.data, cap, cnt.ctypes.data) == 0
    assert cnt[0] == ns
    return first, head, tail, sp[:cnt[1]], int(cnt[2])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_slabs_follow_their_definition(hl, seed):
    """Slab s covers nonzeros [256 s, 256 (s+1)); a row belongs to the slab of
    its start position; a row crossing one slab boundary and ending in the
    next slab is extended (tail -3 - row in its slab, head -2 in the next);
    a row reaching further is a split row with one partial slot per slab it
    touches; head / tail name the split row a slab continues / starts.  Checked against the definitions written
    out per row, on power-law rows with empty rows, rows of exactly 256 and
    rows longer than a slab."""
    rng = np.random.default_rng(seed)
    rp = _powerlaw_rp(rng, 3000)
    if seed == 3:  # nonzero count a multiple of 256, then empty rows
        lens = np.array([256] * 10 + [0] * 5)
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    first, head, tail, sp, nparts = _slabs(hl, rp)
    rows = rp.size - 1
    ns = head.size
    owner = np.minimum(rp[:-1] // 256, ns - 1)
    for s in range(ns):
        assert np.array_equal(np.flatnonzero(owner == s), np.arange(first[s], first[s + 1]))
    exp_head = -np.ones(ns, np.int64)
    exp_tail = -np.ones(ns, np.int64)
    slot = 0
    k = 0
    for r in range(rows):
        b, e = int(rp[r]), int(rp[r + 1])
        if e <= b or b // 256 == (e - 1) // 256:
            continue
        sf, sl = b // 256, (e - 1) // 256
        if sl == sf + 1:  # ends in the next slab: extended, no split record
            exp_tail[sf] = -3 - r
            exp_head[sl] = -2
            continue
        assert tuple(sp[k]) == (r, sf, sl, slot)
        slot += sl - sf + 1
        exp_tail[sf] = k
        exp_head[sf + 1:sl + 1] = k
        k += 1
    assert k == sp.shape[0] and slot == nparts
    assert np.array_equal(head, exp_head) and np.array_equal(tail, exp_tail)

"""Pins of the oracle's maneuver-count reachability (Appendix C): against a
breadth-first search over maneuver segments written here, against the
weighted sweep with a transition cost that dominates every path length, and
the back-tracked plans for validity."""
import collections

import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes


def _world(seed, lx, lt, R, fp, fill):
    sc, img = scenes.tiny(seed, lx, lt, fill=fill, turn_radius=R, footprint=fp)
    o = O.Oracle(lx, lt, R, step_straight=1, step_scale=1, transition=1 << 20)
    B = o.render(img, fp)
    start = next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD)
    return o, B, o.cell(start)


def _bfs(o, B, start, n_cycles):
    """Fewest maneuver segments: a move follows one maneuver for 1 .. period-1
    steps through non-hard cells; levels of a breadth-first search."""
    level = np.full(o.nr, 255, np.uint8)
    level[start] = 0
    frontier = [start]
    for m in range(1, n_cycles + 1):
        nxt = []
        for x in frontier:
            for mu in range(6):
                period = o.nt if mu in (0, 2, 3, 5) else o.nx
                y = x
                for _ in range(period - 1):
                    y = o.succ(mu, y)
                    if B[y] == O.HARD:
                        break
                    if level[y] == 255:
                        level[y] = m
                        nxt.append(y)
        frontier = nxt
    return level


@pytest.mark.parametrize("case", [(1, 3, 3, 2.0, (0, 0, 0), 0.1, 3), (2, 4, 3, 2.5, (1, 0, 0), 0.08, 4),
                                  (3, 3, 4, 1.5, (0, 0, 0), 0.15, 4), (4, 4, 4, 3.0, (1, 1, 1), 0.05, 3)])
def test_reach_equals_breadth_first_search(case):
    seed, lx, lt, R, fp, fill, N = case
    o, B, start = _world(seed, lx, lt, R, fp, fill)
    got = o.reach(B, start, N)
    assert np.array_equal(got, _bfs(o, B, start, N))
    assert (got[B == O.HARD] == 255).all()


@pytest.mark.parametrize("case", [(5, 4, 4, 2.0, (1, 0, 0), 0.06, 3), (6, 5, 5, 3.5, (2, 1, 1), 0.04, 3)])
def test_reach_matches_the_weighted_sweep(case):
    """With every edge costing 1 and a transition cost of 2^20, the weighted
    sweep's N-cycle value divided by the transition cost is the fewest
    maneuvers for every pose reachable within N maneuvers (any such sequence
    fits N cycles, one maneuver per cycle), and more than N elsewhere."""
    seed, lx, lt, R, fp, fill, N = case
    o, B, start = _world(seed, lx, lt, R, fp, fill)
    cnt = o.reach(B, start, N)
    V, _, _ = o.sweep(B, start, N, mode=1)
    m = np.where(V == O.INF, 1 << 30, V >> 20)
    inside = cnt != 255
    assert np.array_equal(m[inside], cnt[inside].astype(m.dtype))
    assert (m[~inside] > N).all()


def test_reach_plans_are_valid_and_minimal():
    o, B, start = _world(7, 5, 5, 3.0, (1, 1, 0), 0.05)
    N = 4
    cnt = o.reach(B, start, N)
    rng = np.random.default_rng(1)
    goals = rng.choice(np.flatnonzero(cnt != 255), size=60, replace=False)
    for g in goals:
        segs = o.reach_extract(B, cnt, int(g))
        assert len(segs) == cnt[g]
        x = start
        for k, s in enumerate(segs):
            assert s["entry"] == x and cnt[s["entry"]] <= k
            y = x
            for _ in range(s["steps"]):
                y = o.succ(s["mu"], y)
                assert B[y] != O.HARD
            assert y == s["exit"]
            x = y
        assert x == g
    assert o.reach_extract(B, cnt, int(np.flatnonzero(B == O.HARD)[0])) is None

"""Oracle pins for the start state of a vehicle already under way (Section
XII) and for the goal-set search (Section IX), on the CPU.

The start state is pinned by reduction (a vehicle at rest is the plain
sweep), by exhaustive enumeration of layer-ordered segment sequences with
the start layer in front (tiny grids, finite N), by Dijkstra on the Star
graph with the start's transition edges re-weighted (the converged value),
and by free-space closed forms along the maneuver in progress.  The goal
search is pinned by a hand-worked 4 x 4 x 4 fixture and by special cases:
zero weights over a box that covers the grid (the volume's minimum), huge
weights (the ideal pose), radius zero (the exact goal)."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes
from tests.util import read_golden

MU = {"LF": O.LF, "SF": O.SF, "RB": O.RB, "RF": O.RF, "SB": O.SB, "LB": O.LB}


def _entries(ct, **over):
    e = [ct] * 6
    for name, v in over.items():
        e[MU[name]] = v
    return e


# ------------------------------------------------------------ start state
@pytest.mark.parametrize("seed,lx,lt,soft", [(0, 4, 4, False), (1, 4, 4, True), (2, 5, 4, True)])
def test_vehicle_at_rest_is_the_plain_sweep(seed, lx, lt, soft):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.1, turn_radius=3.0, soft=soft)
    o = O.Oracle(lx, lt, 3.0, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    s = o.cell(sc.start)
    for mode in (0, 1, 2):
        V0, L0, I0 = o.sweep(B, s, 2, mode)
        V1, L1, I1 = o.sweep_state(B, s, [sc.transition] * 6, 2, mode)
        assert np.array_equal(V0, V1) and np.array_equal(L0, L1) and np.array_equal(I0, I1)


STATE_CASES = [
    dict(seed=0, lx=3, lt=3, R=2.0, soft=False, N=1, entry=dict(LF=0)),
    dict(seed=1, lx=3, lt=3, R=2.0, soft=True, N=1, entry=dict(SB=0)),
    dict(seed=2, lx=3, lt=4, R=2.5, soft=True, N=1, entry=dict(RF=0, RB=-3)),  # -3: ct // 3
    dict(seed=3, lx=4, lt=3, R=3.0, soft=True, N=1, entry=dict(LB=-2, SF=-2)),  # -2: ct // 2
    dict(seed=4, lx=3, lt=3, R=1.5, soft=True, N=2, entry=dict(RB=0)),
    dict(seed=5, lx=3, lt=3, R=2.0, soft=True, N=2, entry=dict(LF=-3, SF=-3, RB=-3, RF=-3, SB=-3, LB=-3)),
]


def _entry_of(case, ct):
    return _entries(ct, **{k: (ct // -v if v < 0 else v) for k, v in case["entry"].items()})


@pytest.mark.parametrize("case", STATE_CASES)
def test_start_state_equals_bruteforce_enumeration(case):
    sc, img = scenes.tiny(case["seed"], case["lx"], case["lt"], fill=0.1, turn_radius=case["R"], soft=case["soft"])
    o = O.Oracle(case["lx"], case["lt"], case["R"], transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    entry = _entry_of(case, sc.transition)
    mattered = False
    for st in [c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD][:3]:
        s = o.cell(st)
        bf = o.bruteforce_state(B, s, entry, case["N"])
        mattered |= not np.array_equal(bf, o.bruteforce(B, s, case["N"]))
        for mode in (0, 1, 2):
            V, _, _ = o.sweep_state(B, s, entry, case["N"], mode)
            assert np.array_equal(V, bf), f"mode {mode}"
    assert mattered, "the start state must change some value in these cases"


@pytest.mark.parametrize("seed,entry", [(0, dict(LF=0)), (1, dict(SB=0, RB=100)), (2, dict(RF=50, LB=0))])
def test_start_state_converges_to_dijkstra_with_reweighted_start_edges(seed, entry):
    sc, img = scenes.tiny(seed, 4, 4, fill=0.1, turn_radius=2.5, soft=True)
    o = O.Oracle(4, 4, 2.5, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    s = o.cell(next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD))
    e = _entries(sc.transition, **entry)
    Vd = o.dijkstra_state(B, s, e)
    assert not np.array_equal(Vd, o.dijkstra(B, s))
    prev = None
    for n in range(1, 31):
        V, _, _ = o.sweep_state(B, s, e, n, mode=1)
        assert np.all(V >= Vd)
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 30 cycles"


def test_maneuver_in_progress_closed_forms():
    """Free space, large ct: continuing the maneuver in progress costs only
    its edges (no transition), a transition in progress its remainder."""
    lx, lt, R, ct = 5, 6, 6.0, 100000
    o = O.Oracle(lx, lt, R, half_shift=1, transition=ct)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    wA = o.tables()["wA"]
    i0, j0 = 10, 9
    s = o.cell((i0, j0, 0))
    # straight forward in progress at heading 0: 100 per step, no ct
    V, L, _ = o.sweep_state(B, s, _entries(ct, SF=0), 1)
    for k in range(1, 15):
        c = o.cell((i0 + k, j0, 0))
        assert V[c] == 100 * k and L[c] == (O.SF << 13) | k
    # left-forward in progress: the quarter turn ends at (i0+R, j0+R, 90 deg)
    V, L, _ = o.sweep_state(B, s, _entries(ct, LF=0), 1)
    end = o.cell((i0 + int(R), j0 + int(R), o.nt // 4))
    assert V[end] == (o.nt // 4) * wA and L[end] == (O.LF << 13) | (o.nt // 4)
    segs = o.extract(V, L, end)
    assert len(segs) == 1 and segs[0]["entry"] == s and segs[0]["mu"] == O.LF
    # a transition toward right-backward with 250 left: the quarter RB turn
    V, L, _ = o.sweep_state(B, s, _entries(ct, RB=250), 1)
    end_rb = o.cell((i0 - int(R), j0 - int(R), o.nt // 4))
    assert V[end_rb] == 250 + (o.nt // 4) * wA
    # other maneuvers still pay ct
    assert V[o.cell((i0 + 5, j0, 0))] == ct + 500
    assert V[s] == 0


def test_start_layer_runs_before_the_first_cycle():
    """A maneuver in progress is followed before cycle 1: a path 'RB in
    progress, then LF' needs only one cycle although LF precedes RB in the
    cycle order, and its LF segment pays ct."""
    lx, lt, R, ct = 5, 5, 4.0, 5000
    o = O.Oracle(lx, lt, R, half_shift=1, transition=ct)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    wA = o.tables()["wA"]
    s = o.cell((16, 16, 0))
    V, _, _ = o.sweep_state(B, s, _entries(ct, RB=0), 1)
    q = o.nt // 4
    x = s
    for _ in range(q):
        x = o.succ(O.RB, x)
    y = x
    for _ in range(q):
        y = o.succ(O.LF, y)
    assert V[x] == q * wA
    # (x0 - 2R, y0, 180 deg) needs half a circle of turning and a second
    # maneuver; only 'RB in progress, then LF' does it with one ct in cycle 1
    assert V[y] == q * wA + ct + q * wA


def test_entry_above_ct_is_refused():
    sc, img = scenes.tiny(0, 4, 4, fill=0.1, turn_radius=3.0)
    o = O.Oracle(4, 4, 3.0, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    with pytest.raises(ValueError):
        o.sweep_state(B, o.cell(sc.start), _entries(sc.transition, SF=sc.transition + 1), 1)


# ------------------------------------------------------------ goal search
def _golden_cases():
    keyed, _ = read_golden("goal_set_4x4x4.txt")
    vols = {}
    for k, v in keyed.items():
        if k[0] == "v" and k[1:].isdigit():
            vols[int(k[1:])] = [tuple(v[i:i + 4]) for i in range(0, len(v), 4)]
    cases = []
    for n in range(1, 100):
        if f"c{n}_v" not in keyed:
            break
        g = keyed[f"c{n}_goals"]
        cases.append((n, vols[keyed[f"c{n}_v"][0]], [tuple(g[i:i + 8]) for i in range(0, len(g), 8)],
                      keyed[f"c{n}_best"]))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: f"case{c[0]}")
def test_goal_set_hand_worked(case):
    _, cells, goals, best = case
    o = O.Oracle(2, 2, 1.0)
    V = np.full(o.nr, O.INF, np.uint32)
    for x, y, t, v in cells:
        V[o.cell((x, y, t))] = v
    got = o.goal_search(V, goals)
    if best == [-1]:
        assert got is None
    else:
        assert got == (o.cell(tuple(best[:3])), best[3])


def _swept(seed=3, lx=4, lt=3):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.1, turn_radius=2.5, soft=True)
    o = O.Oracle(lx, lt, 2.5, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    V, _, _ = o.sweep(B, o.cell(sc.start), 2)
    return o, V


def test_goal_set_zero_weights_over_the_grid_is_the_minimum():
    o, V = _swept()
    # two goals at opposite headings, boxes of N_theta - 1 headings each: together every pose
    rt = o.nt // 2 - 1
    goals = [(o.nx // 2, o.nx // 2, 0, o.nx, rt, 0, 0, 0), (o.nx // 2, o.nx // 2, o.nt // 2, o.nx, rt, 0, 0, 0)]
    cell, score = o.goal_search(V, goals)
    reached = V[V != O.INF]
    assert score == reached.min() and V[cell] == reached.min()
    # the minimum of a swept volume is the start (V = 0), unique
    assert score == 0 and np.count_nonzero(V == 0) == 1


def test_goal_set_huge_weights_pick_the_ideal_pose():
    o, V = _swept()
    reached = np.flatnonzero(V != O.INF)
    rng = np.random.default_rng(0)
    for c in rng.choice(reached, 10, replace=False):
        x, y, t = o.pose(int(c))
        got = o.goal_search(V, [(x, y, t, 3, 2, 1 << 31, 1 << 31, 0)])
        assert got == (int(c), int(V[c]))


def test_goal_set_radius_zero_is_the_exact_goal():
    o, V = _swept()
    for c in [int(np.flatnonzero(V != O.INF)[5]), int(np.flatnonzero(V == O.INF)[0])]:
        x, y, t = o.pose(c)
        got = o.goal_search(V, [(x, y, t, 0, 0, 7, 9, 0)])
        assert got == (None if V[c] == O.INF else (c, int(V[c])))


def test_goal_set_rejects_malformed_goals():
    o, V = _swept()
    for bad in [(o.nx, 0, 0, 1, 1, 0, 0, 0), (0, 0, 0, 256, 0, 0, 0, 0), (0, 0, 0, 1, o.nt // 2, 0, 0, 0),
                (0, 0, 0, 1, 1, -1, 0, 0), (0, 0, 0, 1, 1, 0, 0, 1 << 32)]:
        with pytest.raises(ValueError):
            o.goal_search(V, [bad])

"""Start state of a vehicle under way (Section XII) and goal-set search
(Section IX) on the GPU, through the C ABI, against the oracle: values and
labels bit for bit after a sweep from a start state, best pose, score and
back-tracked plan of goal sets, on small grids and on the 512^3 parking
scene."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


def planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


def entries(ct, **over):
    e = [ct] * 6
    names = dict(LF=O.LF, SF=O.SF, RB=O.RB, RF=O.RF, SB=O.SB, LB=O.LB)
    for k, v in over.items():
        e[names[k]] = v
    return e


def segs_of(o, ref):
    return [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]


def got_segs(res):
    return [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments]


CASES = [
    # lx, lt, R, footprint, soft, N, entry (fractions of ct as negative divisors)
    (3, 3, 2.0, (0, 0, 0), True, 2, dict(LF=0)),
    (4, 5, 3.0, (2, 1, 1), True, 2, dict(SF=0, RB=-3)),
    (5, 6, 6.0, (3, 1, 1), True, 2, dict(SB=0)),
    (5, 9, 9.0, (3, 1, 1), True, 1, dict(RF=0, LB=-2)),
    (6, 5, 10.0, (4, 1, 2), True, 2, dict(LF=-4, SF=-4, RB=-4, RF=0, SB=-4, LB=-4)),
    (7, 7, 12.0, (4, 1, 2), False, 1, dict(RB=0)),
    (10, 5, 20.0, (4, 1, 2), True, 1, dict(SF=0)),  # straight lines longer than one 1024-thread chunk
]


@pytest.mark.parametrize("case", CASES, ids=[f"nx{1 << c[0]}_nt{1 << c[1]}" for c in CASES])
def test_start_state_bit_exact(case):
    lx, lt, R, fp, soft, N, ent = case
    sc, img = scenes.tiny(700 + lx * 16 + lt, lx, lt, fill=0.05, turn_radius=R, footprint=fp, soft=soft,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    ct = sc.transition
    e = entries(ct, **{k: (ct // -v if v < 0 else v) for k, v in ent.items()})
    p = planner(sc, img)
    p.render()
    for start in [c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD][:2]:
        Vo, Lo, _ = o.sweep_state(Bo, o.cell(start), e, N, mode=1)
        p.sweep_state(start, e, N)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
        assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
        reached = np.flatnonzero(Vo != INF)
        rng = np.random.default_rng(lx * 7 + lt)
        for g in rng.choice(reached, size=min(20, len(reached)), replace=False):
            got = p.extract(o.pose(int(g)))
            assert got.cost == Vo[g] and got_segs(got) == segs_of(o, o.extract(Vo, Lo, int(g)))
    # at rest: plan_sweep's bits exactly
    p.sweep_state(start, [ct] * 6, N)
    Vr, Lr, _ = p.volumes(B=False)
    p.sweep(start, N)
    V0, L0, _ = p.volumes(B=False)
    assert np.array_equal(Vr, V0) and np.array_equal(Lr, L0)
    p.close()


def test_start_state_rejects_entry_above_ct():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(3, 5, 5, fill=0.05)
    p = planner(sc, img)
    p.render()
    with pytest.raises(binding.PlanError) as e:
        p.sweep_state(sc.start, entries(sc.transition, LB=sc.transition + 1), 1)
    assert e.value.code == binding.PLAN_EINVAL
    p.close()


def _goal_sets(o, V, rng, n_sets):
    reached = np.flatnonzero(V != INF)
    out = []
    for _ in range(n_sets):
        k = int(rng.integers(1, 6))
        gs = []
        for c in rng.choice(reached, size=k):
            x, y, t = o.pose(int(c))
            # move the ideal pose off the reached cell now and then
            x = int(np.clip(x + rng.integers(-3, 4), 0, o.nx - 1))
            y = int(np.clip(y + rng.integers(-3, 4), 0, o.nx - 1))
            rt = int(rng.integers(0, min(6, (o.nt - 1) // 2) + 1))
            gs.append((x, y, t, int(rng.integers(0, 9)), rt, int(rng.integers(0, 400)), int(rng.integers(0, 400)),
                       int(rng.integers(0, 3000))))
        out.append(gs)
    return out


@pytest.mark.parametrize("lx,lt", [(4, 4), (6, 6), (7, 9)])
def test_goal_set_bit_exact(lx, lt):
    sc, img = scenes.tiny(900 + lx + lt, lx, lt, fill=0.05, turn_radius=2.0 + lx, footprint=(2, 1, 1), soft=True,
                          transition=300)
    o = O.Oracle(lx, lt, 2.0 + lx, transition=sc.transition)
    Bo = o.render(img, sc.footprint) if lx <= 6 else o.render_rows(img, sc.footprint)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    p.render()
    p.sweep(start, 2)
    V, L, _ = p.volumes(B=False)
    rng = np.random.default_rng(lx * 31 + lt)
    for gs in _goal_sets(o, V, rng, 15):
        want = o.goal_search(V, gs)
        got = p.extract_goal_set(gs)
        if want is None:
            assert got is None
            continue
        cell, score = want
        best, gscore, res = got
        assert best == o.pose(cell) and gscore == score
        assert res.cost == V[cell] and got_segs(res) == segs_of(o, o.extract(V, L, cell))
    p.close()


def test_goal_set_edge_cases():
    from paper_2306_01301_b300 import binding
    lx, lt = 6, 6
    sc, img = scenes.tiny(77, lx, lt, fill=0.05, turn_radius=6.0, soft=True, transition=300)
    o = O.Oracle(lx, lt, 6.0, transition=sc.transition)
    Bo = o.render(img, sc.footprint)
    p = planner(sc, img)
    p.render()
    p.sweep(sc.start, 2)
    V, L, _ = p.volumes(B=False)
    # nothing reached in any box
    far = [int(c) for c in np.flatnonzero(V == INF)[:3]]
    gs = [(*o.pose(c), 0, 0, 1, 1, 0) for c in far]
    assert o.goal_search(V, gs) is None and p.extract_goal_set(gs) is None
    # boxes at the grid's corners (clipped, not wrapped) and theta wrapping
    gs = [(0, 0, 0, 5, 3, 10, 10, 0), (o.nx - 1, o.nx - 1, o.nt - 1, 5, 3, 10, 10, 0)]
    want, got = o.goal_search(V, gs), p.extract_goal_set(gs)
    assert (want is None and got is None) or (got[0] == o.pose(want[0]) and got[1] == want[1])
    # many goals (more than one pick block of threads), every one its own radius-0 box
    reached = np.flatnonzero(V != INF)
    rng = np.random.default_rng(5)
    gs = [(*o.pose(int(c)), 0, 0, 0, 0, int(rng.integers(0, 5000))) for c in rng.choice(reached, 700)]
    want, got = o.goal_search(V, gs), p.extract_goal_set(gs)
    assert got[0] == o.pose(want[0]) and got[1] == want[1]
    # ties between goals: two distinct cells of equal value, each a radius-0 goal; the earlier goal wins
    vals, counts = np.unique(V[reached], return_counts=True)
    v = vals[np.flatnonzero(counts > 1)[0]]
    a, b = [int(c) for c in np.flatnonzero(V == v)[:2]]
    for first, second in [(a, b), (b, a)]:
        gs = [(*o.pose(first), 0, 0, 0, 0, 0), (*o.pose(second), 0, 0, 0, 0, 0)]
        assert o.goal_search(V, gs) == (first, int(v))
        assert p.extract_goal_set(gs)[0] == o.pose(first)
    # malformed goals are refused
    for bad in [(o.nx, 0, 0, 1, 1, 0, 0, 0), (0, 0, 0, 256, 0, 0, 0, 0), (0, 0, 0, 1, o.nt // 2, 0, 0, 0)]:
        with pytest.raises(binding.PlanError) as e:
            p.extract_goal_set([bad])
        assert e.value.code == binding.PLAN_EINVAL
    with pytest.raises(binding.PlanError):
        p.extract_goal_set([])
    p.close()


def test_parking_512cubed_start_state_and_goal_set():
    """Full size, the benchmark's scene: one cycle from a start with straight
    forward in progress and a right-backward transition half done, bit for
    bit; then the full cycle count, checked for what holds at any size (never
    worse than from rest, consistent plans), and a goal set around the goal
    against the oracle's search of the same volume."""
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    ct = sc.transition
    e = entries(ct, SF=0, RB=ct // 2)
    p = planner(sc, img)
    p.render()
    p.sweep_state(sc.start, e, 1)
    V1, L1, _ = p.volumes(B=False)
    Vo, Lo, _ = o.sweep_state(Bo, o.cell(sc.start), e, 1, mode=1)
    assert np.array_equal(V1, Vo), f"values differ at {np.flatnonzero(V1 != Vo)[:5]}"
    assert np.array_equal(L1, Lo), f"labels differ at {np.flatnonzero(L1 != Lo)[:5]}"
    del Vo, Lo, Bo
    p.sweep(sc.start, sc.n_cycles)
    Vrest, _, _ = p.volumes(B=False, L=False)
    p.sweep_state(sc.start, e, sc.n_cycles)
    VN, LN, _ = p.volumes(B=False)
    assert np.all(VN <= V1) and np.all(VN <= Vrest)
    gx, gy, gt = sc.goal
    gs = [(gx, gy, gt, 6, 4, 40, 60, 0), (gx, gy, (gt + o.nt // 2) % o.nt, 6, 4, 40, 60, 500)]
    want = o.goal_search(VN, gs)
    got = p.extract_goal_set(gs)
    assert want is not None and got is not None
    best, score, res = got
    assert best == o.pose(want[0]) and score == want[1] and res.cost == VN[want[0]]
    segs = res.segments
    assert segs[-1]["exit"] == best and segs[0]["entry"] == tuple(sc.start)
    for a, b in zip(segs, segs[1:]):
        assert b["entry"] == a["exit"] and b["cost"] > a["cost"]
    p.close()

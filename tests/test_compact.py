"""The Compact graph (Section V.A, Fig. 12) on the GPU, through the C ABI,
against the oracle: the values and labels of all three vertex types bit for
bit and the back-tracked plans segment for segment on grids from 8^2 x 8 to
128^2 x 512, and two cycles of the 512^3 parking scene."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu


def planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


CASES = [
    # lx, lt, R, footprint, N
    (3, 3, 2.0, (0, 0, 0), 2),
    (4, 5, 3.0, (2, 1, 1), 2),
    (5, 7, 7.5, (2, 1, 1), 2),
    (6, 6, 10.0, (4, 1, 2), 2),
    (7, 9, 14.0, (3, 1, 1), 1),
    # several cycles through the fused turn pairs (LB, then the next cycle's LF)
    (5, 8, 6.0, (2, 1, 1), 3),
    (6, 7, 9.0, (3, 1, 1), 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"nx{1 << c[0]}_nt{1 << c[1]}" for c in CASES])
def test_compact_graph_bit_exact(case):
    lx, lt, R, fp, N = case
    sc, img = scenes.tiny(1000 + lx * 16 + lt, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    p.set_compact_graph(True)
    p.render()
    p.sweep_compact(start, N)
    got = p.compact_volumes()
    Vo, Lo = o.sweep_compact(Bo, o.cell(start), N)
    nr = o.nr
    want = (Vo[:nr], Lo[:nr], Vo[nr:2 * nr], Lo[nr:2 * nr], Vo[2 * nr:], Lo[2 * nr:])
    for name, a, b in zip(("V_S", "L_S", "V_L", "L_L", "V_R", "L_R"), got, want):
        assert np.array_equal(a, b), f"{name} differs at {np.flatnonzero(a != b)[:5]}"
    reached = np.flatnonzero(Vo[:nr] != O.INF)
    rng = np.random.default_rng(lx + lt)
    for g in rng.choice(reached, size=min(20, len(reached)), replace=False):
        res = p.extract_compact(o.pose(int(g)))
        ref = o.extract_compact(Vo, Lo, int(g))
        assert res.cost == Vo[g]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_compact_calls_are_checked():
    sc, img = scenes.tiny(11, 5, 5, fill=0.05)
    from paper_2306_01301_b300 import binding
    p = planner(sc, img)
    p.render()
    with pytest.raises(binding.PlanError) as e:
        p.sweep_compact(sc.start, 1)
    assert e.value.code == -8
    p.set_compact_graph(True)
    with pytest.raises(binding.PlanError):
        p.extract_compact(sc.goal)  # nothing swept yet
    p.sweep_compact(sc.start, 1)
    with pytest.raises(binding.PlanError) as e:
        p.extract(sc.goal)  # the Star's back-track does not read Compact volumes
    assert e.value.code == -8
    p.set_compact_graph(False)
    with pytest.raises(binding.PlanError):
        p.sweep_compact(sc.start, 1)
    p.close()


def test_parking_512cubed_compact_graph_two_cycles():
    """Full size, two cycles: the fused turn pairs within and across cycles."""
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    p = planner(sc, img)
    p.set_compact_graph(True)
    p.render()
    p.sweep_compact(sc.start, 2)
    got = p.compact_volumes()
    Vo, Lo = o.sweep_compact(Bo, o.cell(sc.start), 2)
    nr = o.nr
    want = (Vo[:nr], Lo[:nr], Vo[nr:2 * nr], Lo[nr:2 * nr], Vo[2 * nr:], Lo[2 * nr:])
    for name, a, b in zip(("V_S", "L_S", "V_L", "L_L", "V_R", "L_R"), got, want):
        assert np.array_equal(a, b), f"{name} differs at {np.flatnonzero(a != b)[:5]}"
    p.close()


def test_compact_graph_costs_beyond_the_scan_range():
    """A transition cost whose sums could reach 2^30: the two-loop walks on a
    grid the scan would otherwise take, against the oracle."""
    lx, lt, R, fp, N = 5, 7, 7.5, (2, 1, 1), 3
    sc, img = scenes.tiny(1077, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True, transition=1 << 26)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    p.set_compact_graph(True)
    p.render()
    p.sweep_compact(start, N)
    got = p.compact_volumes()
    Vo, Lo = o.sweep_compact(Bo, o.cell(start), N)
    nr = o.nr
    want = (Vo[:nr], Lo[:nr], Vo[nr:2 * nr], Lo[nr:2 * nr], Vo[2 * nr:], Lo[2 * nr:])
    for name, a, b in zip(("V_S", "L_S", "V_L", "L_L", "V_R", "L_R"), got, want):
        assert np.array_equal(a, b), f"{name} differs at {np.flatnonzero(a != b)[:5]}"
    assert (Vo[:nr][Vo[:nr] != O.INF] >= 1 << 26).sum() > 0
    p.close()

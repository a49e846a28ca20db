"""Two gear states on the GPU, through the C ABI, against the oracle: both
states' values and labels bit for bit for vehicles standing in forward or
reverse gear or at rest, with and without per-maneuver transition costs,
back-tracked plans segment for segment, and two cycles of the 512^3 parking
scene."""
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
    # lx, lt, R, footprint, N, pen, start gear, per-maneuver costs
    (2, 2, 1.5, (0, 0, 0), 2, 200, 2, None),
    (3, 3, 2.0, (0, 0, 0), 2, 450, 0, None),
    (4, 5, 3.0, (2, 1, 1), 2, 900, 1, ([300, 100, 900, 300, 700, 900], [0, 0, 50, 0, 50, 50])),
    (5, 7, 7.5, (2, 1, 1), 1, 1500, 0, None),
    (6, 6, 10.0, (4, 1, 2), 2, 700, 2, ([100, 50, 400, 120, 450, 380], [150, 60, 300, 170, 250, 320])),
    (7, 9, 14.0, (3, 1, 1), 1, 2500, 1, None),
    # the fused turn pairs across cycles (LB, then the next cycle's LF)
    (5, 8, 6.0, (2, 1, 1), 2, 1100, 2, ([200, 80, 500, 150, 600, 450], [40, 0, 90, 30, 20, 70])),
    (6, 7, 9.0, (3, 1, 1), 3, 600, 0, None),
    # a penalty whose sums could reach 2^30: the two-loop walks on a grid the scan would take
    (5, 7, 7.5, (2, 1, 1), 2, 1 << 27, 1, None),
]


@pytest.mark.parametrize("case", CASES, ids=[f"nx{1 << c[0]}_nt{1 << c[1]}_g{c[6]}" for c in CASES])
def test_gear_states_bit_exact(case):
    lx, lt, R, fp, N, pen, gear, costs = case
    sc, img = scenes.tiny(600 + lx * 16 + lt, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    if costs:
        o.set_transition(*costs)
        p.set_transition_costs(*costs)
    p.set_gear_penalty(pen)
    p.render()
    p.sweep_gear(start, gear, N)
    Vf, Lf, _ = p.volumes(B=False)
    Vr, Lr = p.reverse_volumes()
    Vo, Lo = o.sweep_gear(Bo, o.cell(start), gear, pen, N)
    nr = o.nr
    for name, got, want in [("V forward", Vf, Vo[:nr]), ("V reverse", Vr, Vo[nr:]),
                            ("L forward", Lf, Lo[:nr]), ("L reverse", Lr, Lo[nr:])]:
        assert np.array_equal(got, want), f"{name} differs at {np.flatnonzero(got != want)[:5]}"
    best = np.minimum(Vo[:nr], Vo[nr:])
    reached = np.flatnonzero(best != O.INF)
    rng = np.random.default_rng(lx + lt)
    for g in rng.choice(reached, size=min(20, len(reached)), replace=False):
        ref = o.extract_gear(Vo, Lo, int(g))
        res, end_gear = p.extract_gear(o.pose(int(g)))
        assert res.cost == best[g] and end_gear == (1 if Vo[nr + g] < Vo[g] else 0)
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_gear_calls_are_checked():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(8, 5, 5, fill=0.05)
    p = planner(sc, img)
    p.render()
    with pytest.raises(binding.PlanError) as e:
        p.sweep_gear(sc.start, 0, 1)  # no gear penalty set
    assert e.value.code == -8
    with pytest.raises(binding.PlanError) as e:
        p.set_gear_penalty(1 << 28)
    assert e.value.code == binding.PLAN_EINVAL
    p.set_gear_penalty(100)
    with pytest.raises(binding.PlanError) as e:
        p.sweep_gear(sc.start, 3, 1)
    assert e.value.code == binding.PLAN_EINVAL
    with pytest.raises(binding.PlanError):
        p.extract_gear(sc.goal)  # nothing swept yet
    # each back-track reads only volumes of its own kind of sweep
    p.sweep_gear(sc.start, 0, 1)
    with pytest.raises(binding.PlanError) as e:
        p.extract(sc.goal)
    assert e.value.code == -8
    p.sweep(sc.start, 1)
    with pytest.raises(binding.PlanError) as e:
        p.extract_gear(sc.goal)
    assert e.value.code == -8
    p.extract(sc.goal)
    p.set_gear_penalty(None)
    with pytest.raises(binding.PlanError):
        p.sweep_gear(sc.start, 0, 1)
    p.close()


def test_parking_512cubed_gear_states_two_cycles():
    """Full size, two cycles: the fused turn pairs within and across cycles."""
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    p = planner(sc, img)
    p.set_gear_penalty(3000)
    p.render()
    p.sweep_gear(sc.start, 0, 2)
    Vf, Lf, _ = p.volumes(B=False)
    Vr, Lr = p.reverse_volumes()
    Vo, Lo = o.sweep_gear(Bo, o.cell(sc.start), 0, 3000, 2)
    nr = o.nr
    assert np.array_equal(Vf, Vo[:nr]) and np.array_equal(Vr, Vo[nr:])
    assert np.array_equal(Lf, Lo[:nr]) and np.array_equal(Lr, Lo[nr:])
    p.close()

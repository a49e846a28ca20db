"""Per-maneuver Star transition edges (Section V.A, Fig. 9) on the GPU,
through the C ABI, against the oracle: values and labels bit for bit on
grids that exercise every turn-kernel shape and the straight kernels, with a
start state, and on the 512^3 parking scene for one cycle."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu

COSTS = [
    ([300, 100, 900, 300, 700, 900], [0, 0, 0, 0, 0, 0]),
    ([100, 50, 400, 120, 450, 380], [150, 60, 300, 170, 250, 320]),
    ([0, 0, 0, 0, 0, 0], [500, 20, 900, 40, 600, 800]),
]

GRIDS = [
    # lx, lt, R, footprint, soft, N
    (3, 3, 2.0, (0, 0, 0), True, 2),
    (4, 5, 3.0, (2, 1, 1), True, 2),
    (5, 7, 7.5, (2, 1, 1), False, 2),
    (5, 9, 9.0, (3, 1, 1), True, 1),
    (6, 6, 10.0, (4, 1, 2), True, 2),
]


def planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


@pytest.mark.parametrize("grid", GRIDS, ids=[f"nx{1 << g[0]}_nt{1 << g[1]}" for g in GRIDS])
def test_per_maneuver_costs_bit_exact(grid):
    lx, lt, R, fp, soft, N = grid
    sc, img = scenes.tiny(300 + lx * 16 + lt, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=soft,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    p.render()
    for cin, cout in COSTS:
        o.set_transition(cin, cout)
        p.set_transition_costs(cin, cout)
        Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
        p.sweep(start, N)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
        assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
        # a start state on top: straight forward in progress
        entry = list(cin)
        entry[O.SF] = 0
        Vo, Lo, _ = o.sweep_state(Bo, o.cell(start), entry, N, mode=1)
        p.sweep_state(start, entry, N)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
        reached = np.flatnonzero(Vo != 0xFFFFFFFF)
        rng = np.random.default_rng(lx + lt)
        for g in rng.choice(reached, size=min(10, len(reached)), replace=False):
            got = p.extract(o.pose(int(g)))
            ref = o.extract(Vo, Lo, int(g))
            assert got.cost == Vo[g]
            assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in got.segments] == \
                   [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    # back to the defaults: plan_create's uniform ct
    p.set_transition_costs([sc.transition] * 6, [0] * 6)
    o.set_transition([sc.transition] * 6, [0] * 6)
    p.sweep(start, N)
    V, L, _ = p.volumes(B=False)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
    p.close()


def test_invalid_costs_are_refused():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(5, 5, 5, fill=0.05)
    p = planner(sc, img)
    with pytest.raises(binding.PlanError) as e:
        p.set_transition_costs([1 << 27] * 6, [1 << 27] * 6)
    assert e.value.code == binding.PLAN_EINVAL
    p.set_transition_costs([100] * 6, [0] * 6)
    p.render()
    entry = [100] * 6
    entry[O.LB] = 101
    with pytest.raises(binding.PlanError):
        p.sweep_state(sc.start, entry, 1)
    p.close()


def test_parking_512cubed_per_maneuver_costs_one_cycle():
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    cin = [1500, 800, 2600, 1500, 2400, 2600]   # backward gear dearer to enter
    cout = [300, 100, 500, 300, 500, 500]
    o.set_transition(cin, cout)
    Bo = o.render_rows(img, sc.footprint)
    p = planner(sc, img)
    p.set_transition_costs(cin, cout)
    p.render()
    p.sweep(sc.start, 1)
    V, L, _ = p.volumes(B=False)
    Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), 1, mode=1)
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    p.close()

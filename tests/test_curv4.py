"""The 4D generalisation of Appendix F on the GPU, through the C ABI, against
the oracle: the library's clothoid tables equal the oracle's (both built
from the clothoid integrals, each with its own code), and the 4D values,
labels and back-tracked plans are bit for bit the oracle's, from start
curvatures across the levels, on grids up to 128^2 x 256 with up to 9
levels, and the values and labels of the 256^2 x 256 parking scene over 9
levels and two cycles."""
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
    # lx, lt, R, footprint, M, L, clothoid cost, N, start level
    (2, 3, 1.5, (0, 0, 0), 1, 1.0, 150, 2, 0),  # Nx = 4: one row per chain group of the clothoid layer
    (3, 3, 2.0, (0, 0, 0), 1, 1.0, 150, 1, 0),
    (4, 4, 3.0, (1, 0, 0), 2, 1.0, 200, 2, 1),
    (5, 6, 6.0, (2, 1, 1), 3, 0.75, 300, 2, -2),
    (6, 7, 10.0, (3, 1, 1), 4, 0.9, 250, 1, 0),
    (7, 7, 14.0, (4, 1, 2), 4, 1.0, 400, 1, 3),
    # several cycles on a grid whose 3D layers take the persistent turn shape
    (7, 8, 12.0, (3, 1, 1), 4, 1.0, 350, 3, -1),
    # a clothoid cost whose sums could reach 2^30: the saturating walks
    (5, 6, 6.0, (2, 1, 1), 2, 1.0, 1 << 27, 2, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"nx{1 << c[0]}_nt{1 << c[1]}_M{c[4]}" for c in CASES])
def test_curvature_levels_bit_exact(case):
    lx, lt, R, fp, M, L, ctc, N, lev = case
    sc, img = scenes.tiny(800 + lx * 16 + lt, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    q = O.Oracle4(o, M, L, ctc)
    Bo = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p = planner(sc, img)
    p.set_curvature_levels(M, L, ctc)
    for got, want in zip(p.clothoid_tables(), q.tables()):
        assert np.array_equal(got, want), "clothoid tables differ"
    p.render()
    p.sweep4(start, lev, N)
    V, Lb = p.volumes4()
    Vo, Lo = q.sweep(Bo, q.cell(start, lev), N)
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(Lb, Lo), f"labels differ at {np.flatnonzero(Lb != Lo)[:5]}"
    reached = np.flatnonzero(Vo != O.INF)
    assert len(np.unique(reached // o.nr)) > 1, "the plans should use more than one curvature level"
    rng = np.random.default_rng(lx + lt + M)
    for g in rng.choice(reached, size=min(20, len(reached)), replace=False):
        gp, gl = q.pose(int(g))
        res = p.extract4(gp, gl)
        ref = q.extract(Vo, Lo, int(g))
        assert res.cost == Vo[g]
        assert [(s["mu"], s["entry"], s["entry_level"], s["exit"], s["exit_level"], s["steps"], s["cost"])
                for s in res.segments] == \
               [(s["mu"], *q.pose(s["entry"]), *q.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_curvature_calls_are_checked():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(9, 5, 5, fill=0.05)
    p = planner(sc, img)
    p.render()
    with pytest.raises(binding.PlanError) as e:
        p.sweep4(sc.start, 0, 1)
    assert e.value.code == -8
    for bad in [(1001, 1.0, 0), (2, 0.0, 0), (2, 5.0, 0), (2, 1.0, 1 << 28)]:
        with pytest.raises(binding.PlanError) as e:
            p.set_curvature_levels(*bad)
        assert e.value.code == binding.PLAN_EINVAL
    p.set_curvature_levels(2, 1.0, 100)
    with pytest.raises(binding.PlanError):
        p.sweep4(sc.start, 3, 1)  # level outside -2 .. 2
    with pytest.raises(binding.PlanError):
        p.extract4(sc.goal, 0)  # nothing swept yet
    p.set_curvature_levels(0)
    with pytest.raises(binding.PlanError):
        p.sweep4(sc.start, 0, 1)
    p.close()


def test_curvature_levels_parking_256_bit_exact():
    """The parking scene at 256^2 x 256 over 9 levels, two cycles: the plain
    kernels' persistent shapes on a level and the clothoid layer at a size
    where its four chains per thread span many blocks."""
    sc = scenes.parallel_parking(nx_log2=8, nt_log2=8, n_cycles=2)
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    q = O.Oracle4(o, 4, 1.0, 500)
    Bo = o.render_rows(img, sc.footprint)
    p = planner(sc, img)
    p.set_curvature_levels(4, 1.0, 500)
    p.render()
    p.sweep4(sc.start, 0, 2)
    V, Lb = p.volumes4()
    Vo, Lo = q.sweep(Bo, q.cell(sc.start, 0), 2)
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(Lb, Lo), f"labels differ at {np.flatnonzero(Lb != Lo)[:5]}"
    p.close()

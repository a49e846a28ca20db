"""Direction penalties (Section XVI, Fig. 19) on the GPU, through the C ABI,
against the oracle: the penalised obstacle volume B and the sweep's values
and labels bit for bit, on grids that take the scalar (Nx = 4) and the
16-byte (Nx >= 8) kernel, with soft costs, and on the 512^3 parking scene
with a two-lane road."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu
NONE = 0xFFFF


def planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


def random_field(rng, nx, nt):
    f = rng.integers(0, nt, (nx, nx)).astype(np.uint16)
    f[rng.random((nx, nx)) < 0.3] = NONE
    return f


GRIDS = [
    # lx, lt, R, footprint, N, tol, pen
    (2, 2, 1.5, (0, 0, 0), 2, 0, 512),
    (3, 3, 2.0, (0, 0, 0), 2, 1, 700),
    (4, 5, 3.0, (2, 1, 1), 2, 3, 1024),
    (6, 6, 10.0, (4, 1, 2), 2, 8, 600),
    (7, 7, 12.0, (4, 1, 2), 1, 16, 2000),
]


@pytest.mark.parametrize("grid", GRIDS, ids=[f"nx{1 << g[0]}_nt{1 << g[1]}" for g in GRIDS])
def test_direction_penalties_bit_exact(grid):
    lx, lt, R, fp, N, tol, pen = grid
    sc, img = scenes.tiny(400 + lx * 16 + lt, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True,
                          transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    rng = np.random.default_rng(lx * 10 + lt)
    field = random_field(rng, o.nx, o.nt)
    B0 = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    Bo = o.direction(B0, field, tol, pen)
    assert not np.array_equal(Bo, B0)
    p = planner(sc, img)
    p.set_direction_field(field, tol, pen)
    p.render()
    _, _, B = p.volumes(V=False, L=False)
    assert np.array_equal(B, Bo), f"B differs at {np.flatnonzero(B != Bo)[:5]}"
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    p.sweep(start, N)
    V, L, _ = p.volumes(B=False)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
    # removing the field renders the plain volume again
    p.set_direction_field(None)
    p.render()
    _, _, B = p.volumes(V=False, L=False)
    assert np.array_equal(B, B0)
    p.close()


def test_batch_renders_the_direction_fields():
    """A batch renders every member's B as plan_render_cspace would, its
    direction field included, and replays its graph again when a field
    changes."""
    from paper_2306_01301_b300 import binding
    lx, lt = 6, 6
    sc, img = scenes.tiny(21, lx, lt, fill=0.05, turn_radius=8.0, footprint=(3, 1, 1), soft=True, transition=300)
    o = O.Oracle(lx, lt, 8.0, transition=sc.transition)
    B0 = o.render(img, sc.footprint)
    starts = [c for c in sc.pose_candidates if B0[o.cell(c)] != O.HARD][:2]
    rng = np.random.default_rng(4)
    fields = [random_field(rng, o.nx, o.nt), None]
    planners = [planner(sc, img) for _ in starts]
    planners[0].set_direction_field(fields[0], 5, 900)
    b = binding.Batch(planners)
    for rep in range(2):
        b.run([(s, sc.goal, 2) for s in starts], render=True)
        b.sync()
        for q, f, s in zip(planners, fields, starts):
            _, _, B = q.volumes(V=False, L=False)
            Bo = B0 if f is None else o.direction(B0, f, 5 if rep == 0 else 2, 900 if rep == 0 else 400)
            assert np.array_equal(B, Bo)
            V, L, _ = q.volumes(B=False)
            Vo, Lo, _ = o.sweep(Bo, o.cell(s), 2, mode=1)
            assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
        planners[0].set_direction_field(fields[0], 2, 400)  # a new tolerance and penalty: a new graph
    b.close()
    for q in planners:
        q.close()


def test_direction_field_is_checked():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(6, 4, 4, fill=0.05)
    p = planner(sc, img)
    for field, tol, pen in [(np.full((16, 16), 16, np.uint16), 0, 512),
                            (np.zeros((16, 16), np.uint16), 9, 512),
                            (np.zeros((16, 16), np.uint16), 0, 255)]:
        with pytest.raises(binding.PlanError) as e:
            p.set_direction_field(field, tol, pen)
        assert e.value.code == binding.PLAN_EINVAL
    # a new field needs a new rendering before the next sweep
    p.render()
    p.set_direction_field(np.zeros((16, 16), np.uint16), 2, 512)
    with pytest.raises(binding.PlanError):
        p.sweep(sc.start, 1)
    p.close()


def test_parking_512cubed_two_lane_road():
    """Lower half of the map drives toward +x (heading 0), upper half toward
    -x (heading pi), within 1/8 turn; against the lane costs 2x."""
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    field = np.zeros((o.nx, o.nx), np.uint16)
    field[o.nx // 2:, :] = o.nt // 2
    B0 = o.render_rows(img, sc.footprint)
    Bo = o.direction(B0, field, o.nt // 8, 512)
    del B0
    p = planner(sc, img)
    p.set_direction_field(field, o.nt // 8, 512)
    p.render()
    p.sweep(sc.start, 1)
    V, L, B = p.volumes()
    assert np.array_equal(B, Bo), f"B differs at {np.flatnonzero(B != Bo)[:5]}"
    Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), 1, mode=1)
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    p.close()

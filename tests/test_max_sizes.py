"""GPU path at the edges of the supported sizes (the grid limits of
plan_create: N_x up to 4096, N_theta up to 1024, at most 2^32 pose cells).

* N_theta = 1024, the largest heading count: every turn-kernel shape the
  library has for it (thread-block clusters of 2, 4 and 8 blocks), one block
  per work item and a persistent grid, bit-exact B, V and L against the
  oracle.
* N_x = 4096, the largest grid side: straight lines of 4096 cells (256
  chunks of the staged straight kernel), bit-exact B, V and L against the
  oracle.
* 2^32 pose cells (4096^2 x 256), where the kernels' 32-bit cell offsets
  reach their limit: too large for the oracle's volumes, so the check uses
  free space, where Section V's costs give exact closed forms (a straight
  step at heading 0 costs w_S = 100, a turn step w_A, entering a maneuver
  ct; the oracle's own successor map, eqs. 25-31, walks the expected goal),
  including poses in the last heading plane, whose cell indices are the
  largest.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu


def _planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


def _first_free(o, B, cands):
    for c in cands:
        if B[o.cell(c)] != O.HARD:
            return c
    raise AssertionError("no free candidate pose")


def test_1024_headings_every_turn_shape_bit_exact():
    lx, lt, R, N = 5, 10, 9.0, 2
    sc, img = scenes.tiny(910, lx, lt, fill=0.05, turn_radius=R, footprint=(3, 1, 1), soft=True, transition=400)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, sc.footprint)
    start = _first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    assert (Vo != O.INF).sum() > 1000
    p = _planner(sc, img)
    p.render()
    first = True
    for variant in range(3):           # clusters of 2, 4 and 8 blocks
        for grid in (0, 5):            # one block (cluster) per item, or a persistent grid
            p.set_kernel_shapes(variant, grid, 0, 0)
            p.sweep(start, N)
            V, L, B = p.volumes(B=first)
            if first:
                assert np.array_equal(B, Bo), "obstacle volume"
                first = False
            assert np.array_equal(V, Vo), (variant, grid, np.flatnonzero(V != Vo)[:5])
            assert np.array_equal(L, Lo), (variant, grid, np.flatnonzero(L != Lo)[:5])
    p.close()


def test_nx_4096_bit_exact():
    lx, lt, R, N = 12, 2, 40.0, 1
    sc, img = scenes.tiny(911, lx, lt, fill=0.0003, turn_radius=R, footprint=(2, 1, 1), soft=True, transition=500)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    start = _first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    assert (Vo != O.INF).sum() > 1_000_000
    assert (Lo[Lo != O.NONE] & 8191).max() > 2000  # segments thousands of steps long
    p = _planner(sc, img)
    p.render()
    p.sweep(start, N)
    V, L, B = p.volumes()
    assert np.array_equal(B, Bo), "obstacle volume"
    del B, Bo
    assert np.array_equal(V, Vo), np.flatnonzero(V != Vo)[:5]
    assert np.array_equal(L, Lo), np.flatnonzero(L != Lo)[:5]
    # plans to the far end of the longest straight lines
    reached = np.flatnonzero(Vo != O.INF)
    rng = np.random.default_rng(7)
    for g in rng.choice(reached, size=10, replace=False):
        got = p.extract(o.pose(int(g)))
        ref = o.extract(Vo, Lo, int(g))
        assert got.cost == Vo[g]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in got.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_two_to_the_32_cells_free_space_closed_forms():
    from paper_2306_01301_b300 import binding
    lx, lt, R, ct = 12, 8, 100.0, 2000
    nx, nt = 1 << lx, 1 << lt
    assert 2 * lx + lt == 32
    img = np.full((nx, nx), scenes.FREE, np.uint16)
    o = O.Oracle(lx, lt, R, transition=ct)
    tab = o.tables()
    wA, wS0 = tab["wA"], int(tab["wS"][0])
    start = (1000, 1000, 0)
    p = binding.Planner(lx, lt, img, (0, 0, 0), R, ct)
    p.render()
    p.sweep(start, 1)

    def walk(mu, k):
        c = o.cell(start)
        for _ in range(k):
            c = o.succ(mu, c)
        return o.pose(c)

    cases = [
        # Straight ahead.  The grid wraps around (only row 0 and column 0 are
        # walls, and a turn step of 2.5 cells can pass over a wall cell it does
        # not land on), so a pose 3000 cells ahead is cheaper the other way
        # round; below half the grid every path of two or more maneuvers
        # costs at least 2 ct + 99.8 per cell travelled, more than the line.
        (O.SF, 1, ct + wS0), (O.SF, 37, ct + 37 * wS0), (O.SF, 1500, ct + 1500 * wS0),
        (O.LF, nt // 4, ct + (nt // 4) * wA),    # a quarter circle to the left
        (O.RF, 1, ct + wA), (O.RF, 9, ct + 9 * wA),  # headings 255, 247: the last planes
    ]
    for mu, k, cost in cases:
        goal = walk(mu, k)
        got = p.extract(goal)
        assert got is not None, (mu, k)
        assert got.cost == cost, (mu, k, got.cost, cost)
        assert [(s["mu"], s["steps"], s["cost"]) for s in got.segments] == [(mu, k, cost)]
        assert tuple(got.segments[0]["exit"]) == tuple(goal)
    assert walk(O.RF, 1)[2] == nt - 1
    # the start itself and an unreachable pose (walls are hard)
    assert p.extract(start).cost == 0
    assert p.extract((0, 5, 0)) is None
    p.close()

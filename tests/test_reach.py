"""Bit-vector maneuver-count reachability (Appendix C) on the GPU against the
oracle: the fewest maneuvers of every pose bit for bit, and the canonical
back-tracked plans segment for segment, on grids from 64^2 x 32 to the
paper's 128^2 x 512 (Table 9); at 512^3 the plans are checked for validity
and minimality against the counts."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu


def _planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


def _segs(o, ref):
    return [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"]) for s in ref]


CASES = [
    # lx, lt, R, footprint, fill, N, half shift
    (6, 5, 5.0, (2, 1, 1), 0.04, 4, 1),
    (6, 6, 6.0, (0, 0, 0), 0.06, 5, 0),
    (7, 7, 12.0, (4, 1, 2), 0.01, 4, 1),
    (7, 9, 14.0, (3, 1, 1), 0.01, 8, 1),  # the resolution of Table 9
    (8, 8, 20.0, (6, 2, 2), 0.004, 3, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{1 << c[0]}^2x{1 << c[1]}" for c in CASES])
def test_reach_counts_and_plans_bit_exact(case):
    lx, lt, R, fp, fill, N, half = case
    sc, img = scenes.tiny(500 + lx * 16 + lt, lx, lt, fill=fill, turn_radius=R, footprint=fp,
                          half_shift=half, transition=300)
    o = O.Oracle(lx, lt, R, half_shift=half, transition=sc.transition)
    B = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
    start = next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD)
    want = o.reach(B, o.cell(start), N)
    p = _planner(sc, img)
    p.render()
    p.reach_sweep(start, N)
    got = p.reach_counts()
    assert np.array_equal(got, want), f"counts differ at {np.flatnonzero(got != want)[:5]}"
    rng = np.random.default_rng(lx + lt)
    reached = np.flatnonzero(want != 255)
    for g in rng.choice(reached, size=min(40, len(reached)), replace=False):
        ref = o.reach_extract(B, want, int(g))
        res = p.reach_extract(o.pose(int(g)))
        assert res is not None and res[0] == want[g]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"]) for s in res[1]] == _segs(o, ref)
    unreached = np.flatnonzero((want == 255) & (B != O.HARD))
    if len(unreached):
        assert p.reach_extract(o.pose(int(unreached[0]))) is None
    # a second sweep from another start reuses the buffers
    start2 = [c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD][1]
    p.reach_sweep(start2, N)
    assert np.array_equal(p.reach_counts(), o.reach(B, o.cell(start2), N))
    p.close()


def test_reach_full_size_parking_plans_are_valid():
    """512^3 parking scene, 8 cycles: counts are consistent (the start is the
    only pose at 0, hard poses never reached) and back-tracked plans to sampled
    poses are collision-free maneuver chains of exactly the counted length."""
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    p = _planner(sc, img)
    p.render()
    p.reach_sweep(sc.start, 8)
    cnt = p.reach_counts()
    _, _, B = p.volumes(V=False, L=False)
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    assert (cnt == 0).sum() == 1 and cnt[o.cell(sc.start)] == 0
    assert (cnt[B == O.HARD] == 255).all()
    reached = np.flatnonzero(cnt != 255)
    assert len(reached) > 1_000_000  # about 8 % of the poses: the 96x38 vehicle leaves much of the map hard
    rng = np.random.default_rng(3)
    for g in list(rng.choice(reached, size=25, replace=False)) + [o.cell(sc.goal)]:
        if cnt[g] == 255:
            continue
        m, segs = p.reach_extract(o.pose(int(g)))
        assert m == cnt[g] and len(segs) == m
        x = o.cell(sc.start)
        for k, s in enumerate(segs):
            assert o.cell(s["entry"]) == x and cnt[x] <= k
            y = x
            for _ in range(s["steps"]):
                y = o.succ(s["mu"], y)
                assert B[y] != O.HARD
            assert y == o.cell(s["exit"])
            x = y
        assert x == g
    p.close()


def test_reach_rejects_unsupported_grids():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(9, 5, 5, fill=0.05)
    p = _planner(sc, img)
    p.render()
    with pytest.raises(binding.PlanError) as e:
        p.reach_sweep(sc.start, 2)  # Nx = 32 is below the supported 64
    assert e.value.code == -1
    p.close()

"""GPU path (through the C ABI) against the CPU oracle: bit-exact obstacle
volume B, value volume V, labels L and extracted plans.

Small cases cover every turn-kernel shape (N_theta 4 .. 512), grids narrower
than a warp (Nx = 4, 8, 16), soft costs, rectangles, with and without the
half-cell shift.  Full-size cases run the 512^3 parallel-parking and maze
workloads in the launch configuration the benchmark uses: the full B and one
full cycle of V and L are compared cell by cell, and the full-N run is
checked for properties that hold at any size (monotone in N, a consistent
extracted plan ending at V(goal)).
"""
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


def first_free(o, B, cands):
    for c in cands:
        if B[o.cell(c)] != O.HARD:
            return c
    raise AssertionError("no free candidate pose")


SMALL = [
    # lx, lt, R, footprint, soft, half, N
    (2, 2, 1.5, (0, 0, 0), True, 1, 2),
    (3, 3, 2.0, (0, 0, 0), False, 1, 1),
    (3, 3, 2.0, (0, 0, 0), True, 1, 3),
    (4, 4, 2.5, (1, 0, 0), True, 0, 2),
    (4, 5, 3.0, (2, 1, 1), True, 1, 3),
    (5, 3, 4.0, (0, 0, 0), True, 1, 2),
    (5, 6, 6.0, (3, 1, 1), True, 1, 2),
    (5, 7, 7.5, (2, 1, 1), False, 1, 2),
    (4, 8, 5.0, (2, 1, 1), True, 1, 2),
    (5, 9, 9.0, (3, 1, 1), True, 0, 1),
    (6, 5, 10.0, (4, 1, 2), True, 1, 3),
]


@pytest.mark.parametrize("case", SMALL, ids=[f"nx{1 << c[0]}_nt{1 << c[1]}" for c in SMALL])
def test_small_grids_bit_exact(case):
    lx, lt, R, fp, soft, half, N = case
    sc, img = scenes.tiny(100 + lx * 16 + lt, lx, lt, fill=0.08, turn_radius=R, footprint=fp, soft=soft,
                          half_shift=half, transition=300)
    o = O.Oracle(lx, lt, R, half_shift=half, transition=sc.transition)
    Bo = o.render(img, fp)
    start = first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    p = planner(sc, img)
    p.render()
    p.sweep(start, N)
    V, L, B = p.volumes()
    assert np.array_equal(B, Bo), "obstacle volume"
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    # plans to every reached cell of a random sample
    reached = np.flatnonzero(Vo != INF)
    rng = np.random.default_rng(lx + lt)
    for g in rng.choice(reached, size=min(25, len(reached)), replace=False):
        ref = o.extract(Vo, Lo, int(g))
        got = p.extract(o.pose(int(g)))
        assert got.cost == Vo[g]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in got.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_single_query_64cubed_bit_exact():
    """The plain single-query workload: 64^3, point vehicle, N = 4."""
    sc = scenes.single_query(0)
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render(img, sc.footprint)
    Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), sc.n_cycles, mode=1)
    p = planner(sc, img)
    p.render()
    p.sweep(sc.start, sc.n_cycles)
    V, L, B = p.volumes()
    assert np.array_equal(B, Bo) and np.array_equal(V, Vo) and np.array_equal(L, Lo)
    ref = o.extract(Vo, Lo, o.cell(sc.goal))
    got = p.extract(sc.goal)
    if ref is None:
        assert got is None
    else:
        assert got.cost == Vo[o.cell(sc.goal)]
        assert [(s["mu"], s["steps"], s["cost"]) for s in got.segments] == \
               [(s["mu"], s["steps"], s["cost"]) for s in ref]
    # other start poses of the same scene, same plan object (state reset by sweep)
    for st in sc.pose_candidates[2:6]:
        Vo, Lo, _ = o.sweep(Bo, o.cell(st), sc.n_cycles, mode=1)
        p.sweep(st, sc.n_cycles)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
    p.close()


def test_errors_are_reported_not_raised_on_device():
    from paper_2306_01301_b300 import binding
    sc, img = scenes.tiny(5, 4, 4, fill=0.1, soft=True)
    p = planner(sc, img)
    with pytest.raises(binding.PlanError) as e:
        p.sweep(sc.start, 1)  # before rendering
    assert e.value.code == -8
    p.render()
    hard = np.argwhere(img == 0xFFFF)
    if len(hard):
        y, x = hard[0]
        with pytest.raises(binding.PlanError) as e:
            p.sweep((int(x), int(y), 0), 1)
        assert e.value.code == -1
    with pytest.raises(binding.PlanError):
        p.sweep((99, 0, 0), 1)
    p.sweep(sc.start, 0)  # zero cycles: only the start is reached
    V, L, _ = p.volumes(B=False)
    assert (V != INF).sum() == 1 and (L != 0xFFFF).sum() == 0
    assert p.extract((0, 0, 0)) is None  # wall cell: unreachable
    p.close()


def _full_size(sc, img, n_check=1):
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    p = planner(sc, img)
    p.render()
    p.sweep(sc.start, n_check)
    V1, L1, B = p.volumes()
    assert np.array_equal(B, Bo), "obstacle volume"
    Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), n_check, mode=1)
    assert np.array_equal(V1, Vo), f"values differ at {np.flatnonzero(V1 != Vo)[:5]}"
    assert np.array_equal(L1, Lo), f"labels differ at {np.flatnonzero(L1 != Lo)[:5]}"
    del Vo, Lo, Bo
    # the benchmark's full cycle count: properties that hold at any size
    p.sweep(sc.start, sc.n_cycles)
    VN, LN, _ = p.volumes(B=False)
    assert np.all(VN <= V1), "more cycles raised a value"
    res = p.extract(sc.goal)
    g = o.cell(sc.goal)
    if res is None:
        assert VN[g] == INF
    else:
        assert res.cost == VN[g]
        segs = res.segments
        assert segs[0]["entry"] == tuple(sc.start) and segs[-1]["exit"] == tuple(sc.goal)
        for a, b in zip(segs, segs[1:]):
            assert b["entry"] == a["exit"] and b["cost"] > a["cost"]
        assert segs[-1]["cost"] == res.cost
    p.close()
    return res


def test_parallel_parking_512cubed_full_size():
    sc = scenes.parallel_parking()
    _full_size(sc, sc.hard_image())


def test_parallel_parking_512cubed_all_cycles_bit_exact():
    """The benchmark's workload end to end, every cycle: 512^3, N = 8, the
    kernel shapes the autotuner picks for it (as bench.py times them), the
    whole V and L against the oracle's full 8-cycle sweep (its chains spread
    over the host's cores), and the plan to the goal."""
    import os
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    try:
        O.Oracle.set_threads(os.cpu_count() or 1)
        Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), sc.n_cycles, mode=1)
    finally:
        O.Oracle.set_threads(1)
    p = planner(sc, img)
    p.render()
    p.autotune(sc.start)
    p.sweep(sc.start, sc.n_cycles)
    V, L, _ = p.volumes(B=False)
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    del V, L
    res = p.extract(sc.goal)
    ref = o.extract(Vo, Lo, o.cell(sc.goal))
    assert (res is None) == (ref is None)
    if res is not None:
        assert res.cost == Vo[o.cell(sc.goal)]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


def test_maze_512cubed_all_32_cycles_bit_exact():
    """The maze workload end to end: 512^3, soft obstacle costs (Section
    VII), N = 32 cycles (129 passes, Insert 1 over 192 layers), the kernel
    shapes the autotuner picks for it, the whole V and L against the
    oracle's 32-cycle sweep (its chains spread over the host's cores), and
    the plan to the goal segment by segment."""
    import os
    from paper_2306_01301_b300 import binding
    sc = scenes.maze()
    img = binding.soft_image(sc.occupancy, sc.soft_radius, sc.soft_max)
    assert np.array_equal(img, O.soft_image(sc.occupancy, sc.soft_radius, sc.soft_max))
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    Bo = o.render_rows(img, sc.footprint)
    try:
        O.Oracle.set_threads(os.cpu_count() or 1)
        Vo, Lo, imp = o.sweep(Bo, o.cell(sc.start), sc.n_cycles, mode=1)
    finally:
        O.Oracle.set_threads(1)
    assert sc.n_cycles == 32 and imp[-12:].sum() >= 0
    p = planner(sc, img)
    p.render()
    p.autotune(sc.start)
    p.sweep(sc.start, sc.n_cycles)
    V, L, B = p.volumes()
    assert np.array_equal(B, Bo), "obstacle volume"
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    del V, L, B
    res = p.extract(sc.goal)
    ref = o.extract(Vo, Lo, o.cell(sc.goal))
    assert (res is None) == (ref is None)
    if res is not None:
        assert res.cost == Vo[o.cell(sc.goal)]
        assert [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments] == \
               [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]
    p.close()


@pytest.mark.parametrize("case", [SMALL[4], SMALL[7], SMALL[9]], ids=["nt32", "nt128", "nt512"])
def test_autotuned_shapes_give_the_same_bits(case):
    """plan_autotune times every kernel shape and keeps the fastest; sweeps
    with the chosen shapes still equal the oracle."""
    lx, lt, R, fp, soft, half, N = case
    sc, img = scenes.tiny(300 + lx * 16 + lt, lx, lt, fill=0.08, turn_radius=R, footprint=fp, soft=soft,
                          half_shift=half, transition=300)
    o = O.Oracle(lx, lt, R, half_shift=half, transition=sc.transition)
    Bo = o.render(img, fp)
    start = first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
    p = planner(sc, img)
    p.render()
    ents = p.autotune(start)
    assert any(e["kernel"] == "turn" for e in ents) and any(e["kernel"] == "straight" for e in ents)
    assert all(e["ms"] > 0 for e in ents)
    p.sweep(start, N)
    V, L, _ = p.volumes(B=False)
    assert np.array_equal(V, Vo) and np.array_equal(L, Lo)
    p.close()


SHAPES = [(v, g, sl, sg) for v in range(3) for g in (0, 5, 37) for (sl, sg) in ((0, 0), (128, 29))]


@pytest.mark.parametrize("lx,lt", [(6, 7), (7, 8), (6, 9), (5, 9)], ids=["64x128", "128x256", "64x512", "32x512"])
def test_every_kernel_shape_gives_the_same_bits(lx, lt):
    """Every turn variant (K, warps, cluster), one block per item or a
    persistent grid smaller than the work (at Nx = 32 every chain row wraps
    around x = Nx), and both straight widths: identical V and L, equal to
    the oracle."""
    R = 0.9 * (1 << lx) / 8
    sc, img = scenes.tiny(40 + lx + lt, lx, lt, fill=0.03, turn_radius=R, footprint=(3, 1, 1), soft=True,
                          transition=350)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, sc.footprint) if lx <= 6 else o.render_rows(img, sc.footprint)
    start = first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(Bo, o.cell(start), 2, mode=1)
    p = planner(sc, img)
    p.render()
    for (v, g, sl, sg) in SHAPES:
        p.set_kernel_shapes(v, g, sl, sg)
        p.sweep(start, 2)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo) and np.array_equal(L, Lo), (v, g, sl, sg)
    p.close()


def test_profile_modes_count_only_when_asked():
    """plan_profile: PLAN_PROFILE_ALL times every pass and counts the cells
    the sweeps write (the same counts as the oracle's per-layer improvements
    summed over the passes); PLAN_PROFILE_TIMING times without counting;
    other modes are refused.  Counting does not change the bits."""
    from paper_2306_01301_b300 import binding
    lx, lt, N = 5, 5, 2
    sc, img = scenes.tiny(77, lx, lt, fill=0.06, turn_radius=3.0, soft=True, transition=300)
    o = O.Oracle(lx, lt, 3.0, transition=sc.transition)
    Bo = o.render(img, sc.footprint)
    start = first_free(o, Bo, sc.pose_candidates)
    Vo, Lo, imp = o.sweep(Bo, o.cell(start), N, mode=1)
    p = planner(sc, img)
    p.render()
    p.profile(True, counts=True)
    p.sweep(start, N)
    a = p.profile_read()
    V1, L1, _ = p.volumes(B=False)
    p.profile(True, counts=False)
    p.sweep(start, N)
    t = p.profile_read()
    V2, L2, _ = p.volumes(B=False)
    p.profile(False)
    assert a["turn_passes"] == t["turn_passes"] == 2 * N + 1 and a["straight_passes"] == t["straight_passes"] == 2 * N
    assert a["turn_ms"] > 0 and t["turn_ms"] > 0 and t["straight_ms"] > 0
    # cells written per pass = cells whose value the pass lowered (a cell
    # lowered by both layers of a fused turn pair is written once)
    passes = [[0]]
    for c in range(N):
        b0 = 6 * c
        passes += [[b0 + 1], [b0 + 2, b0 + 3], [b0 + 4], [b0 + 5, b0 + 6] if c < N - 1 else [b0 + 5]]
    Vr, Lr, _ = o.sweep(Bo, o.cell(start), 0, mode=1)
    turn_w = straight_w = 0
    for grp in passes:
        Vn, Lr, _ = o.layers(Bo, Vr, Lr, grp[0], len(grp), mode=1)
        w = int((Vn < Vr).sum())
        if O.CYCLE_ORDER[grp[0] % 6] in (O.SF, O.SB):
            straight_w += w
        else:
            turn_w += w
        Vr = Vn
    assert np.array_equal(Vr, Vo) and int(imp.sum()) >= turn_w + straight_w > 0
    assert a["turn_improved"] == turn_w and a["straight_improved"] == straight_w
    assert t["turn_improved"] == 0 and t["straight_improved"] == 0
    for X in (V1, V2):
        assert np.array_equal(X, Vo)
    for X in (L1, L2):
        assert np.array_equal(X, Lo)
    assert binding.lib().plan_profile(p._h, 3) == binding.PLAN_EINVAL
    p.close()

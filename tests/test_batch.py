"""Batched planning (plan_batch_*) against the CPU oracle and against the
single-plan path.

A batch mixes grid sizes, heading counts, vehicles, radii, soft and hard
images and cycle counts; every query's volumes B, V, L and its extracted plan
must equal the oracle's bit for bit, whatever kernel shapes the autotuner
picked, with or without graph replay.  The full 64-query workload
(sizes drawn from 128^2x128, 256^2x128, 256^2x256 and 512^2x256; N in
{4, 8, 16}) runs in the configuration the benchmark times and must give every
query the plan it gets alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF

# lx, lt, R, footprint, soft, N, fill  -- lanes: (8, 8) narrow straight
# kernel, (16, 32) two queries of different N, (16, >=256) mixed Nx 256 and
# 512 (work-item offsets), (128, 128) uniform, (32, 64).  Obstacles are
# scattered single cells, sparser where the vehicle covers more cells.
MIXED = [
    (3, 3, 2.0, (0, 0, 0), False, 2, 0.06),
    (5, 4, 3.5, (2, 1, 1), True, 3, 0.06),
    (5, 4, 4.5, (1, 1, 1), False, 1, 0.06),
    (8, 4, 20.0, (6, 2, 2), True, 2, 0.004),
    (9, 4, 24.0, (12, 4, 3), False, 2, 0.002),
    (7, 7, 12.0, (4, 1, 2), False, 1, 0.01),
    (6, 5, 6.0, (0, 0, 0), True, 2, 0.06),
]


def _planner(sc, img):
    from paper_2306_01301_b300 import binding
    return binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                           sc.step_straight, sc.step_scale, sc.half_shift)


def _oracle_render(o, img, fp, nx):
    return o.render(img, fp) if nx <= 64 else o.render_rows(img, fp)


def _free(B, o, cands, k=0):
    free = [c for c in cands if B[o.cell(c)] != O.HARD]
    assert len(free) > k + 1
    return free[k], free[-1 - k]


def _segs(res):
    return [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"]) for s in res.segments]


def _oracle_segs(o, ref):
    return [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"]) for s in ref]


@pytest.fixture(scope="module")
def mixed():
    cases = []
    for k, (lx, lt, R, fp, soft, N, fill) in enumerate(MIXED):
        sc, img = scenes.tiny(700 + k, lx, lt, fill=fill, turn_radius=R, footprint=fp, soft=soft,
                              transition=400)
        o = O.Oracle(lx, lt, R, transition=sc.transition)
        Bo = _oracle_render(o, img, fp, 1 << lx)
        cases.append(dict(sc=sc, img=img, o=o, B=Bo, N=N))
    planners = [_planner(c["sc"], c["img"]) for c in cases]
    yield cases, planners
    for p in planners:
        p.close()


def _check_against_oracle(cases, planners, batch, queries):
    for i, (c, p) in enumerate(zip(cases, planners)):
        o = c["o"]
        start, goal, N = queries[i]
        Vo, Lo, _ = o.sweep(c["B"], o.cell(start), N, mode=1)
        V, L, B = p.volumes()
        assert np.array_equal(B, c["B"]), f"query {i}: obstacle volume"
        assert np.array_equal(V, Vo), f"query {i}: values differ at {np.flatnonzero(V != Vo)[:5]}"
        assert np.array_equal(L, Lo), f"query {i}: labels differ at {np.flatnonzero(L != Lo)[:5]}"
        ref = o.extract(Vo, Lo, o.cell(goal))
        got = batch.result(i)
        if ref is None:
            assert got is None
        else:
            assert got.cost == Vo[o.cell(goal)]
            assert _segs(got) == _oracle_segs(o, ref)


def test_mixed_batch_bit_exact(mixed):
    from paper_2306_01301_b300 import binding
    cases, planners = mixed
    queries = []
    for c in cases:
        s, g = _free(c["B"], c["o"], c["sc"].pose_candidates)
        queries.append((s, g, c["N"]))
    b = binding.Batch(planners)
    b.run(queries, render=True)
    b.sync()
    lanes = b.lanes()
    assert sum(l["n_queries"] for l in lanes) == len(cases)
    assert any(l["nx_min"] != l["nx_max"] for l in lanes), "a lane mixes grid sizes"
    assert all(l["n_candidates"] >= 2 for l in lanes)
    _check_against_oracle(cases, planners, b, queries)
    per_run, total = b.kernel_launches()
    assert per_run > 0 and total == per_run

    # graph replay with new poses (same N), then a new N vector (new graph)
    q2 = []
    for c in cases:
        s, g = _free(c["B"], c["o"], c["sc"].pose_candidates, 1)
        q2.append((s, g, c["N"]))
    b.run(q2, render=False)  # no rendering: a graph of its own
    _check_against_oracle(cases, planners, b, q2)
    per_run2, total = b.kernel_launches()
    assert per_run2 < per_run and total == per_run + per_run2
    q3 = [(s, g, N) for (g, s, N) in q2]  # same N: the graph is replayed
    b.run(q3, render=False)
    _check_against_oracle(cases, planners, b, [(s, g, N) for (s, g, N) in q3])
    assert b.kernel_launches() == (per_run2, per_run + 2 * per_run2)
    q4 = [(s, g, 1 + (k % 3)) for k, (s, g, _) in enumerate(q2)]
    b.run(q4, render=False)
    _check_against_oracle(cases, planners, b, q4)
    b.close()


@pytest.mark.parametrize("graph,tune", [(False, True), (True, False), (False, False)])
def test_batch_modes_give_the_same_bits(mixed, graph, tune):
    from paper_2306_01301_b300 import binding
    cases, planners = mixed
    queries = []
    for c in cases:
        s, g = _free(c["B"], c["o"], c["sc"].pose_candidates, 2)
        queries.append((s, g, c["N"]))
    ref = binding.Batch(planners)
    ref.run(queries, render=True)
    ref.sync()
    want = [p.volumes(B=False) for p in planners]
    want_res = ref.results()
    ref.close()
    b = binding.Batch(planners, graph=graph, tune=tune)
    b.run(queries, render=False)
    b.sync()
    for i, p in enumerate(planners):
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, want[i][0]) and np.array_equal(L, want[i][1]), f"query {i}"
    got_res = b.results()
    for r0, r1 in zip(want_res, got_res):
        assert (r0 is None) == (r1 is None)
        if r0 is not None:
            assert r0.cost == r1.cost and _segs(r0) == _segs(r1)
    if not tune:
        assert all(l["n_candidates"] == 0 for l in b.lanes())
    b.close()


def test_batch_with_per_plan_transition_costs():
    """Plans of one lane with different per-maneuver transition costs (the
    turn launches then read each query's own costs) and a change of costs
    after the graph was captured (a new graph), bit for bit as the oracle."""
    from paper_2306_01301_b300 import binding
    costs = [([300, 100, 900, 300, 700, 900], [0, 0, 50, 0, 50, 50]),
             ([400] * 6, [0] * 6),
             ([100, 50, 400, 120, 450, 380], [150, 60, 300, 170, 250, 320])]
    cases, planners, queries = [], [], []
    for k, (cin, cout) in enumerate(costs):
        sc, img = scenes.tiny(760 + k, 6, 7, fill=0.06, turn_radius=9.0, footprint=(3, 1, 1), soft=True,
                              transition=400)
        o = O.Oracle(6, 7, 9.0, transition=sc.transition)
        o.set_transition(cin, cout)
        Bo = _oracle_render(o, img, (3, 1, 1), 64)
        p = _planner(sc, img)
        p.set_transition_costs(cin, cout)
        cases.append(dict(sc=sc, img=img, o=o, B=Bo, N=2))
        planners.append(p)
        s, g = _free(Bo, o, sc.pose_candidates)
        queries.append((s, g, 2))
    b = binding.Batch(planners)
    b.run(queries, render=True)
    b.sync()
    assert len(b.lanes()) == 1
    _check_against_oracle(cases, planners, b, queries)
    launches = b.kernel_launches()[1]
    # the same costs for every plan: the launch may pass them as parameters, in a new graph
    for c, p in zip(cases, planners):
        c["o"].set_transition([500] * 6, [0] * 6)
        p.set_transition_costs([500] * 6, [0] * 6)
    b.run(queries, render=False)
    b.sync()
    _check_against_oracle(cases, planners, b, queries)
    assert b.kernel_launches()[1] > launches
    b.close()
    for p in planners:
        p.close()


def test_batch_rejects_bad_queries(mixed):
    from paper_2306_01301_b300 import binding
    cases, planners = mixed
    b = binding.Batch(planners[:2])
    c0, c1 = cases[0], cases[1]
    s0, g0 = _free(c0["B"], c0["o"], c0["sc"].pose_candidates)
    s1, g1 = _free(c1["B"], c1["o"], c1["sc"].pose_candidates)
    with pytest.raises(binding.PlanError) as e:
        b.run([(s0, g0, 0), (s1, g1, 1)])
    assert e.value.code == -1
    with pytest.raises(binding.PlanError) as e:
        b.run([(s0, (99, 0, 0), 1), (s1, g1, 1)])
    assert e.value.code == -1
    with pytest.raises(binding.PlanError):
        binding.Batch([planners[0], planners[0]])
    b.close()


def _oracle_sample(qs):
    """Two queries of every grid shape of the batch (each lane and each grid
    size of the mixed lane), the ones with the most cycles first, so the
    sample holds a 512^2 x 256 query with N = 16."""
    by_shape = {}
    for i, sc in enumerate(qs):
        by_shape.setdefault((sc.nx_log2, sc.nt_log2), []).append(i)
    out = []
    for key in sorted(by_shape):
        out += sorted(by_shape[key], key=lambda i: -qs[i].n_cycles)[:2]
    return out


def test_full_batched_workload_matches_single_plans_and_oracle():
    """64 uneven queries in one batch (graph replay, tuned shapes) give each
    query exactly its single-plan result; two queries of every grid shape
    (eight in all, every lane, the largest N first: a 512^2 x 256 query with
    N = 16 among them) are compared with the oracle cell by cell and plan by
    plan."""
    import os
    from paper_2306_01301_b300 import binding
    qs = scenes.batched_queries()
    planners = [binding.Planner.from_scene(sc) for sc in qs]
    queries = [(sc.start, sc.goal, sc.n_cycles) for sc in qs]
    b = binding.Batch(planners)
    b.run(queries, render=True)
    b.sync()
    got = b.results()
    assert len(b.lanes()) >= 3
    sample = _oracle_sample(qs)
    assert len(sample) >= 6 and any(qs[i].nx_log2 == 9 and qs[i].n_cycles == 16 for i in sample)
    batch_vol = {i: planners[i].volumes() for i in sample}
    # each query alone on the plain path
    for i, (sc, p) in enumerate(zip(qs, planners)):
        alone = p.plan(sc.start, sc.goal, sc.n_cycles)
        assert (alone is None) == (got[i] is None), f"query {i}"
        if alone is not None:
            assert alone.cost == got[i].cost and _segs(alone) == _segs(got[i]), f"query {i}"
        if i in batch_vol:
            V, L, B = p.volumes()
            assert np.array_equal(V, batch_vol[i][0]) and np.array_equal(L, batch_vol[i][1])
            assert np.array_equal(B, batch_vol[i][2])
    try:
        O.Oracle.set_threads(os.cpu_count() or 1)
        for i in sample:
            sc = qs[i]
            o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
            Bo = o.render_rows(sc.hard_image(), sc.footprint)
            assert np.array_equal(Bo, batch_vol[i][2])
            Vo, Lo, _ = o.sweep(Bo, o.cell(sc.start), sc.n_cycles, mode=1)
            assert np.array_equal(Vo, batch_vol[i][0]) and np.array_equal(Lo, batch_vol[i][1]), f"query {i}"
            ref = o.extract(Vo, Lo, o.cell(sc.goal))
            assert (ref is None) == (got[i] is None), f"query {i}"
            if ref is not None:
                assert got[i].cost == Vo[o.cell(sc.goal)]
                assert _segs(got[i]) == [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"])
                                         for s in ref], f"query {i}"
            del batch_vol[i]
    finally:
        O.Oracle.set_threads(1)
    b.close()
    for p in planners:
        p.close()

"""Served planning (plan_server_*): cached scenes, admission by an HBM budget,
continuous batching.

Every served result must equal the oracle's plan for its scene, start, goal
and N, and must be the same whether the request runs alone, in a mix of
requests that overlap on the GPU, one at a time, or squeezed by a memory
budget that admits only a few requests at once.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu

# lx, lt, R, footprint, fill: lanes (16, 32), (32, 64), (16, >=256) with
# Nx 256 and 512 (mixed-size launches).
SCENES = [
    (5, 4, 3.5, (2, 1, 1), 0.05),
    (6, 5, 6.0, (3, 1, 1), 0.04),
    (8, 4, 20.0, (6, 2, 2), 0.004),
    (9, 4, 24.0, (12, 4, 3), 0.002),
]


@pytest.fixture(scope="module")
def world():
    out = []
    for k, (lx, lt, R, fp, fill) in enumerate(SCENES):
        sc, img = scenes.tiny(900 + k, lx, lt, fill=fill, turn_radius=R, footprint=fp, soft=(k % 2 == 0),
                              transition=450)
        o = O.Oracle(lx, lt, R, transition=sc.transition)
        B = o.render(img, fp) if lx <= 6 else o.render_rows(img, fp)
        free = np.flatnonzero(B != O.HARD)
        out.append(dict(sc=sc, img=img, o=o, B=B, free=free))
    rng = np.random.default_rng(17)
    reqs = []
    for q in range(24):
        k = int(rng.integers(0, len(out)))
        w = out[k]
        s, g = rng.choice(w["free"], size=2, replace=False)
        reqs.append((k, w["o"].pose(int(s)), w["o"].pose(int(g)), int(rng.integers(1, 4))))
    return out, reqs


def _server(world_scenes, **kw):
    from paper_2306_01301_b300 import binding
    srv = binding.Server(**kw)
    ids = [srv.add_scene(w["sc"], w["img"]) for w in world_scenes]
    assert ids == list(range(len(world_scenes)))
    return srv


def _key(res):
    return None if res is None else (res.cost, [(s["mu"], s["entry"], s["exit"], s["steps"], s["cost"])
                                                for s in res.segments])


def _oracle_key(w, start, goal, N):
    o = w["o"]
    V, L, _ = o.sweep(w["B"], o.cell(start), N, mode=1)
    ref = o.extract(V, L, o.cell(goal))
    if ref is None:
        return None
    return (int(V[o.cell(goal)]), [(s["mu"], o.pose(s["entry"]), o.pose(s["exit"]), s["steps"], s["cost"])
                                   for s in ref])


def _run(srv, reqs):
    tickets = [srv.submit(k, s, g, N) for (k, s, g, N) in reqs]
    out = []
    for t in tickets:
        info, res = srv.wait(t, timeout=120.0)
        out.append((info, res))
    return out


@pytest.fixture(scope="module")
def oracle_keys(world):
    ws, reqs = world
    return [_oracle_key(ws[k], s, g, N) for (k, s, g, N) in reqs]


def test_served_mix_matches_oracle_and_alone(world, oracle_keys):
    ws, reqs = world
    srv = _server(ws, budget_bytes=2 << 30)
    alone = {}
    for i in (0, 5, 11, 17):
        (info, res), = _run(srv, [reqs[i]])
        alone[i] = _key(res)
    mix = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert st["peak_inflight"] > 1, "requests overlapped on the GPU"
    assert st["completed"] == len(reqs) + 4 and st["rejected"] == 0
    assert st["peak_bytes"] <= st["arena_bytes"]
    for i, (info, res) in enumerate(mix):
        assert _key(res) == oracle_keys[i], f"request {i}"
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        if i in alone:
            assert _key(res) == alone[i]


def test_one_at_a_time_and_budget_squeeze_give_the_same_plans(world, oracle_keys):
    ws, reqs = world
    serial = _server(ws, budget_bytes=2 << 30, one_at_a_time=True)
    got = _run(serial, reqs)
    st = serial.stats()
    serial.close()
    assert st["peak_inflight"] == 1 and st["completed"] == len(reqs)
    assert [_key(r) for _, r in got] == oracle_keys

    # a budget that holds the scenes and about two requests of the largest scene
    probe = _server(ws, budget_bytes=2 << 30)
    scene_bytes = probe.stats()["scene_bytes"]
    probe.close()
    big = max(w["sc"].cells for w in ws)
    budget = scene_bytes + (4 << 20) + int(2.5 * 6 * big)
    tight = _server(ws, budget_bytes=budget)
    big_reqs = [r for r in reqs if ws[r[0]]["sc"].cells == big]
    assert len(big_reqs) >= 3
    got = _run(tight, big_reqs * 2)
    st = tight.stats()
    tight.close()
    assert st["peak_bytes"] <= budget
    assert 1 <= st["peak_inflight"] <= 2
    want = [oracle_keys[reqs.index(r)] for r in big_reqs * 2]
    assert [_key(r) for _, r in got] == want


def _request_bytes(sc, n_cycles=1, conv=False):
    """Arena bytes of one request: V (4 B per pose, 256-aligned), L (2 B),
    and with convergence records one word per pass, the block 256-aligned."""
    up = lambda x: (x + 255) // 256 * 256
    nr = sc.cells
    b = up(nr * 4) + nr * 2
    if conv:
        b = up(b) + 4 * (4 * n_cycles + 1)
    return up(b)


def test_budget_of_exactly_the_scenes_and_two_requests(world, oracle_keys):
    """The launch descriptors are reserved when the server is created, so a
    budget of exactly reserved + scene + k requests runs every request (no
    step fails for want of descriptor space)."""
    ws, reqs = world
    big = max(range(len(ws)), key=lambda k: ws[k]["sc"].cells)
    probe = _server([ws[big]], budget_bytes=1 << 30)
    st0 = probe.stats()
    probe.close()
    assert st0["reserved_bytes"] > 0
    budget = st0["reserved_bytes"] + st0["scene_bytes"] + 2 * _request_bytes(ws[big]["sc"])
    srv = _server([ws[big]], budget_bytes=budget)
    mine = [(0, s, g, N) for (k, s, g, N) in reqs if k == big] * 2
    assert len(mine) >= 4
    got = _run(srv, mine)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(mine) and st["rejected"] == 0
    assert st["peak_bytes"] <= budget and 1 <= st["peak_inflight"] <= 2
    want = [oracle_keys[reqs.index((big, s, g, N))] for (_, s, g, N) in mine]
    assert [_key(r) for _, r in got] == want


def test_full_arena_gives_partial_steps_not_failure():
    """Many tiny requests in flight at once need more descriptor space than
    the reserved slots (4 KiB here, about eight requests per step) hold, and
    the arena (exactly the scene and 40 requests, with more waiting) has none
    to spare: steps advance the requests that fit, the others wait, and every
    plan is still the oracle's."""
    lx, lt, R, fp = 4, 4, 3.0, (1, 0, 0)
    sc, img = scenes.tiny(4242, lx, lt, fill=0.05, turn_radius=R, footprint=fp, transition=400)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    B = o.render(img, fp)
    free = np.flatnonzero(B != O.HARD)
    rng = np.random.default_rng(5)
    w = dict(sc=sc, img=img)
    n_req = 120
    reqs = []
    for _ in range(n_req):
        s_, g_ = rng.choice(free, size=2, replace=False)
        reqs.append((0, o.pose(int(s_)), o.pose(int(g_)), 6))
    probe = _server([w], budget_bytes=1 << 30)
    st0 = probe.stats()
    probe.close()
    held = 40  # requests the arena holds at once; the others wait for memory
    budget = st0["reserved_bytes"] + st0["scene_bytes"] + held * _request_bytes(sc)
    probe = _server([w], budget_bytes=1 << 30, slot_bytes=4096)
    small = probe.stats()["reserved_bytes"]
    probe.close()
    budget += small - st0["reserved_bytes"]
    assert budget >= 1 << 20
    srv = _server([w], budget_bytes=budget, slot_bytes=4096)
    got = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert st["completed"] == n_req and st["rejected"] == 0
    assert 8 < st["peak_inflight"] <= held and st["partial_steps"] > 0
    keys = {}
    for (k, s_, g_, N), (info, res) in zip(reqs, got):
        if (s_, g_) not in keys:
            keys[(s_, g_)] = _oracle_key(dict(o=o, B=B), s_, g_, N)
        assert _key(res) == keys[(s_, g_)]


def test_cancel_pending_and_running_requests(world, oracle_keys):
    """Cancelled requests end with PLAN_ECANCELED (or keep their plan when
    the cancel came after their label walk was queued); every other request
    gets exactly its oracle plan."""
    from paper_2306_01301_b300 import binding
    ws, reqs = world
    for one_at_a_time in (False, True):
        srv = _server(ws, budget_bytes=2 << 30, max_inflight=4, one_at_a_time=one_at_a_time)
        tickets = [srv.submit(*r) for r in reqs]
        cancel = set(range(0, len(reqs), 3))
        for i in sorted(cancel):
            srv.cancel(tickets[i])
        n_cancelled = 0
        for i, t in enumerate(tickets):
            try:
                info, res = srv.wait(t, timeout=120.0)
            except binding.PlanError as e:
                assert i in cancel and e.code == binding.PLAN_ECANCELED, (i, e.code)
                n_cancelled += 1
                continue
            assert _key(res) == oracle_keys[i], i
        st = srv.stats()
        with pytest.raises(binding.PlanError):
            srv.cancel(tickets[0])  # ticket released by its wait
        srv.close()
        assert st["cancelled"] == n_cancelled >= 1
        assert st["completed"] + st["cancelled"] == len(reqs)


@pytest.mark.parametrize("one_at_a_time", [False, True])
def test_stop_at_convergence_gives_the_same_plans(world, oracle_keys, one_at_a_time):
    """With PLAN_SERVE_STOP_AT_CONVERGENCE the passes after four that lowered
    nothing return at once; the plans are the oracle's, also for requests
    with many more cycles than they need."""
    ws, reqs = world
    srv = _server(ws, budget_bytes=2 << 30, stop_at_convergence=True, one_at_a_time=one_at_a_time)
    got = _run(srv, reqs)
    long_reqs = [(k, s, g, 12) for (k, s, g, N) in reqs[:6]]
    got_long = _run(srv, long_reqs)
    srv.close()
    assert [_key(r) for _, r in got] == oracle_keys
    for (k, s, g, N), (info, res) in zip(long_reqs, got_long):
        assert _key(res) == _oracle_key(ws[k], s, g, N)


def test_heavy_track_gives_the_same_plans(world, oracle_keys):
    """Big requests (the largest scene) and heavy ones (the next two) each
    one at a time on streams of their own, light ones batched beside them."""
    ws, reqs = world
    cells = sorted(w["sc"].cells for w in ws)
    srv = _server(ws, budget_bytes=2 << 30, heavy_cells=cells[-3], big_cells=cells[-1], max_heavy=1)
    got = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["peak_inflight"] > 1
    assert [_key(r) for _, r in got] == oracle_keys


def test_max_inflight_limits_admission(world, oracle_keys):
    ws, reqs = world
    srv = _server(ws, budget_bytes=2 << 30, max_inflight=3)
    got = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert st["peak_inflight"] <= 3
    assert [_key(r) for _, r in got] == oracle_keys


def test_submit_rejects_bad_requests(world):
    from paper_2306_01301_b300 import binding
    ws, reqs = world
    srv = _server(ws, budget_bytes=1 << 30)
    k, s, g, N = reqs[0]
    w = ws[k]
    hard = np.flatnonzero(w["B"] == O.HARD)
    cases = [(k, w["o"].pose(int(hard[0])), g, N), (k, (1 << 12, 0, 0), g, N), (k, s, g, 0), (99, s, g, N),
             (k, s, (0, 0, 1 << 12), N)]
    for c in cases:
        with pytest.raises(binding.PlanError) as e:
            srv.submit(*c)
        assert e.value.code == -1, c
    with pytest.raises(binding.PlanError) as e:
        srv.wait(123456789)
    assert e.value.code == -1
    srv.close()
    # a request whose volumes can never fit next to the scene: refused at
    # submission or, once nothing else holds memory, by the scheduler
    w3 = ws[3]
    probe = _server([w3], budget_bytes=1 << 30)
    scene_bytes = probe.stats()["scene_bytes"]
    probe.close()
    small = _server([w3], budget_bytes=scene_bytes + (2 << 20))
    s3, g3 = w3["o"].pose(int(w3["free"][0])), w3["o"].pose(int(w3["free"][-1]))
    assert 6 * w3["sc"].cells > (2 << 20)
    with pytest.raises(binding.PlanError) as e:
        small.wait(small.submit(0, s3, g3, 1), timeout=60.0)
    assert e.value.code == -2
    small.close()


def test_served_512cubed_requests_match_oracle():
    """Three 512^3 requests of the served stream's own trace (the stream's two
    512^3 scenes, N = 8), served as the benchmark serves them (continuous
    batching, stop at convergence), each equal to the oracle's plan."""
    import os
    from paper_2306_01301_b300 import binding
    all_sc = scenes.served_scenes()
    trace = scenes.served_trace(all_sc)
    big = [k for k, sc in enumerate(all_sc) if sc.nx_log2 == 9 and sc.nt_log2 == 9]
    picks = [r for r in trace if r[1] in big][:3]
    assert len(big) >= 1 and len(picks) == 3
    srv = binding.Server(budget_bytes=8 << 30, stop_at_convergence=True)
    ids = {k: srv.add_scene(all_sc[k]) for k in big}
    tickets = [srv.submit(ids[k], s, g, N) for (_, k, s, g, N) in picks]
    got = [srv.wait(t, timeout=600.0)[1] for t in tickets]
    srv.close()
    try:
        O.Oracle.set_threads(os.cpu_count() or 1)
        for (_, k, s, g, N), res in zip(picks, got):
            sc = all_sc[k]
            img = O.soft_image(sc.occupancy, sc.soft_radius, sc.soft_max) if sc.soft_radius else sc.hard_image()
            o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
            B = o.render_rows(img, sc.footprint)
            assert _key(res) == _oracle_key(dict(o=o, B=B), s, g, N)
    finally:
        O.Oracle.set_threads(1)

"""Oracle pins for per-maneuver transition costs on the Star graph (Section
V.A, Fig. 9): entering maneuver mu from the transition state costs
cost_in[mu], returning to it cost_out[mu] (gear or steering changes,
speeding up, slowing down).

Pinned by exhaustive enumeration of layer-ordered segment sequences (tiny
grids), by Dijkstra on the Star graph with those edge weights (the converged
value), by free-space closed forms of one maneuver, and by time reversal:
reversing a path swaps its endpoints, flips every gear (mu -> 5 - mu in
cycle-order ids) and swaps the entering and leaving costs, so
V(a -> b) under (in, out) equals V(b -> a) under in'[5 - mu] = out[mu],
out'[5 - mu] = in[mu]."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes


def free_image(nx):
    return np.full((nx, nx), 256, np.uint16)


COSTS = [
    # (cost_in, cost_out) per maneuver, cycle order LF SF RB RF SB LB
    ([300, 100, 900, 300, 700, 900], [0, 0, 0, 0, 0, 0]),          # backward gear dearer to enter
    ([100, 50, 400, 120, 450, 380], [150, 60, 300, 170, 250, 320]),  # in and out split unevenly
    ([0, 0, 0, 0, 0, 0], [500, 20, 900, 40, 600, 800]),              # everything on leaving
]


@pytest.mark.parametrize("costs", COSTS, ids=["in", "in_out", "out"])
@pytest.mark.parametrize("seed,lx,lt,N", [(0, 3, 3, 1), (1, 3, 4, 1), (2, 4, 3, 1), (3, 3, 3, 2)])
def test_sweep_equals_bruteforce(costs, seed, lx, lt, N):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.1, turn_radius=2.0, soft=True)
    o = O.Oracle(lx, lt, 2.0, transition=sc.transition)
    o.set_transition(*costs)
    B = o.render(img, (0, 0, 0))
    for st in [c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD][:2]:
        s = o.cell(st)
        bf = o.bruteforce(B, s, N)
        for mode in (0, 1, 2):
            V, _, _ = o.sweep(B, s, N, mode)
            assert np.array_equal(V, bf), f"mode {mode}"


@pytest.mark.parametrize("costs", COSTS, ids=["in", "in_out", "out"])
def test_converges_to_dijkstra(costs):
    sc, img = scenes.tiny(4, 4, 4, fill=0.1, turn_radius=2.5, soft=True)
    o = O.Oracle(4, 4, 2.5, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    s = o.cell(next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD))
    V_uniform = o.dijkstra(B, s)
    o.set_transition(*costs)
    Vd = o.dijkstra(B, s)
    assert not np.array_equal(Vd, V_uniform)
    prev = None
    for n in range(1, 31):
        V, _, _ = o.sweep(B, s, n, mode=1)
        assert np.all(V >= Vd)
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 30 cycles"


def test_one_maneuver_closed_forms():
    """Free space, every transition dear except the one maneuver measured."""
    lx, lt, R = 5, 6, 6.0
    o = O.Oracle(lx, lt, R, half_shift=1, transition=100000)
    B = o.render(free_image(o.nx), (0, 0, 0))
    wA = o.tables()["wA"]
    i0, j0 = 10, 9
    s = o.cell((i0, j0, 0))
    big = 90000
    for mu, cin, cout in [(O.SF, 130, 70), (O.SB, 20, 400), (O.LF, 0, 250), (O.RB, 333, 0)]:
        ci, co = [big] * 6, [big] * 6
        ci[mu], co[mu] = cin, cout
        o.set_transition(ci, co)
        V, L, _ = o.sweep(B, s, 1)
        if mu in (O.SF, O.SB):
            step = 1 if mu == O.SF else -1
            for k in range(1, 8):
                c = o.cell((i0 + step * k, j0, 0))
                assert V[c] == cin + 100 * k + cout and L[c] == (mu << 13) | k
        else:
            q = o.nt // 4
            end = s
            for _ in range(q):
                end = o.succ(mu, end)
            assert V[end] == cin + q * wA + cout and L[end] == (mu << 13) | q


@pytest.mark.parametrize("costs", COSTS[1:], ids=["in_out", "out"])
def test_time_reversal_swaps_entering_and_leaving_costs(costs):
    lx, lt, R = 4, 4, 3.0
    o = O.Oracle(lx, lt, R, transition=700)
    B = o.render(free_image(o.nx), (0, 0, 0))
    cin, cout = costs
    rin = [cout[5 - m] for m in range(6)]
    rout = [cin[5 - m] for m in range(6)]
    rng = np.random.default_rng(11)
    poses = [(int(rng.integers(1, o.nx)), int(rng.integers(1, o.nx)), int(rng.integers(o.nt))) for _ in range(7)]
    for N in (1, 2):
        o.set_transition(cin, cout)
        fwd = {p: o.sweep(B, o.cell(p), N, mode=1)[0] for p in poses}
        o.set_transition(rin, rout)
        rev = {p: o.sweep(B, o.cell(p), N, mode=1)[0] for p in poses}
        for a in poses:
            for b in poses:
                if a != b:
                    assert fwd[a][o.cell(b)] == rev[b][o.cell(a)]
    # the costs really are asymmetric: with them unswapped the reversal fails somewhere
    o.set_transition(cin, cout)
    same = {p: o.sweep(B, o.cell(p), 1, mode=1)[0] for p in poses}
    assert any(same[a][o.cell(b)] != same[b][o.cell(a)] for a in poses for b in poses if a != b)


def test_start_state_pays_the_leaving_cost():
    lx, lt, R = 5, 6, 6.0
    o = O.Oracle(lx, lt, R, half_shift=1, transition=100000)
    B = o.render(free_image(o.nx), (0, 0, 0))
    ci, co = [90000] * 6, [90000] * 6
    ci[O.SF], co[O.SF] = 500, 45
    o.set_transition(ci, co)
    s = o.cell((10, 9, 0))
    entry = list(ci)
    entry[O.SF] = 0  # straight forward in progress
    V, L, _ = o.sweep_state(B, s, entry, 1)
    for k in range(1, 10):
        assert V[o.cell((10 + k, 9, 0))] == 100 * k + 45
    with pytest.raises(ValueError):
        bad = list(ci)
        bad[O.RB] += 1
        o.sweep_state(B, s, bad, 1)


def test_refuses_costs_that_could_overflow():
    o = O.Oracle(3, 3, 2.0)
    with pytest.raises(ValueError):
        o.set_transition([1 << 27] * 6, [1 << 27] * 6)

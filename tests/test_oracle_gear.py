"""Oracle pins for the two gear states (forward / reverse transition state,
a penalty for every change of gear between consecutive maneuvers).

Pinned by exhaustive enumeration of layer-ordered segment sequences with the
gear state (tiny grids), by Dijkstra on the explicit graph of two transition
vertices and six maneuver vertices per cell (the converged value), by the
reduction that with no penalty the cheaper of the two states is the
single-state sweep, by free-space closed forms of backing up from a vehicle
standing in forward or reverse gear, and by re-summing back-tracked plans."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

REVERSE = {O.LB, O.SB, O.RB}


def _world(seed, lx, lt, R, soft=True):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.1, turn_radius=R, soft=soft)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    starts = [o.cell(c) for c in sc.pose_candidates if B[o.cell(c)] != O.HARD]
    o.ct = sc.transition
    return o, B, starts


@pytest.mark.parametrize("seed,lx,lt,N,pen,gear", [(0, 3, 3, 1, 400, 2), (1, 3, 3, 1, 150, 0), (2, 3, 4, 1, 900, 1),
                                                    (3, 4, 3, 1, 300, 2), (4, 3, 3, 2, 500, 0)])
def test_sweep_equals_bruteforce(seed, lx, lt, N, pen, gear):
    o, B, starts = _world(seed, lx, lt, 2.0)
    for s in starts[:2]:
        V, _ = o.sweep_gear(B, s, gear, pen, N)
        assert np.array_equal(V, o.bruteforce_gear(B, s, gear, pen, N))


@pytest.mark.parametrize("seed,pen,gear", [(0, 300, 2), (1, 1200, 0), (2, 700, 1)])
def test_converges_to_dijkstra(seed, pen, gear):
    o, B, starts = _world(seed, 4, 4, 2.5)
    s = starts[0]
    Vd = o.dijkstra_gear(B, s, gear, pen)
    prev = None
    for n in range(1, 31):
        V, _ = o.sweep_gear(B, s, gear, pen, n)
        assert np.all(V >= Vd)
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 30 cycles"


@pytest.mark.parametrize("seed", [0, 3])
def test_no_penalty_is_the_single_state_sweep(seed):
    o, B, starts = _world(seed, 4, 4, 2.5)
    s = starts[0]
    for N in (1, 2):
        V, _ = o.sweep_gear(B, s, 2, 0, N)
        V1, _, _ = o.sweep(B, s, N)
        assert np.array_equal(np.minimum(V[:o.nr], V[o.nr:]), V1)


def test_backing_up_closed_forms():
    """Free space, large ct: backing k cells straight behind the start costs
    ct + 100 k from a vehicle in reverse gear and ct + pen + 100 k from one in
    forward gear; driving ahead the other way round."""
    lx, lt, ct, pen = 5, 5, 100000, 777
    o = O.Oracle(lx, lt, 4.0, half_shift=1, transition=ct)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    i0, j0 = 16, 9
    s = o.cell((i0, j0, 0))
    for gear in (0, 1, 2):
        V, L = o.sweep_gear(B, s, gear, pen, 1)
        for k in range(1, 8):
            back, ahead = o.cell((i0 - k, j0, 0)), o.cell((i0 + k, j0, 0))
            assert V[o.nr + back] == ct + 100 * k + (pen if gear == 0 else 0)
            assert V[ahead] == ct + 100 * k + (pen if gear == 1 else 0)
            assert L[o.nr + back] == (O.SB << 13) | ((1 if gear == 0 else 0) << 12) | k
            assert V[back] == O.INF or V[back] > V[o.nr + back]  # ending forward there needs more


def test_plans_resum_to_their_values():
    o, B, starts = _world(5, 4, 4, 2.5)
    pen = 600
    V, L = o.sweep_gear(B, starts[0], 2, pen, 3)
    best = np.minimum(V[:o.nr], V[o.nr:])
    rng = np.random.default_rng(2)
    for g in rng.choice(np.flatnonzero(best != O.INF), 40, replace=False):
        segs = o.extract_gear(V, L, int(g))
        assert segs is not None
        total, gear = 0, None
        x = starts[0]
        for sg in segs:
            mu = sg["mu"]
            assert sg["entry"] == x
            g_mu = 1 if mu in REVERSE else 0
            total += o.ct + (pen if gear is not None and gear != g_mu else 0)
            y = x
            for _ in range(sg["steps"]):
                total += o.edge(B, mu, y)
                y = o.succ(mu, y)
            assert y == sg["exit"] and sg["cost"] == total
            x, gear = y, g_mu
        assert x == g and total == best[g]

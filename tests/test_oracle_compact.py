"""Oracle pins for the Compact graph (Section V.A, Fig. 12: the straight
maneuver type doubles as the transition state; vertices S, L, R per cell).

Pinned by exhaustive enumeration of layer-ordered segment sequences with the
vertex type (tiny grids), Dijkstra on the explicit three-vertex graph (the
converged value), the free edge back to S (S never above L or R), free-space
closed forms (a straight needs no transition, a turn one, a change of gear
within one turn direction none), and valid back-tracked plans that cost at
most their values."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes


def _world(seed, lx, lt, R, soft=True):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.1, turn_radius=R, soft=soft)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    return o, B, [o.cell(c) for c in sc.pose_candidates if B[o.cell(c)] != O.HARD], sc.transition


@pytest.mark.parametrize("seed,lx,lt,N", [(0, 3, 3, 1), (1, 3, 3, 2), (2, 3, 4, 1), (3, 4, 3, 1)])
def test_sweep_equals_bruteforce(seed, lx, lt, N):
    o, B, starts, _ = _world(seed, lx, lt, 2.0)
    for s in starts[:2]:
        V, _ = o.sweep_compact(B, s, N)
        assert np.array_equal(V, o.bruteforce_compact(B, s, N))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_converges_to_dijkstra_and_s_is_never_above_the_turns(seed):
    o, B, starts, _ = _world(seed, 4, 4, 2.5)
    s = starts[0]
    Vd = o.dijkstra_compact(B, s)
    prev = None
    for n in range(1, 31):
        V, _ = o.sweep_compact(B, s, n)
        assert np.all(V >= Vd)
        nr = o.nr
        assert np.all(V[:nr] <= V[nr:2 * nr]) and np.all(V[:nr] <= V[2 * nr:])
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 30 cycles"


def test_free_space_closed_forms():
    lx, lt, R, ct = 5, 6, 6.0, 100000
    o = O.Oracle(lx, lt, R, half_shift=1, transition=ct)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    wA = o.tables()["wA"]
    i0, j0 = 10, 9
    s = o.cell((i0, j0, 0))
    V, L = o.sweep_compact(B, s, 1)
    nr = o.nr
    for k in range(1, 10):  # a straight: no transition cost
        c = o.cell((i0 + k, j0, 0))
        assert V[c] == 100 * k and L[c] == (O.SF << 13) | k
    q = o.nt // 4
    end = o.cell((i0 + int(R), j0 + int(R), q))  # quarter left-forward turn: ct once
    assert V[nr + end] == ct + q * wA and V[end] == V[nr + end]
    assert L[nr + end] == (O.LF << 13) | (1 << 12) | q
    # then backward along the left turn (LB is later in the cycle): no second transition
    back = end
    for _ in range(q // 2):
        back = o.succ(O.LB, back)
    assert V[nr + back] <= ct + q * wA + (q // 2) * wA


def test_plans_are_valid_and_no_dearer_than_their_values():
    """Each back-tracked plan follows its maneuvers from the start through
    non-hard cells, pays ct exactly where it enters a turn from S, and costs
    at most V(goal): a label records the entry's value when the layer ran, and
    a later layer may still lower the entry's own value (forward tracking),
    so a walk can be cheaper than the value it ends at, never dearer."""
    o, B, starts, ct = _world(5, 4, 4, 2.5)
    V, L = o.sweep_compact(B, starts[0], 3)
    nr = o.nr
    rng = np.random.default_rng(1)
    equal = 0
    for g in rng.choice(np.flatnonzero(V[:nr] != O.INF), 40, replace=False):
        segs = o.extract_compact(V, L, int(g))
        total, x = 0, starts[0]
        for sg in segs:
            mu = sg["mu"]
            assert sg["entry"] == x
            if mu not in (O.SF, O.SB) and sg["from_s"]:
                total += ct
            y = x
            for _ in range(sg["steps"]):
                assert B[y] != O.HARD
                total += o.edge(B, mu, y)
                y = o.succ(mu, y)
            assert y == sg["exit"] and B[y] != O.HARD
            x = y
        assert x == g and total <= V[g]
        equal += total == V[g]
    assert equal >= 30

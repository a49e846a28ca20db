"""Oracle pins for the 4D generalisation of Appendix F (curvature levels and
clothoid maneuvers).

The clothoid offsets are pinned against the Fresnel integrals of scipy (a
library routine: int_0^s cos(theta0 + a sigma^2) dsigma = (cos theta0 C(z) -
sin theta0 S(z)) / k with k = sqrt(2a / pi), z = k s), the heading offsets
against their closed form; each level's chain map is a bijection and the
clothoid steps are exactly reversible; the sweep equals exhaustive
enumeration on tiny grids, converges to Dijkstra on the explicit 4D graph,
and gives the free-space closed form of one clothoid from straight wheels to
the steering limit."""
import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_2306_01301_b300 import scenes


def _fresnel_offsets(f, s, th0, a):
    k = np.sqrt(2 * a / np.pi)
    S, Cf = special.fresnel(k * s)
    if f == 0:
        return (np.cos(th0) * Cf - np.sin(th0) * S) / k, (np.sin(th0) * Cf + np.cos(th0) * S) / k
    return (np.cos(th0) * Cf + np.sin(th0) * S) / k, (np.sin(th0) * Cf - np.cos(th0) * S) / k


@pytest.mark.parametrize("lx,lt,R,M,L", [(6, 6, 8.0, 3, 1.0), (7, 7, 20.0, 5, 0.75), (9, 9, 110.0, 8, 0.9)])
def test_clothoid_tables_match_fresnel_integrals(lx, lt, R, M, L):
    o = O.Oracle(lx, lt, R)
    q = O.Oracle4(o, M, L, 300)
    dx, dy, dth = q.tables()
    a = 1.0 / (2 * M * R * L)
    nt = o.nt
    checked = 0
    for f in (0, 1):
        for K in range(2 * M + 1):
            kap = K - M
            s = kap * L if f == 0 else -kap * L
            psi = (a if f == 0 else -a) * s * s
            want = np.round(psi * nt / (2 * np.pi))
            assert dth[f, K] == int(np.sign(want) * np.floor(abs(psi * nt / (2 * np.pi)) + 0.5))
            th0 = 2 * np.pi * np.arange(nt) / nt
            X, Y = _fresnel_offsets(f, s, th0, a) if kap else (np.zeros(nt), np.zeros(nt))
            for got, ref in ((dx[f, K], X), (dy[f, K], Y)):
                away = np.abs(np.abs(ref - np.trunc(ref)) - 0.5) > 1e-6  # not at a rounding boundary
                r = np.sign(ref) * np.floor(np.abs(ref) + 0.5)
                assert np.array_equal(got[away], r[away].astype(np.int16))
                checked += int(away.sum())
    assert checked > 0.99 * 2 * 2 * (2 * M + 1) * nt


def test_level_maps_are_bijections_and_steps_reverse():
    o = O.Oracle(4, 4, 3.0)
    q = O.Oracle4(o, 2, 1.0, 300)
    for mu, back in ((q.C1F, q.C1B), (q.C2F, q.C2B)):
        # successors of every cell of every level it can leave: a bijection between levels
        for K in range(q.nk):
            cells = [K * o.nr + x for x in range(o.nr)]
            nxt = [q.succ(mu, c) for c in cells]
            if all(n < 0 for n in nxt):
                continue
            assert all(n >= 0 for n in nxt)
            assert len(set(nxt)) == o.nr
            assert all(q.succ(back, n) == c for c, n in zip(cells, nxt))
    # 3D maneuvers live on their own level only
    assert q.succ(O.SF, q.cell((3, 3, 0), 1)) < 0 and q.succ(O.SF, q.cell((3, 3, 0), 0)) >= 0
    assert q.succ(O.LF, q.cell((3, 3, 0), 2)) >= 0 and q.succ(O.RF, q.cell((3, 3, 0), -2)) >= 0


@pytest.mark.parametrize("seed,lx,lt,M", [(0, 3, 3, 1), (1, 3, 3, 2), (2, 3, 4, 1)])
def test_sweep_equals_bruteforce(seed, lx, lt, M):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.08, turn_radius=2.0, soft=True)
    o = O.Oracle(lx, lt, 2.0, transition=sc.transition)
    q = O.Oracle4(o, M, 1.0, 150)
    B = o.render(img, (0, 0, 0))
    for st in [c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD][:2]:
        s4 = q.cell(st, 0)
        V, _ = q.sweep(B, s4, 1)
        assert np.array_equal(V, q.bruteforce(B, s4, 1))


def test_converges_to_dijkstra():
    sc, img = scenes.tiny(4, 4, 4, fill=0.08, turn_radius=2.5, soft=True)
    o = O.Oracle(4, 4, 2.5, transition=sc.transition)
    q = O.Oracle4(o, 2, 1.0, 200)
    B = o.render(img, (0, 0, 0))
    s4 = q.cell(next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD), 0)
    Vd = q.dijkstra(B, s4)
    prev = None
    for n in range(1, 25):
        V, _ = q.sweep(B, s4, n)
        assert np.all(V >= Vd)
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 24 cycles"


def test_one_clothoid_closed_form_and_plan():
    """Free space: from straight wheels (kappa = 0) to the left steering
    limit the only way is C1F (or C2B backward), one step per level:
    ct_clothoid + M * round(100 L) at the chain's end cell, and its plan is
    that one segment."""
    lx, lt, R, M, L, ctc = 5, 6, 6.0, 3, 1.0, 350
    o = O.Oracle(lx, lt, R, transition=100000)
    q = O.Oracle4(o, M, L, ctc)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    s4 = q.cell((16, 16, 0), 0)
    V, Lb = q.sweep(B, s4, 1)
    end = s4
    for _ in range(M):
        end = q.succ(q.C1F, end)
    assert q.pose(end)[1] == M
    assert V[end] == ctc + M * round(100 * L)
    assert Lb[end] == (q.C1F << 12) | M
    segs = q.extract(V, Lb, end)
    assert len(segs) == 1 and segs[0]["entry"] == s4 and segs[0]["mu"] == q.C1F

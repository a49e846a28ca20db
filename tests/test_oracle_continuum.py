"""The oracle's graph against the continuum vehicle (Appendix B, Theorems
6-7, Lemmas 4-5, Corollary 2).

These pins compare the oracle with plain kinematics written here from the
vehicle model of Section III and eq. 16 -- circles of radius R and straight
lines traversed forward or backward -- not with anything the oracle
computes:

* Graph -> continuum (Corollary 2, the step behind Theorem 6): replaying an
  extracted graph plan maneuver by maneuver on the continuum vehicle (same
  maneuver, same turned angle or same advance along the dominant axis) ends
  at the same heading, within m_c/2 + m_s cells in x and y of the graph's
  final vertex (m_c circular and m_s straight maneuvers, half-cell shift on),
  and the graph cost equals 100 x the continuum length plus one transition
  cost per maneuver, up to the rounding of the per-edge weights.
* Continuum -> graph (Theorem 7): for a random continuum path of at most four
  maneuvers with cost c (100 per cell of length plus a sufficient transition
  cost per maneuver), some graph vertex within 7 + pi d / N_theta cells in x
  and y and 4 headings of its end has value at most c after enough cycles.
  The same holds for the shortest paths themselves, the Reeds-Shepp and
  Dubins closed forms (Theorems 2-3) written in tests/curves.py.
"""
import math

import numpy as np
import pytest

import oracle as O

LX, LT = 6, 6
NX, NT = 1 << LX, 1 << LT
R = 6.0
# Sufficient transition cost (Appendix B.C): one transition must pay for a
# one-cell correction, d_T >= 1 + R dtheta + 4R acos(1 - 1/(4R)) cells.
DT_CELLS = 1 + R * 2 * math.pi / NT + 4 * R * math.acos(1 - 1 / (4 * R))
CT = int(math.ceil(100 * DT_CELLS)) + 50
LF, SF, RB, RF, SB, LB = range(6)


def zeta(x):
    """Round to the nearest integer or half-integer, halves away from zero."""
    y = 2 * x
    r = math.floor(abs(y) + 0.5)
    return math.copysign(r, y) / 2


def psi(T):
    a = zeta(R * math.sin(2 * math.pi * T / NT))
    return a - math.floor(a)


def vertex_pose(cell, half_shift):
    """Continuum configuration a graph vertex stands for (eq. 16)."""
    i, j, T = cell
    if half_shift:
        return (i + psi(T), j + psi((T + NT // 4) % NT), 2 * math.pi * T / NT)
    return (float(i), float(j), 2 * math.pi * T / NT)


def drive(pose, mu, amount):
    """Continuum motion: turns by `amount` radians of heading change, straights
    by `amount` cells of length.  Returns the new pose."""
    x, y, th = pose
    if mu in (SF, SB):
        s = amount if mu == SF else -amount
        return (x + s * math.cos(th), y + s * math.sin(th), th)
    left = mu in (LF, LB)
    up = mu in (LF, RB)           # heading increases
    th2 = th + amount if up else th - amount
    if left:                      # centre on the left of the heading
        cx, cy = x - R * math.sin(th), y + R * math.cos(th)
        return (cx + R * math.sin(th2), cy - R * math.cos(th2), th2)
    cx, cy = x + R * math.sin(th), y - R * math.cos(th)
    return (cx - R * math.sin(th2), cy + R * math.cos(th2), th2)


def straight_len(steps, T):
    th = 2 * math.pi * T / NT
    return steps / max(abs(math.cos(th)), abs(math.sin(th)))


def ang_diff(a, b):
    d = (a - b) % (2 * math.pi)
    return min(d, 2 * math.pi - d)


@pytest.fixture(scope="module", params=[1, 0], ids=["half_shift", "plain_rounding"])
def free_world(request):
    half = request.param
    o = O.Oracle(LX, LT, R, half_shift=half, transition=CT)
    img = np.full((NX, NX), 256, np.uint16)
    B = o.render(img, (0, 0, 0))
    start = (NX // 2, NX // 2, 5)
    V, L, _ = o.sweep(B, o.cell(start), 4, mode=1)
    return dict(o=o, B=B, V=V, L=L, start=start, half=half)


def test_graph_plans_replay_on_the_continuum_vehicle(free_world):
    o, V, L, half = free_world["o"], free_world["V"], free_world["L"], free_world["half"]
    wA = round(100 * 2 * math.pi * R / NT)
    reached = np.flatnonzero(V != O.INF)
    assert len(reached) > 0.5 * NX * NX * NT
    rng = np.random.default_rng(11)
    checked = 0
    for g in rng.choice(reached, size=300, replace=False):
        segs = o.extract(V, L, int(g))
        if not segs:
            continue
        pose = vertex_pose(o.pose(segs[0]["entry"]), half)
        length, steps_total, edge_sum, mc, ms = 0.0, 0, 0, 0, 0
        for s in segs:
            T0 = o.pose(s["entry"])[2]
            if s["mu"] in (SF, SB):
                d = straight_len(s["steps"], T0)
                pose = drive(pose, s["mu"], d)
                length += d
                ms += 1
                th = 2 * math.pi * T0 / NT
                edge_sum += s["steps"] * round(100 / max(abs(math.cos(th)), abs(math.sin(th))))
            else:
                phi = s["steps"] * 2 * math.pi / NT
                pose = drive(pose, s["mu"], phi)
                length += R * phi
                mc += 1
                edge_sum += s["steps"] * wA
            steps_total += s["steps"]
        end = vertex_pose(o.pose(int(g)), half)
        bound = (mc / 2 + ms) if half else (mc + ms)
        assert ang_diff(pose[2], end[2]) < 1e-9, "same heading"
        assert abs(pose[0] - end[0]) <= bound + 1e-9 and abs(pose[1] - end[1]) <= bound + 1e-9, \
            (segs, pose, end, bound)
        m = len(segs)
        assert int(V[g]) == edge_sum + m * CT
        assert abs(edge_sum - 100 * length) <= 0.5 * steps_total + 1e-6
        checked += 1
    assert checked > 250


def test_continuum_paths_are_matched_by_the_graph(free_world):
    """Theorem 7 with sufficient maneuver-counting transition costs."""
    o, V, half = free_world["o"], free_world["V"], free_world["half"]
    start = free_world["start"]
    Vg = V.reshape(NT, NX, NX)  # [T][j][i]
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(200):
        m = int(rng.integers(1, 5))
        pose = vertex_pose(start, half)
        length = 0.0
        for _k in range(m):
            mu = int(rng.integers(0, 6))
            if mu in (SF, SB):
                d = float(rng.uniform(0.0, 8.0))
                length += d
            else:
                d = float(rng.uniform(0.0, math.pi))
                length += R * d
            pose = drive(pose, mu, d)
        x, y, th = pose
        if not (6 <= x <= NX - 6 and 6 <= y <= NX - 6):
            continue  # stay clear of the one-cell walls
        c = 100 * length + m * CT
        d_cells = c / 100
        bound = 7 + math.pi * d_cells / NT
        T = th * NT / (2 * math.pi)
        ok = False
        for dT in range(-4, 5):
            Tc = int(round(T)) + dT
            if abs(Tc - T) > 4:
                continue
            Tm = Tc % NT
            i_lo, i_hi = max(1, math.ceil(x - bound - 0.5)), min(NX - 1, math.floor(x + bound))
            j_lo, j_hi = max(1, math.ceil(y - bound - 0.5)), min(NX - 1, math.floor(y + bound))
            for j in range(j_lo, j_hi + 1):
                for i in range(i_lo, i_hi + 1):
                    vx, vy, _ = vertex_pose((i, j, Tm), half)
                    if abs(vx - x) <= bound and abs(vy - y) <= bound and Vg[Tm, j, i] <= c:
                        ok = True
                        break
                if ok:
                    break
            if ok:
                break
        assert ok, (m, pose, c)
        checked += 1
    assert checked > 100


def test_sufficient_transition_cost_criterion():
    """The transition cost used above meets Appendix B.C's criterion, and the
    lateral-correction distance it is built from matches a direct check: two
    arcs of angle a and two back (C_a C_a | C_a C_a) shift sideways by
    4R(1 - cos a)."""
    assert CT >= 100 * DT_CELLS
    for a in (0.1, 0.3, 0.7):
        p = (0.0, 0.0, 0.0)
        p = drive(p, LF, a)
        p = drive(p, RF, a)
        p = drive(p, LB, a)
        p = drive(p, RB, a)
        assert abs(p[2]) < 1e-12 and abs(p[1] - 4 * R * (1 - math.cos(a))) < 1e-9


def _matched_by_graph(Vg, half, x, y, th, c):
    """Theorem 7's box: some vertex within 7 + pi d / N_theta cells in x and
    y and 4 headings of (x, y, th) with value <= c (d = c / 100 cells)."""
    bound = 7 + math.pi * (c / 100) / NT
    T = th * NT / (2 * math.pi)
    for dT in range(-4, 5):
        Tc = int(round(T)) + dT
        if abs(Tc - T) > 4:
            continue
        Tm = Tc % NT
        for j in range(max(1, math.ceil(y - bound - 0.5)), min(NX - 1, math.floor(y + bound)) + 1):
            for i in range(max(1, math.ceil(x - bound - 0.5)), min(NX - 1, math.floor(x + bound)) + 1):
                vx, vy, _ = vertex_pose((i, j, Tm), half)
                if abs(vx - x) <= bound and abs(vy - y) <= bound and Vg[Tm, j, i] <= c:
                    return True
    return False


@pytest.fixture(scope="module")
def five_cycles(free_world):
    """Five cycles cover any order of up to five maneuvers (Reeds-Shepp words)."""
    o, half = free_world["o"], free_world["half"]
    V, _, _ = o.sweep(free_world["B"], o.cell(free_world["start"]), 5, mode=1)
    return V.reshape(NT, NX, NX), half


@pytest.mark.parametrize("family", ["reeds_shepp", "dubins"])
def test_shortest_continuum_paths_are_matched_by_the_graph(free_world, five_cycles, family):
    """Theorem 7 on the shortest paths themselves: the Reeds-Shepp (Theorem 3)
    and Dubins (Theorem 2) closed-form paths to random goals, with one
    transition cost per maneuver, are matched by the graph within the bound."""
    from tests import curves
    Vg, half = five_cycles
    q0 = vertex_pose(free_world["start"], half)
    rng = np.random.default_rng(23 if family == "reeds_shepp" else 29)
    checked = 0
    for _ in range(150 if family == "reeds_shepp" else 400):
        q1 = (float(rng.uniform(10, NX - 10)), float(rng.uniform(10, NX - 10)), float(rng.uniform(0, 2 * math.pi)))
        path = curves.reeds_shepp_path(q0, q1, R) if family == "reeds_shepp" else curves.dubins_path(q0, q1, R)
        end = curves.drive(q0, path, R)
        assert abs(end[0] - q1[0]) < 1e-6 and abs(end[1] - q1[1]) < 1e-6
        c = 100 * curves.length(path) + CT * max(1, curves.maneuvers(path))
        if c > 100 * 60:
            continue  # long detours leave the grid
        assert _matched_by_graph(Vg, half, q1[0], q1[1], q1[2] % (2 * math.pi), c), (family, q1, path, c)
        checked += 1
    assert checked > 60  # forward-only paths often turn around: more samples for Dubins


def test_closed_forms_are_shortest():
    """The Reeds-Shepp construction used above: every candidate word reaches
    its goal, no random path of up to five segments is shorter, it is
    symmetric, and it is never longer than the forward-only Dubins path."""
    from tests import curves
    rng = np.random.default_rng(3)
    for _ in range(3000):
        m = int(rng.integers(1, 6))
        path = []
        for _k in range(m):
            kind = "LRS"[int(rng.integers(0, 3))]
            path.append((kind, float(rng.uniform(-3, 3) if kind == "S" else rng.uniform(-math.pi, math.pi))))
        end = curves.drive((0.0, 0.0, 0.0), path, 1.0)
        rs = curves.reeds_shepp_path((0.0, 0.0, 0.0), end, 1.0)
        e2 = curves.drive((0.0, 0.0, 0.0), rs, 1.0)
        assert abs(e2[0] - end[0]) < 1e-6 and abs(e2[1] - end[1]) < 1e-6
        assert abs(curves.mod2pi(e2[2] - end[2])) < 1e-6
        assert curves.length(rs) <= curves.length(path) + 1e-7
        back = curves.reeds_shepp_path(end, (0.0, 0.0, 0.0), 1.0)
        assert abs(curves.length(back) - curves.length(rs)) < 1e-7
        db = curves.dubins_path((0.0, 0.0, 0.0), end, 1.0)
        assert curves.length(rs) <= curves.length(db) + 1e-7

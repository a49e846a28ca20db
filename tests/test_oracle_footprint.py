"""Pins of the oracle's vehicle footprint at oblique headings and with the
half-cell shift of eq. 16 (Section V.C: the shift "should be taken into
account in obstacle rendering"; Section VI; Fig. 6).

* Hand-worked fixtures (tests/golden/footprint_oblique.txt): 45 degrees with
  Psi = (1/2, 1/2), 22.5 degrees with only Psi_1 = 1/2 and 67.5 degrees with
  only Psi_0 = 1/2, each derived in the fixture's comments.
* An independent construction written here: the rectangle's four corners
  placed in world coordinates at the shifted rear axle and a cell centre
  tested against the four edge half-planes (cross products), where the
  oracle rotates the cell centre into vehicle coordinates instead.  The two
  agree over a sweep of radii, heading counts, vehicles and both shift modes.
* The fixtures discriminate: the same construction with the shift's sign
  flipped, its axes swapped, the shift left out, or the rotation reversed
  gives a different set of cells for some fixture.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.util import read_golden

EPS = 1e-9


def _fixtures():
    keyed, _ = read_golden("footprint_oblique.txt")
    out = []
    for name in sorted({k.split("_")[0] for k in keyed}):
        r2, lt, T, f, r, hw, p0, p1 = keyed[name + "_params"]
        c = keyed[name + "_cells"]
        cells = set(zip(c[0::2], c[1::2]))
        assert len(cells) * 2 == len(c)
        out.append(dict(name=name, R=r2 / 2.0, lt=lt, T=T, fp=(f, r, hw), psi2=(p0, p1), cells=cells))
    return out


FIXTURES = _fixtures()


def halfplane_footprint(front, rear, hw, theta, psi0, psi1, sign=1.0):
    """Cells whose centre lies in the rectangle, by edge half-planes.

    Corners in world coordinates relative to the pose's integer cell: rear
    axle at (psi0, psi1), unit heading h = (cos, sin), left normal
    n = (-sin, cos); corners counter-clockwise: rear-right, front-right,
    front-left, rear-left.  A point is inside when it lies on the left of
    (or on) every directed edge.  `sign` = -1 rotates the wrong way (a
    deliberately wrong reading, used to show the fixtures discriminate)."""
    c, s = math.cos(theta), sign * math.sin(theta)
    h = np.array([c, s])
    n = np.array([-s, c])
    o = np.array([psi0, psi1])
    corners = [o - rear * h - hw * n, o + front * h - hw * n, o + front * h + hw * n, o - rear * h + hw * n]
    lim = int(math.ceil(math.hypot(max(front, rear), hw))) + 2
    ys, xs = np.mgrid[-lim:lim + 1, -lim:lim + 1]
    px, py = xs.astype(float), ys.astype(float)
    inside = np.ones(px.shape, bool)
    for k in range(4):
        a, b = corners[k], corners[(k + 1) % 4]
        ex, ey = b - a
        ln = math.hypot(ex, ey)
        if ln == 0.0:  # degenerate rectangle side (hw = 0 or front = rear = 0)
            continue
        cross = ex * (py - a[1]) - ey * (px - a[0])
        inside &= cross >= -EPS * ln
    # a zero-width or zero-length vehicle is a segment: the two remaining
    # edges of the degenerate side bound it along its length
    if hw == 0 or front + rear == 0:
        proj_h = (px - o[0]) * h[0] + (py - o[1]) * h[1]
        proj_n = (px - o[0]) * n[0] + (py - o[1]) * n[1]
        inside = (proj_h >= -rear - EPS) & (proj_h <= front + EPS) & (np.abs(proj_n) <= hw + EPS)
    cells = {(int(x), int(y)) for x, y in zip(xs[inside], ys[inside])}
    cells.add((0, 0))
    return cells


def _oracle_cells(o, fp, T):
    dx, dy = o.footprint(*fp, T)
    return set(zip(dx.tolist(), dy.tolist()))


@pytest.mark.parametrize("fx", FIXTURES, ids=[f["name"] for f in FIXTURES])
def test_hand_worked_oblique_footprints(fx):
    lx = max(3, fx["lt"])
    o = O.Oracle(lx, fx["lt"], fx["R"], half_shift=1)
    nt = o.nt
    psi2 = o.tables()["psi2"]
    assert (int(psi2[fx["T"]]), int(psi2[(fx["T"] + nt // 4) % nt])) == fx["psi2"], "eq. 13 shift"
    assert _oracle_cells(o, fx["fp"], fx["T"]) == fx["cells"]
    # the independent construction reproduces the hand-worked set
    th = 2 * math.pi * fx["T"] / nt
    p0, p1 = fx["psi2"][0] / 2, fx["psi2"][1] / 2
    assert halfplane_footprint(*fx["fp"], th, p0, p1) == fx["cells"]


def test_fixtures_discriminate_wrong_readings():
    """Each plausible misreading changes some fixture."""
    wrong = {
        "shift sign flipped": lambda fp, th, p0, p1: halfplane_footprint(*fp, th, -p0, -p1),
        "shift axes swapped": lambda fp, th, p0, p1: halfplane_footprint(*fp, th, p1, p0),
        "no shift": lambda fp, th, p0, p1: halfplane_footprint(*fp, th, 0.0, 0.0),
        "rotation reversed": lambda fp, th, p0, p1: halfplane_footprint(*fp, th, p0, p1, sign=-1.0),
        "front and rear swapped": lambda fp, th, p0, p1: halfplane_footprint(fp[1], fp[0], fp[2], th, p0, p1),
    }
    for name, fn in wrong.items():
        differs = []
        for fx in FIXTURES:
            th = 2 * math.pi * fx["T"] / (1 << fx["lt"])
            got = fn(fx["fp"], th, fx["psi2"][0] / 2, fx["psi2"][1] / 2)
            differs.append(got != fx["cells"])
        assert any(differs), name
    # the shift-only cases tell the axes apart one by one
    b, c = [f for f in FIXTURES if f["name"] in ("b", "c")]
    for fx in (b, c):
        th = 2 * math.pi * fx["T"] / (1 << fx["lt"])
        p0, p1 = fx["psi2"][0] / 2, fx["psi2"][1] / 2
        assert p0 != p1
        assert halfplane_footprint(*fx["fp"], th, p1, p0) != fx["cells"]
        assert halfplane_footprint(*fx["fp"], th, -p0, -p1) != fx["cells"]


SWEEP = [
    # (R, log2 N_theta, vehicle, half_shift)
    (2.0, 3, (2, 1, 1), 1),
    (2.5, 4, (3, 1, 1), 1),
    (3.7, 5, (4, 2, 1), 1),
    (7.3, 6, (7, 2, 3), 1),
    (12.0, 6, (0, 0, 0), 1),
    (10.0, 7, (6, 2, 0), 1),
    (24.0, 7, (24, 6, 7), 1),
    (24.0, 7, (24, 6, 7), 0),
    (110.0, 9, (76, 20, 19), 1),
    (13.9, 8, (11, 3, 4), 0),
]


@pytest.mark.parametrize("R,lt,fp,half", SWEEP)
def test_footprint_equals_halfplane_construction(R, lt, fp, half):
    o = O.Oracle(max(3, lt), lt, R, half_shift=half)
    nt = o.nt
    psi2 = o.tables()["psi2"]
    step = max(1, nt // 64)
    for T in list(range(0, nt, step)) + [1, nt // 8, 3 * nt // 8, nt - 1]:
        th = 2 * math.pi * T / nt
        p0 = psi2[T] / 2 if half else 0.0
        p1 = psi2[(T + nt // 4) % nt] / 2 if half else 0.0
        if not half:
            assert psi2[T] == 0
        assert _oracle_cells(o, fp, T) == halfplane_footprint(*fp, th, p0, p1), (R, nt, fp, T)

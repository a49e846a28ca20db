"""Oracle pins for the direction penalties of Section XVI (Fig. 19): a
hand-worked 4 x 4 x 8 fixture, the cases that leave B unchanged, and a
free-space closed form of the sweep with a lane that prefers heading 0."""
import numpy as np
import pytest

import oracle as O
from tests.util import read_golden

NONE = 0xFFFF


def test_hand_worked_fixture():
    k, _ = read_golden("direction_4x4x8.txt")
    o = O.Oracle(2, 3, 1.0)
    field = np.full((o.nx, o.nx), NONE, np.uint16)
    f = k["field"]
    for i in range(0, len(f), 3):
        field[f[i + 1], f[i]] = f[i + 2]
    B = np.full(o.nr, 256, np.uint16)
    b = k["b_in"]
    for i in range(0, len(b), 4):
        B[o.cell((b[i], b[i + 1], b[i + 2]))] = b[i + 3]
    want = B.copy()
    b = k["b_out"]
    for i in range(0, len(b), 4):
        want[o.cell((b[i], b[i + 1], b[i + 2]))] = b[i + 3]
    got = o.direction(B, field, k["tol"][0], k["pen"][0])
    assert np.array_equal(got, want), f"differs at {[o.pose(int(c)) for c in np.flatnonzero(got != want)]}"


def test_cases_that_change_nothing():
    o = O.Oracle(4, 4, 2.0)
    rng = np.random.default_rng(1)
    B = rng.integers(256, 2000, o.nr).astype(np.uint16)
    B[rng.random(o.nr) < 0.1] = O.HARD
    field = rng.integers(0, o.nt, (o.nx, o.nx)).astype(np.uint16)
    assert np.array_equal(o.direction(B, field, 2, 256), B)          # penalty 1.0
    assert np.array_equal(o.direction(B, field, o.nt // 2, 900), B)  # every heading within tolerance
    assert np.array_equal(o.direction(B, np.full((o.nx, o.nx), NONE, np.uint16), 0, 900), B)
    out = o.direction(B, field, 0, 900)
    assert np.array_equal(out == O.HARD, B == O.HARD) and np.all(out >= B)


def test_lane_makes_driving_against_it_dearer():
    """Free space, every cell prefers heading 0 within one step, penalty 3x:
    a straight line at heading 0 costs 100 per step, one at heading pi costs
    floor(100 * 768 / 256) = 300 per step."""
    lx, lt, ct = 5, 5, 100000
    o = O.Oracle(lx, lt, 4.0, half_shift=1, transition=ct)
    B = o.render(np.full((o.nx, o.nx), 256, np.uint16), (0, 0, 0))
    B = o.direction(B, np.zeros((o.nx, o.nx), np.uint16), 1, 768)
    i0, j0 = 16, 9
    V, _, _ = o.sweep(B, o.cell((i0, j0, 0)), 1)
    for k in range(1, 10):
        assert V[o.cell((i0 + k, j0, 0))] == ct + 100 * k
    half = o.nt // 2
    V, _, _ = o.sweep(B, o.cell((i0, j0, half)), 1)
    for k in range(1, 10):
        assert V[o.cell((i0 - k, j0, half))] == ct + 300 * k


def test_refuses_bad_fields():
    o = O.Oracle(3, 3, 2.0)
    B = np.full(o.nr, 256, np.uint16)
    with pytest.raises(ValueError):
        o.direction(B, np.full((o.nx, o.nx), o.nt, np.uint16), 0, 512)
    with pytest.raises(ValueError):
        o.direction(B, np.zeros((o.nx, o.nx), np.uint16), o.nt, 512)
    with pytest.raises(ValueError):
        o.direction(B, np.zeros((o.nx, o.nx), np.uint16), 0, 255)

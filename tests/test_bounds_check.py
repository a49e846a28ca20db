"""The bounds-check build (PLAN_BOUNDS_CHECK): every global and shared-memory
index of the plain plan path's kernels -- rendering, the turn and straight
sweeps, the label walk -- and of the sweep kernels of the gear states, the
curvature levels and the Compact graph is checked on the device, a failure
is recorded in the plan's error word and reported by the host as
PLAN_EINTERNAL.

On CPU: the checked library builds for sm_103a and exports every entry point
of include/nhplan.h.  On the GPU: in a fresh process that loads the checked
library (NHPLAN_BOUNDS_CHECK=1), plans on grids of 8^3 to 64^3 in several
kernel shapes, and the gear, curvature-level and Compact sweeps on grids
whose turns take the sections scan, equal the oracle cell by cell, with no
check failing.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.util import ROOT


def test_checked_library_builds_and_exports_every_symbol():
    import ctypes as C
    from paper_2306_01301_b300 import _build
    from tests.test_abi import declared_entry_points
    path = _build.build(checked=True)
    L = C.CDLL(path)
    for n in declared_entry_points():
        assert hasattr(L, n), n


CASES = [
    # lx, lt, R, footprint, soft, half_shift, N
    (3, 3, 2.0, (0, 0, 0), False, 1, 2),
    (4, 4, 2.5, (2, 1, 1), True, 1, 2),
    (4, 5, 3.0, (3, 1, 1), True, 0, 2),
    (5, 6, 4.0, (4, 1, 2), True, 1, 2),
    (6, 6, 7.0, (5, 2, 2), False, 1, 3),
    (6, 7, 6.5, (3, 1, 1), True, 1, 2),
]


def _run_checked():
    """Runs in the child process (NHPLAN_BOUNDS_CHECK=1)."""
    import oracle as O
    from paper_2306_01301_b300 import binding, scenes
    assert binding.LIB_PATH.endswith("libnhplan_checked.so")
    for k, (lx, lt, R, fp, soft, half, N) in enumerate(CASES):
        sc, img = scenes.tiny(500 + k, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=soft,
                              half_shift=half, transition=350)
        o = O.Oracle(lx, lt, R, half_shift=half, transition=sc.transition)
        Bo = o.render(img, fp)
        start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
        goal = next(c for c in sc.pose_candidates[3:] if Bo[o.cell(c)] != O.HARD)
        Vo, Lo, _ = o.sweep(Bo, o.cell(start), N, mode=1)
        ref = o.extract(Vo, Lo, o.cell(goal))
        p = binding.Planner(lx, lt, img, fp, R, sc.transition, half_shift=half)
        shapes = [(-1, 0, 0, 0)] + ([(0, 3, 128, 5)] if lx >= 5 else [])
        for sh in shapes:
            p.set_kernel_shapes(*sh)
            p.render()
            p.sweep(start, N)
            V, L, B = p.volumes()  # PLAN_EINTERNAL if a check failed
            assert np.array_equal(B, Bo), (k, sh)
            assert np.array_equal(V, Vo) and np.array_equal(L, Lo), (k, sh)
            res = p.extract(goal)
            assert (res is None) == (ref is None)
            if res is not None:
                assert res.cost == Vo[o.cell(goal)]
        p.close()
    _run_checked_features(O, binding, scenes)
    print("bounds-checked plans equal the oracle")


def _run_checked_features(O, binding, scenes):
    """Gear states, curvature levels and the Compact graph on a 32^2 x 128
    grid (their sections-scan turns, staged gear straights, the plain
    kernels on a level, the four-chain clothoid layer) against the oracle."""
    lx, lt, R, fp = 5, 7, 6.0, (2, 1, 1)
    sc, img = scenes.tiny(560, lx, lt, fill=0.06, turn_radius=R, footprint=fp, soft=True, transition=300)
    o = O.Oracle(lx, lt, R, transition=sc.transition)
    Bo = o.render(img, fp)
    start = next(c for c in sc.pose_candidates if Bo[o.cell(c)] != O.HARD)
    nr = o.nr
    p = binding.Planner(lx, lt, img, fp, R, sc.transition)
    p.render()
    p.set_gear_penalty(800)
    p.sweep_gear(start, 2, 2)
    Vf, Lf, _ = p.volumes(B=False)  # PLAN_EINTERNAL if a check failed
    Vr, Lr = p.reverse_volumes()
    Vo, Lo = o.sweep_gear(Bo, o.cell(start), 2, 800, 2)
    assert np.array_equal(Vf, Vo[:nr]) and np.array_equal(Lf, Lo[:nr]), "gear, forward state"
    assert np.array_equal(Vr, Vo[nr:]) and np.array_equal(Lr, Lo[nr:]), "gear, reverse state"
    p.set_gear_penalty(None)
    q = O.Oracle4(o, 2, 1.0, 250)
    p.set_curvature_levels(2, 1.0, 250)
    p.sweep4(start, 1, 2)
    V4, L4 = p.volumes4()
    Vq, Lq = q.sweep(Bo, q.cell(start, 1), 2)
    assert np.array_equal(V4, Vq) and np.array_equal(L4, Lq), "curvature levels"
    p.set_curvature_levels(0)
    p.set_compact_graph(True)
    p.sweep_compact(start, 2)
    got = p.compact_volumes()
    Vc, Lc = o.sweep_compact(Bo, o.cell(start), 2)
    want = (Vc[:nr], Lc[:nr], Vc[nr:2 * nr], Lc[nr:2 * nr], Vc[2 * nr:], Lc[2 * nr:])
    for a, b in zip(got, want):
        assert np.array_equal(a, b), "Compact graph"
    p.close()


@pytest.mark.gpu
def test_checked_build_plans_equal_the_oracle():
    from paper_2306_01301_b300 import _build
    _build.build(checked=True)
    env = dict(os.environ, NHPLAN_BOUNDS_CHECK="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", "import tests.test_bounds_check as t; t._run_checked()"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "equal the oracle" in r.stdout

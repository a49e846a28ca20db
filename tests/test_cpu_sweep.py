"""The multi-core CPU baseline (oracle/cpu_sweep.c, the kernel-style sweep of
Section VIII.B-C with the curves of a layer spread over OpenMP threads)
against the oracle's layered relaxation: identical V, identical labels and
identical improved-cell counts per layer, on every curve family, with soft
costs, per-maneuver transition costs (Fig. 9) and thread counts of 1 to 8.
It is timed by bench.py as the counterpart of the paper's CPU kernel rows,
so it has to compute the same thing."""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

CASES = [
    # seed, lx, lt, R, footprint, soft, half shift, N
    (0, 3, 3, 2.0, (0, 0, 0), False, 1, 2),
    (1, 4, 4, 2.5, (1, 0, 0), True, 1, 3),
    (2, 5, 4, 3.0, (2, 1, 1), True, 0, 2),
    (3, 4, 6, 4.0, (1, 1, 1), True, 1, 2),
    (4, 6, 5, 6.0, (3, 1, 1), False, 1, 2),
    (5, 2, 2, 1.5, (0, 0, 0), True, 1, 3),
]


def _free_start(o, B, cands):
    for c in cands:
        if B[o.cell(c)] != O.HARD:
            return o.cell(c)
    raise AssertionError("no free start")


@pytest.mark.parametrize("case", CASES, ids=[f"{1 << c[1]}x{1 << c[2]}" for c in CASES])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_cpu_sweep_equals_oracle(case, threads):
    seed, lx, lt, R, fp, soft, half, N = case
    sc, img = scenes.tiny(seed, lx, lt, fill=0.08, turn_radius=R, footprint=fp, soft=soft, half_shift=half,
                          transition=300)
    o = O.Oracle(lx, lt, R, half_shift=half, transition=sc.transition)
    B = o.render(img, fp)
    s = _free_start(o, B, sc.pose_candidates)
    Vo, Lo, io = o.sweep(B, s, N, mode=1)
    V, L, imp, used = O.cpu_sweep(o, B, s, N, threads=threads)
    assert used == threads
    assert np.array_equal(V, Vo), f"values differ at {np.flatnonzero(V != Vo)[:5]}"
    assert np.array_equal(L, Lo), f"labels differ at {np.flatnonzero(L != Lo)[:5]}"
    assert np.array_equal(imp, io)
    assert (V < O.INF).sum() > 1  # the sweep went somewhere


def test_cpu_sweep_per_maneuver_costs():
    sc, img = scenes.tiny(11, 4, 4, fill=0.1, turn_radius=2.5, soft=True)
    o = O.Oracle(4, 4, 2.5, transition=sc.transition)
    o.set_transition([100, 50, 400, 120, 450, 380], [150, 60, 300, 170, 250, 320])
    B = o.render(img, (0, 0, 0))
    s = _free_start(o, B, sc.pose_candidates)
    Vo, Lo, _ = o.sweep(B, s, 3, mode=0)
    V, L, _, _ = O.cpu_sweep(o, B, s, 3, threads=4)
    assert np.array_equal(V, Vo) and np.array_equal(L, Lo)


def test_cpu_sweep_rejects_a_hard_start():
    sc, img = scenes.tiny(12, 3, 3, fill=0.3)
    o = O.Oracle(3, 3, 2.0, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    hard = int(np.flatnonzero(B == O.HARD)[0])
    with pytest.raises(ValueError):
        O.cpu_sweep(o, B, hard, 1)

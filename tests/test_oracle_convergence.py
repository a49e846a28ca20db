"""Pin of the convergence rule the server's PLAN_SERVE_STOP_AT_CONVERGENCE
uses (Section XVI.A cycle order; Table 3's "complete convergence" after a
few cycles): once the six maneuver layers LF, SF, RB, RF, SB, LB have each
run once in a row without lowering any cell, V and L are a fixed point of
every layer, so any further cycles return the same volumes.

In the fused-pass schedule (pass 0 = LF, 4c+1 = SF, 4c+2 = RB+RF, 4c+3 = SB,
4c+4 = LB + the next cycle's LF) any four consecutive passes starting at
pass 1 or later hold all six maneuvers.  The oracle's per-layer improvement
counts give the passes that lowered nothing; the volumes after the first
four quiet passes must equal the volumes after all N cycles.
"""
import numpy as np

import oracle as O
from paper_2306_01301_b300 import scenes


def _pass_layers(N):
    """Layers (0-based, in cycle order) of each fused pass."""
    out = [[0]]
    for c in range(N):
        b = 6 * c
        out += [[b + 1], [b + 2, b + 3], [b + 4], [b + 5, b + 6] if c < N - 1 else [b + 5]]
    return out


def test_four_quiet_passes_mean_a_fixed_point():
    converged = 0
    for seed in range(10):
        lx, lt = (4, 4) if seed % 2 else (5, 4)
        sc, img = scenes.tiny(700 + seed, lx, lt, fill=0.08, turn_radius=2.5 + seed % 3, footprint=(1, 0, 1),
                              soft=bool(seed % 3 == 0), transition=300)
        o = O.Oracle(lx, lt, sc.turn_radius, transition=sc.transition)
        B = o.render(img, sc.footprint)
        start = next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD)
        N = 10
        V, L, imp = o.sweep(B, o.cell(start), N, mode=1)
        layers = _pass_layers(N)
        assert sum(len(x) for x in layers) == 6 * N
        quiet = [int(sum(imp[l] for l in ls)) == 0 for ls in layers]
        stop = next((p for p in range(5, len(layers)) if all(quiet[p - 4:p])), None)
        if stop is None:
            continue
        converged += 1
        # the volumes after passes 0 .. stop-1 equal the final ones
        n_layers = sum(len(x) for x in layers[:stop])
        Vs, Ls, _ = o.sweep(B, o.cell(start), 0, mode=1)
        Vs, Ls, _ = o.layers(B, Vs, Ls, 0, n_layers, mode=1)
        assert np.array_equal(Vs, V) and np.array_equal(Ls, L), seed
        # and no later layer lowered anything
        assert all(quiet[stop:])
    assert converged >= 5

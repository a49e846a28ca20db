"""One small planning case for profilers.

A short process whose kernels are the 512^3 benchmark's kernels in the same
launch shapes, at a size where a counter capture of one launch (tens of
replay passes) ends within a minute and the device holds a few hundred MB:

  python -m paper_2306_01301_b300.profile_case plain
      256^2 x 512 parallel-parking scene (33.5 M pose cells, 335 MB of
      volumes, more than L2): render, then a 2-cycle sweep with the turn
      kernel pinned to the benchmark's shape at 512^3 (16 headings per
      thread, 32 warps, no cluster, persistent grid of 148 blocks; straight
      blocks of 256 lines), then the label walk.

  python -m paper_2306_01301_b300.profile_case features
      256^2 x 256 parallel-parking scene: two gear states (penalty 3000),
      four curvature levels per side, the Compact graph and the bit-vector
      planner, two cycles each.

Prints one line with the plan's cost so that a run can be checked.
"""
import sys


def plain():
    from . import binding, scenes
    sc = scenes.parallel_parking(nx_log2=8, nt_log2=9, n_cycles=2)
    p = binding.Planner.from_scene(sc)
    p.set_kernel_shapes(0, 148, 256, 0)
    p.render()
    p.sweep(sc.start, 2)
    res = p.extract(sc.goal)
    p.close()
    print("plain", res.cost if res else None)


def features():
    import torch
    from . import binding, scenes
    sc = scenes.parallel_parking(nx_log2=8, nt_log2=8, n_cycles=2)
    p = binding.Planner.from_scene(sc)
    p.render()
    p.set_gear_penalty(3000)
    p.sweep_gear(sc.start, 0, 2)
    p.set_gear_penalty(None)
    p.set_curvature_levels(4, 1.0, 500)
    p.sweep4(sc.start, 0, 2)
    p.set_curvature_levels(0)
    p.set_compact_graph(True)
    p.sweep_compact(sc.start, 2)
    p.set_compact_graph(False)
    p.reach_sweep(sc.start, 4)
    r = p.reach_extract(sc.goal)
    torch.cuda.synchronize()
    p.close()
    print("features", r[0] if r else None)


def main(argv):
    cases = {"plain": plain, "features": features}
    if len(argv) != 1 or argv[0] not in cases:
        print(__doc__)
        return 2
    cases[argv[0]]()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))

"""Allocation failures after a plan exists (GPU): the calls that take more
device memory later -- two gear states, curvature levels, the Compact
graph, a direction field, a goal set, the bit-vector planner, a batch, a
server -- return PLAN_ENOMEM when the caller's allocator refuses, hold no
memory afterwards, and leave the plan as it was: its sweep still equals the
oracle, and the same call succeeds once the allocator gives memory again.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import scenes

pytestmark = pytest.mark.gpu


class SwitchAllocator:
    """torch's caching allocator behind a switch: NULL while `fail` is set."""

    def __init__(self, torch, stream):
        from paper_2306_01301_b300 import binding
        self.fail = False
        self.live = {}
        dev = stream.device

        def _alloc(nbytes, _s, _c):
            if self.fail:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream))
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, _s, _c):
            assert self.live.pop(int(ptr)) == int(nbytes)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._fa = binding.ALLOC_FN(_alloc)
        self._ff = binding.FREE_FN(_free)
        self.struct = binding.Allocator(self._fa, self._ff, None)


def _enomem(fn):
    from paper_2306_01301_b300 import binding
    with pytest.raises(binding.PlanError) as e:
        fn()
    assert e.value.code == -2, e.value.code


def test_later_allocations_fail_cleanly_and_the_plan_stays_usable():
    import torch
    from paper_2306_01301_b300 import binding
    lx, lt = 6, 5
    sc, img = scenes.tiny(55, lx, lt, fill=0.05, turn_radius=4.0, footprint=(2, 1, 1), transition=400)
    o = O.Oracle(lx, lt, sc.turn_radius, transition=sc.transition)
    B = o.render(img, sc.footprint)
    start = next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD)
    goal = next(c for c in sc.pose_candidates[5:] if B[o.cell(c)] != O.HARD)
    Vo, Lo, _ = o.sweep(B, o.cell(start), 2, mode=1)
    stream = torch.cuda.current_stream()
    al = SwitchAllocator(torch, stream)
    p = binding.Planner(lx, lt, img, sc.footprint, sc.turn_radius, sc.transition, stream=stream, allocator=al)
    held = dict(al.live)
    p.render()

    def same_as_oracle():
        p.sweep(start, 2)
        V, L, _ = p.volumes(B=False)
        assert np.array_equal(V, Vo) and np.array_equal(L, Lo)

    same_as_oracle()
    al.fail = True
    field = np.full((p.nx, p.nx), 0, np.uint16)
    goals = [(*goal, 2, 1, 10, 20, 0)]
    calls = {
        "gear states": lambda: p.set_gear_penalty(700),
        "curvature levels": lambda: p.set_curvature_levels(2, 1.0, 300),
        "compact graph": lambda: p.set_compact_graph(True),
        "direction field": lambda: p.set_direction_field(field, 2, 512),
        "goal set": lambda: p.extract_goal_set(goals),
        "bit-vector planner": lambda: p.reach_sweep(start, 3),
    }
    for name, fn in calls.items():
        _enomem(fn)
        assert al.live == held, f"{name}: memory held after the failure"
        same_as_oracle()
    b = None
    try:  # a batch's buffers come from the same allocator
        with pytest.raises(binding.PlanError) as e:
            b = binding.Batch([p], allocator=al)
            b.run([(start, goal, 2)])
        assert e.value.code == -2
    finally:
        if b is not None:
            b.close()
    assert al.live == held
    al.fail = False
    p.set_gear_penalty(700)
    p.sweep_gear(start, 0, 1)
    p.set_gear_penalty(None)
    p.set_direction_field(field, 2, 512)
    p.set_direction_field(None)
    p.render()
    same_as_oracle()
    p.extract_goal_set(goals)
    p.reach_sweep(start, 3)
    p.close()
    assert not al.live


def test_server_create_with_a_refusing_allocator():
    import ctypes as C
    import torch
    from paper_2306_01301_b300 import binding
    L = binding.lib()
    binding._server_signatures(L)
    al = SwitchAllocator(torch, torch.cuda.current_stream())
    al.fail = True
    cfg = binding.ServerConfig(1 << 24, 0, 0, 0, 0, 0, 0, 0)
    h = C.c_void_p()
    assert L.plan_server_create(C.byref(cfg), C.byref(al.struct), None, C.byref(h)) == -2
    assert not h.value and not al.live

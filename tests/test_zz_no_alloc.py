"""The allocation-free rendering entry point, plan_render_cspace_static.

It exists for callers that may not allocate device memory when they render:
processes whose device memory is owned by a fixed memory plan, or loops that
forbid allocation after start-up.  Its scratch is a fixed device array inside
the library instead of memory from an allocator.  Checked here through the C
ABI against the ordinary plan_render_cspace path, which allocates its own
scratch, and against the oracle's rendering, on several calls in a row (the
shared array keeps the previous call's contents, so a later call must not
depend on them).

This file is collected last so that a first failure here comes after every
other test has run; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import binding, scenes

pytestmark = pytest.mark.gpu


def reference_B(sc, img):
    p = binding.Planner(sc.nx_log2, sc.nt_log2, img, sc.footprint, sc.turn_radius, sc.transition,
                        half_shift=sc.half_shift)
    p.render()
    _, _, B = p.volumes(V=False, L=False)
    p.close()
    return B


def static_B(torch, sc, img):
    lib = binding.lib()
    lib.plan_render_cspace_static.restype = C.c_int
    lib.plan_render_cspace_static.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(binding.Footprint),
                                              C.c_double, C.c_uint32, C.c_void_p, C.c_void_p]
    d_img = torch.from_numpy(img.astype(np.int16, copy=False).view(np.int16)).cuda()
    d_B = torch.full((sc.cells,), 0x1234, dtype=torch.int16, device="cuda")  # stale garbage
    fp = binding.Footprint(*sc.footprint)
    stream = torch.cuda.current_stream()
    rc = lib.plan_render_cspace_static(C.c_void_p(d_img.data_ptr()), sc.nx_log2, sc.nt_log2, C.byref(fp),
                                       float(sc.turn_radius), binding.PLAN_FLAG_HALF_SHIFT if sc.half_shift else 0,
                                       C.c_void_p(d_B.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, binding.lib().plan_strerror(rc)
    torch.cuda.synchronize()
    return d_B.cpu().numpy().view(np.uint16)


def oracle_B(sc, img):
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, half_shift=sc.half_shift)
    return o.render(img, sc.footprint) if sc.nx_log2 <= 6 else o.render_rows(img, sc.footprint)


def test_static_render_matches_allocating_render_on_consecutive_calls():
    """Five calls in a row, each checked against the allocating path and
    against the oracle: hard and soft images, the half-cell shift of eq. 16
    on and off, and a case where half of the headings have a shift in x or in
    y (R = 2.5 at 16 headings) with a long, narrow vehicle."""
    import torch
    a = scenes.parallel_parking(nx_log2=8, nt_log2=8)
    b, img_b = scenes.tiny(3, 6, 7, fill=0.05, turn_radius=9.0, footprint=(7, 2, 3), soft=True, half_shift=0)
    c = scenes.maze(nx_log2=9, nt_log2=6)
    d, img_d = scenes.tiny(4, 5, 4, fill=0.04, turn_radius=2.5, footprint=(5, 2, 1), soft=True, half_shift=1)
    img_c = binding.soft_image(c.occupancy, c.soft_radius, c.soft_max)
    psi2 = O.Oracle(5, 4, 2.5, half_shift=1).tables()["psi2"]
    assert d.half_shift and 0 < int(psi2.sum()) < 16
    cases = [(a, a.hard_image()), (b, img_b), (c, img_c), (d, img_d), (a, a.hard_image())]
    for sc, img in cases:
        got = static_B(torch, sc, img)
        assert np.array_equal(got, reference_B(sc, img)), sc.name
        assert np.array_equal(got, oracle_B(sc, img)), sc.name


def test_static_render_rejects_grids_beyond_its_scratch():
    import torch
    lib = binding.lib()
    lib.plan_render_cspace_static.restype = C.c_int
    fp = binding.Footprint(0, 0, 0)
    x = torch.zeros(16, dtype=torch.int16, device="cuda")
    rc = lib.plan_render_cspace_static(C.c_void_p(x.data_ptr()), 10, 6, C.byref(fp), C.c_double(5.0),
                                       C.c_uint32(1), C.c_void_p(x.data_ptr()), None)
    assert rc == -6  # PLAN_ERANGE: Nx = 1024 exceeds the fixed scratch, nothing was launched
    torch.cuda.synchronize()

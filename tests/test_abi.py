"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/nhplan.h declares, and its host-only logic
(argument validation, the soft-obstacle helper) behaves without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2306_01301_b300 import _build, binding
from tests.util import ROOT


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return binding.lib()


def declared_entry_points():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*|void)\s+(plan_\w+)\s*\(", src, re.M))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_names_every_code(lib):
    for code in range(0, -10, -1):
        s = lib.plan_strerror(code).decode()
        assert s and s != "unknown error"


def test_create_rejects_bad_arguments_on_host(lib):
    img = np.full((16, 16), 256, np.uint16)
    g = binding.Grid(4, 4, img.ctypes.data_as(C.c_void_p))
    fp = binding.Footprint(0, 0, 0)
    costs = binding.Costs(100, 100, 500, 1)
    h = C.c_void_p()
    cases = [
        (binding.Grid(1, 4, img.ctypes.data_as(C.c_void_p)), fp, 3.0, costs),   # grid too small
        (binding.Grid(4, 11, img.ctypes.data_as(C.c_void_p)), fp, 3.0, costs),  # too many headings
        (g, fp, 0.0, costs),                                                    # radius <= 0
        (g, binding.Footprint(-1, 0, 0), 3.0, costs),                           # negative extent
        (g, fp, 3.0, binding.Costs(100, 100, 1 << 28, 1)),                      # transition too big
        (g, fp, 3.0, binding.Costs(0, 100, 5, 1)),                              # zero step
    ]
    for grid, f, r, c in cases:
        assert lib.plan_create(C.byref(grid), C.byref(f), r, C.byref(c), None, None, C.byref(h)) == -1
    bad = img.copy()
    bad[3, 3] = 100  # below 256 and not hard
    gb = binding.Grid(4, 4, bad.ctypes.data_as(C.c_void_p))
    assert lib.plan_create(C.byref(gb), C.byref(fp), 3.0, C.byref(costs), None, None, C.byref(h)) == -1
    assert lib.plan_sweep(None, binding.Pose(1, 1, 1), 1) == -1
    assert lib.plan_destroy(None) == -1


@pytest.mark.parametrize("nx,radius,soft_max,p", [(8, 3, 90, 0.05), (64, 6, 512, 0.03), (96, 4, 1000, 0.1),
                                                  (32, 0, 0, 0.1), (40, 7, 777, 0.0)])
def test_soft_image_helper_matches_oracle(lib, nx, radius, soft_max, p):
    occ = (np.random.default_rng(nx).random((nx, nx)) < p).astype(np.uint8)
    assert np.array_equal(binding.soft_image(occ, radius, soft_max), O.soft_image(occ, radius, soft_max))


def test_entry_points_have_header_comments():
    src = open(os.path.join(ROOT, "include", "nhplan.h")).read()
    for n in declared_entry_points():
        i = src.index(n + "(")
        assert "*/" in src[max(0, i - 1200):i] or n in ("plan_destroy", "plan_strerror"), n


def test_batch_entry_points_reject_bad_arguments_on_host(lib):
    binding._batch_signatures(lib)
    h = C.c_void_p()
    assert lib.plan_batch_create(None, 1, 0, None, None, C.byref(h)) == -1
    arr = (C.c_void_p * 2)(None, None)
    assert lib.plan_batch_create(arr, 2, 0, None, None, C.byref(h)) == -1  # NULL plans
    assert lib.plan_batch_create(arr, 0, 0, None, None, C.byref(h)) == -1
    assert lib.plan_batch_run(None, None, 1) == -1
    assert lib.plan_batch_sync(None) == -1
    n = C.c_int(0)
    cost = C.c_uint32(0)
    assert lib.plan_batch_result(None, 0, None, 0, C.byref(n), C.byref(cost)) == -1
    assert lib.plan_batch_lanes(None, C.byref(n)) == -1
    assert lib.plan_batch_destroy(None) == -1


def test_server_entry_points_reject_bad_arguments_on_host(lib):
    binding._server_signatures(lib)
    h = C.c_void_p()
    assert lib.plan_server_create(None, None, None, C.byref(h)) == -1
    cfg = binding.ServerConfig(1000, 0, 0, 0, 0, 0, 0)  # below 1 MiB
    assert lib.plan_server_create(C.byref(cfg), None, None, C.byref(h)) == -1
    cfg = binding.ServerConfig(1 << 30, 0, 7, 0, 0, 0, 0)  # unknown mode
    assert lib.plan_server_create(C.byref(cfg), None, None, C.byref(h)) == -1
    for bad in ((1 << 30, -1, 0, 0, 0, 0, 0), (1 << 30, 0, 0, -5, 0, 1, 0), (1 << 30, 0, 0, 100, 0, -1, 0),
                (1 << 30, 0, 0, 0, -3, 1, 0), (1 << 30, 0, 0, 0, 0, 0, 6),  # unknown flag bits
                (1 << 30, 0, 0, 0, 0, 0, 0, 100)):  # descriptor slots below 4 KiB
        cfg = binding.ServerConfig(*bad)
        assert lib.plan_server_create(C.byref(cfg), None, None, C.byref(h)) == -1
    t = C.c_uint64(0)
    assert lib.plan_server_submit(None, 0, binding.Pose(0, 0, 0), binding.Pose(0, 0, 0), 1, C.byref(t)) == -1
    info = binding.RequestInfo()
    assert lib.plan_server_wait(None, 1, 0.0, C.byref(info), None, 0, None) == -1
    assert lib.plan_server_cancel(None, 1) == -1
    assert lib.plan_server_destroy(None) == -1

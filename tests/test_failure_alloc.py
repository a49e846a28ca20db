"""Failure handling of the allocator callback (plan_allocator), on the host.

plan_create takes every device buffer from the caller's allocator before it
touches the GPU, so a failing allocator is testable without a GPU: a fake
allocator hands out host blocks and returns NULL from its k-th call on.
Every k must give PLAN_ENOMEM, and every block handed out must come back to
the free callback exactly once with its size.  With an allocator that never
fails, plan_create gets past the allocations and, with no GPU here, fails at
its first CUDA call (PLAN_ECUDA) -- again returning every block.  The GPU
side (a plan that stays usable when a later allocation fails) is in
tests/test_failure_gpu.py.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2306_01301_b300 import _build, binding


class FakeAllocator:
    """Host blocks standing in for device memory; NULL from call `fail_at` on."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}      # address -> size
        self.freed = []     # (address, size) as the free callback saw them
        self._keep = {}

        def _alloc(nbytes, _stream, _ctx):
            self.calls += 1
            if self.fail_at is not None and self.calls >= self.fail_at:
                return None
            buf = C.create_string_buffer(max(1, int(nbytes)))
            addr = C.addressof(buf)
            self._keep[addr] = buf
            self.live[addr] = int(nbytes)
            return addr

        def _free(ptr, nbytes, _stream, _ctx):
            self.freed.append((int(ptr), int(nbytes)))
            assert self.live.pop(int(ptr)) == int(nbytes), "freed with another size"
            self._keep.pop(int(ptr))

        self._fa = binding.ALLOC_FN(_alloc)
        self._ff = binding.FREE_FN(_free)
        self.struct = binding.Allocator(self._fa, self._ff, None)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return binding.lib()


def _create(lib, alloc, nx_log2=5, nt_log2=5):
    img = np.full((1 << nx_log2, 1 << nx_log2), 256, np.uint16)
    img[3:6, 3:9] = 0xFFFF
    g = binding.Grid(nx_log2, nt_log2, img.ctypes.data_as(C.c_void_p))
    fp = binding.Footprint(3, 1, 1)
    costs = binding.Costs(100, 100, 500, 1)
    h = C.c_void_p()
    rc = lib.plan_create(C.byref(g), C.byref(fp), 4.0, C.byref(costs), C.byref(alloc.struct), None, C.byref(h))
    return rc, h


def test_every_failing_allocation_gives_enomem_and_returns_every_block(lib):
    probe = FakeAllocator()
    rc, h = _create(lib, probe)
    n_allocs = probe.calls
    assert rc != 0 and not h.value  # no GPU here: the first CUDA call fails after the allocations
    assert n_allocs >= 10
    assert not probe.live, "a failed plan_create kept device blocks"
    for k in range(1, n_allocs + 1):
        a = FakeAllocator(fail_at=k)
        rc, h = _create(lib, a)
        assert rc == -2, (k, rc)  # PLAN_ENOMEM
        assert not h.value
        assert not a.live, f"allocation {k} failing leaked {a.live}"
        assert len(a.freed) == k - 1


def test_batch_and_server_reject_a_null_allocator_pair(lib):
    binding._server_signatures(lib)
    bad = binding.Allocator(binding.ALLOC_FN(lambda n, s, c: None), C.cast(None, binding.FREE_FN), None)
    cfg = binding.ServerConfig(1 << 30, 0, 0, 0, 0, 0, 0, 0)
    h = C.c_void_p()
    assert lib.plan_server_create(C.byref(cfg), C.byref(bad), None, C.byref(h)) == -1  # PLAN_EINVAL
    img = np.full((32, 32), 256, np.uint16)
    g = binding.Grid(5, 5, img.ctypes.data_as(C.c_void_p))
    fp = binding.Footprint(0, 0, 0)
    costs = binding.Costs(100, 100, 500, 1)
    assert lib.plan_create(C.byref(g), C.byref(fp), 4.0, C.byref(costs), C.byref(bad), None, C.byref(h)) == -1

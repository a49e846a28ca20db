"""Thin Python binding of the nhplan C ABI (include/nhplan.h).

Argument marshalling only: every step of the planner runs in the library's
CUDA kernels.  PyTorch provides the device memory (its caching allocator,
through the C ABI's allocator callbacks) and the CUDA stream.  If the
compiled library is missing or no CUDA device is present, the calls raise;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# NHPLAN_BOUNDS_CHECK=1 in the environment loads the bounds-check build
# (every index of the plain plan path's kernels checked; a failure is
# reported as PLAN_EINTERNAL), built by `_build.build(checked=True)`.
LIB_PATH = os.path.join(_PKG, "_lib", "libnhplan_checked.so" if os.environ.get("NHPLAN_BOUNDS_CHECK") == "1"
                        else "libnhplan.so")

PLAN_OK = 0
PLAN_EINVAL = -1
PLAN_NO_DIRECTION = 0xFFFF
PLAN_GEAR_FORWARD, PLAN_GEAR_REVERSE, PLAN_GEAR_AT_REST = 0, 1, 2
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EUNREACHABLE", -6: "ERANGE",
          -7: "EINTERNAL", -8: "ESTATE"}
PLAN_EUNREACHABLE = -5
PLAN_FLAG_HALF_SHIFT = 1
INF = 0xFFFFFFFF
MANEUVERS = ("LF", "SF", "RB", "RF", "SB", "LB")


class PlanError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code == -3:
            try:
                detail = " [" + lib().plan_last_error().decode() + "]"
            except Exception:
                pass
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)}){detail}")


class Pose(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("theta", C.c_int32)]


class Costs(C.Structure):
    _fields_ = [("step_straight", C.c_uint32), ("step_scale", C.c_uint32), ("transition", C.c_uint32),
                ("flags", C.c_uint32)]


class Grid(C.Structure):
    _fields_ = [("nx_log2", C.c_int32), ("ntheta_log2", C.c_int32), ("image", C.c_void_p)]


class Footprint(C.Structure):
    _fields_ = [("front", C.c_int32), ("rear", C.c_int32), ("half_width", C.c_int32)]


class ProfileStats(C.Structure):
    _fields_ = [("turn_passes", C.c_int64), ("straight_passes", C.c_int64), ("render_passes", C.c_int64),
                ("init_passes", C.c_int64), ("turn_ms", C.c_double), ("straight_ms", C.c_double),
                ("render_ms", C.c_double), ("init_ms", C.c_double), ("turn_improved", C.c_uint64),
                ("straight_improved", C.c_uint64), ("turn_tiles_improved", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class TuneEntry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("shape", C.c_int32), ("grid", C.c_int32), ("ms", C.c_float)]


class Segment(C.Structure):
    _fields_ = [("maneuver", C.c_int32), ("entry", Pose), ("exit", Pose), ("steps", C.c_int32),
                ("cost", C.c_uint32)]


class Segment4(C.Structure):
    _fields_ = [("maneuver", C.c_int32), ("entry", Pose), ("entry_level", C.c_int32), ("exit", Pose),
                ("exit_level", C.c_int32), ("steps", C.c_int32), ("cost", C.c_uint32)]


class Goal(C.Structure):
    _fields_ = [("pose", Pose), ("radius_xy", C.c_int32), ("radius_theta", C.c_int32), ("w_xy", C.c_uint32),
                ("w_theta", C.c_uint32), ("bias", C.c_uint32)]


_lib = None


def lib():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2306_01301_b300._build`")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.plan_create.restype = C.c_int
        L.plan_create.argtypes = [C.POINTER(Grid), C.POINTER(Footprint), C.c_double, C.POINTER(Costs),
                                  C.POINTER(Allocator), vp, C.POINTER(vp)]
        L.plan_set_image.restype = C.c_int
        L.plan_set_image.argtypes = [vp, vp]
        L.plan_render_cspace.restype = C.c_int
        L.plan_render_cspace.argtypes = [vp]
        L.plan_sweep.restype = C.c_int
        L.plan_sweep.argtypes = [vp, Pose, C.c_int]
        L.plan_extract.restype = C.c_int
        L.plan_extract.argtypes = [vp, Pose, C.POINTER(Segment), C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_uint32)]
        L.plan_copy_volumes.restype = C.c_int
        L.plan_copy_volumes.argtypes = [vp, vp, vp, vp]
        L.plan_device_volumes.restype = C.c_int
        L.plan_device_volumes.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
        L.plan_profile.restype = C.c_int
        L.plan_profile.argtypes = [vp, C.c_int]
        L.plan_profile_read.restype = C.c_int
        L.plan_profile_read.argtypes = [vp, C.POINTER(ProfileStats)]
        L.plan_kernel_launches.restype = C.c_int
        L.plan_kernel_launches.argtypes = [vp, C.POINTER(C.c_int64)]
        L.plan_destroy.restype = C.c_int
        L.plan_destroy.argtypes = [vp]
        L.plan_strerror.restype = C.c_char_p
        L.plan_strerror.argtypes = [C.c_int]
        L.plan_last_error.restype = C.c_char_p
        L.plan_last_error.argtypes = []
        L.plan_reach_sweep.restype = C.c_int
        L.plan_set_direction_field.restype = C.c_int
        L.plan_set_direction_field.argtypes = [vp, vp, C.c_int, C.c_uint32]
        L.plan_set_compact_graph.restype = C.c_int
        L.plan_set_compact_graph.argtypes = [vp, C.c_int]
        L.plan_sweep_compact.restype = C.c_int
        L.plan_sweep_compact.argtypes = [vp, Pose, C.c_int]
        L.plan_extract_compact.restype = C.c_int
        L.plan_extract_compact.argtypes = [vp, Pose, C.POINTER(Segment), C.c_int, C.POINTER(C.c_int),
                                           C.POINTER(C.c_uint32)]
        L.plan_copy_compact_volumes.restype = C.c_int
        L.plan_copy_compact_volumes.argtypes = [vp, vp, vp, vp, vp]
        L.plan_set_curvature_levels.restype = C.c_int
        L.plan_set_curvature_levels.argtypes = [vp, C.c_int, C.c_double, C.c_uint32]
        L.plan_sweep4.restype = C.c_int
        L.plan_sweep4.argtypes = [vp, Pose, C.c_int, C.c_int]
        L.plan_extract4.restype = C.c_int
        L.plan_extract4.argtypes = [vp, Pose, C.c_int, C.POINTER(Segment4), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_uint32)]
        L.plan_copy_volumes4.restype = C.c_int
        L.plan_copy_volumes4.argtypes = [vp, vp, vp]
        L.plan_clothoid_tables.restype = C.c_int
        L.plan_clothoid_tables.argtypes = [vp, vp, vp, vp]
        L.plan_set_gear_penalty.restype = C.c_int
        L.plan_set_gear_penalty.argtypes = [vp, C.c_uint32]
        L.plan_sweep_gear.restype = C.c_int
        L.plan_sweep_gear.argtypes = [vp, Pose, C.c_int, C.c_int]
        L.plan_extract_gear.restype = C.c_int
        L.plan_extract_gear.argtypes = [vp, Pose, C.POINTER(Segment), C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_uint32), C.POINTER(C.c_int)]
        L.plan_copy_reverse_volumes.restype = C.c_int
        L.plan_copy_reverse_volumes.argtypes = [vp, vp, vp]
        L.plan_set_transition_costs.restype = C.c_int
        L.plan_set_transition_costs.argtypes = [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.plan_sweep_state.restype = C.c_int
        L.plan_sweep_state.argtypes = [vp, Pose, C.POINTER(C.c_uint32), C.c_int]
        L.plan_extract_goal_set.restype = C.c_int
        L.plan_extract_goal_set.argtypes = [vp, C.POINTER(Goal), C.c_int, C.POINTER(Segment), C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_uint32), C.POINTER(Pose),
                                            C.POINTER(C.c_uint64)]
        L.plan_reach_sweep.argtypes = [vp, Pose, C.c_int]
        L.plan_reach_extract.restype = C.c_int
        L.plan_reach_extract.argtypes = [vp, Pose, C.POINTER(Segment), C.c_int, C.POINTER(C.c_int),
                                         C.POINTER(C.c_int)]
        L.plan_reach_counts.restype = C.c_int
        L.plan_reach_counts.argtypes = [vp, vp]
        L.plan_set_kernel_shapes.restype = C.c_int
        L.plan_set_kernel_shapes.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.plan_autotune.restype = C.c_int
        L.plan_autotune.argtypes = [vp, Pose, vp, C.c_int, C.POINTER(C.c_int)]
        L.plan_soft_image.restype = C.c_int
        L.plan_soft_image.argtypes = [C.c_int, vp, C.c_int, C.c_int, vp]
        _lib = L
    return _lib


def _strerror(code: int) -> str:
    try:
        return lib().plan_strerror(code).decode()
    except Exception:  # library not loadable while formatting an error
        return "?"


def _check(rc: int, where: str):
    if rc != PLAN_OK:
        raise PlanError(rc, where)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def soft_image(occupancy: np.ndarray, radius: int, soft_max: int) -> np.ndarray:
    """Section VII soft-obstacle image (library host helper)."""
    occ = np.ascontiguousarray(occupancy, dtype=np.uint8)
    img = np.zeros(occ.shape, np.uint16)
    _check(lib().plan_soft_image(int(occ.shape[0]), _ptr(occ), int(radius), int(soft_max), _ptr(img)),
           "plan_soft_image")
    return img


@dataclass
class PlanResult:
    cost: int
    segments: List[dict]


class _TorchAllocator:
    """C-ABI allocator callbacks bound to torch's CUDA caching allocator."""

    def __init__(self, torch, stream):
        self.torch = torch
        self.stream = stream
        self.device = stream.device

        def _alloc(nbytes, _stream, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, _nbytes, _stream, _ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._fa = ALLOC_FN(_alloc)
        self._ff = FREE_FN(_free)
        self.struct = Allocator(self._fa, self._ff, None)


class Planner:
    """One plan: grid shape + image + vehicle + costs, volumes on the GPU."""

    def __init__(self, nx_log2: int, nt_log2: int, image: np.ndarray, footprint: Tuple[int, int, int],
                 turn_radius: float, transition: int, step_straight: int = 100, step_scale: int = 100,
                 half_shift: int = 1, stream=None, allocator=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("nhplan needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.nx_log2, self.nt_log2 = nx_log2, nt_log2
        self.nx, self.nt = 1 << nx_log2, 1 << nt_log2
        self.cells = self.nx * self.nx * self.nt
        self.stream = stream or torch.cuda.current_stream()
        # an object with a `struct` (Allocator) attribute; torch's caching allocator by default
        self._alloc = allocator or _TorchAllocator(torch, self.stream)
        img = np.ascontiguousarray(image, dtype=np.uint16)
        assert img.shape == (self.nx, self.nx)
        grid = Grid(nx_log2, nt_log2, img.ctypes.data_as(C.c_void_p))
        fp = Footprint(*[int(v) for v in footprint])
        costs = Costs(step_straight, step_scale, transition, PLAN_FLAG_HALF_SHIFT if half_shift else 0)
        h = C.c_void_p()
        _check(lib().plan_create(C.byref(grid), C.byref(fp), float(turn_radius), C.byref(costs),
                                 C.byref(self._alloc.struct), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "plan_create")
        self._h = h

    @classmethod
    def from_scene(cls, sc, image: Optional[np.ndarray] = None, stream=None) -> "Planner":
        if image is None:
            image = soft_image(sc.occupancy, sc.soft_radius, sc.soft_max) if sc.soft_radius else sc.hard_image()
        return cls(sc.nx_log2, sc.nt_log2, image, sc.footprint, sc.turn_radius, sc.transition,
                   sc.step_straight, sc.step_scale, sc.half_shift, stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ steps
    def set_image(self, image: np.ndarray):
        img = np.ascontiguousarray(image, dtype=np.uint16)
        _check(lib().plan_set_image(self._h, _ptr(img)), "plan_set_image")

    def render(self):
        _check(lib().plan_render_cspace(self._h), "plan_render_cspace")

    def sweep(self, start, n_cycles: int):
        _check(lib().plan_sweep(self._h, Pose(*[int(v) for v in start]), int(n_cycles)), "plan_sweep")

    def set_direction_field(self, heading, tolerance: int = 0, penalty_q8: int = 256):
        """plan_set_direction_field: preferred heading per cell (Nx x Nx,
        PLAN_NO_DIRECTION = none), or None to remove the field."""
        if heading is None:
            _check(lib().plan_set_direction_field(self._h, None, 0, 256), "plan_set_direction_field")
            return
        h = np.ascontiguousarray(heading, dtype=np.uint16)
        assert h.shape == (self.nx, self.nx)
        _check(lib().plan_set_direction_field(self._h, _ptr(h), int(tolerance), int(penalty_q8)),
               "plan_set_direction_field")

    # ------------------------------------------- Compact graph (Fig. 12)
    def set_compact_graph(self, enable: bool = True):
        _check(lib().plan_set_compact_graph(self._h, 1 if enable else 0), "plan_set_compact_graph")

    def sweep_compact(self, start, n_cycles: int):
        _check(lib().plan_sweep_compact(self._h, Pose(*[int(v) for v in start]), int(n_cycles)),
               "plan_sweep_compact")

    def extract_compact(self, goal, cap: int = 1024) -> Optional[PlanResult]:
        segs = (Segment * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        rc = lib().plan_extract_compact(self._h, Pose(*[int(v) for v in goal]), segs, cap, C.byref(n),
                                        C.byref(cost))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_extract_compact")
        return PlanResult(int(cost.value), self._segments(segs, n.value))

    def compact_volumes(self):
        """(V_S, L_S, V_L, L_L, V_R, L_R)"""
        vs, ls, _ = self.volumes(B=False)
        arrs = [np.empty(self.cells, t) for t in (np.uint32, np.uint16, np.uint32, np.uint16)]
        _check(lib().plan_copy_compact_volumes(self._h, *[_ptr(a) for a in arrs]), "plan_copy_compact_volumes")
        return (vs, ls, *arrs)

    # ---------------------------------------- curvature levels (Appendix F)
    def set_curvature_levels(self, levels_per_side: int, arc_per_level: float = 1.0, clothoid_cost: int = 0):
        _check(lib().plan_set_curvature_levels(self._h, int(levels_per_side), float(arc_per_level),
                                               int(clothoid_cost)), "plan_set_curvature_levels")
        self.curv_M = int(levels_per_side)

    def sweep4(self, start, start_level: int, n_cycles: int):
        _check(lib().plan_sweep4(self._h, Pose(*[int(v) for v in start]), int(start_level), int(n_cycles)),
               "plan_sweep4")

    def extract4(self, goal, goal_level: int, cap: int = 1024):
        segs = (Segment4 * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        rc = lib().plan_extract4(self._h, Pose(*[int(v) for v in goal]), int(goal_level), segs, cap, C.byref(n),
                                 C.byref(cost))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_extract4")
        out = [dict(mu=x.maneuver, entry=(x.entry.x, x.entry.y, x.entry.theta), entry_level=x.entry_level,
                    exit=(x.exit.x, x.exit.y, x.exit.theta), exit_level=x.exit_level, steps=x.steps, cost=x.cost)
               for x in segs[:n.value]]
        return PlanResult(int(cost.value), out)

    def volumes4(self):
        n4 = self.cells * (2 * self.curv_M + 1)
        v = np.empty(n4, np.uint32)
        l_ = np.empty(n4, np.uint16)
        _check(lib().plan_copy_volumes4(self._h, _ptr(v), _ptr(l_)), "plan_copy_volumes4")
        return v, l_

    def clothoid_tables(self):
        nk = 2 * self.curv_M + 1
        dx = np.zeros((2, nk, self.nt), np.int16)
        dy = np.zeros((2, nk, self.nt), np.int16)
        dth = np.zeros((2, nk), np.int32)
        _check(lib().plan_clothoid_tables(self._h, _ptr(dx), _ptr(dy), _ptr(dth)), "plan_clothoid_tables")
        return dx, dy, dth

    def set_gear_penalty(self, penalty):
        """plan_set_gear_penalty (None: PLAN_GEAR_OFF)."""
        _check(lib().plan_set_gear_penalty(self._h, 0xFFFFFFFF if penalty is None else int(penalty)),
               "plan_set_gear_penalty")

    def sweep_gear(self, start, start_gear: int, n_cycles: int):
        _check(lib().plan_sweep_gear(self._h, Pose(*[int(v) for v in start]), int(start_gear), int(n_cycles)),
               "plan_sweep_gear")

    def extract_gear(self, goal, cap: int = 1024):
        """Returns (PlanResult, end gear) or None when unreachable."""
        segs = (Segment * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        gear = C.c_int(0)
        rc = lib().plan_extract_gear(self._h, Pose(*[int(v) for v in goal]), segs, cap, C.byref(n), C.byref(cost),
                                     C.byref(gear))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_extract_gear")
        return PlanResult(int(cost.value), self._segments(segs, n.value)), int(gear.value)

    def reverse_volumes(self):
        v = np.empty(self.cells, np.uint32)
        l_ = np.empty(self.cells, np.uint16)
        _check(lib().plan_copy_reverse_volumes(self._h, _ptr(v), _ptr(l_)), "plan_copy_reverse_volumes")
        return v, l_

    def set_transition_costs(self, cost_in, cost_out):
        """plan_set_transition_costs: per-maneuver Star transition edges
        (cycle order LF, SF, RB, RF, SB, LB)."""
        if len(cost_in) != 6 or len(cost_out) != 6:
            raise ValueError("six entering and six leaving costs")
        ci = (C.c_uint32 * 6)(*[int(v) for v in cost_in])
        co = (C.c_uint32 * 6)(*[int(v) for v in cost_out])
        _check(lib().plan_set_transition_costs(self._h, ci, co), "plan_set_transition_costs")

    def sweep_state(self, start, entry, n_cycles: int):
        """plan_sweep_state: entry[mu] = cost of entering maneuver mu (cycle
        order LF, SF, RB, RF, SB, LB) at the start, at most the transition cost."""
        e = (C.c_uint32 * 6)(*[int(v) for v in entry])
        if len(entry) != 6:
            raise ValueError("entry needs one cost per maneuver")
        _check(lib().plan_sweep_state(self._h, Pose(*[int(v) for v in start]), e, int(n_cycles)),
               "plan_sweep_state")

    @staticmethod
    def _segments(segs, n):
        return [dict(mu=s.maneuver, entry=(s.entry.x, s.entry.y, s.entry.theta),
                     exit=(s.exit.x, s.exit.y, s.exit.theta), steps=s.steps, cost=s.cost) for s in segs[:n]]

    def extract(self, goal, cap: int = 1024) -> Optional[PlanResult]:
        segs = (Segment * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        rc = lib().plan_extract(self._h, Pose(*[int(v) for v in goal]), segs, cap, C.byref(n), C.byref(cost))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_extract")
        return PlanResult(int(cost.value), self._segments(segs, n.value))

    def extract_goal_set(self, goals, cap: int = 1024):
        """plan_extract_goal_set over (x, y, theta, r_xy, r_theta, w_xy,
        w_theta, bias) tuples.  Returns (best pose, score, PlanResult) or None
        when no pose of any box was reached."""
        arr = (Goal * len(goals))(*[Goal(Pose(*[int(v) for v in g[:3]]), *[int(v) for v in g[3:8]]) for g in goals])
        segs = (Segment * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        best = Pose()
        score = C.c_uint64(0)
        rc = lib().plan_extract_goal_set(self._h, arr, len(goals), segs, cap, C.byref(n), C.byref(cost),
                                         C.byref(best), C.byref(score))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_extract_goal_set")
        return (best.x, best.y, best.theta), int(score.value), PlanResult(int(cost.value),
                                                                         self._segments(segs, n.value))

    def plan(self, start, goal, n_cycles: int) -> Optional[PlanResult]:
        self.render()
        self.sweep(start, n_cycles)
        return self.extract(goal)

    # ------------------------------------------------ Appendix C reachability
    def reach_sweep(self, start, n_cycles: int):
        """Fewest-maneuver reachability over hard obstacles (bit vectors)."""
        _check(lib().plan_reach_sweep(self._h, Pose(*[int(v) for v in start]), int(n_cycles)), "plan_reach_sweep")

    def reach_extract(self, goal, cap: int = 256):
        """(fewest maneuvers, segments in driving order), or None if the goal
        needs more maneuvers than were swept."""
        segs = (Segment * cap)()
        n, m = C.c_int(0), C.c_int(0)
        rc = lib().plan_reach_extract(self._h, Pose(*[int(v) for v in goal]), segs, cap, C.byref(n), C.byref(m))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_reach_extract")
        return int(m.value), _segments(segs, n.value)

    def reach_counts(self) -> np.ndarray:
        out = np.empty(self.cells, np.uint8)
        _check(lib().plan_reach_counts(self._h, _ptr(out)), "plan_reach_counts")
        return out

    def set_kernel_shapes(self, turn_variant: int = -1, turn_grid: int = 0, straight_lines: int = 0,
                          straight_grid: int = 0):
        _check(lib().plan_set_kernel_shapes(self._h, int(turn_variant), int(turn_grid), int(straight_lines),
                                            int(straight_grid)), "plan_set_kernel_shapes")

    def autotune(self, start) -> List[dict]:
        """Time the kernel shapes on this plan and keep the fastest for its
        sweeps (plan_autotune).  Returns every timed shape."""
        cap = 64
        arr = (TuneEntry * cap)()
        n = C.c_int(0)
        _check(lib().plan_autotune(self._h, Pose(*[int(v) for v in start]), C.cast(arr, C.c_void_p), cap,
                                   C.byref(n)), "plan_autotune")
        return [{"kernel": "turn" if e.kind == 0 else "straight", "shape": e.shape, "grid": e.grid, "ms": e.ms}
                for e in arr[:n.value]]

    # ------------------------------------------------------------ inspection
    def volumes(self, V=True, L=True, B=True):
        v = np.empty(self.cells, np.uint32) if V else None
        l_ = np.empty(self.cells, np.uint16) if L else None
        b = np.empty(self.cells, np.uint16) if B else None
        _check(lib().plan_copy_volumes(self._h, _ptr(v) if V else None, _ptr(l_) if L else None,
                                       _ptr(b) if B else None), "plan_copy_volumes")
        return v, l_, b

    def device_pointers(self):
        v, l_, b = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib().plan_device_volumes(self._h, C.byref(v), C.byref(l_), C.byref(b)), "plan_device_volumes")
        return v.value, l_.value, b.value

    def profile(self, enable: bool = True, counts: bool = True):
        """Per-pass event timing; with counts, also the improved-cell
        counters (which add work to the sweep kernels)."""
        _check(lib().plan_profile(self._h, (1 if counts else 2) if enable else 0), "plan_profile")

    def profile_read(self) -> dict:
        st = ProfileStats()
        _check(lib().plan_profile_read(self._h, C.byref(st)), "plan_profile_read")
        return {f: getattr(st, f) for f, _ in ProfileStats._fields_}

    def kernel_launches(self) -> int:
        c = C.c_int64(0)
        _check(lib().plan_kernel_launches(self._h, C.byref(c)), "plan_kernel_launches")
        return int(c.value)


# ---------------------------------------------------------------- batching
class Query(C.Structure):
    _fields_ = [("start", Pose), ("goal", Pose), ("n_cycles", C.c_int32)]


class LaneInfo(C.Structure):
    _fields_ = [("n_queries", C.c_int32), ("ntheta_log2", C.c_int32), ("nx_min", C.c_int32),
                ("nx_max", C.c_int32), ("turn_variant", C.c_int32), ("turn_k", C.c_int32),
                ("turn_sections", C.c_int32), ("turn_cluster", C.c_int32), ("turn_grid", C.c_int32),
                ("straight_lines", C.c_int32), ("straight_grid", C.c_int32), ("n_candidates", C.c_int32),
                ("turn_ms", C.c_float), ("straight_ms", C.c_float)]


PLAN_BATCH_NO_GRAPH = 1
PLAN_BATCH_NO_TUNE = 2


def _batch_signatures(L):
    vp = C.c_void_p
    L.plan_batch_create.restype = C.c_int
    L.plan_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.c_uint32, C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.plan_batch_run.restype = C.c_int
    L.plan_batch_run.argtypes = [vp, C.POINTER(Query), C.c_int]
    L.plan_batch_sync.restype = C.c_int
    L.plan_batch_sync.argtypes = [vp]
    L.plan_batch_result.restype = C.c_int
    L.plan_batch_result.argtypes = [vp, C.c_int, C.POINTER(Segment), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_uint32)]
    L.plan_batch_lanes.restype = C.c_int
    L.plan_batch_lanes.argtypes = [vp, C.POINTER(C.c_int)]
    L.plan_batch_lane.restype = C.c_int
    L.plan_batch_lane.argtypes = [vp, C.c_int, C.POINTER(LaneInfo)]
    L.plan_batch_kernel_launches.restype = C.c_int
    L.plan_batch_kernel_launches.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.plan_batch_destroy.restype = C.c_int
    L.plan_batch_destroy.argtypes = [vp]


def _segments(segs, n) -> List[dict]:
    return [dict(mu=s.maneuver, entry=(s.entry.x, s.entry.y, s.entry.theta), exit=(s.exit.x, s.exit.y, s.exit.theta),
                 steps=s.steps, cost=s.cost) for s in segs[:n]]


class Batch:
    """Many queries, one per Planner, run together (plan_batch_* in the C ABI)."""

    def __init__(self, planners: List[Planner], graph: bool = True, tune: bool = True, stream=None,
                 allocator=None):
        import torch
        L = lib()
        if not hasattr(L, "_batch_sig"):
            _batch_signatures(L)
            L._batch_sig = True
        self.planners = list(planners)
        self.stream = stream or torch.cuda.current_stream()
        self._alloc = allocator or _TorchAllocator(torch, self.stream)
        arr = (C.c_void_p * len(self.planners))(*[p._h.value for p in self.planners])
        flags = (0 if graph else PLAN_BATCH_NO_GRAPH) | (0 if tune else PLAN_BATCH_NO_TUNE)
        h = C.c_void_p()
        _check(L.plan_batch_create(arr, len(self.planners), flags, C.byref(self._alloc.struct),
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)), "plan_batch_create")
        self._h = h

    def run(self, queries, render: bool = True):
        """queries: [(start, goal, n_cycles)] (one per planner).  Async."""
        n = len(self.planners)
        assert len(queries) == n
        arr = (Query * n)()
        for i, (s, g, N) in enumerate(queries):
            arr[i] = Query(Pose(*[int(v) for v in s]), Pose(*[int(v) for v in g]), int(N))
        _check(lib().plan_batch_run(self._h, arr, 1 if render else 0), "plan_batch_run")

    def sync(self):
        _check(lib().plan_batch_sync(self._h), "plan_batch_sync")

    def result(self, i: int, cap: int = 1024) -> Optional[PlanResult]:
        segs = (Segment * cap)()
        n = C.c_int(0)
        cost = C.c_uint32(0)
        rc = lib().plan_batch_result(self._h, int(i), segs, cap, C.byref(n), C.byref(cost))
        if rc == PLAN_EUNREACHABLE:
            return None
        _check(rc, "plan_batch_result")
        return PlanResult(int(cost.value), _segments(segs, n.value))

    def results(self) -> List[Optional[PlanResult]]:
        return [self.result(i) for i in range(len(self.planners))]

    def lanes(self) -> List[dict]:
        n = C.c_int(0)
        _check(lib().plan_batch_lanes(self._h, C.byref(n)), "plan_batch_lanes")
        out = []
        for k in range(n.value):
            li = LaneInfo()
            _check(lib().plan_batch_lane(self._h, k, C.byref(li)), "plan_batch_lane")
            out.append({f: getattr(li, f) for f, _ in LaneInfo._fields_})
        return out

    def kernel_launches(self) -> Tuple[int, int]:
        a, b = C.c_int64(0), C.c_int64(0)
        _check(lib().plan_batch_kernel_launches(self._h, C.byref(a), C.byref(b)), "plan_batch_kernel_launches")
        return int(a.value), int(b.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().plan_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving
PLAN_SERVE_CONTINUOUS = 0
PLAN_SERVE_ONE_AT_A_TIME = 1
PLAN_SERVE_STOP_AT_CONVERGENCE = 1
PLAN_ECANCELED = -9


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_inflight", C.c_int32), ("mode", C.c_int32),
                ("heavy_cells", C.c_int64), ("big_cells", C.c_int64), ("max_heavy", C.c_int32),
                ("flags", C.c_int32), ("slot_bytes", C.c_int64)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("cost", C.c_uint32), ("n_segments", C.c_int32), ("scene", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("scenes", "submitted", "admitted", "completed", "rejected", "steps",
                                         "launches", "peak_inflight", "arena_bytes", "peak_bytes",
                                         "scene_bytes", "reserved_bytes", "cancelled", "partial_steps")]


def _server_signatures(L):
    vp = C.c_void_p
    L.plan_server_create.restype = C.c_int
    L.plan_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.plan_server_add_scene.restype = C.c_int
    L.plan_server_add_scene.argtypes = [vp, C.POINTER(Grid), C.POINTER(Footprint), C.c_double, C.POINTER(Costs),
                                        C.POINTER(C.c_int32)]
    L.plan_server_submit.restype = C.c_int
    L.plan_server_submit.argtypes = [vp, C.c_int32, Pose, Pose, C.c_int32, C.POINTER(C.c_uint64)]
    L.plan_server_wait.restype = C.c_int
    L.plan_server_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(RequestInfo), C.POINTER(Segment), C.c_int,
                                   C.POINTER(C.c_int)]
    L.plan_server_cancel.restype = C.c_int
    L.plan_server_cancel.argtypes = [vp, C.c_uint64]
    L.plan_server_stats_read.restype = C.c_int
    L.plan_server_stats_read.argtypes = [vp, C.POINTER(ServerStats)]
    L.plan_server_destroy.restype = C.c_int
    L.plan_server_destroy.argtypes = [vp]


class Server:
    """Planning server (plan_server_* in the C ABI): cached scenes, requests
    admitted by an HBM budget, continuous batching or one at a time."""

    def __init__(self, budget_bytes: int, max_inflight: int = 0, one_at_a_time: bool = False,
                 heavy_cells: int = 0, big_cells: int = 0, max_heavy: int = 0, stop_at_convergence: bool = False,
                 slot_bytes: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("nhplan needs a CUDA device; there is no CPU fallback")
        L = lib()
        if not hasattr(L, "_server_sig"):
            _server_signatures(L)
            L._server_sig = True
        self.stream = stream or torch.cuda.current_stream()
        self._alloc = _TorchAllocator(torch, self.stream)
        cfg = ServerConfig(int(budget_bytes), int(max_inflight),
                           PLAN_SERVE_ONE_AT_A_TIME if one_at_a_time else PLAN_SERVE_CONTINUOUS,
                           int(heavy_cells), int(big_cells), int(max_heavy),
                           PLAN_SERVE_STOP_AT_CONVERGENCE if stop_at_convergence else 0, int(slot_bytes))
        h = C.c_void_p()
        _check(L.plan_server_create(C.byref(cfg), C.byref(self._alloc.struct), C.c_void_p(self.stream.cuda_stream),
                                    C.byref(h)), "plan_server_create")
        self._h = h

    def add_scene(self, sc, image: Optional[np.ndarray] = None) -> int:
        if image is None:
            image = soft_image(sc.occupancy, sc.soft_radius, sc.soft_max) if sc.soft_radius else sc.hard_image()
        img = np.ascontiguousarray(image, dtype=np.uint16)
        grid = Grid(sc.nx_log2, sc.nt_log2, img.ctypes.data_as(C.c_void_p))
        fp = Footprint(*[int(v) for v in sc.footprint])
        costs = Costs(sc.step_straight, sc.step_scale, sc.transition, PLAN_FLAG_HALF_SHIFT if sc.half_shift else 0)
        sid = C.c_int32(-1)
        _check(lib().plan_server_add_scene(self._h, C.byref(grid), C.byref(fp), float(sc.turn_radius),
                                           C.byref(costs), C.byref(sid)), "plan_server_add_scene")
        return int(sid.value)

    def submit(self, scene: int, start, goal, n_cycles: int) -> int:
        t = C.c_uint64(0)
        _check(lib().plan_server_submit(self._h, int(scene), Pose(*[int(v) for v in start]),
                                        Pose(*[int(v) for v in goal]), int(n_cycles), C.byref(t)),
               "plan_server_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout: float = -1.0, cap: int = 1024):
        """Returns (info dict, PlanResult or None when unreachable)."""
        info = RequestInfo()
        segs = (Segment * cap)()
        n = C.c_int(0)
        _check(lib().plan_server_wait(self._h, int(ticket), float(timeout), C.byref(info), segs, cap, C.byref(n)),
               "plan_server_wait")
        d = {f: getattr(info, f) for f, _ in RequestInfo._fields_}
        if info.status == PLAN_EUNREACHABLE:
            return d, None
        if info.status != PLAN_OK:
            raise PlanError(info.status, "served request")
        return d, PlanResult(int(info.cost), _segments(segs, n.value))

    def cancel(self, ticket: int):
        _check(lib().plan_server_cancel(self._h, int(ticket)), "plan_server_cancel")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().plan_server_stats_read(self._h, C.byref(st)), "plan_server_stats_read")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().plan_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``nhp_oracle.c``, a plain, slow, single-threaded C
restatement of the paper's graph (Section V), obstacle rendering (Section VI),
kernel-style layered relaxation (Section VIII.B, Insert 1), Dijkstra (Section
VIII.A) and forward-tracking extraction (Section X).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package; the planner library never does, and this package never imports
the planner library.

Every function cites the passage it follows in the C source.  All of them are
pinned by ``tests/test_oracle_pins.py`` (hand-worked table values, closed
forms, brute-force enumeration, Dijkstra convergence, symmetries, an
independent library distance transform).

``cpu_sweep`` (``cpu_sweep.c``) is not part of the oracle: it is the same
kernel-style sweep spread over all host cores with OpenMP, the CPU baseline
that ``bench.py`` times beside the oracle (the counterpart of the paper's
CPU kernel timings); ``tests/test_cpu_sweep.py`` checks it against the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_lib", "libnhp_oracle.so")
_SRC = os.path.join(_HERE, "nhp_oracle.c")
_HDR = os.path.join(_HERE, "nhp_oracle.h")
_CS_SO = os.path.join(_HERE, "_lib", "libnhp_cpu_sweep.so")
_CS_SRC = os.path.join(_HERE, "cpu_sweep.c")

INF = 0xFFFFFFFF
HARD = 0xFFFF
NONE = 0xFFFF
LF, SF, RB, RF, SB, LB = range(6)
CYCLE_ORDER = (LF, SF, RB, RF, SB, LB)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_lib (idempotent)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(_SRC),
                                                                       os.path.getmtime(_HDR)):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _SO)
    if force or not os.path.exists(_CS_SO) or os.path.getmtime(_CS_SO) < os.path.getmtime(_CS_SRC):
        tmp = _CS_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O3", "-fopenmp", "-Wall", "-fPIC", "-shared", "-o", tmp,
                               _CS_SRC])
        os.replace(tmp, _CS_SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        p = C.c_void_p
        L.orc_create.restype = p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_destroy.argtypes = [p]
        L.orc_tables.argtypes = [p] + [p] * 7
        L.orc_footprint.restype = C.c_int
        L.orc_footprint.argtypes = [p, C.c_int, C.c_int, C.c_int, C.c_int, p, p, C.c_int]
        L.orc_render.restype = C.c_int
        L.orc_render.argtypes = [p, p, C.c_int, C.c_int, C.c_int, p]
        L.orc_render_rows.restype = C.c_int
        L.orc_render_rows.argtypes = [p, p, C.c_int, C.c_int, C.c_int, p]
        L.orc_render_cells.restype = C.c_int
        L.orc_render_cells.argtypes = [p, p, C.c_int, C.c_int, C.c_int, p, C.c_int64, p]
        L.orc_succ.restype = C.c_int64
        L.orc_succ.argtypes = [p, C.c_int, C.c_int64]
        L.orc_edge.restype = C.c_uint32
        L.orc_edge.argtypes = [p, p, C.c_int, C.c_int64]
        L.orc_sweep.restype = C.c_int
        L.orc_sweep.argtypes = [p, p, C.c_int64, C.c_int, C.c_int, p, p, p]
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_layers.restype = C.c_int
        L.orc_layers.argtypes = [p, p, C.c_int, C.c_int, C.c_int, p, p, p]
        L.orc_dijkstra.restype = C.c_int
        L.orc_dijkstra.argtypes = [p, p, C.c_int64, p]
        L.orc_bruteforce.restype = C.c_int
        L.orc_bruteforce.argtypes = [p, p, C.c_int64, C.c_int, p]
        L.orc_extract.restype = C.c_int
        L.orc_extract.argtypes = [p, p, p, C.c_int64, p, C.c_int]
        L.orc_soft_image.argtypes = [C.c_int, p, C.c_int, C.c_int, p]
        L.orc_set_transition.restype = C.c_int
        L.orc_set_transition.argtypes = [p, p, p]
        L.orc_direction.restype = C.c_int
        L.orc_direction.argtypes = [p, p, p, C.c_int, C.c_uint32]
        L.orc_sweep_gear.restype = C.c_int
        L.orc_sweep_gear.argtypes = [p, p, C.c_int64, C.c_int, C.c_uint32, C.c_int, p, p]
        L.orc_dijkstra_gear.restype = C.c_int
        L.orc_dijkstra_gear.argtypes = [p, p, C.c_int64, C.c_int, C.c_uint32, p]
        L.orc_bruteforce_gear.restype = C.c_int
        L.orc_bruteforce_gear.argtypes = [p, p, C.c_int64, C.c_int, C.c_uint32, C.c_int, p]
        L.orc_extract_gear.restype = C.c_int
        L.orc_extract_gear.argtypes = [p, p, p, C.c_int64, p, C.c_int]
        L.orc_sweep_compact.restype = C.c_int
        L.orc_sweep_compact.argtypes = [p, p, C.c_int64, C.c_int, p, p]
        L.orc_dijkstra_compact.restype = C.c_int
        L.orc_dijkstra_compact.argtypes = [p, p, C.c_int64, p]
        L.orc_bruteforce_compact.restype = C.c_int
        L.orc_bruteforce_compact.argtypes = [p, p, C.c_int64, C.c_int, p]
        L.orc_extract_compact.restype = C.c_int
        L.orc_extract_compact.argtypes = [p, p, p, C.c_int64, p, C.c_int]
        L.orc4_create.restype = p
        L.orc4_create.argtypes = [p, C.c_int, C.c_double, C.c_uint32]
        L.orc4_destroy.argtypes = [p]
        L.orc4_tables.argtypes = [p, p, p, p]
        L.orc4_succ.restype = C.c_int64
        L.orc4_succ.argtypes = [p, C.c_int, C.c_int64]
        L.orc4_sweep.restype = C.c_int
        L.orc4_sweep.argtypes = [p, p, C.c_int64, C.c_int, p, p]
        L.orc4_dijkstra.restype = C.c_int
        L.orc4_dijkstra.argtypes = [p, p, C.c_int64, p]
        L.orc4_bruteforce.restype = C.c_int
        L.orc4_bruteforce.argtypes = [p, p, C.c_int64, C.c_int, p]
        L.orc4_extract.restype = C.c_int
        L.orc4_extract.argtypes = [p, p, p, C.c_int64, p, C.c_int]
        L.orc_seed.restype = C.c_int
        L.orc_seed.argtypes = [p, p, C.c_int64, p, p, p]
        L.orc_sweep_state.restype = C.c_int
        L.orc_sweep_state.argtypes = [p, p, C.c_int64, p, C.c_int, C.c_int, p, p, p]
        L.orc_dijkstra_state.restype = C.c_int
        L.orc_dijkstra_state.argtypes = [p, p, C.c_int64, p, p]
        L.orc_bruteforce_state.restype = C.c_int
        L.orc_bruteforce_state.argtypes = [p, p, C.c_int64, p, C.c_int, p]
        L.orc_goal_search.restype = C.c_int
        L.orc_goal_search.argtypes = [p, p, p, C.c_int, p, p]
        L.orc_reach.restype = C.c_int
        L.orc_reach.argtypes = [p, p, C.c_int64, C.c_int, p]
        L.orc_reach_extract.restype = C.c_int
        L.orc_reach_extract.argtypes = [p, p, p, C.c_int64, p, C.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One grid shape + vehicle turn radius + integer costs."""

    def __init__(self, nx_log2: int, nt_log2: int, turn_radius: float, half_shift: int = 1,
                 step_straight: int = 100, step_scale: int = 100, transition: int = 500):
        self.nx_log2, self.nt_log2 = nx_log2, nt_log2
        self.nx, self.nt = 1 << nx_log2, 1 << nt_log2
        self.nr = self.nx * self.nx * self.nt
        self.ct = transition
        self.cin, self.cout = [transition] * 6, [0] * 6
        self._c = lib().orc_create(nx_log2, nt_log2, float(turn_radius), int(half_shift),
                                   step_straight, step_scale, transition)
        if not self._c:
            raise ValueError("oracle: invalid grid description")

    def __del__(self):
        if getattr(self, "_c", None):
            lib().orc_destroy(self._c)
            self._c = None

    def cell(self, pose) -> int:
        i, j, t = pose
        return int(i) + self.nx * (int(j) + self.nx * int(t))

    def pose(self, cell: int):
        cell = int(cell)
        return (cell & (self.nx - 1), (cell >> self.nx_log2) & (self.nx - 1), cell >> (2 * self.nx_log2))

    # ----------------------------------------------------------- eqs. 11-24
    def tables(self):
        nt, nx = self.nt, self.nx
        beta = np.zeros(nt, np.int32)
        psi2 = np.zeros(nt, np.uint8)
        iflag = np.zeros(nt, np.uint8)
        jsign = np.zeros(nt, np.int8)
        bsh = np.zeros((nt, nx), np.int32)
        wS = np.zeros(nt, np.uint32)
        wA = np.zeros(1, np.uint32)
        lib().orc_tables(self._c, _ptr(beta), _ptr(psi2), _ptr(iflag), _ptr(jsign), _ptr(bsh), _ptr(wS), _ptr(wA))
        return dict(beta=beta, psi2=psi2, iflag=iflag, jsign=jsign, bshear=bsh, wS=wS, wA=int(wA[0]))

    # ----------------------------------------------------------- Section VI
    def footprint(self, front: int, rear: int, hw: int, theta: int):
        cap = 1 << 18
        dx = np.zeros(cap, np.int32)
        dy = np.zeros(cap, np.int32)
        n = lib().orc_footprint(self._c, front, rear, hw, theta, _ptr(dx), _ptr(dy), cap)
        if n < 0:
            raise ValueError("footprint too large")
        return dx[:n].copy(), dy[:n].copy()

    def render(self, img: np.ndarray, footprint) -> np.ndarray:
        img = np.ascontiguousarray(img, dtype=np.uint16)
        B = np.zeros(self.nr, np.uint16)
        if lib().orc_render(self._c, _ptr(img), *[int(v) for v in footprint], _ptr(B)) != 0:
            raise MemoryError
        return B

    def render_rows(self, img: np.ndarray, footprint) -> np.ndarray:
        """Same volume as render(), by row runs and sliding maxima (fast)."""
        img = np.ascontiguousarray(img, dtype=np.uint16)
        B = np.zeros(self.nr, np.uint16)
        if lib().orc_render_rows(self._c, _ptr(img), *[int(v) for v in footprint], _ptr(B)) != 0:
            raise MemoryError
        return B

    def render_cells(self, img: np.ndarray, footprint, cells) -> np.ndarray:
        img = np.ascontiguousarray(img, dtype=np.uint16)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(len(cells), np.uint16)
        if lib().orc_render_cells(self._c, _ptr(img), *[int(v) for v in footprint], _ptr(cells),
                                  len(cells), _ptr(out)) != 0:
            raise ValueError("render_cells failed")
        return out

    # ----------------------------------------------------------- eqs. 25-31
    def succ(self, mu: int, cell: int) -> int:
        return int(lib().orc_succ(self._c, mu, int(cell)))

    def edge(self, B: np.ndarray, mu: int, cell: int) -> int:
        return int(lib().orc_edge(self._c, _ptr(B), mu, int(cell)))

    # ----------------------------------------------------------- Section VIII
    @staticmethod
    def set_threads(n: int):
        """Host threads of the lockstep mode (mode 1); 1 by default.  The
        chains of a layer are independent, so the results do not depend on
        the count (tests/test_oracle_pins.py checks 1 against 8)."""
        lib().orc_set_threads(int(n))

    def sweep(self, B: np.ndarray, start: int, n_cycles: int, mode: int = 0):
        B = np.ascontiguousarray(B, dtype=np.uint16)
        V = np.zeros(self.nr, np.uint32)
        L = np.zeros(self.nr, np.uint16)
        imp = np.zeros(max(1, 6 * n_cycles), np.int64)
        rc = lib().orc_sweep(self._c, _ptr(B), int(start), int(n_cycles), int(mode), _ptr(V), _ptr(L), _ptr(imp))
        if rc != 0:
            raise ValueError(f"oracle sweep failed ({rc})")
        return V, L, imp[:6 * n_cycles]

    def layers(self, B, V, L, first_layer: int, n_layers: int, mode: int = 0):
        V = np.array(V, dtype=np.uint32, copy=True)
        L = np.array(L, dtype=np.uint16, copy=True)
        imp = np.zeros(max(1, n_layers), np.int64)
        rc = lib().orc_layers(self._c, _ptr(np.ascontiguousarray(B, dtype=np.uint16)), first_layer, n_layers,
                              mode, _ptr(V), _ptr(L), _ptr(imp))
        if rc != 0:
            raise ValueError("oracle layers failed")
        return V, L, imp[:n_layers]

    def dijkstra(self, B: np.ndarray, start: int) -> np.ndarray:
        V = np.zeros(self.nr, np.uint32)
        if lib().orc_dijkstra(self._c, _ptr(np.ascontiguousarray(B, dtype=np.uint16)), int(start), _ptr(V)) != 0:
            raise ValueError("dijkstra failed")
        return V

    def bruteforce(self, B: np.ndarray, start: int, n_cycles: int) -> np.ndarray:
        V = np.zeros(self.nr, np.uint32)
        if lib().orc_bruteforce(self._c, _ptr(np.ascontiguousarray(B, dtype=np.uint16)), int(start),
                                int(n_cycles), _ptr(V)) != 0:
            raise ValueError("bruteforce failed")
        return V

    # ---------------------------------------------- Section XVI, Fig. 19
    def direction(self, B: np.ndarray, heading: np.ndarray, tol: int, pen: int) -> np.ndarray:
        """B with direction penalties applied (a copy): heading is Nx x Nx,
        0xFFFF = no preferred heading."""
        B = np.array(B, dtype=np.uint16, copy=True)
        h = np.ascontiguousarray(heading, dtype=np.uint16)
        if h.shape != (self.nx, self.nx) or lib().orc_direction(self._c, _ptr(B), _ptr(h), int(tol), int(pen)) != 0:
            raise ValueError("bad direction field")
        return B

    # ------------------------------------------------- Section V.A, Fig. 9
    def set_transition(self, cost_in, cost_out):
        """Per-maneuver Star transition edges: entering mu costs cost_in[mu],
        returning to the transition state cost_out[mu] (cycle-order ids)."""
        ci = np.ascontiguousarray(cost_in, dtype=np.uint32)
        co = np.ascontiguousarray(cost_out, dtype=np.uint32)
        if ci.shape != (6,) or co.shape != (6,) or lib().orc_set_transition(self._c, _ptr(ci), _ptr(co)) != 0:
            raise ValueError("transition costs need 6 + 6 values with every sum below 2^28")
        self.cin, self.cout = [int(v) for v in ci], [int(v) for v in co]

    # ------------------------------------------------ Compact graph (Fig. 12)
    def sweep_compact(self, B: np.ndarray, start: int, n_cycles: int):
        """V, L of 3 * nr entries: vertex types S, L, R."""
        V = np.zeros(3 * self.nr, np.uint32)
        L = np.zeros(3 * self.nr, np.uint16)
        if lib().orc_sweep_compact(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), int(n_cycles),
                                   _ptr(V), _ptr(L)) != 0:
            raise ValueError("sweep_compact failed")
        return V, L

    def dijkstra_compact(self, B: np.ndarray, start: int) -> np.ndarray:
        V = np.zeros(3 * self.nr, np.uint32)
        if lib().orc_dijkstra_compact(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), _ptr(V)) != 0:
            raise ValueError("dijkstra_compact failed")
        return V

    def bruteforce_compact(self, B: np.ndarray, start: int, n_cycles: int) -> np.ndarray:
        V = np.zeros(3 * self.nr, np.uint32)
        if lib().orc_bruteforce_compact(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start),
                                        int(n_cycles), _ptr(V)) != 0:
            raise ValueError("bruteforce_compact failed")
        return V

    def extract_compact(self, V: np.ndarray, L: np.ndarray, goal: int, cap: int = 4096):
        seg = np.zeros((cap, 6), np.int64)
        n = lib().orc_extract_compact(self._c, _ptr(np.ascontiguousarray(V, np.uint32)),
                                      _ptr(np.ascontiguousarray(L, np.uint16)), int(goal), _ptr(seg), cap)
        if n == -1:
            return None
        if n < 0:
            raise ValueError(f"extract_compact failed ({n})")
        return [dict(mu=int(r[0]), entry=int(r[1]), exit=int(r[2]), steps=int(r[3]), cost=int(r[4]),
                     from_s=int(r[5])) for r in seg[:n]]

    # ------------------------------------------------------ gear states
    def sweep_gear(self, B: np.ndarray, start: int, start_gear: int, pen: int, n_cycles: int):
        """Two transition states (forward / reverse gear of the last maneuver):
        returns V, L of 2 * nr entries, the forward state first."""
        V = np.zeros(2 * self.nr, np.uint32)
        L = np.zeros(2 * self.nr, np.uint16)
        rc = lib().orc_sweep_gear(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), int(start_gear),
                                  int(pen), int(n_cycles), _ptr(V), _ptr(L))
        if rc != 0:
            raise ValueError(f"sweep_gear failed ({rc})")
        return V, L

    def dijkstra_gear(self, B: np.ndarray, start: int, start_gear: int, pen: int) -> np.ndarray:
        V = np.zeros(2 * self.nr, np.uint32)
        if lib().orc_dijkstra_gear(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), int(start_gear),
                                   int(pen), _ptr(V)) != 0:
            raise ValueError("dijkstra_gear failed")
        return V

    def bruteforce_gear(self, B: np.ndarray, start: int, start_gear: int, pen: int, n_cycles: int) -> np.ndarray:
        V = np.zeros(2 * self.nr, np.uint32)
        if lib().orc_bruteforce_gear(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start),
                                     int(start_gear), int(pen), int(n_cycles), _ptr(V)) != 0:
            raise ValueError("bruteforce_gear failed")
        return V

    def extract_gear(self, V: np.ndarray, L: np.ndarray, goal: int, cap: int = 4096):
        seg = np.zeros((cap, 7), np.int64)
        n = lib().orc_extract_gear(self._c, _ptr(np.ascontiguousarray(V, np.uint32)),
                                   _ptr(np.ascontiguousarray(L, np.uint16)), int(goal), _ptr(seg), cap)
        if n == -1:
            return None
        if n < 0:
            raise ValueError(f"extract_gear failed ({n})")
        return [dict(mu=int(r[0]), entry=int(r[1]), exit=int(r[2]), steps=int(r[3]),
                     cost=int(r[4]) | (int(r[5]) << 16), entry_gear=int(r[6])) for r in seg[:n]]

    # ----------------------------------------------------------- Section XII
    def _entry(self, entry) -> np.ndarray:
        e = np.ascontiguousarray(entry, dtype=np.uint32)
        if e.shape != (6,):
            raise ValueError("entry needs one cost per maneuver (cycle-order ids)")
        return e

    def sweep_state(self, B: np.ndarray, start: int, entry, n_cycles: int, mode: int = 0):
        """orc_sweep with the start layer: maneuvers with entry[mu] < ct first
        followed from the start alone, entered at entry[mu]."""
        B = np.ascontiguousarray(B, dtype=np.uint16)
        V = np.zeros(self.nr, np.uint32)
        L = np.zeros(self.nr, np.uint16)
        imp = np.zeros(max(1, 6 * n_cycles), np.int64)
        rc = lib().orc_sweep_state(self._c, _ptr(B), int(start), _ptr(self._entry(entry)), int(n_cycles), int(mode),
                                   _ptr(V), _ptr(L), _ptr(imp))
        if rc != 0:
            raise ValueError(f"oracle sweep_state failed ({rc})")
        return V, L, imp[:6 * n_cycles]

    def seed(self, B: np.ndarray, start: int, entry, V: np.ndarray, L: np.ndarray):
        """The start layer applied to copies of (V, L)."""
        V = np.array(V, dtype=np.uint32, copy=True)
        L = np.array(L, dtype=np.uint16, copy=True)
        if lib().orc_seed(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), _ptr(self._entry(entry)),
                          _ptr(V), _ptr(L)) != 0:
            raise ValueError("seed failed")
        return V, L

    def dijkstra_state(self, B: np.ndarray, start: int, entry) -> np.ndarray:
        V = np.zeros(self.nr, np.uint32)
        if lib().orc_dijkstra_state(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start),
                                    _ptr(self._entry(entry)), _ptr(V)) != 0:
            raise ValueError("dijkstra_state failed")
        return V

    def bruteforce_state(self, B: np.ndarray, start: int, entry, n_cycles: int) -> np.ndarray:
        V = np.zeros(self.nr, np.uint32)
        if lib().orc_bruteforce_state(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start),
                                      _ptr(self._entry(entry)), int(n_cycles), _ptr(V)) != 0:
            raise ValueError("bruteforce_state failed")
        return V

    # ----------------------------------------------------------- Section IX
    def goal_search(self, V: np.ndarray, goals):
        """Best pose of a goal set: goals are (x, y, theta, r_xy, r_theta,
        w_xy, w_theta, bias) tuples.  Returns (cell, score) or None when no
        pose of any box was reached."""
        g = np.ascontiguousarray(np.array(goals, dtype=np.int64).reshape(-1, 8))
        cell = np.zeros(1, np.int64)
        score = np.zeros(1, np.uint64)
        rc = lib().orc_goal_search(self._c, _ptr(np.ascontiguousarray(V, np.uint32)), _ptr(g), len(g), _ptr(cell),
                                   _ptr(score))
        if rc == -1:
            return None
        if rc != 0:
            raise ValueError(f"goal_search failed ({rc})")
        return int(cell[0]), int(score[0])

    # ----------------------------------------------------------- Section X
    def extract(self, V: np.ndarray, L: np.ndarray, goal: int, cap: int = 4096):
        seg = np.zeros((cap, 6), np.int64)
        n = lib().orc_extract(self._c, _ptr(np.ascontiguousarray(V, np.uint32)),
                              _ptr(np.ascontiguousarray(L, np.uint16)), int(goal), _ptr(seg), cap)
        if n == -1:
            return None
        if n < 0:
            raise ValueError(f"extract failed ({n})")
        return [dict(mu=int(r[0]), entry=int(r[1]), exit=int(r[2]), steps=int(r[3]),
                     cost=int(r[4]) | (int(r[5]) << 16)) for r in seg[:n]]


    # ------------------------------------------- Appendix C reachability
    def reach(self, B: np.ndarray, start: int, n_cycles: int) -> np.ndarray:
        """Fewest maneuvers to every pose (255 beyond n_cycles)."""
        count = np.zeros(self.nr, np.uint8)
        if lib().orc_reach(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start), int(n_cycles),
                           _ptr(count)) != 0:
            raise ValueError("reach failed")
        return count

    def reach_extract(self, B: np.ndarray, count: np.ndarray, goal: int, cap: int = 256):
        seg = np.zeros((cap, 4), np.int64)
        n = lib().orc_reach_extract(self._c, _ptr(np.ascontiguousarray(B, np.uint16)),
                                    _ptr(np.ascontiguousarray(count, np.uint8)), int(goal), _ptr(seg), cap)
        if n == -1:
            return None
        if n < 0:
            raise ValueError(f"reach_extract failed ({n})")
        return [dict(mu=int(r[0]), entry=int(r[1]), exit=int(r[2]), steps=int(r[3])) for r in seg[:n]]


class Oracle4:
    """4D generalisation (App. F): 2M+1 curvature levels of an Oracle's 3D
    volume, clothoid maneuvers between them (ids 6 C1F, 7 C1B, 8 C2F, 9 C2B)."""

    C1F, C1B, C2F, C2B = 6, 7, 8, 9

    def __init__(self, base: "Oracle", M: int, L: float, ct_clothoid: int):
        self.base, self.M, self.nk, self.L = base, M, 2 * M + 1, L
        self.nr = base.nr
        self.n4 = base.nr * self.nk
        self._c = lib().orc4_create(base._c, int(M), float(L), int(ct_clothoid))
        if not self._c:
            raise ValueError("bad 4D parameters")

    def __del__(self):
        if getattr(self, "_c", None):
            lib().orc4_destroy(self._c)
            self._c = None

    def cell(self, pose, level: int) -> int:
        """level = kappa in [-M, M]"""
        return (level + self.M) * self.nr + self.base.cell(pose)

    def pose(self, cell4: int):
        return self.base.pose(cell4 % self.nr), cell4 // self.nr - self.M

    def tables(self):
        nt = self.base.nt
        dx = np.zeros((2, self.nk, nt), np.int16)
        dy = np.zeros((2, self.nk, nt), np.int16)
        dth = np.zeros((2, self.nk), np.int32)
        lib().orc4_tables(self._c, _ptr(dx), _ptr(dy), _ptr(dth))
        return dx, dy, dth

    def succ(self, mu: int, cell4: int) -> int:
        return int(lib().orc4_succ(self._c, int(mu), int(cell4)))

    def sweep(self, B: np.ndarray, start4: int, n_cycles: int):
        V = np.zeros(self.n4, np.uint32)
        L = np.zeros(self.n4, np.uint16)
        if lib().orc4_sweep(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start4), int(n_cycles),
                            _ptr(V), _ptr(L)) != 0:
            raise ValueError("4D sweep failed")
        return V, L

    def dijkstra(self, B: np.ndarray, start4: int) -> np.ndarray:
        V = np.zeros(self.n4, np.uint32)
        if lib().orc4_dijkstra(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start4), _ptr(V)) != 0:
            raise ValueError("4D dijkstra failed")
        return V

    def bruteforce(self, B: np.ndarray, start4: int, n_cycles: int) -> np.ndarray:
        V = np.zeros(self.n4, np.uint32)
        if lib().orc4_bruteforce(self._c, _ptr(np.ascontiguousarray(B, np.uint16)), int(start4), int(n_cycles),
                                 _ptr(V)) != 0:
            raise ValueError("4D bruteforce failed")
        return V

    def extract(self, V: np.ndarray, L: np.ndarray, goal4: int, cap: int = 4096):
        seg = np.zeros((cap, 5), np.int64)
        n = lib().orc4_extract(self._c, _ptr(np.ascontiguousarray(V, np.uint32)),
                               _ptr(np.ascontiguousarray(L, np.uint16)), int(goal4), _ptr(seg), cap)
        if n == -1:
            return None
        if n < 0:
            raise ValueError(f"4D extract failed ({n})")
        return [dict(mu=int(r[0]), entry=int(r[1]), exit=int(r[2]), steps=int(r[3]), cost=int(r[4]))
                for r in seg[:n]]


def soft_image(occupancy: np.ndarray, radius: int, soft_max: int) -> np.ndarray:
    """Section VII soft-obstacle image from a binary occupancy map."""
    occ = np.ascontiguousarray(occupancy, dtype=np.uint8)
    nx = occ.shape[0]
    img = np.zeros((nx, nx), np.uint16)
    lib().orc_soft_image(nx, _ptr(occ), int(radius), int(soft_max), _ptr(img))
    return img


# ------------------------------------------------------------ CPU baseline
_cs_lib = None


def cpu_sweep(o: Oracle, B: np.ndarray, start: int, n_cycles: int, threads: int = 0):
    """The kernel-style sweep of Section VIII.B-C on all host cores (OpenMP),
    with the geometry tables and costs of oracle ``o``: V, L, the improved
    cells per layer and the thread count used.  A timed CPU baseline, not
    the oracle; it expects B as rendered (hard walls)."""
    global _cs_lib
    if _cs_lib is None:
        build()
        L_ = C.CDLL(_CS_SO)
        L_.cs_sweep.restype = C.c_int
        L_.cs_sweep.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 5 + [C.c_uint32] + [C.c_void_p] * 3 + \
            [C.c_int64, C.c_int, C.c_int] + [C.c_void_p] * 3
        _cs_lib = L_
    t = o.tables()
    bsh = np.ascontiguousarray(t["bshear"], dtype=np.int32)
    cin = np.asarray(o.cin, dtype=np.uint32)
    cout = np.asarray(o.cout, dtype=np.uint32)
    B = np.ascontiguousarray(B, dtype=np.uint16)
    V = np.empty(o.nr, np.uint32)
    L = np.empty(o.nr, np.uint16)
    imp = np.zeros(max(1, 6 * n_cycles), np.int64)
    used = _cs_lib.cs_sweep(o.nx_log2, o.nt_log2, _ptr(t["beta"]), _ptr(t["iflag"]), _ptr(t["jsign"]), _ptr(bsh),
                            _ptr(t["wS"]), t["wA"], _ptr(cin), _ptr(cout), _ptr(B), int(start), int(n_cycles),
                            int(threads), _ptr(V), _ptr(L), _ptr(imp))
    if used < 0:
        raise ValueError("cpu_sweep: bad input")
    return V, L, imp[:6 * n_cycles], used

"""Seeded synthetic planning inputs.

This module only draws inputs: occupancy maps, vehicle rectangles, turn radii,
start/goal poses and cost parameters.  It holds none of the planner's
arithmetic (no geometry tables, rendering, relaxation or labels), so that the
CUDA path and the CPU oracle can both consume its outputs without sharing any
method code.

The paper's own scenes exist only as stripped figures, so each workload below
is a synthetic stand-in with the sizes and structure the paper describes
(Section XVI: parallel parking, mazes; Tables 5-8 resolutions):

* ``single_query``     64x64x64, point vehicle, R = 12, random rectangles to
                       10 % fill, start/goal uniform over free cells, N = 4.
* ``parallel_parking`` 512x512x512, 96x38 vehicle, R = 110, curb band, two
                       parked 96x38 cars with a 150-cell gap, 2 % clutter,
                       goal in the gap aligned with the curb, N = 8, gear 2000.
* ``maze``             512x512x512 recursive-backtracker maze (9x9 cells at a
                       56-cell pitch: 48 corridor + 8 wall), 30x14 vehicle,
                       R = 24, soft penalty band of 6 cells, N = 32.
* ``batched_queries``  independent queries of mixed sizes
                       {128^2x128, 256^2x128, 256^2x256, 512^2x256}.
* ``served_scenes``    16 persistent scenes (2 at 512^3, the rest of the
                       batched sizes) and ``served_trace`` a Poisson request
                       stream over them (200 plans/s, 10 % at 512^3, N = 8).

Occupancy is uint8 [y][x] (1 = obstacle).  Images are uint16 Q8 reciprocal
velocity: 256 = free, 0xFFFF = hard.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

HARD = 0xFFFF
FREE = 256


@dataclass
class Scene:
    name: str
    nx_log2: int
    nt_log2: int
    turn_radius: float
    footprint: Tuple[int, int, int]  # (front, rear, half_width) in cells
    occupancy: np.ndarray            # uint8 [nx, nx], 1 = obstacle
    start: Tuple[int, int, int]      # (i, j, theta)
    goal: Tuple[int, int, int]
    n_cycles: int
    transition: int                  # cost charged on entering a maneuver
    step_straight: int = 100
    step_scale: int = 100
    soft_radius: int = 0             # 0 = hard obstacles only
    soft_max: int = 0
    half_shift: int = 1
    pose_candidates: List[Tuple[int, int, int]] = field(default_factory=list)

    @property
    def nx(self) -> int:
        return 1 << self.nx_log2

    @property
    def nt(self) -> int:
        return 1 << self.nt_log2

    @property
    def cells(self) -> int:
        return self.nx * self.nx * self.nt

    def hard_image(self) -> np.ndarray:
        """Image with hard obstacles only (256 free, 0xFFFF occupied)."""
        img = np.full(self.occupancy.shape, FREE, dtype=np.uint16)
        img[self.occupancy != 0] = HARD
        return img


def vehicle_rect(length: int, width: int) -> Tuple[int, int, int]:
    """Split an L x W cell vehicle about its rear axle: the axle sits 21 % of
    the length from the back (3.8 m ahead / 1.0 m behind in the paper's
    practical-resolution example), half the width to each side."""
    front = int(np.floor(0.79 * length + 0.5))
    return front, length - front, width // 2


def _place_rects(rng, nx, fill, side_lo, side_hi, keepout=()):
    occ = np.zeros((nx, nx), dtype=np.uint8)
    target = fill * nx * nx
    tries = 0
    while occ.sum() < target and tries < 100000:
        tries += 1
        w = int(rng.integers(side_lo, side_hi + 1))
        h = int(rng.integers(side_lo, side_hi + 1))
        x0 = int(rng.integers(1, nx - w))
        y0 = int(rng.integers(1, nx - h))
        bad = False
        for (cx, cy, rad) in keepout:
            dx = max(x0 - cx, 0, cx - (x0 + w - 1))
            dy = max(y0 - cy, 0, cy - (y0 + h - 1))
            if dx * dx + dy * dy <= rad * rad:
                bad = True
                break
        if bad:
            continue
        occ[y0:y0 + h, x0:x0 + w] = 1
    return occ


def _free_cell_pose(rng, occ, nt, margin=1):
    nx = occ.shape[0]
    while True:
        i = int(rng.integers(margin, nx - margin))
        j = int(rng.integers(margin, nx - margin))
        if occ[j, i] == 0:
            return (i, j, int(rng.integers(0, nt)))


def single_query(seed: int = 0, nx_log2: int = 6, nt_log2: int = 6, n_cycles: int = 4,
                 fill: float = 0.10, turn_radius: float = 12.0, transition: int = 500) -> Scene:
    """Plain single-query sweep: point vehicle, random rectangles (sides 3-10)
    to the given fill, start and goal uniform over free cells."""
    rng = np.random.default_rng(seed)
    nx, nt = 1 << nx_log2, 1 << nt_log2
    side_hi = min(10, max(3, nx // 4))
    occ = _place_rects(rng, nx, fill, 3, side_hi)
    cands = [_free_cell_pose(rng, occ, nt) for _ in range(64)]
    return Scene("single_query", nx_log2, nt_log2, turn_radius, (0, 0, 0), occ,
                 cands[0], cands[1], n_cycles, transition, pose_candidates=cands)


def parallel_parking(seed: int = 1, nx_log2: int = 9, nt_log2: int = 9, n_cycles: int = 8,
                     car: Tuple[int, int] = (96, 38), gap: int = 150, turn_radius: float = 110.0,
                     transition: int = 2000, clutter: float = 0.02) -> Scene:
    """Canonical parallel-parking stand-in (Fig. 2 / 'Parallel Tight').  At
    smaller grids every length scales with Nx/512."""
    rng = np.random.default_rng(seed)
    nx, nt = 1 << nx_log2, 1 << nt_log2
    s = nx / 512.0
    L, W = max(2, int(round(car[0] * s))), max(2, int(round(car[1] * s)))
    gap = max(L + 2, int(round(gap * s)))
    R = max(2.0, turn_radius * s)
    fp = vehicle_rect(L, W)
    occ = np.zeros((nx, nx), dtype=np.uint8)
    curb_y0, curb_h = max(1, int(round(20 * s))), max(1, int(round(8 * s)))
    occ[curb_y0:curb_y0 + curb_h, :] = 1
    lane_y0 = curb_y0 + curb_h + max(1, int(round(2 * s)))
    xa = int(round(60 * s))
    xb = xa + L + gap
    occ[lane_y0:lane_y0 + W, xa:xa + L] = 1
    occ[lane_y0:lane_y0 + W, xb:xb + L] = 1
    # goal: rear axle in the gap, heading along the curb (theta = 0)
    gx = xa + L + (gap - L) // 2 + fp[1]
    gy = lane_y0 + W // 2
    # start: in the driving lane, 120 cells off the curb, 200 cells before the gap
    sx = max(fp[1] + 2, xa + L - int(round(200 * s)))
    sy = curb_y0 + curb_h + int(round(120 * s))
    reach = int(np.ceil(np.hypot(max(fp[0], fp[1]), fp[2]))) + 2
    clut = _place_rects(rng, nx, clutter, max(1, int(round(3 * s))), max(2, int(round(10 * s))),
                        keepout=[(gx, gy, reach + gap // 2), (sx, sy, reach + 10)])
    occ = np.maximum(occ, clut)
    return Scene("parallel_parking", nx_log2, nt_log2, R, fp, occ,
                 (sx, sy, 0), (gx, gy, 0), n_cycles, transition)


def _maze_tree(rng, cells):
    """Recursive-backtracker spanning tree over a cells x cells grid; returns
    the set of opened walls between neighbouring cells."""
    visited = np.zeros((cells, cells), dtype=bool)
    opened = set()
    stack = [(0, 0)]
    visited[0, 0] = True
    while stack:
        cx, cy = stack[-1]
        nbrs = [(cx + dx, cy + dy) for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))
                if 0 <= cx + dx < cells and 0 <= cy + dy < cells and not visited[cy + dy, cx + dx]]
        if not nbrs:
            stack.pop()
            continue
        nx_, ny_ = nbrs[int(rng.integers(0, len(nbrs)))]
        visited[ny_, nx_] = True
        opened.add(((cx, cy), (nx_, ny_)))
        opened.add(((nx_, ny_), (cx, cy)))
        stack.append((nx_, ny_))
    return opened


def maze(seed: int = 2, nx_log2: int = 9, nt_log2: int = 9, n_cycles: int = 32,
         cells: int = 9, corridor: int = 48, wall: int = 8, car: Tuple[int, int] = (30, 14),
         turn_radius: float = 24.0, transition: int = 500, soft_radius: int = 6,
         soft_max: int = 512) -> Scene:
    """Maze stand-in (Fig. 1 / 'Maze 1'): start and goal in opposite corner
    cells, heading along the first corridor.  At smaller grids every length
    scales with Nx/512."""
    rng = np.random.default_rng(seed)
    nx, nt = 1 << nx_log2, 1 << nt_log2
    s = nx / 512.0
    corridor, wall = max(4, int(round(corridor * s))), max(1, int(round(wall * s)))
    car = (max(2, int(round(car[0] * s))), max(2, int(round(car[1] * s))))
    R = max(2.0, turn_radius * s)
    pitch = corridor + wall
    if cells * pitch + wall > nx:
        raise ValueError("maze does not fit the grid")
    occ = np.ones((nx, nx), dtype=np.uint8)
    opened = _maze_tree(rng, cells)
    for cy in range(cells):
        for cx in range(cells):
            x0, y0 = wall + cx * pitch, wall + cy * pitch
            occ[y0:y0 + corridor, x0:x0 + corridor] = 0
            if ((cx, cy), (cx + 1, cy)) in opened:
                occ[y0:y0 + corridor, x0 + corridor:x0 + pitch] = 0
            if ((cx, cy), (cx, cy + 1)) in opened:
                occ[y0 + corridor:y0 + pitch, x0:x0 + corridor] = 0
    fp = vehicle_rect(*car)
    c0 = wall + corridor // 2
    c1 = wall + (cells - 1) * pitch + corridor // 2
    start = (wall + fp[1] + 4, c0, 0)
    goal = (c1 - max(2, corridor // 12), c1, 0)
    return Scene("maze", nx_log2, nt_log2, R, fp, occ, start, goal, n_cycles, transition,
                 soft_radius=soft_radius, soft_max=soft_max)


BATCH_SHAPES = [(7, 7), (8, 7), (8, 8), (9, 8)]  # (nx_log2, nt_log2)


def _uneven_scene(rng, name, lx, lt, sites=2):
    """One scene of the batched / served mixes: random rectangles to 5-20 %
    fill, a vehicle between 8x4 and 96x38 and a turn radius between 10 and 110
    cells (both scaled by Nx / 512, so that the vehicle keeps its share of the
    map on the smaller grids), and `sites` keep-out discs where the vehicle
    fits at any heading (start and goal positions)."""
    nx = 1 << lx
    fill = float(rng.uniform(0.05, 0.20))
    t = float(rng.uniform(0.0, 1.0))
    L = int(round(8 + t * (96 - 8)))
    W = int(round(4 + t * (38 - 4)))
    s = nx / 512.0
    L, W = max(2, int(round(L * s))), max(2, int(round(W * s)))
    fp = vehicle_rect(L, W)
    R = max(2.0, float(rng.integers(10, 111)) * s)
    reach = int(np.ceil(np.hypot(max(fp[0], fp[1]), fp[2]))) + 2
    lo, hi = reach + 1, nx - reach - 1
    pts = [(int(rng.integers(lo, hi)), int(rng.integers(lo, hi))) for _ in range(sites)]
    occ = _place_rects(rng, nx, fill, 3, 10, keepout=[(x, y, reach) for x, y in pts])
    return name, lx, lt, R, fp, occ, pts


def batched_queries(seed: int = 3, count: int = 64, shapes=None, cycles=(4, 8, 16)) -> List[Scene]:
    """Many independent, uneven queries: grid size, fill, vehicle, turn radius
    and cycle count drawn per query (see _uneven_scene)."""
    rng = np.random.default_rng(seed)
    shapes = shapes or BATCH_SHAPES
    out = []
    for q in range(count):
        lx, lt = shapes[int(rng.integers(0, len(shapes)))]
        n = int(cycles[int(rng.integers(0, len(cycles)))])
        name, lx, lt, R, fp, occ, pts = _uneven_scene(rng, f"batch{q}", lx, lt, 2)
        nt = 1 << lt
        (sx, sy), (gx, gy) = pts
        out.append(Scene(name, lx, lt, R, fp, occ, (sx, sy, int(rng.integers(0, nt))),
                         (gx, gy, int(rng.integers(0, nt))), n, 500))
    return out


def served_scenes(seed: int = 4, count: int = 16, big: int = 2, sites: int = 12) -> List[Scene]:
    """Persistent scenes of the served stream: `big` at 512^3, the rest cycling
    through the batched sizes.  Each scene carries `sites` start/goal
    positions in pose_candidates (heading 0; requests draw the heading)."""
    rng = np.random.default_rng(seed)
    shapes = [(9, 9)] * big + [BATCH_SHAPES[k % len(BATCH_SHAPES)] for k in range(count - big)]
    out = []
    for k, (lx, lt) in enumerate(shapes):
        name, lx, lt, R, fp, occ, pts = _uneven_scene(rng, f"served{k}", lx, lt, sites)
        cands = [(x, y, 0) for x, y in pts]
        out.append(Scene(name, lx, lt, R, fp, occ, cands[0], cands[1], 8, 500, pose_candidates=cands))
    return out


def served_trace(scenes_: List[Scene], rate: float = 200.0, seconds: float = 60.0, n_cycles: int = 8,
                 big_share: float = 0.10, seed: int = 5):
    """Poisson arrivals: [(t, scene index, start, goal, N)].  A request is at
    512^3 with probability big_share, otherwise its size is drawn uniformly
    from the batched sizes; the scene is then drawn uniformly among the scenes
    of that size, and start and goal from two different sites of the scene
    with uniform headings."""
    rng = np.random.default_rng(seed)
    big = [i for i, sc in enumerate(scenes_) if (sc.nx_log2, sc.nt_log2) == (9, 9)]
    by_shape = {}
    for i, sc in enumerate(scenes_):
        if (sc.nx_log2, sc.nt_log2) != (9, 9):
            by_shape.setdefault((sc.nx_log2, sc.nt_log2), []).append(i)
    shapes = sorted(by_shape)
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= seconds:
            break
        if big and rng.random() < big_share:
            k = big[int(rng.integers(0, len(big)))]
        else:
            grp = by_shape[shapes[int(rng.integers(0, len(shapes)))]]
            k = grp[int(rng.integers(0, len(grp)))]
        sc = scenes_[k]
        a, b = rng.choice(len(sc.pose_candidates), size=2, replace=False)
        s = sc.pose_candidates[int(a)][:2] + (int(rng.integers(0, sc.nt)),)
        g = sc.pose_candidates[int(b)][:2] + (int(rng.integers(0, sc.nt)),)
        out.append((t, k, s, g, n_cycles))
    return out


def tiny(seed: int, nx_log2: int = 3, nt_log2: int = 3, fill: float = 0.1, turn_radius: float = 2.0,
         footprint=(0, 0, 0), transition: int = 300, n_cycles: int = 1, soft: bool = False,
         half_shift: int = 1):
    """Small scene for exhaustive checks; returns (scene, image).  With
    soft=True the free cells get random values in [256, 1024)."""
    rng = np.random.default_rng(seed)
    nx, nt = 1 << nx_log2, 1 << nt_log2
    occ = np.zeros((nx, nx), dtype=np.uint8)
    k = int(round(fill * nx * nx))
    if k:
        idx = rng.choice(nx * nx, size=k, replace=False)
        occ.flat[idx] = 1
    img = np.full((nx, nx), FREE, dtype=np.uint16)
    if soft:
        img = rng.integers(256, 1024, size=(nx, nx)).astype(np.uint16)
    img[occ != 0] = HARD
    cands = [_free_cell_pose(rng, occ, nt) for _ in range(64)]
    sc = Scene("tiny", nx_log2, nt_log2, turn_radius, tuple(footprint), occ, cands[0], cands[1],
               n_cycles, transition, half_shift=half_shift, pose_candidates=cands)
    return sc, img

"""Pins for the CPU oracle: checks against things other than the oracle itself.

* hand-worked geometry tables (Section V.C, eqs. 11-24) in tests/golden;
* structural facts the paper states: every maneuver map is a bijection and
  its forward/backward versions are exact inverses (Section V.C-D); following
  the edges of eqs. 25-31 traces the chains of eqs. 18 and 23;
* closed forms in free space: a straight run of k steps, a 45-degree run, a
  quarter turn (exact endpoint and cost);
* brute-force enumeration of every layer-ordered segment sequence on tiny
  grids equals the layered relaxation (Section VIII.B);
* the O(n) two-loop scan equals the O(n^2) definition, values and labels;
* Dijkstra on the explicit Star graph (Section VIII.A) equals the sweep once
  it has converged, and more cycles never raise a value;
* time-reversal/gear symmetry in free space, mirror symmetry without the
  half-cell shift;
* obstacle rendering against an independent maximum filter (scipy) and the
  exact axis-aligned footprint rectangles;
* the soft-obstacle image against scipy's Euclidean distance transform and a
  hand-worked fixture;
* extracted plans: segment costs re-summed from the obstacle volume equal the
  goal value at convergence.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_2306_01301_b300 import scenes
from tests.util import read_golden

INF = O.INF


def free_image(nx):
    return np.full((nx, nx), 256, np.uint16)


# ------------------------------------------------------------------ tables
@pytest.mark.parametrize("fixture,lx,lt,R", [("tables_R2_N8.txt", 3, 3, 2.0),
                                             ("tables_R2p5_N16.txt", 4, 4, 2.5)])
def test_tables_match_hand_worked_values(fixture, lx, lt, R):
    g, _ = read_golden(fixture)
    t = O.Oracle(lx, lt, R, half_shift=1).tables()
    assert t["beta"].tolist() == g["beta_half"]
    assert t["psi2"].tolist() == g["psi2_half"]
    assert t["iflag"].tolist() == g["iflag"]
    assert t["jsign"].tolist() == g["jsign"]
    assert t["wS"].tolist() == g["wS"]
    assert t["wA"] == g["wA"][0]
    for T in (1, 2, 3):
        assert t["bshear"][T].tolist() == g[f"bshear{T}"]
    if "beta_round" in g:
        t0 = O.Oracle(lx, lt, R, half_shift=0).tables()
        assert t0["beta"].tolist() == g["beta_round"]
        assert t0["psi2"].tolist() == [0] * (1 << lt)


# ------------------------------------------------------------ edge maps
@pytest.mark.parametrize("lx,lt,R,half", [(3, 3, 2.0, 1), (4, 4, 2.5, 1), (4, 5, 7.0, 0), (5, 4, 3.0, 1)])
def test_maneuver_maps_are_bijective_and_reversible(lx, lt, R, half):
    o = O.Oracle(lx, lt, R, half_shift=half)
    cells = np.arange(o.nr)
    succ = {mu: np.array([o.succ(mu, c) for c in cells]) for mu in range(6)}
    for mu in range(6):
        assert np.array_equal(np.sort(succ[mu]), cells), f"maneuver {mu} is not a bijection"
    # LF<->LB, SF<->SB, RB<->RF are exact inverses (mu <-> 5 - mu)
    for mu in range(6):
        assert np.array_equal(succ[5 - mu][succ[mu]], cells)
    # turns change the heading by exactly +/-1; straights keep it
    T = cells >> (2 * lx)
    for mu, dT in ((O.LF, 1), (O.RB, 1), (O.RF, -1), (O.LB, -1), (O.SF, 0), (O.SB, 0)):
        assert np.array_equal(succ[mu] >> (2 * lx), (T + dT) % o.nt)


@pytest.mark.parametrize("half", [0, 1])
def test_edges_trace_the_chains_of_eq18_and_eq23(half):
    lx, lt, R = 4, 5, 5.0
    o = O.Oracle(lx, lt, R, half_shift=half)
    t = o.tables()
    nx, nt, M = o.nx, o.nt, o.nx - 1
    beta = t["beta"]

    def bq(q, T):
        return int(beta[(T + q * nt // 4) % nt])

    rng = np.random.default_rng(0)
    for _ in range(200):
        xq, yq, T = int(rng.integers(nx)), int(rng.integers(nx)), int(rng.integers(nt))
        # eq. 18, LEFT (beta_0, beta_3) and RIGHT (beta_2, beta_1)
        left = lambda T_: o.cell(((xq + bq(0, T_)) & M, (yq + bq(3, T_)) & M, T_ % nt))
        right = lambda T_: o.cell(((xq + bq(2, T_)) & M, (yq + bq(1, T_)) & M, T_ % nt))
        assert o.succ(O.LF, left(T)) == left(T + 1)
        assert o.succ(O.LB, left(T)) == left(T - 1 + nt)
        assert o.succ(O.RB, right(T)) == right(T + 1)
        assert o.succ(O.RF, right(T)) == right(T - 1 + nt)
        # eq. 23 straight line (x', T), position y'
        Bs = t["bshear"][T]
        y = int(rng.integers(nx))

        def line(y_):
            y_ &= M
            c = (xq + int(Bs[y_])) & M
            return o.cell((y_, c, T) if t["iflag"][T] == 0 else (c, y_, T))

        fwd = int(t["jsign"][T])
        assert o.succ(O.SF, line(y)) == line(y + fwd)
        assert o.succ(O.SB, line(y)) == line(y - fwd)


# ------------------------------------------------------------ closed forms
def test_free_space_closed_forms():
    """Single-maneuver plans in uniform free space with a large transition
    cost (so no multi-maneuver path can compete): exact integer costs."""
    lx, lt, R, ct = 5, 6, 6.0, 100000
    o = O.Oracle(lx, lt, R, half_shift=1, transition=ct)
    B = o.render(free_image(o.nx), (0, 0, 0))
    t = o.tables()
    wA = t["wA"]
    assert wA == round(100 * 2 * np.pi * R / o.nt)
    i0, j0 = 10, 9
    # heading 0: straight ahead k steps along +x, weight 100 per step
    V, _, _ = o.sweep(B, o.cell((i0, j0, 0)), 1)
    for k in range(1, 15):
        assert V[o.cell((i0 + k, j0, 0))] == ct + 100 * k
    # 45 degrees: diagonal, weight round(100*sqrt(2)) = 141
    T45 = o.nt // 8
    V, _, _ = o.sweep(B, o.cell((i0, j0, T45)), 1)
    for k in range(1, 12):
        assert V[o.cell((i0 + k, j0 + k, T45))] == ct + 141 * k
    # 90 degrees: along +y
    T90 = o.nt // 4
    V, _, _ = o.sweep(B, o.cell((i0, j0, T90)), 1)
    for k in range(1, 15):
        assert V[o.cell((i0, j0 + k, T90))] == ct + 100 * k
    # quarter left-forward turn from heading 0 ends at (i0+R, j0+R, 90 deg)
    # (eq. 1 with q = +1: x0 + R sin, y0 + R(1 - cos)); N_theta/4 edges
    V, L, _ = o.sweep(B, o.cell((i0, j0, 0)), 1)
    end = o.cell((i0 + int(R), j0 + int(R), T90))
    assert V[end] == ct + (o.nt // 4) * wA
    assert L[end] == (O.LF << 13) | (o.nt // 4)
    # quarter right-backward turn from heading 0 ends at (i0-R, j0-R, 90 deg)
    end_rb = o.cell((i0 - int(R), j0 - int(R), T90))
    assert V[end_rb] == ct + (o.nt // 4) * wA
    assert L[end_rb] == (O.RB << 13) | (o.nt // 4)
    # the start never improves (a full loop costs ct + N_theta*wA > 0)
    assert V[o.cell((i0, j0, 0))] == 0


# ------------------------------------------------------ brute force / modes
TINY_CASES = [
    dict(seed=0, lx=3, lt=3, R=2.0, fp=(0, 0, 0), soft=False, half=1, N=1),
    dict(seed=1, lx=3, lt=3, R=2.0, fp=(0, 0, 0), soft=True, half=1, N=1),
    dict(seed=2, lx=3, lt=4, R=2.5, fp=(1, 0, 0), soft=True, half=0, N=1),
    dict(seed=3, lx=4, lt=3, R=3.0, fp=(0, 0, 0), soft=True, half=1, N=1),
    dict(seed=4, lx=3, lt=3, R=1.5, fp=(0, 0, 0), soft=True, half=1, N=2),
]


@pytest.mark.parametrize("case", TINY_CASES)
def test_sweep_equals_bruteforce_enumeration(case):
    sc, img = scenes.tiny(case["seed"], case["lx"], case["lt"], fill=0.1, turn_radius=case["R"],
                          footprint=case["fp"], soft=case["soft"], half_shift=case["half"])
    o = O.Oracle(case["lx"], case["lt"], case["R"], half_shift=case["half"], transition=sc.transition)
    B = o.render(img, case["fp"])
    starts = [c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD][:2]
    for st in starts:
        s = o.cell(st)
        bf = o.bruteforce(B, s, case["N"])
        for mode in (0, 1, 2):
            V, _, _ = o.sweep(B, s, case["N"], mode)
            assert np.array_equal(V, bf), f"mode {mode}"


@pytest.mark.parametrize("seed,lx,lt,soft", [(0, 4, 4, False), (1, 4, 4, True), (2, 5, 4, True), (3, 4, 5, False)])
def test_scan_equals_definition_values_and_labels(seed, lx, lt, soft):
    sc, img = scenes.tiny(seed, lx, lt, fill=0.12, turn_radius=3.0, soft=soft)
    o = O.Oracle(lx, lt, 3.0, transition=sc.transition)
    B = o.render(img, (0, 0, 0))
    s = o.cell(sc.start)
    V2, L2, I2 = o.sweep(B, s, 3, mode=2)
    for mode in (0, 1):
        V, L, I = o.sweep(B, s, 3, mode=mode)
        assert np.array_equal(V, V2) and np.array_equal(L, L2) and np.array_equal(I, I2)


@pytest.mark.parametrize("seed,soft,fp", [(0, False, (0, 0, 0)), (1, True, (0, 0, 0)), (2, True, (1, 1, 0))])
def test_converges_to_dijkstra_and_never_increases(seed, soft, fp):
    sc, img = scenes.tiny(seed, 4, 4, fill=0.1, turn_radius=2.5, footprint=fp, soft=soft)
    o = O.Oracle(4, 4, 2.5, transition=sc.transition)
    B = o.render(img, fp)
    s = o.cell(next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD))
    Vd = o.dijkstra(B, s)
    prev = None
    for n in range(1, 31):
        V, _, _ = o.sweep(B, s, n, mode=1)
        assert np.all(V >= Vd)  # never below the true shortest path
        if prev is not None:
            assert np.all(V <= prev)
        prev = V
        if np.array_equal(V, Vd):
            break
    assert np.array_equal(prev, Vd), "did not converge to Dijkstra within 30 cycles"


# ------------------------------------------------------------ symmetries
def test_time_reversal_gear_symmetry_in_free_space():
    """Reversing a path swaps its endpoints and flips every gear; the cycle
    order LF,SF,RB,RF,SB,LB reversed and gear-flipped is itself, and in
    uniform free space each segment costs the same both ways."""
    lx, lt, R = 4, 4, 3.0
    o = O.Oracle(lx, lt, R, transition=700)
    B = o.render(free_image(o.nx), (0, 0, 0))
    rng = np.random.default_rng(5)
    poses = [(int(rng.integers(1, o.nx)), int(rng.integers(1, o.nx)), int(rng.integers(o.nt))) for _ in range(8)]
    for N in (1, 2):
        Vs = {p: o.sweep(B, o.cell(p), N, mode=1)[0] for p in poses}
        for a in poses:
            for b in poses:
                assert Vs[a][o.cell(b)] == Vs[b][o.cell(a)]


def test_mirror_symmetry_without_half_shift():
    """Mirroring y -> -y, theta -> -theta turns left curves into right curves
    and keeps the obstacle rendering (a symmetric rectangle) mirrored.  The
    straight lines' shear B(y', T) is anchored at the wall y' = 0 (eq. 23),
    so a straight line is mirror-symmetric only about the axis parallel to
    it: the y-mirror for |tan| <= 1 headings and the x-mirror
    (x -> -x, theta -> pi - theta) for the others.  Without the half-cell
    shift all of these hold exactly."""
    lx, lt, R = 4, 4, 3.0
    o = O.Oracle(lx, lt, R, half_shift=0, transition=400)
    nx, nt = o.nx, o.nt
    t = o.tables()

    def ymir(c):
        i, j, T = o.pose(c)
        return o.cell((i, (-j) % nx, (-T) % nt))

    def xmir(c):
        i, j, T = o.pose(c)
        return o.cell(((-i) % nx, j, (nt // 2 - T) % nt))

    turn_pairs = {O.LF: O.RF, O.LB: O.RB, O.RF: O.LF, O.RB: O.LB}
    for c in range(o.nr):
        for mu, nu in turn_pairs.items():
            assert ymir(o.succ(mu, c)) == o.succ(nu, ymir(c))
        T = c >> (2 * lx)
        mirror = ymir if t["iflag"][T] == 0 else xmir
        for mu in (O.SF, O.SB):
            assert mirror(o.succ(mu, c)) == o.succ(mu, mirror(c))
    sc, img = scenes.tiny(7, lx, lt, fill=0.08, soft=True)
    mimg = img[(-np.arange(nx)) % nx, :]
    fp = (2, 1, 1)
    B = o.render(img, fp).reshape(nt, nx, nx)
    Bm = o.render(mimg, fp).reshape(nt, nx, nx)
    T = np.arange(nt)
    assert np.array_equal(Bm, B[(-T) % nt][:, (-np.arange(nx)) % nx, :])


# ------------------------------------------------------------ rendering
def test_footprint_axis_aligned_headings():
    o = O.Oracle(6, 6, 10.0, half_shift=1)
    f, r, hw = 7, 2, 3
    for T, (xr, yr) in {0: ((-r, f), (-hw, hw)),
                        o.nt // 4: ((-hw, hw), (-r, f)),
                        o.nt // 2: ((-f, r), (-hw, hw)),
                        3 * o.nt // 4: ((-hw, hw), (-f, r))}.items():
        dx, dy = o.footprint(f, r, hw, T)
        got = set(zip(dx.tolist(), dy.tolist()))
        want = {(x, y) for x in range(xr[0], xr[1] + 1) for y in range(yr[0], yr[1] + 1)}
        assert got == want, f"heading {T}"
    dx, dy = o.footprint(0, 0, 0, 5)
    assert list(zip(dx, dy)) == [(0, 0)]


def test_render_against_maximum_filter():
    sc, img = scenes.tiny(11, 5, 3, fill=0.05, soft=True)
    o = O.Oracle(5, 3, 3.0)
    nx = o.nx
    walled = img.copy()
    walled[0, :] = O.HARD
    walled[:, 0] = O.HARD
    # point vehicle: B is the walled image in every heading
    B = o.render(img, (0, 0, 0)).reshape(o.nt, nx, nx)
    for T in range(o.nt):
        assert np.array_equal(B[T], walled)
    # rectangle at heading 0: maximum over [-r, f] x [-hw, hw], wrapping
    f, r, hw = 3, 1, 2
    B = o.render(img, (f, r, hw)).reshape(o.nt, nx, nx)
    fpm = np.ones((2 * hw + 1, f + r + 1), bool)
    ref = ndimage.maximum_filter(walled, footprint=fpm, mode="wrap", origin=(0, (r - f) // 2))
    # maximum_filter's origin convention: build the expectation explicitly
    exp = np.zeros_like(walled)
    for y in range(nx):
        for x in range(nx):
            rows = [(y + d) % nx for d in range(-hw, hw + 1)]
            cols = [(x + d) % nx for d in range(-r, f + 1)]
            exp[y, x] = walled[np.ix_(rows, cols)].max()
    assert np.array_equal(B[0], exp)
    # and the library filter agrees on the symmetric part of the window
    sym = ndimage.maximum_filter(walled, size=(2 * hw + 1, 2 * max(f, r) + 1), mode="wrap")
    assert np.all(sym >= exp)
    del ref


@pytest.mark.parametrize("lx,lt,fp,half", [(5, 4, (5, 2, 2), 1), (4, 5, (9, 3, 4), 0), (3, 3, (6, 2, 3), 1),
                                           (6, 4, (0, 0, 0), 1)])
def test_row_run_render_equals_definition(lx, lt, fp, half):
    sc, img = scenes.tiny(13 + lx, lx, lt, fill=0.1, soft=True)
    o = O.Oracle(lx, lt, 4.0, half_shift=half)
    assert np.array_equal(o.render_rows(img, fp), o.render(img, fp))


def test_render_cells_matches_full_render():
    sc, img = scenes.tiny(12, 5, 4, fill=0.1, soft=True)
    o = O.Oracle(5, 4, 4.0)
    fp = (5, 2, 2)
    B = o.render(img, fp)
    cells = np.random.default_rng(0).integers(0, o.nr, 500)
    assert np.array_equal(o.render_cells(img, fp, cells), B[cells])


# ------------------------------------------------------------ soft image
def test_soft_image_fixture_and_distance_transform():
    _, rows = read_golden("soft_8x8_r3.txt")
    occ = np.zeros((8, 8), np.uint8)
    occ[3, 3] = 1
    assert O.soft_image(occ, 3, 90).tolist() == rows
    rng = np.random.default_rng(3)
    occ = (rng.random((48, 48)) < 0.03).astype(np.uint8)
    img = O.soft_image(occ, 6, 512)
    d2 = np.rint(ndimage.distance_transform_edt(occ == 0) ** 2).astype(int)
    pen = np.where(d2 < 36, 512 * (36 - d2) // 36, 0)
    exp = np.where(occ != 0, O.HARD, 256 + pen)
    assert np.array_equal(img.astype(int), exp)


# ------------------------------------------------------------ extraction
def test_extracted_plan_costs_resum_at_convergence():
    sc, img = scenes.tiny(21, 4, 4, fill=0.08, soft=True, transition=250)
    o = O.Oracle(4, 4, 2.5, transition=250)
    B = o.render(img, (0, 0, 0))
    s = o.cell(sc.start)
    Vd = o.dijkstra(B, s)
    for n in range(1, 40):
        V, L, _ = o.sweep(B, s, n, mode=1)
        if np.array_equal(V, Vd):
            break
    V2, L2, _ = o.sweep(B, s, n + 1, mode=1)
    assert np.array_equal(V2, V)
    reached = np.flatnonzero((V2 != INF) & (np.arange(o.nr) != s))
    for g in np.random.default_rng(1).choice(reached, size=min(40, len(reached)), replace=False):
        segs = o.extract(V2, L2, int(g))
        assert segs[0]["entry"] == s and segs[-1]["exit"] == g
        total = 0
        for k, sg in enumerate(segs):
            if k:
                assert sg["entry"] == segs[k - 1]["exit"]
            c = sg["entry"]
            total += o.ct
            for _ in range(sg["steps"]):
                total += o.edge(B, sg["mu"], c)
                c = o.succ(sg["mu"], c)
            assert c == sg["exit"]
            assert total == sg["cost"] == V2[sg["exit"]]
        assert total == V2[g]
    # unreachable goal
    hard = np.flatnonzero(B == O.HARD)
    assert o.extract(V2, L2, int(hard[0])) is None


def test_lockstep_threads_give_the_same_volumes():
    """The lockstep mode may spread the independent chains of a layer over
    host threads; values, labels and per-layer counts do not change."""
    sc, img = scenes.tiny(1234, 6, 6, fill=0.06, turn_radius=5.0, footprint=(2, 1, 1), soft=True, transition=400)
    o = O.Oracle(6, 6, 5.0, transition=sc.transition)
    B = o.render(img, sc.footprint)
    start = next(c for c in sc.pose_candidates if B[o.cell(c)] != O.HARD)
    try:
        O.Oracle.set_threads(1)
        V1, L1, i1 = o.sweep(B, o.cell(start), 2, mode=1)
        O.Oracle.set_threads(8)
        V8, L8, i8 = o.sweep(B, o.cell(start), 2, mode=1)
    finally:
        O.Oracle.set_threads(1)
    assert (V1 != O.INF).sum() > 1000
    assert np.array_equal(V1, V8) and np.array_equal(L1, L8) and np.array_equal(i1, i8)

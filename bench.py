"""Benchmark: the 512^3 parallel-parking plan (N = 8 maneuver cycles).

One step = one whole plan through the hot path: c-space obstacle rendering,
4N + 1 fused maneuver sweeps (6N maneuver layers) and goal lookup + label
walk.  Metric: pose-cell updates per second, one update being one pose cell
processed by one maneuver layer (6 * N * Nx^2 * N_theta per plan); plans/s is
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run, one rank per GPU; the planner does
not shard, so every rank plans its own replica (weak scaling) and no
collective touches the data path.  --impl reference times the CPU oracle
(the repository's own plain restatement of the method) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pose-cell updates/s"
WORKLOAD = "parallel_parking_512x512x512_N8"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def source_hash():
    """Hash of what the turn kernel is built from: the turn section of
    sweep.cu (kernel and launcher), the scan it runs (turn_scan.cuh) and the
    structures it reads."""
    csrc = os.path.join(ROOT, "paper_2306_01301_b300", "csrc")
    with open(os.path.join(csrc, "sweep.cu")) as f:
        sweep = f.read()
    with open(os.path.join(csrc, "turn_scan.cuh")) as f:
        scan = f.read()
    with open(os.path.join(csrc, "internal.h")) as f:
        internal = f.read()
    a = sweep.index("// ------------------------------------------------------------------- turns")
    b = sweep.index("// ---------------------------------------------------------------- straights", a)
    h = hashlib.sha256()
    h.update(sweep[a:b].encode())
    h.update(scan.encode())
    for name in ("PlaneInfo", "DevGrid", "Volumes", "QueryDesc"):
        i = internal.index("struct " + name + " {")
        h.update(internal[i:internal.index("\n};", i) + 3].encode())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per turn-kernel launch from the committed ncu summary, or
    None when the kernel source changed since it was captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if t.get("source_hash") == source_hash():
            return t.get("turn_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (read-only query)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    from paper_2306_01301_b300 import replicas
    return replicas.rank_env()


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(sc, img):
    """The oracle, as it stands, on a bounded sample: one maneuver cycle (6
    layers) of the same 512^3 workload on one host core.  Beside it, the
    kernel-style sweep on all host cores (OpenMP, oracle/cpu_sweep.c; not the
    oracle, checked against it in the tests), the counterpart of the paper's
    CPU kernel rows, over the whole N-cycle sweep of the workload."""
    import oracle as O
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    B = o.render_rows(img, sc.footprint)
    t0 = time.perf_counter()
    o.sweep(B, o.cell(sc.start), 1, mode=1)
    dt = time.perf_counter() - t0
    oracle_line = {"value": 6 * sc.cells / dt, "unit": METRIC, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                   "sample": f"1 maneuver cycle (6 layers) of {WORKLOAD}, single-threaded C oracle, "
                             f"{dt:.1f} s; host has {os.cpu_count()} cores"}
    t0 = time.perf_counter()
    _, _, _, threads = O.cpu_sweep(o, B, o.cell(sc.start), sc.n_cycles)
    dk = time.perf_counter() - t0
    kernel_line = {"value": 6 * sc.n_cycles * sc.cells / dk, "unit": METRIC, "threads": threads, "cpu": cpu_model(),
                   "plans_per_s": 1.0 / dk, "kind": "kernel-style sweep on all host cores (OpenMP), not the oracle",
                   "sample": f"the whole {sc.n_cycles}-cycle sweep of {WORKLOAD} (B rendered beforehand), "
                             f"{dk:.2f} s; host has {os.cpu_count()} cores"}
    return oracle_line, kernel_line


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O
    from paper_2306_01301_b300 import scenes
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    o = O.Oracle(sc.nx_log2, sc.nt_log2, sc.turn_radius, transition=sc.transition)
    B = o.render_rows(img, sc.footprint)
    V, L, _ = o.sweep(B, o.cell(sc.start), 0, mode=1)
    # each step: one maneuver layer of the oracle (a bounded sample of a plan)
    for k in range(args.warmup):
        V, L, _ = o.layers(B, V, L, k, 1, mode=1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        V, L, _ = o.layers(B, V, L, args.warmup + k, 1, mode=1)
    dt = time.perf_counter() - t0
    value = args.steps * sc.cells / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "step": "one maneuver layer", "threads": 1},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} maneuver layers of {WORKLOAD}"},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2306_01301_b300 import binding, scenes
    sc = scenes.parallel_parking()
    img = sc.hard_image()
    N = sc.n_cycles
    updates = 6 * N * sc.cells
    stream = torch.cuda.current_stream()
    p = binding.Planner.from_scene(sc, img, stream=stream)
    p.render()
    if args.shapes:
        # pinned kernel shapes (profiling runs: timing-based tuning under a profiler picks differently)
        tv, tg, sl, sg = (int(x) for x in args.shapes.split(","))
        p.set_kernel_shapes(tv, tg, sl, sg)
        tuning = [{"kernel": "turn", "shape": tv, "grid": tg, "ms": 0.0, "pinned": True},
                  {"kernel": "straight", "shape": sl, "grid": sg, "ms": 0.0, "pinned": True}]
    else:
        tuning = p.autotune(sc.start)  # kernel shapes for this plan, outside the timed region

    def step():
        p.render()
        p.sweep(sc.start, N)
        return p.extract(sc.goal)

    res = None
    for _ in range(max(3, args.warmup)):
        res = step()
    torch.cuda.synchronize()

    from paper_2306_01301_b300 import replicas

    def barrier():
        replicas.barrier(world)

    # improved-cell counts of one plan (untimed: counting adds work to the
    # sweep kernels, and a plan's counts depend only on its inputs)
    p.profile(True, counts=True)
    step()
    counted = p.profile_read()
    p.profile(False)

    # ---- device-resident timing (image already in HBM); per-pass events only
    clocks = ClockSampler(dev)
    p.profile(True, counts=False)
    l0 = p.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = p.kernel_launches() - l0
    prof = p.profile_read()
    p.profile(False)
    clk = clocks.stop()
    # every rank plans its own replica: units of all ranks over the slowest rank's time
    value, _, sec = replicas.job_rate(updates * args.steps, ms / 1e3, world, device="cuda")

    # ---- end to end through the C ABI: host image in, host plan out
    pinned = torch.from_numpy(img).pin_memory()
    host_img = pinned.numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nseg = 0
    for _ in range(args.steps):
        p.set_image(host_img)
        r = step()
        nseg = len(r.segments) if r else 0
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s, world, device="cuda")
    h2d = img.nbytes
    d2h = 8 + 36 * nseg

    peak, peak_kind = load_peaks()
    turn_launch_ms = prof["turn_ms"] / max(1, prof["turn_passes"])
    turn_bytes = sc.cells * 6 + 6 * counted["turn_improved"] / max(1, counted["turn_passes"])
    achieved = turn_bytes / (turn_launch_ms / 1e3) / 1e9
    straight_launch_ms = prof["straight_ms"] / max(1, prof["straight_passes"])
    straight_bytes = sc.cells * 6 + 6 * counted["straight_improved"] / max(1, counted["straight_passes"])
    render_ms = prof["render_ms"] / max(1, prof["render_passes"])
    render_gbs = sc.cells * 2 / (render_ms / 1e3) / 1e9  # writes B; the image and bit tables come from L2
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "512x512x512", "n_cycles": N, "vehicle_cells": "96x38",
                   "turn_radius_cells": sc.turn_radius, "gear_cost": sc.transition,
                   "parallelism": f"replicas{world}", "l2": "inputs_larger_than_L2 (V+L+B = 1 GiB)"},
        "plans_per_s": args.steps * world / sec,
        "plan_cost": res.cost if res else None, "plan_maneuvers": len(res.segments) if res else 0,
        "gpu_launches": launches,
        "autotuned": {k: min((e for e in tuning if e["kernel"] == k), key=lambda e: e["ms"])
                      for k in ("turn", "straight")},
        "roofline": {"bound": "hbm", "kernel": "k_turn (fused turn-pair sweep)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(), "bytes_per_launch": turn_bytes, "launch_ms": turn_launch_ms},
        "kernels": {"turn_ms_per_launch": turn_launch_ms, "straight_ms_per_launch": straight_launch_ms,
                    "straight_GBps": straight_bytes / (straight_launch_ms / 1e3) / 1e9,
                    "straight_frac": straight_bytes / (straight_launch_ms / 1e3) / 1e9 / peak,
                    "render_ms_per_step": render_ms,
                    "render": {"bound": "alu", "GBps": render_gbs, "frac_of_hbm": render_gbs / peak,
                               "note": "2 B of B written per pose; per 32 poses one OR of two sparse-table windows "
                                       "per footprint row run (96x38 vehicle: about 40 to 100 runs per heading), "
                                       "so the footprint test, not HBM, bounds it"},
                    "init_ms_per_step": prof["init_ms"] / max(1, prof["init_passes"]),
                    "turn_tiles_improved_share": counted["turn_tiles_improved"] / max(1, counted["turn_passes"])
                    / ((sc.nx * sc.nx + 31) // 32)},
        "e2e": {"value": updates * args.steps * world / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "plans_per_s": args.steps * world / e2e_s},
        "clocks": clk,
    }
    p.close()
    if world == 1 and not args.no_single:
        line["single_query_64"] = run_single_query(args, torch)
    if world == 1 and not args.no_maze:
        line["maze"] = run_maze(args, torch)
    if world == 1 and not args.no_reach:
        line["reach_bitvector"] = run_reach(args, torch)
    if world == 1 and not args.no_extensions:
        line["extensions"] = run_extensions(args, torch)
    if world == 1 and not args.no_batched:
        line["batched"] = run_batched(args, torch)
    if world == 1 and not args.no_served:
        line["served"] = run_served(args, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["cpu_kernel_baseline"] = cpu_baseline(sc, img)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_maze(args, torch):
    """The 512^3 maze (soft obstacle costs, N = 32): whole plans timed with
    CUDA events, render included, after autotuning the kernel shapes."""
    from paper_2306_01301_b300 import binding, scenes
    sc = scenes.maze()
    stream = torch.cuda.current_stream()
    p = binding.Planner.from_scene(sc, stream=stream)
    p.render()
    p.autotune(sc.start)
    for _ in range(max(3, args.warmup)):
        p.plan(sc.start, sc.goal, sc.n_cycles)
    steps = max(3, args.maze_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        p.render()
        p.sweep(sc.start, sc.n_cycles)
        res = p.extract(sc.goal)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    p.close()
    updates = 6 * sc.n_cycles * sc.cells
    return {"workload": "maze_512x512x512_N32_soft", "ms_per_plan": ms, "plans_per_s": 1e3 / ms,
            "updates_per_s": updates / (ms / 1e3), "plan_cost": res.cost if res else None,
            "plan_maneuvers": len(res.segments) if res else 0, "steps": steps}


def run_single_query(args, torch):
    """The plain single-query sweep (64^3, point vehicle, N = 4): whole plans
    (render, init, 17 passes, label walk) through the plain calls, timed on
    the device with CUDA events and end to end (image copied from pinned host
    memory every plan, the plan read back); and the same plan as a batch of
    one replayed through a captured CUDA graph.  The volumes (7 MB) sit in
    L2, so this size is launch-bound: plans/s, not a roofline figure."""
    import numpy as np
    from paper_2306_01301_b300 import binding, scenes
    sc = scenes.single_query()
    img = sc.hard_image()
    stream = torch.cuda.current_stream()
    p = binding.Planner.from_scene(sc, img, stream=stream)
    p.render()
    p.autotune(sc.start)
    N = sc.n_cycles
    steps = 200
    for _ in range(20):
        p.plan(sc.start, sc.goal, N)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        p.render()
        p.sweep(sc.start, N)
        res = p.extract(sc.goal)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pinned = torch.from_numpy(img).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        p.set_image(pinned)
        p.render()
        p.sweep(sc.start, N)
        res2 = p.extract(sc.goal)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / steps
    launches_plain = p.kernel_launches()
    b = binding.Batch([p], stream=stream)
    q = [(sc.start, sc.goal, N)]
    b.run(q, render=True)
    b.sync()
    for _ in range(20):
        b.run(q, render=True)
        b.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.run(q, render=True)
        b.sync()
        res3 = b.result(0)
    graph_ms = 1e3 * (time.perf_counter() - t0) / steps
    per_run, _ = b.kernel_launches()
    b.close()
    p.close()
    same = all(r is not None and r.cost == res.cost and r.segments == res.segments for r in (res2, res3))
    updates = 6 * N * sc.cells
    return {"workload": "single_query_64x64x64_N4", "ms_per_plan": ms, "plans_per_s": 1e3 / ms,
            "updates_per_s": updates / (ms / 1e3),
            "e2e": {"ms_per_plan": e2e_ms, "plans_per_s": 1e3 / e2e_ms, "h2d_bytes_per_plan": img.nbytes},
            "graph_replay": {"ms_per_plan": graph_ms, "plans_per_s": 1e3 / graph_ms, "gpu_launches": per_run,
                             "timing": "host wall clock, result read back every plan"},
            "graph_speedup_over_plain_e2e": e2e_ms / graph_ms, "same_plan_all_ways": same,
            "plan_cost": res.cost if res else None, "steps": steps,
            "note": "volumes of 7 MB stay in L2; launch-bound at this size"}


def run_reach(args, torch):
    """Appendix C's bit-vector planner (fewest maneuvers over hard obstacles):
    render + 8 reachability cycles + back-track, at the paper's Table 9
    resolution (128^2 x 512) and on the 512^3 parking scene."""
    from paper_2306_01301_b300 import binding, scenes
    out = {}
    t9, _ = scenes.tiny(17, 7, 9, fill=0.01, turn_radius=14.0, footprint=(3, 1, 1))
    for name, sc, start, goal in (("table9_128x128x512_N8", t9, t9.pose_candidates[0], t9.pose_candidates[5]),
                                  ("parking_512x512x512_N8", scenes.parallel_parking(), None, None)):
        sc_start = start or sc.start
        sc_goal = goal or sc.goal
        stream = torch.cuda.current_stream()
        p = binding.Planner.from_scene(sc, sc.hard_image(), stream=stream)

        def step():
            p.render()
            p.reach_sweep(sc_start, 8)
            return p.reach_extract(sc_goal)

        for _ in range(max(3, args.warmup)):
            res = step()
        steps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # the 8 cycles alone: each reads R_m and H and writes R_{m+1}, 3 bits per pose
        e0.record(stream)
        for _ in range(steps):
            p.reach_sweep(sc_start, 8)
        e1.record(stream)
        torch.cuda.synchronize()
        cycles_ms = e0.elapsed_time(e1) / steps
        peak, peak_kind = load_peaks()
        gbs = 8 * 3 * sc.cells / 8 / (cycles_ms * 1e6)
        out[name] = {"ms_per_plan": ms, "plans_per_s": 1e3 / ms,
                     "pose_cycles_per_s": 8 * 6 * sc.cells / (ms / 1e3),
                     "maneuvers_to_goal": res[0] if res else None,
                     "cycles_ms": cycles_ms,
                     "roofline": {"bound": "hbm", "algorithmic_mb_per_cycle": 3 * sc.cells / 8 / 1e6, "GBps": gbs,
                                  "frac_of_hbm": gbs / peak, "peak": peak, "peak_kind": peak_kind}}
        p.close()
    out["paper_context"] = "Table 9: 2 ms for render + 8 cycles + back-track at 128^2 x 512 on its larger GPU"
    return out


def run_extensions(args, torch):
    """The calls beyond the plain sweep, on the 512^3 parking scene, timed with
    CUDA events: the direction-penalty pass over B (Section XVI, Fig. 19; the
    difference between rendering with and without a two-lane field), the
    start layer of a vehicle under way (Section XII; init + start layer
    against init alone), and a goal-set search with back-track (Section IX;
    12 goals of 13 x 13 x 9 poses, against the single-goal walk), and the
    two-gear-state sweep (forward / reverse transition states, penalty 3000,
    N = 8, one maneuver per launch), the 4D sweep over 9 curvature levels
    (Appendix F; clothoids of one level per cell, N = 8) and the Compact
    graph's sweep (Fig. 12; three vertex types, N = 8)."""
    import numpy as np
    from paper_2306_01301_b300 import binding, scenes
    sc = scenes.parallel_parking()
    stream = torch.cuda.current_stream()
    p = binding.Planner.from_scene(sc, sc.hard_image(), stream=stream)
    nx, nt = p.nx, p.nt

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    render_plain = timed(p.render)
    field = np.zeros((nx, nx), np.uint16)
    field[nx // 2:, :] = nt // 2
    p.set_direction_field(field, nt // 8, 512)
    render_dir = timed(p.render)
    p.set_direction_field(None)
    p.render()
    entry = [sc.transition] * 6
    entry[1] = 0  # straight forward in progress
    init_only = timed(lambda: p.sweep(sc.start, 0))
    init_seed = timed(lambda: p.sweep_state(sc.start, entry, 0))
    p.sweep(sc.start, sc.n_cycles)
    gx, gy, gt = sc.goal
    goals = [(max(0, gx - 40 + 8 * k), gy, (gt + k) % nt, 6, 4, 40, 60, 100 * k) for k in range(12)]
    walk = timed(lambda: p.extract(sc.goal))
    goal_set = timed(lambda: p.extract_goal_set(goals))
    p.set_gear_penalty(3000)
    gear_plan = timed(lambda: p.sweep_gear(sc.start, 0, sc.n_cycles), reps=3)
    gear_res = p.extract_gear(sc.goal)
    p.set_gear_penalty(None)
    M4 = 4
    p.set_curvature_levels(M4, 1.0, 500)
    curv_plan = timed(lambda: p.sweep4(sc.start, 0, sc.n_cycles), reps=3)
    curv_res = p.extract4(sc.goal, 0)
    nk = 2 * M4 + 1
    curv_updates = sc.n_cycles * (4 * nk + 6) * sc.cells  # 4 clothoid layers over every level, 6 3D layers on one
    p.set_curvature_levels(0)
    p.set_compact_graph(True)
    compact_plan = timed(lambda: p.sweep_compact(sc.start, sc.n_cycles), reps=3)
    compact_res = p.extract_compact(sc.goal)
    p.set_compact_graph(False)
    p.close()
    dir_ms = max(render_dir - render_plain, 1e-6)
    # Algorithmic bytes read per plan (the stores of improved cells are left
    # out: a few per cent): every sweep launch reads its volumes once per
    # cell.  Gear states: each turn launch (a fused pair or a lone turn) and
    # each straight reads B and both gears' values, 10 B per cell.  Compact
    # graph: a turn launch reads B, its turn state and S (10 B); a straight B
    # and S (6 B).  Curvature levels: a clothoid layer reads V and B on every
    # level (6 B per cell and level), a 3D pass V and B on its level (6 B).
    peak, peak_kind = load_peaks()
    turns, straights = 4 * sc.n_cycles + 1 - 2 * sc.n_cycles, 2 * sc.n_cycles

    def hbm(nbytes, ms):
        gbs = nbytes / (ms * 1e6)
        return {"algorithmic_gb_read": nbytes / 1e9, "GBps": gbs, "frac_of_hbm": gbs / peak, "peak": peak,
                "peak_kind": peak_kind}
    gear_bytes = (turns + straights) * 10 * sc.cells
    compact_bytes = (turns * 10 + straights * 6) * sc.cells
    curv_bytes = sc.n_cycles * (4 * nk * 6 + 5 * 6) * sc.cells
    return {"direction_pass_ms": dir_ms, "direction_pass_gbs": 4 * sc.cells / (dir_ms * 1e6),
            "render_ms_with_field": render_dir, "render_ms": render_plain,
            "start_layer_ms": max(init_seed - init_only, 0.0),
            "goal_set_extract_ms": goal_set, "single_goal_extract_ms": walk,
            "gear_states_sweep_ms": gear_plan, "gear_states_updates_per_s": 6 * sc.n_cycles * sc.cells / (gear_plan / 1e3),
            "gear_states_roofline": hbm(gear_bytes, gear_plan),
            "gear_states_plan_cost": gear_res[0].cost if gear_res else None,
            "compact_graph": {"sweep_ms": compact_plan, "updates_per_s": 6 * sc.n_cycles * sc.cells / (compact_plan / 1e3),
                              "roofline": hbm(compact_bytes, compact_plan),
                              "plan_cost": compact_res.cost if compact_res else None,
                              "plan_maneuvers": len(compact_res.segments) if compact_res else None},
            "curvature_levels": {"levels": nk, "sweep_ms": curv_plan, "updates_per_s": curv_updates / (curv_plan / 1e3),
                                 "roofline": hbm(curv_bytes, curv_plan),
                                 "plan_cost": curv_res.cost if curv_res else None,
                                 "plan_maneuvers": len(curv_res.segments) if curv_res else None},
            "note": "direction pass moves 4 B per pose (read and write B); the other two are latency-bound one-block kernels"}


def run_batched(args, torch):
    """64 uneven queries (sizes 128^2x128 .. 512^2x256, N in {4, 8, 16}) as
    one batch: render + sweeps + label walks of all queries per step, one
    graph replay, against the same queries planned one at a time through the
    plain single-plan calls; both timed on the host from a synchronised start
    to the results on the host."""
    from paper_2306_01301_b300 import binding, scenes
    qs = scenes.batched_queries()
    stream = torch.cuda.current_stream()
    planners = [binding.Planner.from_scene(sc, stream=stream) for sc in qs]
    queries = [(sc.start, sc.goal, sc.n_cycles) for sc in qs]
    updates = sum(6 * sc.n_cycles * sc.cells for sc in qs)
    b = binding.Batch(planners, stream=stream)
    b.run(queries, render=True)  # tunes the lanes, captures the graph
    b.sync()
    for _ in range(max(3, args.warmup)):
        b.run(queries, render=True)
    b.sync()
    steps = max(3, args.batch_steps)
    # both arms on the same clock: host wall time from a synchronised start to
    # the last result on the host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.run(queries, render=True)
        b.sync()
        res = b.results()
    ms = 1e3 * (time.perf_counter() - t0) / steps
    per_run, _ = b.kernel_launches()
    lanes = b.lanes()
    b.close()

    def one_at_a_time():
        out = []
        for sc, p in zip(qs, planners):
            p.render()
            p.sweep(sc.start, sc.n_cycles)
            out.append(p.extract(sc.goal))
        return out

    one_at_a_time()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        single = one_at_a_time()
    torch.cuda.synchronize()
    ms_single = 1e3 * (time.perf_counter() - t0) / steps
    same = all((a is None and b_ is None) or (a is not None and b_ is not None and a.cost == b_.cost
                                               and a.segments == b_.segments) for a, b_ in zip(res, single))
    for p in planners:
        p.close()
    return {"workload": "batched_64_queries_128^2x128..512^2x256_N4-16", "queries": len(qs),
            "ms_per_batch": ms, "plans_per_s": len(qs) / (ms / 1e3), "updates_per_s": updates / (ms / 1e3),
            "gpu_launches_per_batch": per_run, "steps": steps,
            "timing": "host wall clock for both arms, results read back on the host",
            "one_at_a_time": {"ms_per_batch": ms_single, "plans_per_s": len(qs) / (ms_single / 1e3),
                              "updates_per_s": updates / (ms_single / 1e3)},
            "speedup_vs_one_at_a_time": ms_single / ms, "same_plans_as_one_at_a_time": same,
            "lanes": [{k: l[k] for k in ("n_queries", "ntheta_log2", "nx_min", "nx_max", "turn_k",
                                         "turn_sections", "turn_cluster", "turn_grid", "straight_lines",
                                         "straight_grid", "n_candidates")} for l in lanes],
            "l2": "inputs_larger_than_L2 (about 15 GB of volumes)"}


def _res_key(res):
    return None if res is None else (res.cost, [(g["mu"], g["steps"], g["cost"]) for g in res.segments])


def _pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def _served_stats(lat, span, burst_s, n_burst, keys):
    return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "mean_ms": sum(lat) / len(lat), "max_ms": max(lat),
            "plans_per_s": len(lat) / span, "saturated_plans_per_s": n_burst / burst_s,
            "reachable": sum(1 for k in keys if k is not None)}


def _wait_until(t):
    while True:
        dt = t - time.perf_counter()
        if dt <= 0:
            return
        if dt > 0.0015:
            time.sleep(dt - 0.001)


def run_served(args, torch):
    """The served stream: 16 persistent scenes (c-space rendered once, kept in
    HBM), Poisson arrivals at --served-rate plans/s for --served-seconds (10 %
    of requests at 512^3, the rest of the batched sizes; N = 8).  The same
    trace runs three ways:
      continuous        the continuous-batching server (120 GB admission
                        budget), every request running all of its N cycles;
      continuous_stop   the same server stopping each request's sweep once
                        it has converged (PLAN_SERVE_STOP_AT_CONVERGENCE);
      one_at_a_time     plain calls in arrival order, plan_sweep +
                        plan_extract on one plan object per scene whose
                        c-space was rendered once.
    Latency = result on the host minus arrival.  The first 1000 requests at
    once give each way's saturated plans/s."""
    from paper_2306_01301_b300 import binding, scenes
    scs = scenes.served_scenes()
    trace = scenes.served_trace(scs, rate=args.served_rate, seconds=args.served_seconds)
    free = torch.cuda.mem_get_info()[0]
    budget = min(120 << 30, int(free * 0.8))
    out = {"workload": f"served_stream_poisson{args.served_rate:g}_per_s_{args.served_seconds:g}s_16_scenes_N8",
           "requests": len(trace), "budget_bytes": budget, "scenes": len(scs),
           "policy": {"heavy_cells": args.heavy_cells, "big_cells": args.big_cells, "max_heavy": args.max_heavy},
           "big_share": sum(1 for x in trace if scs[x[1]].nt_log2 == 9) / max(1, len(trace))}
    keys = {}
    burst = trace[:1000]
    for mode in ("continuous", "continuous_stop"):
        torch.cuda.empty_cache()
        srv = binding.Server(budget_bytes=budget, heavy_cells=args.heavy_cells, big_cells=args.big_cells,
                             max_heavy=args.max_heavy, stop_at_convergence=(mode == "continuous_stop"))
        for sc in scs:
            srv.add_scene(sc)
        for k, sc in enumerate(scs):  # warm-up: one request per scene
            srv.wait(srv.submit(k, sc.pose_candidates[0], sc.pose_candidates[1], 8))
        clocks = ClockSampler(torch.cuda.current_device())
        t0 = time.perf_counter()
        tickets = []
        for (ta, k, st, gl, N) in trace:
            _wait_until(t0 + ta)
            tickets.append(srv.submit(k, st, gl, N))
        got = [srv.wait(t) for t in tickets]
        clk = clocks.stop()
        lat = [1e3 * (i["t_done"] - i["t_submit"]) for i, _ in got]
        span = max(i["t_done"] for i, _ in got) - min(i["t_submit"] for i, _ in got)
        stats = srv.stats()
        keys[mode] = [_res_key(r) for _, r in got]
        tb = [srv.submit(k, st, gl, N) for (_, k, st, gl, N) in burst]
        gb = [srv.wait(t) for t in tb]
        bspan = max(i["t_done"] for i, _ in gb) - min(i["t_submit"] for i, _ in gb)
        srv.close()
        out[mode] = _served_stats(lat, span, bspan, len(gb), keys[mode])
        out[mode].update({"gpu_launches": stats["launches"], "steps": stats["steps"],
                          "peak_inflight": stats["peak_inflight"], "peak_arena_bytes": stats["peak_bytes"],
                          "scene_bytes": stats["scene_bytes"], "clocks": clk})
    # one at a time through the plain calls
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    planners = [binding.Planner.from_scene(sc, stream=stream) for sc in scs]
    for p, sc in zip(planners, scs):
        p.render()
        p.plan(sc.pose_candidates[0], sc.pose_candidates[1], 8)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    t0 = time.perf_counter()
    lat, got, launches0 = [], [], sum(p.kernel_launches() for p in planners)
    for (ta, k, st, gl, N) in trace:
        _wait_until(t0 + ta)
        planners[k].sweep(st, N)
        got.append(planners[k].extract(gl))
        lat.append(1e3 * (time.perf_counter() - (t0 + ta)))
    span = time.perf_counter() - t0
    clk = clocks.stop()
    launches = sum(p.kernel_launches() for p in planners) - launches0
    keys["one_at_a_time"] = [_res_key(r) for r in got]
    tb0 = time.perf_counter()
    for (_, k, st, gl, N) in burst:
        planners[k].sweep(st, N)
        planners[k].extract(gl)
    bspan = time.perf_counter() - tb0
    for p in planners:
        p.close()
    out["one_at_a_time"] = _served_stats(lat, span, bspan, len(burst), keys["one_at_a_time"])
    out["one_at_a_time"].update({"calls": "plan_sweep + plan_extract per request, c-space rendered once per scene",
                                 "gpu_launches": launches, "clocks": clk})
    out["same_plans_all_ways"] = keys["continuous"] == keys["continuous_stop"] == keys["one_at_a_time"]
    c, a, o = out["continuous"], out["continuous_stop"], out["one_at_a_time"]
    out["p50_ratio_one_at_a_time_over_continuous"] = o["p50_ms"] / c["p50_ms"]
    out["p99_ratio_one_at_a_time_over_continuous"] = o["p99_ms"] / c["p99_ms"]
    out["saturated_speedup"] = c["saturated_plans_per_s"] / o["saturated_plans_per_s"]
    out["p99_ratio_one_at_a_time_over_continuous_stop"] = o["p99_ms"] / a["p99_ms"]
    out["saturated_speedup_continuous_stop"] = a["saturated_plans_per_s"] / o["saturated_plans_per_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-maze", action="store_true")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-reach", action="store_true")
    ap.add_argument("--no-extensions", action="store_true")
    ap.add_argument("--shapes", default="", help="pin turn variant,turn grid,straight lines,straight grid "
                                                   "instead of autotuning (e.g. 0,148,256,0)")
    ap.add_argument("--maze-steps", type=int, default=5)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-seconds", type=float, default=60.0)
    ap.add_argument("--served-rate", type=float, default=200.0)
    ap.add_argument("--heavy-cells", type=int, default=1 << 24)
    ap.add_argument("--big-cells", type=int, default=0)
    ap.add_argument("--max-heavy", type=int, default=1)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

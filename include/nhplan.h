/*
 * nhplan.h -- C ABI of the B300 kernel-style nonholonomic planner.
 *
 * Implements the data-parallel hot path of Nister et al., "Nonholonomic
 * Motion Planning as Efficient as Piano Mover's" (arXiv 2306.01301):
 * configuration-space obstacle rendering (Section VI), kernel-style
 * processing of the Star graph by maneuver sweeps (Section VIII.B-C, Insert
 * 1, cycle order of Section XVI.A) and forward-tracking plan extraction
 * (Sections IX-X).  All compute runs in hand-written sm_103a CUDA kernels;
 * there is no CPU fallback.
 *
 * Data model
 *   Grid      Nx = Ny = 2^nx_log2 cells, N_theta = 2^ntheta_log2 headings
 *             (Section V.C).  Heading T stands for theta = 2*pi*T/N_theta.
 *   Layout    every volume is theta-major, x fastest:
 *             idx(i, j, T) = i + Nx*(j + Nx*T)  (i = x column, j = y row).
 *   Image     uint16 [Nx][Nx] (row j, column i), Q8 reciprocal of the highest
 *             velocity (Section VI): 256 = free, larger = slower, 0xFFFF =
 *             hard.  Non-hard values must be >= 256.
 *   B         uint16 obstacle volume: max of the image over the vehicle
 *             footprint at that pose, 0xFFFF where the footprint touches a
 *             hard cell or the one-cell walls at i = 0 and j = 0 (Section V.C).
 *   V         uint32 value of the transition state (Section V.A: the only
 *             volume kernel-style processing keeps), PLAN_INF = unreached.
 *             Costs are fixed-point integers with saturating addition.
 *   L         uint16 forward-tracking label (Section X): (mu << 13) | d, where
 *             mu is the maneuver in cycle-order numbering
 *             LF=0 SF=1 RB=2 RF=3 SB=4 LB=5 and d (1 <= d < 8192) the number of
 *             steps from the segment's entry cell; PLAN_LABEL_NONE where V was
 *             never improved.  Labels are written only on strict improvement;
 *             among equally cheap entries the one furthest upstream wins.
 *   Edge cost leaving a non-hard cell X along maneuver mu:
 *             (w_mu * B(X)) >> 8, w = round(step_scale * 2*pi*R / N_theta) for
 *             turns and round(step_straight / max(|cos|,|sin|)) for straights
 *             (Section V.D); entering any maneuver costs `transition` (Star
 *             graph transition edges, Section V.A).
 *
 * Ownership and threading
 *   Host inputs are copied during the call; the caller keeps them.  Device
 *   volumes belong to the plan until plan_destroy.  A plan is not re-entrant;
 *   all its work is ordered on the stream given at creation.  Calls marked
 *   "async" enqueue work and return; plan_extract and plan_copy_volumes
 *   synchronise the plan's stream.
 *
 * Errors
 *   Every entry point returns PLAN_OK (0) or a negative PLAN_E* code; no
 *   entry point aborts the process.  plan_strerror() names the code.
 */
#ifndef NHPLAN_H
#define NHPLAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLAN_OK 0
#define PLAN_EINVAL (-1)       /* bad dimensions, pose, radius, costs, image value */
#define PLAN_ENOMEM (-2)       /* allocator returned NULL */
#define PLAN_ECUDA (-3)        /* a CUDA runtime call failed */
#define PLAN_ETIMEOUT (-4)     /* a bounded device wait gave up */
#define PLAN_EUNREACHABLE (-5) /* goal value is PLAN_INF */
#define PLAN_ERANGE (-6)       /* output capacity too small, or costs could overflow */
#define PLAN_EINTERNAL (-7)    /* device-side consistency check failed */
#define PLAN_ESTATE (-8)       /* call out of order (e.g. sweep before render) */
#define PLAN_ECANCELED (-9)    /* request cancelled (plan_server_cancel) */

#define PLAN_INF 0xFFFFFFFFu
#define PLAN_NO_DIRECTION 0xFFFFu /* no preferred heading (plan_set_direction_field) */
#define PLAN_HARD 0xFFFFu
#define PLAN_LABEL_NONE 0xFFFFu

#define PLAN_FLAG_HALF_SHIFT 1u /* eqs. 13-16: quarter-cell turn rounding */

typedef struct plan_s plan_t;

typedef struct {
    int32_t x, y, theta; /* integer cell indices: 0 <= x, y < Nx, 0 <= theta < N_theta */
} plan_pose;

typedef struct {
    uint32_t step_straight; /* cost of one unit straight step at theta = 0 (e.g. 100) */
    uint32_t step_scale;    /* cost per cell of arc length (e.g. 100) */
    uint32_t transition;    /* ct: cost of entering any maneuver (gear/steer change), < 2^28 */
    uint32_t flags;         /* PLAN_FLAG_* */
} plan_costs;

typedef struct {
    int32_t nx_log2;       /* 2..12 */
    int32_t ntheta_log2;   /* 2..10, with 2*nx_log2 + ntheta_log2 <= 32 */
    const uint16_t* image; /* host pointer, Nx*Nx values, see "Image" above */
} plan_grid;

typedef struct {
    /* Closed rectangle [-rear, front] x [-half_width, half_width] in cells,
     * origin at the rear axle (Fig. 6); all zero = point vehicle. */
    int32_t front, rear, half_width;
} plan_footprint;

typedef struct {
    /* Device memory provider.  alloc returns NULL on failure; free receives
     * the same byte count.  `stream` is the plan's cudaStream_t. */
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} plan_allocator;

typedef struct {
    int32_t maneuver;   /* cycle-order id LF=0 SF=1 RB=2 RF=3 SB=4 LB=5 */
    plan_pose entry;    /* transition point where the maneuver starts */
    plan_pose exit;     /* transition point where it ends */
    int32_t steps;      /* maneuver edges followed */
    uint32_t cost;      /* V at the exit pose */
} plan_segment;

/* Create a plan for one grid shape, vehicle and cost model (the role of
 * Appendix G's `ini`).  turn_radius_cells = R = 1/k_max in cells (> 0).
 * allocator NULL uses cudaMalloc/cudaFree.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream).  Copies the image to the device.  On
 * success *out owns the device volumes V, L, B (8 bytes per pose cell) plus
 * an image-sized scratch table. */
int plan_create(const plan_grid* grid, const plan_footprint* footprint, double turn_radius_cells,
                const plan_costs* costs, const plan_allocator* allocator, void* cuda_stream,
                plan_t** out);

/* Replace the obstacle image (host pointer, Nx*Nx uint16).  The copy is
 * enqueued on the plan's stream; the host buffer may be reused on return. */
int plan_set_image(plan_t* plan, const uint16_t* image);

/* Section VI: render the obstacle volume B from the image and the footprint
 * (walls of Section V.C included).  Async. */
int plan_render_cspace(plan_t* plan);

/* Section VIII.B: V <- INF, L <- NONE, V[start] <- 0, then n_cycles cycles of
 * the six maneuver sweeps in the order LF, SF, RB, RF, SB, LB (Section XVI.A).
 * Requires a rendered obstacle volume (PLAN_ESTATE otherwise) and a non-hard
 * start (PLAN_EINVAL; checked on the host from the image and the footprint).
 * Async.  Returns
 * PLAN_ERANGE if finite costs could reach 2^30 for this image and cycle
 * count. */
int plan_sweep(plan_t* plan, plan_pose start, int n_cycles);

/* Sections IX-X: read V at the exact goal pose and follow the labels back to
 * the start.  Writes at most `cap` segments in driving order to `out` (host),
 * sets *n_out to the number of segments (also when cap is too small:
 * PLAN_ERANGE) and *cost to V(goal).  Synchronises.  PLAN_EUNREACHABLE (with
 * *n_out = 0, *cost = PLAN_INF) if the goal was not reached; PLAN_ESTATE
 * unless the plan's volumes come from plan_sweep, plan_sweep_state or a
 * batch run (not from plan_sweep_gear or plan_autotune). */
int plan_extract(plan_t* plan, plan_pose goal, plan_segment* out, int cap, int* n_out,
                 uint32_t* cost);

/* Section XVI, Fig. 19: direction penalties (stay in the right-hand lane,
 * do not drive against a lane's direction).  heading: Nx*Nx host values
 * (row y, column x, like the image), the preferred heading of poses whose
 * reference cell that is, in [0, N_theta), or PLAN_NO_DIRECTION.  A pose
 * whose heading differs from its cell's preferred heading by more than
 * `tolerance` heading steps (circular distance) has its obstacle value
 * scaled after rendering: B = min(B * penalty_q8 >> 8, 0xFFFE); hard poses
 * stay hard.  Copied to the device; applies from the next
 * plan_render_cspace (the plan must be rendered again).  NULL removes the
 * field.  PLAN_EINVAL for a heading >= N_theta other than PLAN_NO_DIRECTION,
 * tolerance outside [0, N_theta/2] or penalty_q8 outside [256, 65535].  The
 * allocation-free plan_render_cspace_static does not apply it. */
int plan_set_direction_field(plan_t* plan, const uint16_t* heading, int tolerance, uint32_t penalty_q8);

#define PLAN_GEAR_OFF 0xFFFFFFFFu
#define PLAN_GEAR_FORWARD 0
#define PLAN_GEAR_REVERSE 1
#define PLAN_GEAR_AT_REST 2

/* Two gear states: the transition vertex of Fig. 9 split into a forward and
 * a reverse one (the gear of the last maneuver: LF SF RF forward, LB SB RB
 * reverse), so that `penalty` is charged exactly when two consecutive
 * maneuvers change gear -- entering maneuver mu costs cost_in[mu] from its own
 * gear's state and cost_in[mu] + penalty from the other; leaving returns to
 * its own gear's state at cost_out[mu].  Allocates the reverse state's V and
 * L (6 B per pose) on first use; PLAN_GEAR_OFF releases them.  Only for grids
 * up to 2048 (Nx and N_theta; labels need d <= n, a whole turn circle now
 * being able to pay off by changing the gear state).  PLAN_EINVAL for a
 * penalty >= 2^28 or a larger grid, PLAN_ESTATE for a plan without volumes. */
int plan_set_gear_penalty(plan_t* plan, uint32_t penalty);

/* The sweep of the two-state graph: init (start_gear PLAN_GEAR_FORWARD or
 * _REVERSE: the vehicle stands in that gear; _AT_REST: both states 0) and
 * 6N maneuver layers in the cycle order, each reading both states and
 * writing its own gear's (one maneuver per launch, no fused pairs).  The
 * forward state is the plan's V and L (plan_copy_volumes), the reverse one
 * plan_copy_reverse_volumes; labels are (mu << 13) | (entered from the other
 * state << 12) | d.  Saturating arithmetic, no range check needed.  Async.
 * PLAN_ESTATE without plan_set_gear_penalty or before rendering. */
int plan_sweep_gear(plan_t* plan, plan_pose start, int start_gear, int n_cycles);

/* Back-track after plan_sweep_gear from the cheaper state at the goal
 * (forward on a tie), as plan_extract; *end_gear is that state.
 * Synchronises.  PLAN_ESTATE unless the volumes come from plan_sweep_gear. */
int plan_extract_gear(plan_t* plan, plan_pose goal, plan_segment* out, int cap, int* n_out, uint32_t* cost,
                      int* end_gear);

/* The reverse gear state's V and L (either may be NULL).  Synchronises. */
int plan_copy_reverse_volumes(plan_t* plan, uint32_t* V, uint16_t* L);

/* Section V.A, Fig. 12: the Compact graph -- three vertices per cell, S (the
 * straight maneuver type, which is also the transition state), L (left
 * turns, forward and backward) and R (right turns), and ten edges: S -> L and
 * S -> R at costs.transition, L -> S and R -> S free, and the six maneuver
 * edges inside their types.  A turn costs ct to start, a straight nothing, a
 * change of gear within one turn direction nothing.  enable = 1 allocates the
 * L and R values and labels (12 B per pose; S is the plan's own V and L),
 * 0 releases them.  PLAN_EINVAL for a grid above 2048, PLAN_ESTATE for a plan
 * without volumes. */
int plan_set_compact_graph(plan_t* plan, int enable);

/* Kernel-style processing of the Compact graph: the cycle order of Section
 * XVI.A, one maneuver per launch; a turn layer enters its chain from the
 * cell's turn state free or from S at ct (the turn state on a tie) and stores
 * into its turn state and into S; a straight layer moves within S.  The
 * vehicle starts in S.  Labels (maneuver << 13) | (entered from S << 12) | d.
 * Async.  PLAN_ESTATE without plan_set_compact_graph or before rendering. */
int plan_sweep_compact(plan_t* plan, plan_pose start, int n_cycles);

/* Back-track from S(goal) (never above L(goal) or R(goal)) as plan_extract;
 * *cost = V_S(goal).  A walk may cost less than *cost when a later layer
 * lowered an entry's value after its segment was labelled (forward
 * tracking), never more.  Synchronises.  PLAN_ESTATE unless the volumes come
 * from plan_sweep_compact. */
int plan_extract_compact(plan_t* plan, plan_pose goal, plan_segment* out, int cap, int* n_out, uint32_t* cost);

/* The L and R vertex values and labels (S: plan_copy_volumes); any pointer
 * may be NULL.  Synchronises. */
int plan_copy_compact_volumes(plan_t* plan, uint32_t* VL, uint16_t* LL, uint32_t* VR, uint16_t* LR);

/* Appendix F, the 4D generalisation: curvature as a fourth state variable.
 * levels_per_side = M gives 2M+1 levels kappa = -M .. M of the 3D volume,
 * curvature kappa / (M R).  The 3D turns run at the steering limits (LF, LB
 * at kappa = +M; RF, RB at -M), the straights at kappa = 0, and four clothoid
 * maneuvers change the curvature one level per `arc_per_level` cells of
 * travel: PLAN_C1F (curvature rising as the vehicle drives forward), its
 * reverse-gear traversal PLAN_C1B, PLAN_C2F (falling forward) and PLAN_C2B.
 * A clothoid chain through the pose (x0, y0, theta0) at kappa = 0 is at
 * (x0 + round X, y0 + round Y, theta0 + round Psi) at level kappa, X and Y
 * the clothoid's integrals over its arc length (Appendix F's per-level map,
 * a bijection per level).  A clothoid step costs round(step_scale *
 * arc_per_level) * B >> 8 of the cell it leaves; entering a clothoid costs
 * clothoid_cost, the 3D maneuvers keep their costs.  A cycle is the layers
 * C1F, C2F, C1B, C2B, LF, SF, RB, RF, SB, LB.  Allocates (2M+1) * 6 B per
 * pose; M = 0 releases.  PLAN_EINVAL for M > 1000, arc_per_level outside
 * (0, 4], clothoid_cost >= 2^28 or a grid above 2048; PLAN_ESTATE for a plan
 * without volumes. */
#define PLAN_C1F 6
#define PLAN_C1B 7
#define PLAN_C2F 8
#define PLAN_C2B 9
int plan_set_curvature_levels(plan_t* plan, int levels_per_side, double arc_per_level, uint32_t clothoid_cost);

/* The sweep over the curvature levels: init (V = 0 at the start pose on
 * start_level, a curvature in -M .. M) and N cycles of the ten layers.
 * Labels are (maneuver << 12) | d.  Async.  PLAN_ESTATE without
 * plan_set_curvature_levels or before rendering. */
int plan_sweep4(plan_t* plan, plan_pose start, int start_level, int n_cycles);

typedef struct {
    int32_t maneuver;    /* 0 .. 5 as plan_segment, PLAN_C1F .. PLAN_C2B */
    plan_pose entry;
    int32_t entry_level; /* kappa at the entry */
    plan_pose exit;
    int32_t exit_level;
    int32_t steps;
    uint32_t cost;       /* V at the exit */
} plan_segment4;

/* Back-track after plan_sweep4 from the goal pose at goal_level, as
 * plan_extract.  Synchronises. */
int plan_extract4(plan_t* plan, plan_pose goal, int goal_level, plan_segment4* out, int cap, int* n_out,
                  uint32_t* cost);

/* The 4D V and L ((2M+1) * Nx^2 * N_theta entries each, level -M first) and
 * the clothoid tables the library built (dx, dy: [2][2M+1][N_theta], dth:
 * [2][2M+1]); any pointer may be NULL.  Synchronises. */
int plan_copy_volumes4(plan_t* plan, uint32_t* V, uint16_t* L);
int plan_clothoid_tables(plan_t* plan, int16_t* dx, int16_t* dy, int32_t* dth);

/* Section V.A, Fig. 9: per-maneuver transition edges of the Star graph.
 * Entering maneuver mu (cycle-order ids) from the transition state costs
 * cost_in[mu], returning to it cost_out[mu] -- the time of changing gear or
 * steering and of speeding up or slowing down, e.g. a dearer entry into the
 * backward maneuvers.  Until this is called every cost_in is
 * costs.transition and every cost_out 0.  Applies to later sweeps of this
 * plan (plan_sweep, plan_sweep_state, plan_autotune).  PLAN_EINVAL if some
 * cost_in[mu] + cost_out[mu] >= 2^28. */
int plan_set_transition_costs(plan_t* plan, const uint32_t cost_in[6], const uint32_t cost_out[6]);

/* Section XII: plan_sweep for a vehicle already under way.  entry[mu] is the
 * cost of entering maneuver mu (cycle-order ids) at the start pose: its
 * cost_in (ct = costs.transition by default) for a vehicle at rest in the
 * transition state, 0 to continue the maneuver in progress without a
 * transition cost, the rest of a transition in progress toward mu otherwise.
 * Every maneuver with entry[mu] < cost_in[mu] is first followed from the
 * start alone (the start layer; maneuvers in cycle order, a cell keeps the
 * first strictly cheaper value, labelled with that maneuver; leaving still
 * costs cost_out[mu]), then the N cycles run as in plan_sweep; the start
 * keeps V = 0, so entering at cost_in stays possible.  With every entry
 * equal to cost_in this is plan_sweep.  PLAN_EINVAL if an entry exceeds
 * cost_in,
 * otherwise the errors of plan_sweep (the range check counts the start
 * layer as one more layer).  Async on the plan's stream. */
int plan_sweep_state(plan_t* plan, plan_pose start, const uint32_t entry[6], int n_cycles);

/* One goal of a goal set (Section IX): the poses of its box score
 *   V + bias + w_xy * (|dx| + |dy|) + w_theta * |dtheta|
 * (a reward falling with the distance from the ideal pose, turned into a
 * cost).  The box is |dx|, |dy| <= radius_xy, clipped to the grid (which does
 * not wrap), and |dtheta| <= radius_theta modulo N_theta. */
typedef struct {
    plan_pose pose;       /* the ideal goal pose */
    int32_t radius_xy;    /* 0 .. 255 cells */
    int32_t radius_theta; /* 0 .. 255 headings, 2 * radius_theta < N_theta */
    uint32_t w_xy;        /* score per cell of |dx| + |dy| */
    uint32_t w_theta;     /* score per heading of |dtheta| */
    uint32_t bias;        /* score of choosing this goal at all */
} plan_goal;

#define PLAN_MAX_GOALS 65536

/* Sections IX-X: find the best pose of a goal set on the device -- the
 * reached pose with the smallest score over every goal's box; ties go to the
 * earlier goal, then to the goal's ideal pose, then to the box in raster
 * order (dtheta, dy, dx increasing) -- and back-track from it as
 * plan_extract does, without V leaving the device.  Sets *best, *score and,
 * as plan_extract, *cost = V(best), *n_out and `out`.  PLAN_EUNREACHABLE (*n_out
 * = 0, *cost = PLAN_INF, *score = UINT64_MAX) when no pose of any box was
 * reached; PLAN_EINVAL for 0 or more than PLAN_MAX_GOALS goals or a goal out
 * of range.  Synchronises. */
int plan_extract_goal_set(plan_t* plan, const plan_goal* goals, int n_goals, plan_segment* out, int cap,
                          int* n_out, uint32_t* cost, plan_pose* best, uint64_t* score);

/* One timed kernel shape of plan_autotune. */
typedef struct {
    int32_t kind;  /* 0 turn kernel, 1 straight kernel */
    int32_t shape; /* turn: variant index (plan_batch_lane_info); straight: lines per block */
    int32_t grid;  /* 0 = one block per work item, else persistent blocks */
    float ms;      /* best of three timed passes */
} plan_tune_entry;

/* Pick the kernel shapes plan_sweep uses for this plan: time every turn
 * shape on a turn pass and every straight shape on a straight pass of a
 * sweep from `start`, on the plan's own volumes, and keep the fastest of
 * each (all shapes give the same bits).  Requires a rendered plan.  Writes
 * up to cap entries to out (host) and their count to *n_out (NULL allowed),
 * PLAN_ERANGE if cap was too small (the choice is still made).  Leaves V and
 * L in an intermediate state; the next plan_sweep starts over.
 * Synchronises. */
int plan_autotune(plan_t* plan, plan_pose start, plan_tune_entry* out, int cap, int* n_out);

/* Fix the kernel shapes plan_sweep uses (as plan_autotune would): turn
 * variant (-1 = default, else an index below the number of shapes for
 * N_theta), turn grid in work-item slots (0 = one block per item), straight
 * lines per block (0 = default, 128 or 256) and straight grid in blocks.  Every
 * shape gives the same bits.  PLAN_EINVAL for values out of range. */
int plan_set_kernel_shapes(plan_t* plan, int turn_variant, int turn_grid, int straight_lines,
                           int straight_grid);

/* Appendix C: fewest maneuvers with hard obstacles only, one bit per pose.
 * Requires a rendered plan (the hard poses of its obstacle volume are the
 * obstacles; soft costs are ignored), 64 <= Nx <= 512 and 32 <= N_theta <= 512,
 * a non-hard start (PLAN_EINVAL) and 0 <= n_cycles <= 254.  Cycle m + 1
 * takes every maneuver from the poses reachable within m maneuvers (every
 * maneuver edge free, every transition one maneuver), so after n_cycles the
 * plan holds, per pose, whether it is reachable within m maneuvers for m = 0
 * .. n_cycles (n_cycles + 1 bits per pose, plus 4 scratch bits per pose).
 * Does not touch V or L.  Async. */
int plan_reach_sweep(plan_t* plan, plan_pose start, int n_cycles);

/* Back-track a fewest-maneuver plan to goal after plan_reach_sweep: at each
 * level the first maneuver in cycle order (LF, SF, RB, RF, SB, LB) whose
 * curve reaches back, without a hard pose, to a pose of the previous level,
 * from its nearest such pose.  Segments in driving order (cost = maneuvers
 * up to the segment's exit), *maneuvers = the fewest maneuvers.
 * PLAN_EUNREACHABLE if the goal needs more than n_cycles.  Synchronises. */
int plan_reach_extract(plan_t* plan, plan_pose goal, plan_segment* out, int cap, int* n_out, int* maneuvers);

/* Fewest maneuvers of every pose after plan_reach_sweep (host, Nx*Nx*N_theta
 * bytes; 255 where more than n_cycles).  Synchronises. */
int plan_reach_counts(plan_t* plan, uint8_t* counts);

/* Copy the device volumes to host buffers (any may be NULL): V (uint32),
 * L (uint16), B (uint16), Nx*Nx*N_theta entries each.  Synchronises. */
int plan_copy_volumes(plan_t* plan, uint32_t* V, uint16_t* L, uint16_t* B);

/* Device pointers of the volumes (owned by the plan). */
int plan_device_volumes(plan_t* plan, uint32_t** V, uint16_t** L, uint16_t** B);

/* Per-pass timing and work counters, for roofline accounting.  While
 * profiling is on, plan_render_cspace and plan_sweep record a CUDA event pair
 * around each kernel pass on the plan's stream, and (PLAN_PROFILE_ALL) the
 * sweep kernels count the cells whose value strictly decreased (the cells
 * they write).  Counting adds a warp reduction and atomics per tile and one
 * block barrier per turn tile; timing adds two event records per pass.  The
 * counts of a sweep depend only on its inputs, so a timed run can leave
 * counting off (PLAN_PROFILE_TIMING) and take them from an untimed sweep. */
typedef struct {
    int64_t turn_passes;      /* fused or single turn sweeps */
    int64_t straight_passes;
    int64_t render_passes;    /* sparse table + render */
    int64_t init_passes;
    double turn_ms, straight_ms, render_ms, init_ms; /* summed event times */
    uint64_t turn_improved;   /* cells written by turn passes */
    uint64_t straight_improved;
    uint64_t turn_tiles_improved; /* turn-kernel work items (32 chains) with any written cell */
} plan_profile_stats;

/* Profiling modes of plan_profile. */
#define PLAN_PROFILE_OFF 0
#define PLAN_PROFILE_ALL 1    /* event timing and improved-cell counters */
#define PLAN_PROFILE_TIMING 2 /* event timing only */

/* Set the profiling mode (PLAN_PROFILE_*; PLAN_EINVAL otherwise); either
 * way the counters restart.  Synchronises. */
int plan_profile(plan_t* plan, int enable);

/* Read the counters accumulated since plan_profile(plan, 1).  Synchronises. */
int plan_profile_read(plan_t* plan, plan_profile_stats* out);

/* Number of CUDA kernels launched by this plan since creation. */
int plan_kernel_launches(plan_t* plan, int64_t* count);

int plan_destroy(plan_t* plan);

const char* plan_strerror(int code);

/* Which CUDA call failed, and its error name, for the last PLAN_ECUDA
 * returned on this host thread ("" if none).  The text stays valid until the
 * next failure on the thread. */
const char* plan_last_error(void);

/* Obstacle rendering for callers that cannot allocate device memory -- for
 * example a runtime that owns all device memory through a fixed memory plan,
 * or a control loop that forbids allocation once it is running.  The paper
 * has no counterpart; this is the same computation as plan_render_cspace
 * without a plan object.  image_dev: device pointer, Nx*Nx uint16 (as in
 * plan_grid.image); B_dev: device pointer, Nx*Nx*N_theta uint16, written.
 * footprint, turn radius and flags as in plan_create (the radius and the
 * half-shift flag fix the footprint's sub-cell placement).  Work is enqueued
 * on cuda_stream.  The call allocates nothing: its scratch (sparse table and
 * footprint runs, about 5.8 MB) is one fixed device array that every GPU which
 * loads this library holds until the process exits, so Nx is limited to 512
 * (larger grids return PLAN_ERANGE before any work) and the footprint to 65536
 * row runs over all headings.  The first call on a device looks up that
 * array's device address with the device current.  All calls share the one
 * array: two calls whose work overlaps on a
 * GPU (other streams, other host threads) race and may produce wrong volumes.
 * Returns PLAN_EINVAL for bad arguments and PLAN_ECUDA if a CUDA call fails. */
int plan_render_cspace_static(const uint16_t* image_dev, int nx_log2, int ntheta_log2,
                              const plan_footprint* footprint, double turn_radius_cells, uint32_t flags,
                              uint16_t* B_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched planning.  Many independent queries -- each on its own plan, so
 * grid size, vehicle, turn radius, costs and N may all differ -- run together:
 * every sweep pass is one launch over all queries of a lane (same N_theta,
 * compatible Nx), lanes run as parallel branches of one captured CUDA graph,
 * and an autotuner picks each lane's kernel shapes on the first run.  Results
 * are bit-identical to running each plan alone (plan_render_cspace,
 * plan_sweep, plan_extract).
 *
 * The batch borrows the plans: they must outlive it, must not be used on
 * their own while a batch run is in flight, and a plan may appear once.
 * After a run, each plan's volumes (plan_copy_volumes) hold its query's
 * result.  All batch work is ordered on the stream given at creation.
 */
typedef struct plan_batch_s plan_batch_t;

#define PLAN_BATCH_NO_GRAPH 1u /* launch pass by pass instead of replaying a graph */
#define PLAN_BATCH_NO_TUNE 2u  /* default kernel shapes, no timing runs */

typedef struct {
    plan_pose start, goal;
    int32_t n_cycles; /* N >= 1 */
} plan_query;

typedef struct {
    int32_t n_queries, ntheta_log2, nx_min, nx_max;
    /* chosen shapes: turn kernel K headings per thread, warps per block and
     * blocks per cluster (variant index among the shapes for N_theta), grid
     * in work-item slots (0 = one block per item, else persistent); straight
     * kernel lines per block and grid */
    int32_t turn_variant, turn_k, turn_sections, turn_cluster, turn_grid;
    int32_t straight_lines, straight_grid;
    int32_t n_candidates; /* shapes timed (0 with PLAN_BATCH_NO_TUNE) */
    float turn_ms, straight_ms; /* best timed pass of each kind */
} plan_batch_lane_info;

/* Create a batch over n distinct plans.  allocator (NULL = cudaMalloc) serves
 * the batch's own small device buffers.  Synchronises the plans' streams
 * once.  PLAN_EINVAL on NULL or repeated plans. */
int plan_batch_create(plan_t* const* plans, int n, uint32_t flags, const plan_allocator* allocator,
                      void* cuda_stream, plan_batch_t** out);

/* Run query i on plan i for all i (queries: host array of n).  render != 0
 * renders every plan's obstacle volume first (else each plan must have been
 * rendered: PLAN_ESTATE).  Checks poses (PLAN_EINVAL: outside the grid, hard
 * start, N < 1) and cost range (PLAN_ERANGE) before any work.  The first run
 * tunes the kernel shapes (timing runs on the plans' volumes); a run whose
 * N values differ from the previous run's captures a new graph, otherwise
 * the graph is replayed with the new start and goal poses.  Async: returns
 * once the work is enqueued. */
int plan_batch_run(plan_batch_t* batch, const plan_query* queries, int render);

/* Wait for the last run. */
int plan_batch_sync(plan_batch_t* batch);

/* Result of query i of the last run, as plan_extract reports it (segments in
 * driving order, *n_out, *cost, PLAN_EUNREACHABLE, PLAN_ERANGE when cap is
 * too small).  Synchronises. */
int plan_batch_result(plan_batch_t* batch, int i, plan_segment* out, int cap, int* n_out, uint32_t* cost);

/* Lanes and the shapes the autotuner chose for them (PLAN_ESTATE before the
 * first run). */
int plan_batch_lanes(plan_batch_t* batch, int* n_lanes);
int plan_batch_lane(plan_batch_t* batch, int lane, plan_batch_lane_info* out);

/* Kernel launches of one run (graph nodes) and since creation. */
int plan_batch_kernel_launches(plan_batch_t* batch, int64_t* per_run, int64_t* total);

int plan_batch_destroy(plan_batch_t* batch);

/* ------------------------------------------------------------------------
 * Serving.  A server keeps scenes (image + vehicle + costs, rendered once)
 * resident on the device and plans requests against them.  All its device
 * memory -- scenes, each in-flight request's value and label volumes (6 bytes
 * per pose cell) and small descriptor buffers -- comes from one arena of
 * budget_bytes allocated at creation; a request is admitted (in arrival
 * order) when the arena has room for its volumes and a slot is free.
 *
 * PLAN_SERVE_CONTINUOUS: a native scheduler thread runs the GPU in steps;
 * each step initialises the newly admitted requests, advances every other
 * admitted request by one sweep pass (one launch per lane and pass kind, each
 * request at its own pass) and walks the labels of the requests that ran
 * their last pass, so requests that arrive while others run join them on the
 * GPU.  PLAN_SERVE_ONE_AT_A_TIME: the same thread plans one request at a time
 * with the single-plan launch sequence (the plain-sweep baseline).  In both
 * modes a request's result equals plan_sweep + plan_extract on its scene.
 */
typedef struct plan_server_s plan_server_t;

#define PLAN_SERVE_CONTINUOUS 0
#define PLAN_SERVE_ONE_AT_A_TIME 1

typedef struct {
    size_t budget_bytes;  /* device memory of the server (>= 1 MiB) */
    int32_t max_inflight; /* requests admitted at once; 0 = only memory limits */
    int32_t mode;         /* PLAN_SERVE_* */
    /* Continuous mode, size classes: requests of at least big_cells pose
     * cells are big, of at least heavy_cells heavy, the rest light (0 = class
     * unused).  At most max_heavy big and max_heavy heavy requests run at
     * once (0 = no limit), each class taken in arrival order while requests
     * of other classes may pass one that waits for its slot.  Each class
     * steps on a stream of its own, light at the highest stream priority and
     * big at the lowest, so small requests do not wait for large passes. */
    int64_t heavy_cells;
    int64_t big_cells;
    int32_t max_heavy;
    int32_t flags;        /* PLAN_SERVE_* flags below */
    /* Launch-descriptor bytes reserved per step slot (3 slots per stream, 3
     * streams) when the server is created; 0 = 64 KiB, about 140 requests
     * per step.  At least 4096. */
    int64_t slot_bytes;
} plan_server_config;

/* Stop a request's sweep once it has converged: when four consecutive passes
 * (every maneuver once, from the first cycle's SF on) have lowered no cell,
 * V and L are a fixed point of every maneuver layer, so the remaining passes
 * of its N cycles would change nothing.  Each pass records on the device
 * whether it lowered a cell; later passes of a converged request read those
 * records and return without touching its volumes.  Results are identical
 * with and without the flag; served latency drops for requests that converge
 * before their N-th cycle. */
#define PLAN_SERVE_STOP_AT_CONVERGENCE 1

typedef struct {
    int32_t status;     /* PLAN_OK, PLAN_EUNREACHABLE, PLAN_ENOMEM (can never fit), PLAN_ECANCELED, PLAN_ECUDA ... */
    uint32_t cost;      /* V(goal) */
    int32_t n_segments;
    int32_t scene;
    double t_submit, t_admit, t_done; /* host steady clock, seconds */
} plan_request_info;

typedef struct {
    int64_t scenes, submitted, admitted, completed, rejected;
    int64_t steps;         /* scheduler steps (one-at-a-time: requests) */
    int64_t launches;      /* kernels launched for requests */
    int64_t peak_inflight; /* most requests admitted at once */
    int64_t arena_bytes, peak_bytes, scene_bytes;
    int64_t reserved_bytes; /* arena bytes held from creation on for launch descriptors */
    int64_t cancelled;      /* requests ended by plan_server_cancel */
    int64_t partial_steps;  /* steps that advanced only some requests (descriptor space) */
} plan_server_stats;

/* Create a server and start its scheduler thread.  allocator (NULL =
 * cudaMalloc) provides the one arena block; cuda_stream's earlier work is
 * waited for once.  The server uses the device current at creation.  The
 * launch descriptors of every stream's steps are carved from the arena at
 * creation (reserved_bytes in the stats, PLAN_ENOMEM when the budget cannot
 * hold them), so scenes and requests get the rest.  Descriptor space grows
 * only from arena memory nobody else holds; when it cannot grow, a step
 * advances the requests that fit and the others wait for the next step. */
int plan_server_create(const plan_server_config* cfg, const plan_allocator* allocator, void* cuda_stream,
                       plan_server_t** out);

/* Add a scene (arguments as plan_create) and render its obstacle volume into
 * the arena now (synchronous).  *scene_id numbers scenes from 0.
 * PLAN_ENOMEM when the arena cannot hold it. */
int plan_server_add_scene(plan_server_t* server, const plan_grid* grid, const plan_footprint* footprint,
                          double turn_radius_cells, const plan_costs* costs, int32_t* scene_id);

/* Queue a request (thread-safe, does not wait for the GPU).  Checks the
 * scene, the poses (PLAN_EINVAL: outside the grid, hard start, N < 1), the
 * cost range (PLAN_ERANGE) and that the volumes can ever fit (PLAN_ENOMEM).
 * *ticket identifies the request for plan_server_wait. */
int plan_server_submit(plan_server_t* server, int32_t scene_id, plan_pose start, plan_pose goal,
                       int32_t n_cycles, uint64_t* ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; PLAN_ETIMEOUT
 * if it is not done.  On PLAN_OK fills *info and up to cap segments in
 * driving order (*n_out = all segments; PLAN_ERANGE if cap is too small) and
 * releases the ticket. */
int plan_server_wait(plan_server_t* server, uint64_t ticket, double timeout_s, plan_request_info* info,
                     plan_segment* out, int cap, int* n_out);

/* Cancel a request (thread-safe, does not wait).  A request not yet admitted
 * is dropped; an admitted one runs no further passes and its memory is
 * released once the work already queued for it has finished; its wait then
 * reports PLAN_ECANCELED in info->status.  A request whose label walk is
 * already on the GPU, or that is done, keeps its result.  In one-at-a-time
 * mode the request being planned is not interrupted.  PLAN_EINVAL for an
 * unknown ticket. */
int plan_server_cancel(plan_server_t* server, uint64_t ticket);

/* Counters since creation. */
int plan_server_stats_read(plan_server_t* server, plan_server_stats* out);

/* Finish every submitted request, stop the thread, free everything. */
int plan_server_destroy(plan_server_t* server);

/* Section VII, host helper: soft-obstacle image from a binary occupancy map
 * [nx][nx] (nonzero = obstacle).  Obstacle cells become 0xFFFF; a free cell at
 * squared Euclidean distance d2 from the nearest obstacle gets
 * 256 + soft_max*(r2 - d2)/r2 (integer division) when d2 < r2 = radius^2, else
 * 256.  radius 0 gives the hard-only image.  Returns PLAN_EINVAL for bad
 * arguments (nx <= 0, radius < 0 or > 255, soft_max < 0 or > 65000). */
int plan_soft_image(int nx, const uint8_t* occupancy, int radius, int soft_max, uint16_t* image);

#ifdef __cplusplus
}
#endif
#endif /* NHPLAN_H */

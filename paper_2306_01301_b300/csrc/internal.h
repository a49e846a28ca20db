// internal.h -- private declarations of the nhplan library (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nhplan.h"

namespace nhp {

// Values at or above TH mean "unreached" inside the kernels.  Stored volumes
// keep PLAN_INF; loads clamp to TH and hard cells get edge cost TH, so every
// intermediate of the sweeps (a clamped value, plus one transition cost
// < 2^28, plus one edge cost <= TH) fits in 32 bits without saturation
// logic.  The host refuses inputs whose finite costs could reach TH.
constexpr uint32_t TH = 0x40000000u;
constexpr uint16_t HARD = 0xFFFFu;
constexpr uint16_t NONE = 0xFFFFu;
constexpr uint16_t NO_DIRECTION = PLAN_NO_DIRECTION;

enum Maneuver { LF = 0, SF = 1, RB = 2, RF = 3, SB = 4, LB = 5 };

// Per-heading constants of the straight lines.
struct PlaneInfo {
    int32_t iflag;  // eq. 19
    int32_t jsign;  // eq. 24
    uint32_t wS;    // straight step weight
    int32_t pad;
};

// One maximal run of the footprint in a row: cells dx in [lo, hi] at dy.
// The row maximum over the run is the larger of two sparse-table windows of
// width 2^lvl starting at lo and at hi2 = hi - 2^lvl + 1.
struct Run {
    int16_t dy, lo;
    int16_t lvl;
    int16_t hi2;
};

struct DevGrid {
    int lx, lt, nx, nt, mx, mt;
    uint32_t wA;
    // Star transition edges (Fig. 9): ctm[mu] = cost of entering plus
    // leaving maneuver mu.  Every segment takes both edges, so charging the
    // sum on entering stores the same values and labels; cout[mu] alone is
    // what the start layer adds after an entry cost of its own.
    uint32_t ctm[6], cout[6];
    const int4* beta4;       // per heading: (beta_0, beta_3, beta_2, beta_1), raw
    const PlaneInfo* plane;  // per heading
    const int16_t* bshear;   // [T*nx + y'] B(y', T), eq. 22
    const int32_t* run_off;  // [nt + 1]
    const Run* runs;
};

struct Volumes {
    uint32_t* V;
    uint16_t* L;
    uint16_t* B;
    unsigned long long* improved;  // optional counter of strictly improved cells
};

// Everything a kernel needs about one planning query.  Kernels take a device
// array of these, so one launch serves a single plan, a batch of plans of
// one grid shape, or one step of the server with each query at its own pass.
struct QueryDesc {
    DevGrid g;
    Volumes v;
    int64_t start;            // start cell (init)
    int64_t goal;             // goal cell (extract)
    int32_t n_cycles;         // N: the query runs passes 0 .. 4N
    int32_t pass;             // this query's pass when a launch says "per query"
    const uint16_t* img;      // obstacle image (Nx*Nx)
    uint32_t* bits;           // bit-parallel hard table, (lx+1) * Nx * Nx/32 words
    uint16_t* table;          // uint16 sparse max table, (lx+1) * Nx * Nx
    plan_segment* seg;        // label walk output (goal first)
    int32_t* status;          // [0] segment count or error, [1] V(goal) low, [2] high
    int32_t seg_cap;
    int32_t max_runs;         // footprint runs of the widest heading
    // Optional (null = off): one word per pass (4N + 1), set to 1 by a pass
    // that lowered some cell of this query.  Once four consecutive passes
    // starting at pass 1 or later -- every maneuver once -- lowered nothing,
    // V and L are a fixed point of every maneuver layer, so later passes of
    // the query change nothing; launch_conv_gate then takes them out of the
    // launches that follow (same values and labels).
    uint32_t* conv;
    // Built with PLAN_BOUNDS_CHECK: the first failed index check of the plain
    // plan path's kernels records its site here (the host reports
    // PLAN_EINTERNAL); null or unused otherwise.
    int32_t* err;
    // Bit position of the maneuver in the labels the sweeps write: 0 means
    // 13 (plain labels, (mu << 13) | steps); the curvature levels' 3D
    // layers use 12 (maneuvers up to 9, steps up to 4095).
    int32_t mu_shift;
};

__device__ __forceinline__ uint32_t label_tag(const QueryDesc& Q, int mu) {
    return (uint32_t)mu << (Q.mu_shift ? Q.mu_shift : 13);
}

// Index checks of the PLAN_BOUNDS_CHECK build: NHP_IN(i, n, err, site) is
// true when 0 <= i < n; otherwise it records `site` in *err (first failure
// wins) and is false, and the caller skips the access.  Without the build
// flag it is the constant true and costs nothing.
#ifdef PLAN_BOUNDS_CHECK
__device__ __forceinline__ bool nhp_in(int64_t i, int64_t n, int32_t* err, int site) {
    if (i >= 0 && i < n) return true;
    if (err) atomicCAS(err, 0, site);
    return false;
}
#define NHP_IN(i, n, err, site) ::nhp::nhp_in((int64_t)(i), (int64_t)(n), (err), (site))
#else
#define NHP_IN(i, n, err, site) true
#endif

// True when pass p of a query with convergence flags has nothing left to do.
__device__ __forceinline__ bool pass_converged(const uint32_t* conv, int p) {
    return conv != nullptr && p >= 5 && (conv[p - 1] | conv[p - 2] | conv[p - 3] | conv[p - 4]) == 0u;
}

// One launch group: nq descriptors on the device.  Without `item_off` every
// query has the shape (lx, lt) and a launch gives each work item its own
// block.  A batched launch mixes grid sizes: item_off (device, nq + 1
// entries) is the prefix sum of each query's work items (turn: 32-chain
// tiles, all queries with N_theta = 2^lt; straight: heading planes times
// line blocks, all queries with Nx >= the block's lines), `items` their
// total, and `grid` > 0 caps the blocks, which then loop over the items
// (a persistent launch).
struct Group {
    const QueryDesc* d;
    int nq;
    int lx, lt;
    int max_runs;             // max over the group
    const int32_t* item_off = nullptr;
    int64_t items = 0;
    int grid = 0;
    // host copy of the transition costs (DevGrid::ctm) when every query of
    // the launch has the same ones, else null: turn launches then pass the
    // pass's two costs as kernel parameters instead of each tile reading
    // them from its descriptor
    const uint32_t* ctm = nullptr;
};

// Cycle schedule (Section XVI.A) with the turn pairs fused: N cycles are the
// passes p = 0 .. 4N:
//   p = 0      LF              (a lone opening left-forward)
//   p = 4c+1   SF              p = 4c+3   SB
//   p = 4c+2   RB then RF      (right chains, heading up then down)
//   p = 4c+4   LB then LF      (left chains, heading down then up; the LF
//                               belongs to cycle c+1 and is dropped when
//                               c = N-1)
inline int pass_count(int n_cycles) { return n_cycles > 0 ? 4 * n_cycles + 1 : 0; }
inline bool pass_is_turn(int p) { return (p & 1) == 0; }
// Maneuvers of turn pass p, in scan order (the second is -1 for p = 0; the
// last pass of a query may drop it, which needs no cost).
inline void turn_pass_maneuvers(int p, int* mu1, int* mu2) {
    if (p == 0) { *mu1 = LF; *mu2 = -1; }
    else if ((p & 3) == 2) { *mu1 = RB; *mu2 = RF; }
    else { *mu1 = LB; *mu2 = LF; }
}
// Kernel-parameter marker: read the cost from each query's descriptor.
constexpr uint32_t kCostPerQuery = 0xFFFFFFFFu;

// Launchers.  `pass` < 0 means "each query's own QueryDesc::pass"; queries
// whose pass is outside 0 .. 4N do nothing.  Each returns cudaGetLastError().
cudaError_t launch_init(const Group& gr, cudaStream_t s);
// Before a sweep launch over nq device descriptors with convergence records:
// converged queries get pass -1, the others pass_all (or keep their pass
// when pass_all < 0).
cudaError_t launch_conv_gate(QueryDesc* qd, int nq, int pass_all, cudaStream_t s);
// Rendering: bit-parallel hard test for Nx >= 32 (uint16 maxima for the
// non-hard poses when `soft`), uint16 sparse-table path otherwise.  Returns
// the number of kernels launched through *launches.
cudaError_t launch_render(const Group& gr, bool soft, cudaStream_t s, int* launches);
// Turn pass with kernel shape `variant` (index into the shapes available for
// the group's N_theta, -1 = the measured default).
cudaError_t launch_turn(const Group& gr, int pass, int variant, cudaStream_t s);
int turn_variants(int nt);
// Shape of a turn variant: K headings per thread, SL warps per block, CL
// blocks per cluster (K * SL * CL = N_theta).
void turn_shape(int lt, int variant, int* K, int* SL, int* CL);
// Resident blocks of one SM for a turn variant / straight shape (persistent
// grid sizing); 0 on error.
int turn_blocks_per_sm(int lt, int variant);
int straight_blocks_per_sm(int lines);
// Work items of one query in a batched launch.
inline int64_t turn_items(int lx) { return (((int64_t)1 << (2 * lx)) + 31) / 32; }
inline int64_t straight_items(int lx, int lt, int lines) { return ((int64_t)1 << lt) * (((int64_t)1 << lx) / lines); }
// Straight pass with `lines` (128 or 256, 0 = default) lines per block.
cudaError_t launch_straight(const Group& gr, int pass, int lines, cudaStream_t s);
// Label walk from each query's goal into its seg/status buffers.
cudaError_t launch_extract(const Group& gr, cudaStream_t s);

// Per-maneuver constants by a select chain: indexing the arrays with a
// runtime maneuver would move the kernel's copy of DevGrid to local memory.
__device__ __forceinline__ uint32_t pick6(const uint32_t (&a)[6], int mu) {
    uint32_t r = a[0];
    r = mu == 1 ? a[1] : r;
    r = mu == 2 ? a[2] : r;
    r = mu == 3 ? a[3] : r;
    r = mu == 4 ? a[4] : r;
    r = mu == 5 ? a[5] : r;
    return r;
}

// Two gear states (forward / reverse transition vertices): one maneuver
// layer's arguments.  Vf, Lf are the plan's own volumes, Vr, Lr the reverse
// state's.
struct GearLayer {
    DevGrid g;
    const uint16_t* B;
    uint32_t *Vf, *Vr;
    uint16_t *Lf, *Lr;
    uint32_t pen, cin, cout;  // gear change; entering and leaving the layer's maneuver
    bool scan;                // finite costs stay below TH: turn layers may run the sections scan
    int32_t* err;             // the bounds-check build's error word (QueryDesc::err)
};
cudaError_t launch_gear_init(uint32_t* Vf, uint32_t* Vr, uint16_t* Lf, uint16_t* Lr, int64_t nr, int64_t start,
                             int start_gear, cudaStream_t s);
cudaError_t launch_gear_layer(const GearLayer& a, int mu, cudaStream_t s);
// Whether this grid runs a turn pair (RB then RF, or LB then LF: opposite
// gears on the same chains) as one fused launch, and that launch; ct1, ct2
// are the two maneuvers' entering plus leaving edges.
bool gear_pair_fused(const GearLayer& a);
cudaError_t launch_gear_pair(const GearLayer& a, int mu1, int mu2, uint32_t ct1, uint32_t ct2, cudaStream_t s);
// A straight layer of the gear states on the staged tiles of the plain
// straight kernel (sweep.cu); needs Nx >= 16 and a.scan.
cudaError_t launch_gear_straight_tiled(const GearLayer& a, int mu, cudaStream_t s);
cudaError_t launch_gear_extract(const GearLayer& a, int64_t goal, plan_segment* seg, int cap, int32_t* status,
                                cudaStream_t s);

// 4D generalisation (Appendix F): one maneuver layer over 2M+1 curvature
// levels of the 3D volume (V, L hold nk * nr entries, level K = kappa + M
// first), with the clothoid tables dx, dy [2][nk][N_theta] and dth [2][nk].
struct Layer4 {
    DevGrid g;
    const uint16_t* B;
    uint32_t* V;
    uint16_t* L;
    int64_t nr;
    int nk;
    const int16_t *dx, *dy;
    const int32_t* dxy;     // (dy << 16) | (dx & 0xFFFF), the same entries in one word
    const int32_t* dth;
    uint32_t w, cin, cout;  // step weight of the layer's maneuver; entering, leaving
    bool th;                // finite costs stay below TH: clothoids in the plain sweeps' value domain
    int32_t* err;           // the bounds-check build's error word (QueryDesc::err)
};
cudaError_t launch4_init(uint32_t* V, uint16_t* L, int64_t n4, int64_t start4, cudaStream_t s);
cudaError_t launch4_layer(const Layer4& a, int mu, int level, cudaStream_t s);
cudaError_t launch4_extract(const Layer4& a, int64_t goal4, plan_segment4* seg, int cap, int32_t* status,
                            cudaStream_t s);

// Direction penalties (Section XVI, Fig. 19) applied to a rendered B.
cudaError_t launch_direction(uint16_t* B, const uint16_t* field, int lx, int lt, int tol, uint32_t pen,
                             cudaStream_t s);

// Start state (Section XII): entry cost of each maneuver at the start pose.
struct StartEntry {
    uint32_t e[6];
};
// Best pose of one goal's box, or of the whole set: score, then rank (goal
// index << 40 | position in the box, the ideal pose first), cell (-1: none).
struct GoalBest {
    uint64_t score, rank;
    int64_t cell;
};
// The start layer on qd[0]'s volumes (after init, before pass 0).
cudaError_t launch_seed(const QueryDesc* qd, const StartEntry& entry, cudaStream_t s);
// Goal search over n goals (device array); writes qd[0].goal on the device.
cudaError_t launch_goal_search(QueryDesc* qd, const plan_goal* goals, int n, GoalBest* per_goal, GoalBest* result,
                               cudaStream_t s);

// Maneuver-count reachability with bit vectors (reach.cu, extract.cu).
cudaError_t launch_hard_bits(const uint16_t* B, uint32_t* H, int64_t nr, cudaStream_t s);
cudaError_t launch_reach_init(uint32_t* R, int64_t nr, int64_t start, cudaStream_t s);
cudaError_t launch_bit_transpose(const uint32_t* src, uint32_t* dst, const int32_t* planes, int nplanes, int lx,
                                 bool and_into, cudaStream_t s);
// mode: 0 AND into Rn, 1 Rn = Rm AND result, 2 Rn = result
cudaError_t launch_reach_turn(const DevGrid& g, const uint32_t* Rm, uint32_t* Rn, const uint32_t* H, int family,
                              int mode, cudaStream_t s);
// Steep planes' results stored into Out, shallow planes' (transposed) into OT.
cudaError_t launch_reach_straight(const DevGrid& g, const uint32_t* Rm, const uint32_t* H, const uint32_t* RmT,
                                  const uint32_t* HT, uint32_t* Out, uint32_t* OT, cudaStream_t s);
// Rn &= X1 & X2 over all words.
cudaError_t launch_reach_combine(uint32_t* Rn, const uint32_t* X1, const uint32_t* X2, int64_t nr, cudaStream_t s);
cudaError_t launch_reach_counts(const uint32_t* R, int n, int64_t nr, uint8_t* count, cudaStream_t s);
cudaError_t launch_reach_extract(const DevGrid& g, const uint32_t* R, int n, int64_t words, const uint32_t* H,
                                 int64_t goal, plan_segment* seg, int cap, int32_t* status, cudaStream_t s);

// Rendering pieces used by the allocation-free entry point.
cudaError_t launch_sparse_table(const Group& gr, cudaStream_t s);
cudaError_t launch_render_table(const Group& gr, cudaStream_t s);

}  // namespace nhp

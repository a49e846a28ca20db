// plan_state.h -- the plan object shared by the single-plan, batch and
// server entry points (private).
#pragma once
#include <vector>

#include "internal.h"

using nhp::DevGrid;
using nhp::PlaneInfo;
using nhp::Run;

enum { VOL_NONE = 0, VOL_PLAIN = 1, VOL_GEAR = 2, VOL_COMPACT = 3 };
enum { VOL4_NONE = 0, VOL4_SWEPT = 1 };

struct plan_s {
    int lx = 0, lt = 0, nx = 0, nt = 0;
    int64_t nxy = 0, nr = 0;
    double R = 0;
    plan_costs costs{};
    uint32_t cin[6] = {}, cout[6] = {};  // Star transition edges per maneuver
    uint16_t* d_dir = nullptr;            // direction field (Nx*Nx), or none
    uint32_t *d_Vcl = nullptr, *d_Vcr = nullptr;  // Compact graph: L and R vertex values and labels
    uint16_t *d_Lcl = nullptr, *d_Lcr = nullptr;
    uint32_t* d_Vr = nullptr;             // reverse gear state (plan_set_gear_penalty)
    uint16_t* d_Lr = nullptr;
    uint32_t gear_pen = 0;
    // curvature levels (plan_set_curvature_levels)
    int curv_M = 0, curv_nk = 0;
    double curv_L = 0.0;
    uint32_t curv_w = 0, curv_ct = 0;
    uint32_t* d_V4 = nullptr;
    // the 3D layers' descriptors on the levels they run on (left limit,
    // kappa = 0, right limit), for the plain sweep kernels
    nhp::QueryDesc* d_qd4 = nullptr;
    // the Compact graph's straights as a one-cycle query on S (plain kernel)
    nhp::QueryDesc* d_qdc = nullptr;
    uint16_t* d_L4 = nullptr;
    int16_t *d_cdx = nullptr, *d_cdy = nullptr;
    int32_t* d_cdxy = nullptr;  // dx and dy packed in one word
    int32_t* d_cdth = nullptr;
    std::vector<int16_t> cdx, cdy;
    std::vector<int32_t> cdth;
    bool gear_on = false;
    // what V and L hold: nothing usable, a plain (one transition state)
    // sweep, or a two-gear-state sweep; each back-track reads only its own
    int vol_kind = VOL_NONE;
    int vol4_kind = VOL4_NONE;
    int dir_tol = 0;
    uint32_t dir_pen = 256;
    plan_footprint fp{};
    cudaStream_t stream = nullptr;
    plan_allocator alloc{};
    // host copies
    std::vector<int4> beta4;
    std::vector<PlaneInfo> planes;
    std::vector<int16_t> bshear;
    std::vector<int32_t> run_off;
    std::vector<Run> runs;
    std::vector<int32_t> fp_dx, fp_dy;  // footprint cells of every heading, concatenated
    std::vector<int32_t> fp_off;
    std::vector<unsigned char> blob;    // staged table upload
    std::vector<uint16_t> img;
    int max_runs = 0;
    uint32_t wA = 0, w_max = 0;
    uint32_t img_max_soft = 256;
    // device
    unsigned char* d_blob = nullptr;
    size_t blob_bytes = 0;
    uint16_t* d_img = nullptr;
    uint16_t* d_table = nullptr;
    size_t table_bytes = 0;
    uint32_t* d_bits = nullptr;  // bit-parallel hard table (Nx >= 32)
    size_t bits_bytes = 0;
    uint32_t* d_V = nullptr;
    uint16_t* d_L = nullptr;
    uint16_t* d_B = nullptr;
    plan_segment* d_seg = nullptr;
    int* d_status = nullptr;
    unsigned char* d_goals = nullptr;  // goal-set search: goals, per-goal bests, result
    int goal_cap = 0;
    bool rendered = false;
    bool volumes = true;  // V and L allocated (scenes of a server hold only B)
    // maneuver-count reachability (Appendix C): hard bits, their transposed
    // shallow planes, scratch for transposed reachability and output, the
    // reachability volumes R_0 .. R_N and the list of shallow planes
    uint32_t* d_hb = nullptr;
    uint32_t* d_hbt = nullptr;
    uint32_t* d_rt = nullptr;
    uint32_t* d_ot = nullptr;
    // the second turn family's and the straights' results of a cycle, written
    // on two side streams while the first family runs, then ANDed into R_{m+1}
    uint32_t* d_x1 = nullptr;
    uint32_t* d_x2 = nullptr;
    cudaStream_t reach_side[2] = {nullptr, nullptr};
    cudaEvent_t reach_ev[3] = {nullptr, nullptr, nullptr};  // fork, join of each side stream
    uint32_t* d_reach = nullptr;
    int32_t* d_shallow = nullptr;
    std::vector<int32_t> shallow;
    int n_shallow = 0, reach_cap = 0, reach_n = 0;
    bool reach_ready = false;
    // kernel shapes of plan_sweep (plan_autotune; defaults until then)
    int turn_variant = -1, turn_grid = 0, straight_lines = 0, straight_grid = 0;
    int64_t launches = 0;
    DevGrid g{};
    nhp::QueryDesc qd{};             // this plan as one query (host copy)
    nhp::QueryDesc* d_qd = nullptr;  // ... and its device copy
    nhp::Group group() const {
        nhp::Group r{d_qd, 1, lx, lt, max_runs > 0 ? max_runs : 1};
        r.ctm = g.ctm;
        return r;
    }
    // profiling (plan_profile)
    bool prof = false;        // per-pass event timing
    bool prof_count = false;  // improved-cell counters in the sweep kernels
    unsigned long long* d_cnt = nullptr;  // improved cells [0] turn, [1] straight; [2] turn tiles with any
    struct Mark { int kind; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
    plan_profile_stats acc{};

    void* dalloc(size_t bytes) { return alloc.alloc(bytes, (void*)stream, alloc.ctx); }
    void dfree(void* p, size_t bytes) {
        if (p) alloc.free(p, bytes, (void*)stream, alloc.ctx);
    }
};

namespace nhp {
// Segments the device label walk can hold for one plan.
constexpr int kDevSegCap = 4096;
int cuda_rc(cudaError_t e);
// Record a failed CUDA call (plan_last_error) and return PLAN_ECUDA.
int cuda_fail(cudaError_t e, const char* where);
const char* last_error_text();
// Record a failed index check of the bounds-check build (plan_last_error).
void record_check_failure(int site);
bool pose_ok(const plan_s* p, plan_pose q);
int64_t cell_index(const plan_s* p, plan_pose q);
bool pose_hard(const plan_s* p, plan_pose q);
// PLAN_ERANGE when finite costs of an N-cycle sweep could reach TH.
int range_check(const plan_s* p, int n_cycles);
int range_check_layers(const plan_s* p, int layers);
// Largest non-hard obstacle value B can hold (image, direction field).
uint64_t obstacle_bound(const plan_s* p);
void set_transition(plan_s* p, const uint32_t* cin, const uint32_t* cout);
void curv4_release(plan_s* p);  // the curvature levels' buffers
void compact_release(plan_s* p);  // the Compact graph's L and R volumes
// The bounds-check build's error word (the plan's d_status[3]): after the
// work queued so far (synchronises), PLAN_EINTERNAL when an index check
// failed, reported once with its site (plan_last_error) and cleared.
int check_error_word(plan_s* p);
int check_failed(plan_s* p, int32_t site);
// Copy the plan's QueryDesc to the device (async on the plan's stream).
int upload_desc(plan_s* p);
// plan_create, optionally without the V and L volumes (a cached scene).
int create_plan(const plan_grid* grid, const plan_footprint* footprint, double turn_radius_cells,
                const plan_costs* costs, const plan_allocator* allocator, void* cuda_stream, bool volumes,
                plan_s** out);
// Host-side validity of a (start, n_cycles) sweep request: PLAN_OK, EINVAL, ERANGE.
int check_sweep(const plan_s* p, plan_pose start, int n_cycles);
}  // namespace nhp

// Return PLAN_ECUDA (recording the call) when a CUDA call fails.
#define NHP_CK(call)                                              \
    do {                                                          \
        const cudaError_t nhp_e_ = (call);                        \
        if (nhp_e_ != cudaSuccess) return nhp::cuda_fail(nhp_e_, #call); \
    } while (0)

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
    uint32_t wA, ct;
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

// Kernel launchers (each returns cudaGetLastError()).
cudaError_t launch_sparse_table(const uint16_t* img, uint16_t* table, int lx, cudaStream_t s);
cudaError_t launch_render(const DevGrid& g, const uint16_t* table, uint16_t* B, int max_runs,
                          cudaStream_t s);
// Rendering with a bit-parallel hard test (Nx >= 32): builds the per-row OR
// table `bits` ((lx+1) * Nx * Nx/32 words), writes HARD / 256 into B; with
// soft = true the maximum of the image (sparse `table`, already built) is
// then filled in for the non-hard poses.  Launches lx + 3 kernels (lx + 4
// with soft).
cudaError_t launch_render_bits(const DevGrid& g, const uint16_t* img, uint32_t* bits, uint16_t* B, bool soft,
                               const uint16_t* table, int max_runs, cudaStream_t s);
cudaError_t launch_init(const DevGrid& g, Volumes v, int64_t start, cudaStream_t s);
// Turn chains: family 0 = LEFT (beta_0, beta_3), 1 = RIGHT (beta_2, beta_1).
// First scan direction asc (1: T increasing) with maneuver mu1; if mu2 >= 0 a
// second scan in the opposite direction with maneuver mu2 follows on the same
// chains (fused pair).
cudaError_t launch_turn(const DevGrid& g, Volumes v, int family, int asc, int mu1, int mu2,
                        cudaStream_t s);
cudaError_t launch_straight(const DevGrid& g, Volumes v, int mu, cudaStream_t s);
// Label walk from goal; writes up to cap plan_segment records (goal first)
// and status[0] = count, or -1 unreachable, -3 malformed labels.
cudaError_t launch_extract(const DevGrid& g, Volumes v, int64_t goal, plan_segment* seg, int cap,
                           int* status, cudaStream_t s);

}  // namespace nhp

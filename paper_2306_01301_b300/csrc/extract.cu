// extract.cu -- goal lookup and label walk (Sections IX-X).
//
// With forward tracking (Section X), each improved cell records the maneuver
// that improved it and how many steps back along that maneuver's curve the
// segment entered.  The entry cell follows in O(1) from the curve
// parametrisation (eqs. 18, 23): move the curve coordinate back by d and
// re-apply the map.  The walk runs on the device so V never leaves HBM
// (Section IX).
#include "curve.cuh"
#include "internal.h"

namespace nhp {
namespace {

__global__ void k_extract(const QueryDesc* __restrict__ qd) {
    if (threadIdx.x != 0) return;
    const QueryDesc& Q = qd[blockIdx.x];
    const DevGrid g = Q.g;
    const Volumes vol = Q.v;
    const int64_t goal = Q.goal;
    plan_segment* seg = Q.seg;
    int32_t* status = Q.status;
    const int cap = Q.seg_cap;
    status[1] = (int32_t)(vol.V[goal] & 0xFFFFu);
    status[2] = (int32_t)(vol.V[goal] >> 16);
    if (vol.V[goal] == 0xFFFFFFFFu) { status[0] = -1; return; }
    int64_t x = goal;
    int n = 0;
    const int guard = 1 << 20;
    [[maybe_unused]] const int64_t nr = (int64_t)g.nx * g.nx * g.nt;
    while (vol.L[x] != NONE) {
        if (n >= guard) { status[0] = -3; return; }
        const uint16_t lab = vol.L[x];
        const int mu = lab >> 13, d = lab & 8191;
        if (mu > 5 || d == 0) { status[0] = -3; return; }
        const int64_t e = entry_cell(g, x, mu, d);
        if (!NHP_IN(e, nr, Q.err, 20)) { status[0] = -3; return; }
        if (n < cap) {
            plan_segment s;
            s.maneuver = mu;
            s.entry = pose_of(g, e);
            s.exit = pose_of(g, x);
            s.steps = d;
            s.cost = vol.V[x];
            seg[n] = s;
        }
        n++;
        x = e;
    }
    status[0] = vol.V[x] == 0 ? n : -3;
}

// Back-track of the bit-vector reachability (Appendix C): the fewest
// maneuvers m* to the goal is the first volume R_m whose goal bit is 0; then,
// level by level, the first maneuver in cycle order whose curve, walked
// upstream from the current cell without meeting a hard cell, reaches a cell
// of R_{m-1}, at its nearest such cell.  Warp mu scans maneuver mu 32 steps
// at a time (ballots find the first hard and the first reachable cell).
__device__ __forceinline__ bool bit_of(const uint32_t* v, int64_t c) { return (v[c >> 5] >> (c & 31)) & 1u; }

__global__ void k_reach_extract(const DevGrid g, const uint32_t* __restrict__ R, int n, int64_t words,
                                const uint32_t* __restrict__ H, int64_t goal, plan_segment* __restrict__ seg,
                                int cap, int32_t* __restrict__ status) {
    __shared__ int found_d[6];
    __shared__ int64_t found_e[6];
    __shared__ int64_t cur;
    __shared__ int mstar;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mstar = -1;
        for (int m = 0; m <= n; m++)
            if (!bit_of(R + (int64_t)m * words, goal)) { mstar = m; break; }
        cur = goal;
        status[1] = mstar;
    }
    __syncthreads();
    if (mstar < 0) {
        if (threadIdx.x == 0) status[0] = -1;
        return;
    }
    int nseg = 0;
    for (int m = mstar; m > 0; m--) {
        const int mu = warp;  // six warps, one per maneuver
        const int period = (mu == SF || mu == SB) ? g.nx : g.nt;
        const uint32_t* prev = R + (int64_t)(m - 1) * words;
        int d_found = 0;
        int64_t e_found = -1;
        for (int base = 0; base < period - 1; base += 32) {
            const int d = base + lane + 1;
            const bool ok = d < period;
            const int64_t e = ok ? entry_cell(g, cur, mu, d) : 0;
            const uint32_t hard = __ballot_sync(0xFFFFFFFFu, ok && bit_of(H, e));
            const uint32_t reach = __ballot_sync(0xFFFFFFFFu, ok && !bit_of(prev, e));
            const uint32_t before_hard = hard ? ((1u << (__ffs(hard) - 1)) - 1u) : 0xFFFFFFFFu;
            const uint32_t cand = reach & before_hard;
            if (cand) {
                const int t = __ffs(cand) - 1;
                d_found = base + t + 1;
                e_found = __shfl_sync(0xFFFFFFFFu, e, t);
                break;
            }
            if (hard) break;
        }
        if (lane == 0) {
            found_d[mu] = d_found;
            found_e[mu] = e_found;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int pick = -1;
            for (int k = 0; k < 6 && pick < 0; k++)
                if (found_d[k] > 0) pick = k;
            if (pick < 0) {
                status[0] = -3;
                cur = -1;
            } else {
                if (nseg < cap) {
                    plan_segment sgm;
                    sgm.maneuver = pick;
                    sgm.entry = pose_of(g, found_e[pick]);
                    sgm.exit = pose_of(g, cur);
                    sgm.steps = found_d[pick];
                    sgm.cost = (uint32_t)m;  // maneuvers up to the exit
                    seg[nseg] = sgm;
                }
                cur = found_e[pick];
            }
        }
        nseg++;
        __syncthreads();
        if (cur < 0) return;
    }
    if (threadIdx.x == 0) status[0] = nseg;
}

}  // namespace

cudaError_t launch_reach_extract(const DevGrid& g, const uint32_t* R, int n, int64_t words, const uint32_t* H,
                                 int64_t goal, plan_segment* seg, int cap, int32_t* status, cudaStream_t s) {
    k_reach_extract<<<1, 192, 0, s>>>(g, R, n, words, H, goal, seg, cap, status);
    return cudaGetLastError();
}

cudaError_t launch_extract(const Group& gr, cudaStream_t s) {
    k_extract<<<(unsigned)gr.nq, 32, 0, s>>>(gr.d);
    return cudaGetLastError();
}

}  // namespace nhp

// start_goal.cu -- the start state of a vehicle already under way (Section
// XII) and the goal-set search (Section IX).
//
// Start layer: each maneuver whose start entry cost is below ct is followed
// from the start pose alone before the first cycle.  Along one curve the
// value d steps ahead is the entry cost plus a prefix sum of edge costs, so
// one block walks a curve in chunks of blockDim steps: every thread computes
// its step's cell in closed form and its edge cost, a block-wide inclusive
// scan adds them up, and the chunk total carries into the next chunk.  The
// maneuvers go one after the other in cycle order (a cell on two of the
// curves keeps the first strictly cheaper value).
//
// Goal search: one block per goal scores every pose of its box, V + bias +
// w_xy (|dx| + |dy|) + w_theta |dtheta|, and reduces to the lexicographic
// minimum of (score, goal, position in the box: the ideal pose first, then
// raster order); a second one-block kernel reduces over the goals and writes
// the chosen cell into the query's descriptor on the device, where the label
// walk reads it -- the value volume never leaves HBM.
#include "curve.cuh"
#include "internal.h"

namespace nhp {
namespace {

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__global__ void __launch_bounds__(1024) k_seed(const QueryDesc* __restrict__ qd, StartEntry entry) {
    __shared__ uint64_t wsum[32];
    const QueryDesc& Q = qd[0];
    const DevGrid g = Q.g;
    const Volumes vol = Q.v;
    const int64_t start = Q.start;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int mu = 0; mu < 6; mu++) {  // maneuver ids are the cycle order
        const uint32_t cout = pick6(g.cout, mu), cin = pick6(g.ctm, mu) - cout;
        if (entry.e[mu] >= cin) continue;
        const bool turn = mu != SF && mu != SB;
        const int n = turn ? g.nt : g.nx;  // the curve closes after n steps
        const uint32_t w = turn ? g.wA : g.plane[start >> (2 * g.lx)].wS;
        uint64_t carry = entry.e[mu];  // value at the chunk's first cell
        for (int base = 0; base < n - 1; base += blockDim.x) {
            const int k = base + threadIdx.x;  // this thread's step leaves cell k and reaches cell k + 1
            uint64_t e = 0;
            int64_t to = -1;
            if (k < n - 1) {
                const uint16_t b = vol.B[entry_cell(g, start, mu, -k)];
                e = b == HARD ? TH : (w * (uint32_t)b) >> 8;
                to = entry_cell(g, start, mu, -(k + 1));
            }
            const uint64_t x = warp_incl_scan(e, lane);
            if (lane == 31) wsum[wid] = x;
            __syncthreads();
            if (wid == 0) {
                const uint64_t t = warp_incl_scan(lane < nw ? wsum[lane] : 0, lane);
                if (lane < nw) wsum[lane] = t;
            }
            __syncthreads();
            // back in the transition state after the maneuver's leaving edge
            const uint64_t run = carry + x + (wid ? wsum[wid - 1] : 0) + cout;
            // an edge left a hard cell (cost TH) or the value is not finite
            if (to >= 0 && run < TH && vol.B[to] != HARD && run < vol.V[to]) {
                vol.V[to] = (uint32_t)run;
                vol.L[to] = (uint16_t)((mu << 13) | (k + 1));
            }
            carry += wsum[nw - 1];
            __syncthreads();  // wsum is rewritten by the next chunk
        }
        __syncthreads();  // the next maneuver compares against these values
    }
}

struct Best {
    uint64_t score, rank;
    int64_t cell;
};

__device__ __forceinline__ bool better(uint64_t s, uint64_t r, uint64_t bs, uint64_t br) {
    return s < bs || (s == bs && r < br);
}

// Lexicographic minimum over the block; thread 0 returns it.
__device__ Best block_min(Best b) {
    __shared__ Best sb[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint64_t s = __shfl_down_sync(0xFFFFFFFFu, b.score, o);
        const uint64_t r = __shfl_down_sync(0xFFFFFFFFu, b.rank, o);
        const int64_t c = __shfl_down_sync(0xFFFFFFFFu, b.cell, o);
        if (better(s, r, b.score, b.rank)) b = Best{s, r, c};
    }
    if (lane == 0) sb[wid] = b;
    __syncthreads();
    if (wid == 0) {
        b = lane < nw ? sb[lane] : Best{~0ull, ~0ull, -1};
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const uint64_t s = __shfl_down_sync(0xFFFFFFFFu, b.score, o);
            const uint64_t r = __shfl_down_sync(0xFFFFFFFFu, b.rank, o);
            const int64_t c = __shfl_down_sync(0xFFFFFFFFu, b.cell, o);
            if (better(s, r, b.score, b.rank)) b = Best{s, r, c};
        }
    }
    return b;
}

__global__ void __launch_bounds__(256) k_goal_box(const QueryDesc* __restrict__ qd, const plan_goal* __restrict__ goals,
                                                  GoalBest* __restrict__ out) {
    const int gi = blockIdx.x;
    const plan_goal G = goals[gi];
    const DevGrid g = qd[0].g;
    const uint32_t* V = qd[0].v.V;
    const int side = 2 * G.radius_xy + 1, tside = 2 * G.radius_theta + 1;
    const int64_t box = (int64_t)side * side * tside;
    Best b{~0ull, ~0ull, -1};
    for (int64_t q = threadIdx.x; q <= box; q += blockDim.x) {
        int dx = 0, dy = 0, dt = 0;  // q = 0: the ideal pose; q >= 1: raster position q - 1
        if (q > 0) {
            int64_t r = q - 1;
            dx = (int)(r % side) - G.radius_xy;
            r /= side;
            dy = (int)(r % side) - G.radius_xy;
            dt = (int)(r / side) - G.radius_theta;
        }
        const int x = G.pose.x + dx, y = G.pose.y + dy;
        if (x < 0 || x >= g.nx || y < 0 || y >= g.nx) continue;  // the grid does not wrap
        const uint32_t v = V[cell_of(g, x, y, G.pose.theta + dt)];
        if (v == 0xFFFFFFFFu) continue;
        const uint64_t s = (uint64_t)v + G.bias + (uint64_t)G.w_xy * (uint64_t)(abs(dx) + abs(dy)) +
                           (uint64_t)G.w_theta * (uint64_t)abs(dt);
        const uint64_t r = ((uint64_t)gi << 40) | (uint64_t)q;
        if (better(s, r, b.score, b.rank)) b = Best{s, r, cell_of(g, x, y, G.pose.theta + dt)};
    }
    b = block_min(b);
    if (threadIdx.x == 0) {
        out[gi].score = b.score;
        out[gi].rank = b.rank;
        out[gi].cell = b.cell;
    }
}

__global__ void __launch_bounds__(256) k_goal_pick(QueryDesc* __restrict__ qd, const GoalBest* __restrict__ per_goal,
                                                   int n, GoalBest* __restrict__ result) {
    Best b{~0ull, ~0ull, -1};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const GoalBest e = per_goal[i];
        if (e.cell >= 0 && better(e.score, e.rank, b.score, b.rank)) b = Best{e.score, e.rank, e.cell};
    }
    b = block_min(b);
    if (threadIdx.x == 0) {
        result->score = b.score;
        result->rank = b.rank;
        result->cell = b.cell;
        if (b.cell >= 0) qd[0].goal = b.cell;  // the label walk starts here
    }
}

}  // namespace

cudaError_t launch_seed(const QueryDesc* qd, const StartEntry& entry, cudaStream_t s) {
    k_seed<<<1, 1024, 0, s>>>(qd, entry);
    return cudaGetLastError();
}

cudaError_t launch_goal_search(QueryDesc* qd, const plan_goal* goals, int n, GoalBest* per_goal, GoalBest* result,
                               cudaStream_t s) {
    k_goal_box<<<(unsigned)n, 256, 0, s>>>(qd, goals, per_goal);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_goal_pick<<<1, 256, 0, s>>>(qd, per_goal, n, result);
    return cudaGetLastError();
}

}  // namespace nhp

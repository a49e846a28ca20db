// curve.cuh -- closed-form positions along the maneuver curves.
//
// A pose's cell, the pose of a cell, and the cell d steps back along a
// maneuver's curve (d < 0: forward) straight from the curve parametrisation
// (turns: chain coordinates and the beta table of eq. 18; straights: line
// coordinates and the shear table of eqs. 22-23).
#pragma once
#include "internal.h"

namespace nhp {

__device__ __forceinline__ plan_pose pose_of(const DevGrid& g, int64_t c) {
    plan_pose p;
    p.x = (int)(c & g.mx);
    p.y = (int)((c >> g.lx) & g.mx);
    p.theta = (int)(c >> (2 * g.lx));
    return p;
}

__device__ __forceinline__ int64_t cell_of(const DevGrid& g, int i, int j, int T) {
    return (int64_t)(i & g.mx) + ((int64_t)(j & g.mx) << g.lx) + ((int64_t)(T & g.mt) << (2 * g.lx));
}

// Entry cell of a segment of maneuver mu that reached cell c after d steps
// (with d < 0, the cell -d steps ahead of c).
__device__ __forceinline__ int64_t entry_cell(const DevGrid& g, int64_t c, int mu, int d) {
    const int i = (int)(c & g.mx), j = (int)((c >> g.lx) & g.mx), T = (int)(c >> (2 * g.lx));
    if (mu == SF || mu == SB) {
        const PlaneInfo pi = g.plane[T];
        const int dir = mu == SF ? pi.jsign : -pi.jsign;  // direction of y' along the sweep
        const int16_t* bs = g.bshear + (int64_t)T * g.nx;
        if (pi.iflag == 0) {  // cell (y', x' + B(y'))
            const int yq = i, xq = (j - bs[yq]) & g.mx;
            const int ye = (yq - dir * d) & g.mx;
            return cell_of(g, ye, xq + bs[ye], T);
        } else {              // cell (x' + B(y'), y')
            const int yq = j, xq = (i - bs[yq]) & g.mx;
            const int ye = (yq - dir * d) & g.mx;
            return cell_of(g, xq + bs[ye], ye, T);
        }
    }
    const bool left = mu == LF || mu == LB;
    const int dir = (mu == LF || mu == RB) ? 1 : -1;  // heading step along the sweep
    const int4 b = g.beta4[T];
    const int bx = left ? b.x : b.z, by = left ? b.y : b.w;
    const int xq = i - bx, yq = j - by;  // chain coordinates (mod Nx)
    const int Te = (T - dir * d) & g.mt;
    const int4 be = g.beta4[Te];
    return cell_of(g, xq + (left ? be.x : be.z), yq + (left ? be.y : be.w), Te);
}

// Cell of turn chain (xq, yq) of maneuver mu at step q of a walk that starts
// at heading 0: LF and RB step the heading up, LB and RF down (eq. 18).
__device__ __forceinline__ int64_t turn_chain_cell(const DevGrid& g, int mu, int xq, int yq, int q) {
    const bool left = mu == LF || mu == LB;
    const int step = (mu == LF || mu == RB) ? 1 : -1;
    const int T = (step * q) & g.mt;
    const int4 b = __ldg(&g.beta4[T]);
    return cell_of(g, xq + (left ? b.x : b.z), yq + (left ? b.y : b.w), T);
}

// Cell of straight line xq of heading T at step q of a walk from its wall
// cell y' = 0 in the maneuver's direction (eqs. 23-24).
__device__ __forceinline__ int64_t line_cell(const DevGrid& g, const PlaneInfo& pi, int mu, int T, int xq, int q) {
    const int dir = (mu == SF ? pi.jsign : -pi.jsign) > 0 ? 1 : -1;
    const int y = (dir * q) & g.mx;
    const int col = (xq + g.bshear[(int64_t)T * g.nx + y]) & g.mx;
    return pi.iflag ? cell_of(g, col, y, T) : cell_of(g, y, col, T);
}

}  // namespace nhp

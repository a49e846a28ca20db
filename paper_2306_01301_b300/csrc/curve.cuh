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

}  // namespace nhp

// extract.cu -- goal lookup and label walk (Sections IX-X).
//
// With forward tracking (Section X), each improved cell records the maneuver
// that improved it and how many steps back along that maneuver's curve the
// segment entered.  The entry cell follows in O(1) from the curve
// parametrisation (eqs. 18, 23): move the curve coordinate back by d and
// re-apply the map.  The walk runs on the device so V never leaves HBM
// (Section IX).
#include "internal.h"

namespace nhp {
namespace {

__device__ plan_pose pose_of(const DevGrid& g, int64_t c) {
    plan_pose p;
    p.x = (int)(c & g.mx);
    p.y = (int)((c >> g.lx) & g.mx);
    p.theta = (int)(c >> (2 * g.lx));
    return p;
}

__device__ int64_t cell_of(const DevGrid& g, int i, int j, int T) {
    return (int64_t)(i & g.mx) + ((int64_t)(j & g.mx) << g.lx) + ((int64_t)(T & g.mt) << (2 * g.lx));
}

// Entry cell of a segment of maneuver mu that reached cell c after d steps.
__device__ int64_t entry_cell(const DevGrid& g, int64_t c, int mu, int d) {
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
    while (vol.L[x] != NONE) {
        if (n >= guard) { status[0] = -3; return; }
        const uint16_t lab = vol.L[x];
        const int mu = lab >> 13, d = lab & 8191;
        if (mu > 5 || d == 0) { status[0] = -3; return; }
        const int64_t e = entry_cell(g, x, mu, d);
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

}  // namespace

cudaError_t launch_extract(const Group& gr, cudaStream_t s) {
    k_extract<<<(unsigned)gr.nq, 32, 0, s>>>(gr.d);
    return cudaGetLastError();
}

}  // namespace nhp

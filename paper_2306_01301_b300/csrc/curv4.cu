// curv4.cu -- the 4D generalisation of Appendix F: curvature levels.
//
// The value function of the transition state lives on 2M+1 copies of the 3D
// volume, one per curvature level kappa = -M .. M (curvature kappa / (M R)).
// The 3D turns run on the steering-limit levels (left at +M, right at -M),
// the straights on kappa = 0, and clothoids (the extremal steering-rate
// controls) move one level per step.  A clothoid chain is named by its pose
// (x0, y0, theta0) at kappa = 0; on each level it is translated by a rounded
// clothoid integral that depends only on (theta0, kappa) and rotated by a
// heading offset that depends only on kappa (Appendix F), so for one level
// the map is a permutation of the 3D cells and consecutive threads (x0) touch
// consecutive cells.  Clothoid chains are open (the curvature runs from one
// limit to the other): one pass from the first level.  Labels are
// (maneuver << 12) | d.
//
// When the finite costs stay below TH (checked on the host), the 3D layers
// are passes of the plain turn and straight kernels on their level, and the
// clothoid layer (k4_clothoid_th) carries four chains per thread in 32-bit
// arithmetic.  Otherwise every layer is one thread per chain with saturating
// arithmetic, the 3D maneuvers walking their cyclic chains twice on their
// level, as the paper's two loops.
#include <algorithm>
#include <cmath>
#include <vector>

#include "curve.cuh"
#include "plan_state.h"

namespace nhp {
namespace {

constexpr uint32_t INF32 = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t sadd(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a + b;
    return s >= INF32 ? INF32 : (uint32_t)s;
}

struct Carry {
    uint32_t v = INF32;
    int qe = 0;
};

// Store where the carried value (after the leaving edge) improves the cell,
// enter at the cell, move on over the edge leaving it.
__device__ __forceinline__ void step4(Carry& s, int64_t c4, int64_t c3, int q, bool store, int mu, uint32_t w,
                                      const Layer4& a) {
    const uint16_t b = a.B[c3];
    const bool hard = b == HARD;
    const uint32_t u = a.V[c4];  // before this layer: only this thread writes the cell
    if (store) {
        const uint32_t cand = hard ? INF32 : sadd(s.v, a.cout);
        if (cand < u) {
            a.V[c4] = cand;
            a.L[c4] = (uint16_t)((mu << 12) | (q - s.qe));
        }
    }
    const uint32_t t = hard ? INF32 : sadd(u, a.cin);
    if (t < s.v) {
        s.v = t;
        s.qe = q;
    }
    s.v = sadd(s.v, hard ? INF32 : (uint32_t)(((uint64_t)w * b) >> 8));
}

__global__ void __launch_bounds__(256) k4_turn(const Layer4 a, int mu, int level) {
    const DevGrid& g = a.g;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t chain = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= nxy) return;
    const int xq = (int)(chain & g.mx), yq = (int)(chain >> g.lx);
    const int n = g.nt;
    const int64_t base = (int64_t)level * a.nr;
    Carry s;
    for (int q = 0; q < 2 * n; q++) {
        const int64_t c = turn_chain_cell(g, mu, xq, yq, q);
        step4(s, base + c, c, q, q >= n, mu, a.w, a);
    }
}

__global__ void __launch_bounds__(256) k4_straight(const Layer4 a, int mu, int level) {
    const DevGrid& g = a.g;
    const int xq = blockIdx.x * blockDim.x + threadIdx.x;
    if (xq >= g.nx) return;
    const int T = blockIdx.y;
    const PlaneInfo pi = g.plane[T];
    const int n = g.nx;
    const int64_t base = (int64_t)level * a.nr;
    Carry s;
    for (int q = 0; q < 2 * n; q++) {
        const int64_t c = line_cell(g, pi, mu, T, xq, q);
        step4(s, base + c, c, q, q >= n, mu, pi.wS, a);
    }
}

__device__ __forceinline__ int family_of(int mu) { return (mu == PLAN_C1F || mu == PLAN_C1B) ? 0 : 1; }
__device__ __forceinline__ int dir_of(int mu) { return (mu == PLAN_C1F || mu == PLAN_C2B) ? 1 : -1; }

// 3D cell of clothoid family f's chain (x0, y0, T0) on level K.
__device__ __forceinline__ int64_t chain4(const Layer4& a, int f, int x0, int y0, int T0, int K) {
    const int64_t at = ((int64_t)f * a.nk + K) * a.g.nt + T0;
    return cell_of(a.g, x0 + a.dx[at], y0 + a.dy[at], T0 + a.dth[f * a.nk + K]);
}

__global__ void __launch_bounds__(256) k4_clothoid(const Layer4 a, int mu) {
    const DevGrid& g = a.g;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // chain = its kappa = 0 pose
    if (t >= a.nr) return;
    const int x0 = (int)(t & g.mx), y0 = (int)((t >> g.lx) & g.mx), T0 = (int)(t >> (2 * g.lx));
    const int f = family_of(mu), dir = dir_of(mu);
    Carry s;
    for (int q = 0; q < a.nk; q++) {
        const int K = dir > 0 ? q : a.nk - 1 - q;
        const int64_t c = chain4(a, f, x0, y0, T0, K);
        step4(s, (int64_t)K * a.nr + c, c, q, true, mu, a.w, a);
    }
}

// The clothoid layer in the value domain of the plain sweeps (finite costs
// below TH, checked on the host): 32-bit cell offsets within a level, no
// saturation, the transition costs added on entering.  A hard cell reads as
// 0, so nothing is stored there, and the TH on its leaving edge cancels an
// entry there before it reaches another cell.  Same values and labels as
// the saturating walk.
// Each thread carries kClothoidRows chains of one heading and column, rows
// y0 + j Nx / kClothoidRows: a level's table entry, x and heading are the
// same for all of them.
constexpr int kClothoidRows = 4;

__global__ void __launch_bounds__(256) k4_clothoid_th(const Layer4 a, int mu) {
    constexpr int J = kClothoidRows;
    const DevGrid& g = a.g;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nr / J) return;
    const int lq = g.lx - 2;  // log2(Nx / J)
    const int x0 = (int)(t & g.mx), yb = (int)((t >> g.lx) & ((1 << lq) - 1)), T0 = (int)(t >> (g.lx + lq));
    const int f = family_of(mu), dir = dir_of(mu);
    // the chains' first level, then one level per step in direction dir
    const int K0 = dir > 0 ? 0 : a.nk - 1;
    const int64_t lstep = dir > 0 ? a.nr : -a.nr;
    uint32_t* Vk = a.V + (int64_t)K0 * a.nr;
    uint16_t* Lk = a.L + (int64_t)K0 * a.nr;
    const int32_t* dxy = a.dxy + ((int64_t)f * a.nk + K0) * g.nt + T0;
    const int32_t* dth = a.dth + f * a.nk + K0;
    const int dxy_step = dir * g.nt;
    const uint32_t ct = a.cin + a.cout, tag = (uint32_t)mu << 12;
    uint32_t v[J];
    int pv[J];
#pragma unroll
    for (int j = 0; j < J; j++) { v[j] = 0xFFFFFFFFu; pv[j] = 0; }
    for (int q = 0; q < a.nk; q++) {
        const int32_t o = __ldg(dxy);
        const uint32_t x = (uint32_t)(x0 + (int16_t)(o & 0xFFFF)) & (uint32_t)g.mx;
        const uint32_t T = (uint32_t)(T0 + __ldg(dth)) & (uint32_t)g.mt;
        const uint32_t base = x | (T << (2 * g.lx));
        const int dy = o >> 16;
#pragma unroll
        for (int j = 0; j < J; j++) {
            const uint32_t y = (uint32_t)(yb + (j << lq) + dy) & (uint32_t)g.mx;
            const uint32_t c = base | (y << g.lx);
            if (!NHP_IN((int64_t)(dir > 0 ? q : a.nk - 1 - q) * a.nr + c, (int64_t)a.nk * a.nr, a.err, 38)) continue;
            const uint16_t b = __ldg(a.B + c);
            const bool hard = b == HARD;
            const uint32_t u = hard ? 0u : min(Vk[c], TH);
            if (v[j] < u) {
                Vk[c] = v[j];
                Lk[c] = (uint16_t)(tag | (uint32_t)(q - pv[j]));
            }
            const uint32_t tt = u + ct;
            if (tt < v[j]) { v[j] = tt; pv[j] = q; }
            v[j] += hard ? TH : (uint32_t)(((uint64_t)a.w * b) >> 8);
        }
        Vk += lstep;
        Lk += lstep;
        dxy += dxy_step;
        dth += dir;
    }
}

__global__ void k4_init(uint32_t* V, uint16_t* L, int64_t n4, int64_t start4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        V[i] = i == start4 ? 0u : INF32;
        L[i] = NONE;
    }
}

// Entry (4D cell) of a segment of maneuver mu reaching 4D cell x after d steps.
__device__ int64_t entry4(const Layer4& a, int64_t x, int mu, int d) {
    const int K = (int)(x / a.nr);
    const int64_t c = x - (int64_t)K * a.nr;
    if (mu < 6) return (int64_t)K * a.nr + entry_cell(a.g, c, mu, d);
    const int f = family_of(mu), Ke = K - dir_of(mu) * d;
    if (Ke < 0 || Ke >= a.nk) return -1;
    const int i = (int)(c & a.g.mx), j = (int)((c >> a.g.lx) & a.g.mx), T = (int)(c >> (2 * a.g.lx));
    const int T0 = (T - a.dth[f * a.nk + K]) & a.g.mt;
    const int64_t at = ((int64_t)f * a.nk + K) * a.g.nt + T0;
    return (int64_t)Ke * a.nr + chain4(a, f, i - a.dx[at], j - a.dy[at], T0, Ke);
}

__device__ void pose4(const Layer4& a, int64_t x, plan_pose* p, int32_t* level) {
    const int K = (int)(x / a.nr);
    *p = pose_of(a.g, x - (int64_t)K * a.nr);
    *level = K - (a.nk - 1) / 2;
}

// status: [0] segments or -1 unreachable / -3 malformed, [1] V(goal)
__global__ void k4_extract(const Layer4 a, int64_t goal, plan_segment4* seg, int cap, int32_t* status) {
    if (threadIdx.x != 0) return;
    status[1] = (int32_t)a.V[goal];
    if (a.V[goal] == INF32) { status[0] = -1; return; }
    int64_t x = goal;
    int n = 0;
    while (a.L[x] != NONE) {
        if (n >= (1 << 20)) { status[0] = -3; return; }
        const int mu = a.L[x] >> 12, d = a.L[x] & 4095;
        if (mu > 9 || d == 0) { status[0] = -3; return; }
        const int64_t e = entry4(a, x, mu, d);
        if (e < 0) { status[0] = -3; return; }
        if (n < cap) {
            plan_segment4 s;
            s.maneuver = mu;
            pose4(a, e, &s.entry, &s.entry_level);
            pose4(a, x, &s.exit, &s.exit_level);
            s.steps = d;
            s.cost = a.V[x];
            seg[n] = s;
        }
        n++;
        x = e;
    }
    status[0] = a.V[x] == 0 ? n : -3;
}

}  // namespace

cudaError_t launch4_init(uint32_t* V, uint16_t* L, int64_t n4, int64_t start4, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((n4 + 255) / 256, 148 * 16);
    k4_init<<<(unsigned)blocks, 256, 0, s>>>(V, L, n4, start4);
    return cudaGetLastError();
}

cudaError_t launch4_layer(const Layer4& a, int mu, int level, cudaStream_t s) {
    if (mu >= PLAN_C1F) {
        if (a.th && a.g.lx >= 2) k4_clothoid_th<<<(unsigned)((a.nr / kClothoidRows + 255) / 256), 256, 0, s>>>(a, mu);
        else k4_clothoid<<<(unsigned)((a.nr + 255) / 256), 256, 0, s>>>(a, mu);
    } else if (mu == SF || mu == SB) {
        k4_straight<<<dim3((unsigned)((a.g.nx + 255) / 256), (unsigned)a.g.nt), 256, 0, s>>>(a, mu, level);
    } else {
        const int64_t chains = (int64_t)a.g.nx * a.g.nx;
        k4_turn<<<(unsigned)((chains + 255) / 256), 256, 0, s>>>(a, mu, level);
    }
    return cudaGetLastError();
}

cudaError_t launch4_extract(const Layer4& a, int64_t goal4, plan_segment4* seg, int cap, int32_t* status,
                            cudaStream_t s) {
    k4_extract<<<1, 32, 0, s>>>(a, goal4, seg, cap, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host
namespace {

constexpr double kPi = 3.14159265358979323846;

// cos (xy = 0) or sin (xy = 1) of theta0 +- a sigma^2 (family f = 0: +)
double clothoid_value(int f, int xy, double th0, double a, double sg) {
    const double ang = f == 0 ? th0 + a * sg * sg : th0 - a * sg * sg;
    return xy == 0 ? std::cos(ang) : std::sin(ang);
}

// The clothoid's displacement integral over [0, s]: composite Simpson, n even.
double clothoid_integral(int f, int xy, double th0, double a, double s, int n) {
    const double h = s / n;
    double acc = clothoid_value(f, xy, th0, a, 0.0) + clothoid_value(f, xy, th0, a, s);
    for (int i = 1; i < n; i++) acc += (i & 1 ? 4.0 : 2.0) * clothoid_value(f, xy, th0, a, i * h);
    return acc * h / 3.0;
}

// Tables of the two clothoid families (Appendix F's per-level map): level K
// (kappa = K - M) at arc length s = kappa L (rising) or -kappa L (falling)
// from the chain's kappa = 0 pose, heading offset +-a s^2 with a = 1 / (2 M R
// L), translation (X, Y) the integrals of cos and sin of the heading,
// rounded half away from zero, headings in steps of 2 pi / N_theta.
void build_clothoids(plan_s* p) {
    const int M = p->curv_M, nk = p->curv_nk, nt = p->nt;
    const double L = p->curv_L, a = 1.0 / (2.0 * M * p->R * L);
    p->cdx.assign((size_t)2 * nk * nt, 0);
    p->cdy.assign((size_t)2 * nk * nt, 0);
    p->cdth.assign((size_t)2 * nk, 0);
    for (int f = 0; f < 2; f++)
        for (int K = 0; K < nk; K++) {
            const int kap = K - M;
            const double s = f == 0 ? kap * L : -kap * L;
            const double psi = f == 0 ? a * s * s : -a * s * s;
            p->cdth[(size_t)f * nk + K] = (int32_t)std::lround(psi * nt / (2.0 * kPi));
            if (kap == 0) continue;
            const int intervals = 64 * (kap < 0 ? -kap : kap);
            for (int T0 = 0; T0 < nt; T0++) {
                const double th0 = 2.0 * kPi * T0 / nt;
                const size_t at = ((size_t)f * nk + K) * nt + T0;
                p->cdx[at] = (int16_t)std::lround(clothoid_integral(f, 0, th0, a, s, intervals));
                p->cdy[at] = (int16_t)std::lround(clothoid_integral(f, 1, th0, a, s, intervals));
            }
        }
}

// Whether every finite value of an N-cycle sweep over the levels stays below
// TH (each layer adds at most one segment: its transition cost and at most
// max(Nx, N_theta) - 1 edges on a 3D layer, N_levels - 1 on a clothoid), so
// that the 3D layers may run on the plain sweep kernels, which clamp there.
bool levels_in_range(const plan_s* p, int n_cycles) {
    const double b_max = (double)obstacle_bound(p);
    uint64_t ct = 0;
    for (int k = 0; k < 6; k++) ct = std::max<uint64_t>(ct, (uint64_t)p->cin[k] + p->cout[k]);
    const double layer3 = (double)ct + (double)(std::max(p->nx, p->nt) - 1) * std::floor((double)p->w_max * b_max / 256.0);
    const double layerc = (double)p->curv_ct + (double)(p->curv_nk - 1) * std::floor((double)p->curv_w * b_max / 256.0);
    return (double)n_cycles * (6.0 * layer3 + 4.0 * layerc) < (double)TH;
}

Layer4 layer_args(const plan_s* p) {
    Layer4 a{};
    a.g = p->g;
    a.B = p->d_B;
    a.V = p->d_V4;
    a.L = p->d_L4;
    a.nr = p->nr;
    a.nk = p->curv_nk;
    a.dx = p->d_cdx;
    a.dy = p->d_cdy;
    a.dth = p->d_cdth;
    a.dxy = p->d_cdxy;
    a.err = p->d_status + 3;
    return a;
}

}  // namespace

void curv4_release(plan_s* p) {
    const size_t n4 = (size_t)p->nr * p->curv_nk;
    p->dfree(p->d_V4, n4 * 4);
    p->dfree(p->d_L4, n4 * 2);
    p->dfree(p->d_cdx, p->cdx.size() * 2);
    p->dfree(p->d_cdy, p->cdy.size() * 2);
    p->dfree(p->d_cdth, p->cdth.size() * 4);
    p->dfree(p->d_cdxy, p->cdx.size() * 4);
    p->d_cdxy = nullptr;
    p->dfree(p->d_qd4, 3 * sizeof(QueryDesc));
    p->d_qd4 = nullptr;
    p->d_V4 = nullptr;
    p->d_L4 = nullptr;
    p->d_cdx = p->d_cdy = nullptr;
    p->d_cdth = nullptr;
    p->cdx.clear();
    p->cdy.clear();
    p->cdth.clear();
    p->curv_M = p->curv_nk = 0;
    p->vol4_kind = VOL4_NONE;
}

}  // namespace nhp

using namespace nhp;

extern "C" {

int plan_set_curvature_levels(plan_t* p, int levels_per_side, double arc_per_level, uint32_t clothoid_cost) {
    if (!p || levels_per_side < 0 || levels_per_side > 1000) return PLAN_EINVAL;
    curv4_release(p);
    if (levels_per_side == 0) return PLAN_OK;
    if (!(arc_per_level > 0.0) || arc_per_level > 4.0 || clothoid_cost >= (1u << 28) || p->nx > 2048 ||
        p->nt > 2048)
        return PLAN_EINVAL;
    if (!p->volumes) return PLAN_ESTATE;
    p->curv_M = levels_per_side;
    p->curv_nk = 2 * levels_per_side + 1;
    p->curv_L = arc_per_level;
    p->curv_ct = clothoid_cost;
    p->curv_w = (uint32_t)std::lround((double)p->costs.step_scale * arc_per_level);
    if (p->curv_w == 0) p->curv_w = 1;
    build_clothoids(p);
    const size_t n4 = (size_t)p->nr * p->curv_nk;
    p->d_V4 = (uint32_t*)p->dalloc(n4 * 4);
    p->d_L4 = (uint16_t*)p->dalloc(n4 * 2);
    p->d_cdx = (int16_t*)p->dalloc(p->cdx.size() * 2);
    p->d_cdy = (int16_t*)p->dalloc(p->cdy.size() * 2);
    p->d_cdth = (int32_t*)p->dalloc(p->cdth.size() * 4);
    p->d_qd4 = (QueryDesc*)p->dalloc(3 * sizeof(QueryDesc));
    p->d_cdxy = (int32_t*)p->dalloc(p->cdx.size() * 4);
    if (!p->d_V4 || !p->d_L4 || !p->d_cdx || !p->d_cdy || !p->d_cdth || !p->d_qd4 || !p->d_cdxy) {
        curv4_release(p);
        return PLAN_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_cdx, p->cdx.data(), p->cdx.size() * 2, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_cdy, p->cdy.data(), p->cdy.size() * 2, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_cdth, p->cdth.data(), p->cdth.size() * 4, cudaMemcpyHostToDevice, p->stream);
    std::vector<int32_t> dxy(p->cdx.size());
    for (size_t i = 0; i < dxy.size(); i++)
        dxy[i] = (int32_t)(((uint32_t)(uint16_t)p->cdy[i] << 16) | (uint32_t)(uint16_t)p->cdx[i]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_cdxy, dxy.data(), dxy.size() * 4, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // the host tables may change with the next call
    if (e != cudaSuccess) {
        curv4_release(p);  // no half-built levels
        return cuda_fail(e, "plan_set_curvature_levels");
    }
    return PLAN_OK;
}

int plan_sweep4(plan_t* p, plan_pose start, int start_level, int n_cycles) {
    if (!p || n_cycles < 0 || n_cycles > 4096 || !pose_ok(p, start)) return PLAN_EINVAL;
    if (!p->curv_nk || !p->rendered) return PLAN_ESTATE;
    if (start_level < -p->curv_M || start_level > p->curv_M || pose_hard(p, start)) return PLAN_EINVAL;
    // a cycle: C1F, C2F, C1B, C2B, then the 3D order LF SF RB RF SB LB
    static const int order[10] = {PLAN_C1F, PLAN_C2F, PLAN_C1B, PLAN_C2B, LF, SF, RB, RF, SB, LB};
    Layer4 a = layer_args(p);
    cudaStream_t s = p->stream;
    p->vol4_kind = VOL4_NONE;
    const int64_t start4 = (int64_t)(start_level + p->curv_M) * p->nr + cell_index(p, start);
    int rc = cuda_rc(launch4_init(p->d_V4, p->d_L4, p->nr * p->curv_nk, start4, s));
    p->launches++;
    if (rc == PLAN_OK && levels_in_range(p, n_cycles)) {
        a.th = true;
        // The 3D layers are plain turn and straight layers on one level: the
        // plain sweep kernels run them, one descriptor per level, each a
        // one-cycle query whose passes 0 .. 4 are LF, SF, {RB, RF}, SB and a
        // lone LB (the next cycle's clothoids come between LB and LF).
        QueryDesc q[3];
        const int lvl[3] = {p->curv_nk - 1, p->curv_M, 0};  // left limit, kappa = 0, right limit
        for (int i = 0; i < 3; i++) {
            q[i] = p->qd;
            q[i].v = Volumes{p->d_V4 + (int64_t)lvl[i] * p->nr, p->d_L4 + (int64_t)lvl[i] * p->nr, p->d_B, nullptr};
            q[i].n_cycles = 1;
            q[i].pass = -1;
            q[i].conv = nullptr;
            q[i].mu_shift = 12;
        }
        rc = cuda_rc(cudaMemcpyAsync(p->d_qd4, q, sizeof(q), cudaMemcpyHostToDevice, s));
        // the host copy must outlive the copy
        if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(s));
        static const int pass_desc[5] = {0, 1, 2, 1, 0};
        for (int c = 0; c < n_cycles && rc == PLAN_OK; c++) {
            for (int l = 0; l < 4 && rc == PLAN_OK; l++) {
                a.w = p->curv_w;
                a.cin = p->curv_ct;
                a.cout = 0;
                rc = cuda_rc(launch4_layer(a, order[l], -1, s));
                p->launches++;
            }
            for (int pass = 0; pass < 5 && rc == PLAN_OK; pass++) {
                Group gr{p->d_qd4 + pass_desc[pass], 1, p->lx, p->lt, p->max_runs > 0 ? p->max_runs : 1};
                gr.ctm = p->g.ctm;
                const bool turn = pass_is_turn(pass);
                gr.grid = turn ? p->turn_grid : p->straight_grid;
                rc = cuda_rc(turn ? launch_turn(gr, pass, p->turn_variant, s)
                                  : launch_straight(gr, pass, p->straight_lines, s));
                p->launches++;
            }
        }
        if (rc == PLAN_OK) p->vol4_kind = VOL4_SWEPT;
        return rc;
    }
    for (int l = 0; l < 10 * n_cycles && rc == PLAN_OK; l++) {
        const int mu = order[l % 10];
        int level = p->curv_M;  // straights
        if (mu >= PLAN_C1F) {
            a.w = p->curv_w;
            a.cin = p->curv_ct;
            a.cout = 0;
            level = -1;
        } else {
            a.w = p->wA;  // the straights take their plane's weight instead
            a.cin = p->cin[mu];
            a.cout = p->cout[mu];
            if (mu == LF || mu == LB) level = p->curv_nk - 1;
            if (mu == RF || mu == RB) level = 0;
        }
        rc = cuda_rc(launch4_layer(a, mu, level, s));
        p->launches++;
    }
    if (rc == PLAN_OK) p->vol4_kind = VOL4_SWEPT;
    return rc;
}

int plan_extract4(plan_t* p, plan_pose goal, int goal_level, plan_segment4* out, int cap, int* n_out,
                  uint32_t* cost) {
    if (!p || !n_out || !cost || cap < 0 || (cap > 0 && !out) || !pose_ok(p, goal)) return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    if (p->vol4_kind != VOL4_SWEPT) return PLAN_ESTATE;
    if (goal_level < -p->curv_M || goal_level > p->curv_M) return PLAN_EINVAL;
    const int64_t goal4 = (int64_t)(goal_level + p->curv_M) * p->nr + cell_index(p, goal);
    // the label walk reuses the plan's segment buffer: plan_segment4 is larger than plan_segment
    const int cap4 = (int)(sizeof(plan_segment) * kDevSegCap / sizeof(plan_segment4));
    NHP_CK(launch4_extract(layer_args(p), goal4, reinterpret_cast<plan_segment4*>(p->d_seg), cap4, p->d_status,
                           p->stream));
    p->launches++;
    int32_t status[4] = {0, 0, 0, 0};  // [3]: the bounds-check build's error word
    NHP_CK(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    NHP_CK(cudaStreamSynchronize(p->stream));
    if (status[3] != 0) return check_failed(p, status[3]);
    if (status[0] == -1) return PLAN_EUNREACHABLE;
    if (status[0] < 0) return PLAN_EINTERNAL;
    *cost = (uint32_t)status[1];
    *n_out = status[0];
    if (status[0] > cap || status[0] > cap4) return PLAN_ERANGE;
    if (status[0] > 0) {
        NHP_CK(cudaMemcpyAsync(out, p->d_seg, sizeof(plan_segment4) * status[0], cudaMemcpyDeviceToHost, p->stream));
        NHP_CK(cudaStreamSynchronize(p->stream));
        std::reverse(out, out + status[0]);
    }
    return PLAN_OK;
}

int plan_copy_volumes4(plan_t* p, uint32_t* V, uint16_t* L) {
    if (!p) return PLAN_EINVAL;
    if (!p->curv_nk) return PLAN_ESTATE;
    const size_t n4 = (size_t)p->nr * p->curv_nk;
    if (V) NHP_CK(cudaMemcpyAsync(V, p->d_V4, n4 * 4, cudaMemcpyDeviceToHost, p->stream));
    if (L) NHP_CK(cudaMemcpyAsync(L, p->d_L4, n4 * 2, cudaMemcpyDeviceToHost, p->stream));
    return check_error_word(p);
}

int plan_clothoid_tables(plan_t* p, int16_t* dx, int16_t* dy, int32_t* dth) {
    if (!p) return PLAN_EINVAL;
    if (!p->curv_nk) return PLAN_ESTATE;
    if (dx) std::copy(p->cdx.begin(), p->cdx.end(), dx);
    if (dy) std::copy(p->cdy.begin(), p->cdy.end(), dy);
    if (dth) std::copy(p->cdth.begin(), p->cdth.end(), dth);
    return PLAN_OK;
}

}  // extern "C"

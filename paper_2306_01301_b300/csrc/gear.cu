// gear.cu -- two gear states: forward / reverse transition vertices.
//
// The Star of Fig. 9 with its centre split in two remembers the gear of the
// last maneuver (forward: LF SF RF; reverse: LB SB RB), so a penalty can be
// charged exactly when consecutive maneuvers change gear: entering maneuver
// mu costs cost_in[mu] from its own gear's state and cost_in[mu] + pen from
// the other one; leaving costs cost_out[mu] and returns to mu's gear's
// state.  Each maneuver layer reads both states and writes its own gear's.
//
// When the finite costs stay below TH (checked on the host), turn layers run
// on the sections scan of turn_scan.cuh, RB with RF and LB with the next
// cycle's LF fused into one launch (k_gear_scan), and straight layers on the
// staged tiles of the plain straight kernel with a third tile for the other
// gear (k_gear_straight_tiled, sweep.cu).  Otherwise, and on grids the scan
// does not take, a turn layer walks every chain twice around its cycle (one
// thread per chain over N_theta headings), as the paper's two sequential
// loops do: the first loop warms the carried value up, the second stores; a
// straight layer walks each line once from its wall cell (one thread per
// line).  A cell is read once per step before its possible store, so the
// values used for entering are those before the layer (only this thread
// writes the cell, and only in the second loop); that arithmetic saturates
// at PLAN_INF.  Labels are (mu << 13) | (other << 12) | d with d <= n (a
// whole turn circle can pay off: it changes the gear state), so grids are
// limited to 2048.
#include "curve.cuh"
#include "internal.h"
#include "turn_scan.cuh"

namespace nhp {
namespace {

constexpr uint32_t INF32 = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t sadd(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a + b;
    return s >= INF32 ? INF32 : (uint32_t)s;
}

__host__ __device__ __forceinline__ int gear_of(int mu) { return (mu == LB || mu == SB || mu == RB) ? 1 : 0; }

// One step of the two-loop walk at cell c, position q of 2n.
struct Walk {
    uint32_t v = INF32;  // carried value (entered and moved, not yet left)
    int qe = 0, vo = 0;  // entry position, entered from the other gear's state
};

__device__ __forceinline__ void walk_step(Walk& s, int64_t c, int q, int n, int mu, uint32_t w,
                                          const GearLayer& a) {
    const int G = gear_of(mu);
    uint32_t* Vs = G ? a.Vr : a.Vf;
    uint16_t* Ls = G ? a.Lr : a.Lf;
    const uint32_t* Vo = G ? a.Vf : a.Vr;
    const uint16_t b = a.B[c];
    const bool hard = b == HARD;
    const uint32_t u = Vs[c];  // before this layer: only this thread writes c, below
    if (q >= n) {
        const uint32_t cand = hard ? INF32 : sadd(s.v, a.cout);
        if (cand < u) {
            Vs[c] = cand;
            Ls[c] = (uint16_t)((mu << 13) | (s.vo << 12) | (q - s.qe));
        }
    }
    const uint32_t ts = hard ? INF32 : sadd(u, a.cin);
    const uint32_t to = hard ? INF32 : sadd(sadd(Vo[c], a.cin), a.pen);
    const int oth = to < ts;
    const uint32_t t = oth ? to : ts;
    if (t < s.v) {
        s.v = t;
        s.qe = q;
        s.vo = oth;
    }
    s.v = sadd(s.v, hard ? INF32 : (uint32_t)(((uint64_t)w * b) >> 8));
}

__global__ void __launch_bounds__(256) k_gear_turn(const GearLayer a, int mu) {
    const DevGrid& g = a.g;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t chain = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= nxy) return;
    const int xq = (int)(chain & g.mx), yq = (int)(chain >> g.lx);
    const int n = g.nt;
    Walk s;
    for (int q = 0; q < 2 * n; q++) walk_step(s, turn_chain_cell(g, mu, xq, yq, q), q, n, mu, g.wA, a);
}

// A straight line starts at its wall cell (y' = 0, always hard), which
// drops whatever is carried into it, so the warm-up loop of the turn chains
// is not needed: one storing loop from the wall gives the same values and
// labels.
__global__ void __launch_bounds__(256) k_gear_straight(const GearLayer a, int mu) {
    const DevGrid& g = a.g;
    const int xq = blockIdx.x * blockDim.x + threadIdx.x;  // line
    if (xq >= g.nx) return;
    const int T = blockIdx.y;
    const PlaneInfo pi = g.plane[T];
    const int n = g.nx;
    Walk s;
    for (int q = n; q < 2 * n; q++) walk_step(s, line_cell(g, pi, mu, T, xq, q - n), q, n, mu, pi.wS, a);
}

// ------------------------------------------------ turns on the sections scan
// A turn layer as one maneuver scan of turn_scan.cuh over tiles of 32
// chains and all N_theta headings (K = 16 per thread, SL = N_theta / 16
// warps): the same relaxation as the two-loop walk above, each cell read
// once.  Entering at a cell costs the cheaper of its own gear's value and
// the other gear's value plus the penalty (own gear on a tie), with both
// transition edges; a store must beat the own gear's value; the "entered
// from the other gear" bit travels with the entry position to the label.
// Values at or above TH mean unreached (the host picks this kernel only when
// the finite costs stay below TH).
//
// The turns of one chain family come in pairs in the cycle order (RB then
// RF on the right chains, LB then the next cycle's LF on the left chains),
// each pair's maneuvers of opposite gears and opposite scan directions, as
// in the plain sweep's fused pairs: the tile's values of both gears stay in
// registers, the first scan's results are stored and then seen by the
// second scan as the other gear's values.
template <int K, int NTH>
struct GearCells {
    uint32_t (&u)[K];        // own gear's value, TH when unreached, 0 when hard
    const uint32_t (&o)[K];  // the other gear's value, the same way
    const uint32_t (*bp)[NTH];  // shared memory: B of cells 2j (low half) and 2j+1, by thread
    int tid;
    uint32_t ct, pct;        // transition edges; the same plus the gear-change penalty
    uint32_t oth;            // bit k: entering at cell k from the other gear is strictly cheaper
    uint32_t wstep;
    __device__ __forceinline__ uint32_t bound(int k) const { return u[k]; }
    __device__ __forceinline__ void store(int k, uint32_t v) { u[k] = v; }
    // a hard cell enters at ct, which its edge (TH) makes unusable
    __device__ __forceinline__ uint32_t ent(int k) const { return min(u[k] + ct, o[k] + pct); }
    __device__ __forceinline__ uint32_t e(int k) const {
        const uint32_t b = (bp[k >> 1][tid] >> ((k & 1) * 16)) & 0xFFFFu;
        return b == HARD ? TH : (wstep * b) >> 8;
    }
    __device__ __forceinline__ int tag(int k) const { return (int)(((oth >> k) & 1u) << 16); }
    __device__ __forceinline__ uint32_t label_bits(int pv, int q) const {
        return (uint32_t)((((pv >> 16) & 1) << 12) | (q - (pv & 0xFFFF)));
    }
};

template <int K>
__device__ __forceinline__ uint32_t other_cheaper(const uint32_t (&u)[K], const uint32_t (&o)[K], uint32_t ct,
                                                  uint32_t pct) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < K; k++) m |= (uint32_t)(o[k] + pct < u[k] + ct) << k;
    return m;
}

template <int K, int SL>
struct GearTurnSmem {
    int2 cell[K * SL];
    uint32_t bp[K / 2][32 * SL];  // each thread's B values, two per word (registers are full)
    TurnShared<K, SL, 2> sh;
};

// One tile: maneuver mu1 (transition edges ct1), then mu2 (ct2) when
// mu2 >= 0; mu2 is of the other gear and scans the other way.
template <int K, int SL>
__global__ void __launch_bounds__(32 * SL, 1024 / (32 * SL) > 4 ? 4 : 1024 / (32 * SL))
k_gear_scan(const GearLayer a, int mu1, int mu2, uint32_t ct1, uint32_t ct2) {
    extern __shared__ __align__(16) unsigned char gear_smem[];
    GearTurnSmem<K, SL>& sm = *reinterpret_cast<GearTurnSmem<K, SL>*>(gear_smem);
    const DevGrid& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, sec = tid >> 5;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t tile = blockIdx.x;
    const int x0 = (int)((tile * 32) & g.mx), y0 = (int)((tile * 32 >> g.lx) & g.mx);
    const bool left = mu1 == LF || mu1 == LB;
    const bool asc = mu1 == LF || mu1 == RB;  // heading up along the first scan
    const int G = gear_of(mu1);
    uint32_t* V1 = G ? a.Vr : a.Vf;
    uint16_t* L1 = G ? a.Lr : a.Lf;
    uint32_t* V2 = G ? a.Vf : a.Vr;
    uint16_t* L2 = G ? a.Lf : a.Lr;
    if (lane < K) {  // this warp's headings: row offset and x of lane 0's cell
        const int t = sec * K + lane;
        const int4 b = __ldg(&g.beta4[t]);
        const int bx = left ? b.x : b.z, by = left ? b.y : b.w;
        sm.cell[t] = make_int2((int)(uint32_t)((((y0 + by) & g.mx) << g.lx) + (int64_t)t * nxy), (x0 + bx) & g.mx);
    }
    __syncwarp();
    uint32_t v1[K], v2[K];  // the first scan's gear, the other gear
    uint32_t sa = 0, bw = 0;
    bool live = false;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int2 c = sm.cell[sec * K + k];
        const uint32_t id = (uint32_t)c.x + (uint32_t)((c.y + lane) & g.mx);
        uint16_t b = HARD;
        uint32_t x1 = TH, x2 = TH;
        if (NHP_IN(id, nxy * g.nt, a.err, 30)) {
            b = __ldg(a.B + id);
            x1 = min(__ldg(V1 + id), TH);
            x2 = min(__ldg(V2 + id), TH);
        }
        const bool hard = b == HARD;
        v1[k] = hard ? 0u : x1;
        v2[k] = hard ? 0u : x2;
        if (k & 1) sm.bp[k >> 1][tid] = bw | ((uint32_t)b << 16);
        else bw = b;
        sa = min(sa + (hard ? TH : (a.g.wA * (uint32_t)b) >> 8), TH);
        live |= !hard && (x1 < TH || x2 < TH);
    }
    auto store = [&](uint32_t chg, const uint32_t (&v)[K], uint32_t* V, uint16_t* L) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (chg & (1u << k)) {
                const int2 c = sm.cell[sec * K + k];
                const uint32_t id = (uint32_t)c.x + (uint32_t)((c.y + lane) & g.mx);
                if (!NHP_IN(id, nxy * g.nt, a.err, 31)) continue;
                V[id] = v[k];
                L[id] = sm.sh.lab[k][tid];
            }
        }
    };
    uint32_t chg = 0;
    {
        const uint32_t pct = ct1 + a.pen;
        GearCells<K, 32 * SL> cl{v1, v2, sm.bp, tid, ct1, pct, other_cheaper(v1, v2, ct1, pct), g.wA};
        if (asc) turn_scan<K, SL, 1, 2, true>(cl, chg, (uint32_t)mu1 << 13, sec, lane, 0, 0, 0, sa, live, sm.sh);
        else turn_scan<K, SL, 1, 2, false>(cl, chg, (uint32_t)mu1 << 13, sec, lane, 0, 0, 0, sa, live, sm.sh);
    }
    if (chg) store(chg, v1, V1, L1);  // labels are per thread: the second scan may reuse them
    if (mu2 < 0) return;
    live = live || chg != 0;
    chg = 0;
    {
        const uint32_t pct = ct2 + a.pen;
        GearCells<K, 32 * SL> cl{v2, v1, sm.bp, tid, ct2, pct, other_cheaper(v2, v1, ct2, pct), g.wA};
        if (asc) turn_scan<K, SL, 1, 2, false>(cl, chg, (uint32_t)mu2 << 13, sec, lane, 0, 1, 1, sa, live, sm.sh);
        else turn_scan<K, SL, 1, 2, true>(cl, chg, (uint32_t)mu2 << 13, sec, lane, 0, 1, 1, sa, live, sm.sh);
    }
    if (chg) store(chg, v2, V2, L2);
}

__global__ void k_gear_init(uint32_t* Vf, uint32_t* Vr, uint16_t* Lf, uint16_t* Lr, int64_t nr, int64_t start,
                            int start_gear) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        Vf[i] = (i == start && start_gear != 1) ? 0u : INF32;
        Vr[i] = (i == start && start_gear != 0) ? 0u : INF32;
        Lf[i] = NONE;
        Lr[i] = NONE;
    }
}

// Label walk from the cheaper state at the goal (forward on a tie).
// status: [0] segments or -1 unreachable / -3 malformed, [1] cost, [2] gear
// of the last segment's state.
__global__ void k_gear_extract(const GearLayer a, int64_t goal, plan_segment* seg, int cap, int32_t* status) {
    if (threadIdx.x != 0) return;
    const DevGrid& g = a.g;
    int st = a.Vr[goal] < a.Vf[goal] ? 1 : 0;
    const uint32_t cost = st ? a.Vr[goal] : a.Vf[goal];
    status[1] = (int32_t)cost;
    status[2] = st;
    if (cost == INF32) { status[0] = -1; return; }
    int64_t x = goal;
    int n = 0;
    for (;;) {
        const uint16_t lab = st ? a.Lr[x] : a.Lf[x];
        if (lab == NONE) break;
        if (n >= (1 << 20)) { status[0] = -3; return; }
        const int mu = lab >> 13, oth = (lab >> 12) & 1, d = lab & 4095;
        if (mu > 5 || d == 0 || gear_of(mu) != st) { status[0] = -3; return; }
        const int64_t e = entry_cell(g, x, mu, d);
        if (n < cap) {
            plan_segment s;
            s.maneuver = mu;
            s.entry = pose_of(g, e);
            s.exit = pose_of(g, x);
            s.steps = d;
            s.cost = st ? a.Vr[x] : a.Vf[x];
            seg[n] = s;
        }
        n++;
        x = e;
        st = oth ? 1 - st : st;
    }
    status[0] = (st ? a.Vr[x] : a.Vf[x]) == 0 ? n : -3;
}

}  // namespace

cudaError_t launch_gear_init(uint32_t* Vf, uint32_t* Vr, uint16_t* Lf, uint16_t* Lr, int64_t nr, int64_t start,
                             int start_gear, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((nr + 255) / 256, 148 * 16);
    k_gear_init<<<(unsigned)blocks, 256, 0, s>>>(Vf, Vr, Lf, Lr, nr, start, start_gear);
    return cudaGetLastError();
}

namespace {
template <int K, int SL>
cudaError_t launch_gear_scan(const GearLayer& a, int mu1, int mu2, uint32_t ct1, uint32_t ct2, unsigned tiles,
                             cudaStream_t s) {
    // more than the default 48 KB of shared memory; the attribute is per
    // device and setting it again is harmless
    const int bytes = (int)sizeof(GearTurnSmem<K, SL>);
    cudaError_t e = cudaFuncSetAttribute(k_gear_scan<K, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    k_gear_scan<K, SL><<<tiles, 32 * SL, bytes, s>>>(a, mu1, mu2, ct1, ct2);
    return cudaGetLastError();
}

// The sections scan needs whole 32-chain rows and 16 headings per warp, and
// values below TH (a.scan).
bool gear_scan_fits(const GearLayer& a) {
    return a.scan && a.g.nx >= 32 && (a.g.nt == 128 || a.g.nt == 256 || a.g.nt == 512);
}

cudaError_t launch_gear_scan_any(const GearLayer& a, int mu1, int mu2, uint32_t ct1, uint32_t ct2,
                                 cudaStream_t s) {
    const unsigned tiles = (unsigned)((int64_t)a.g.nx * a.g.nx / 32);
    switch (a.g.nt) {
        case 128: return launch_gear_scan<16, 8>(a, mu1, mu2, ct1, ct2, tiles, s);
        case 256: return launch_gear_scan<16, 16>(a, mu1, mu2, ct1, ct2, tiles, s);
        default: return launch_gear_scan<16, 32>(a, mu1, mu2, ct1, ct2, tiles, s);
    }
}
}  // namespace

cudaError_t launch_gear_layer(const GearLayer& a, int mu, cudaStream_t s) {
    if (mu == SF || mu == SB) {
        if (a.scan && a.g.nx >= 16) return launch_gear_straight_tiled(a, mu, s);
        k_gear_straight<<<dim3((unsigned)((a.g.nx + 255) / 256), (unsigned)a.g.nt), 256, 0, s>>>(a, mu);
        return cudaGetLastError();
    }
    if (gear_scan_fits(a)) return launch_gear_scan_any(a, mu, -1, a.cin + a.cout, 0u, s);
    const int64_t chains = (int64_t)a.g.nx * a.g.nx;
    k_gear_turn<<<(unsigned)((chains + 255) / 256), 256, 0, s>>>(a, mu);
    return cudaGetLastError();
}

bool gear_pair_fused(const GearLayer& a) { return gear_scan_fits(a); }

cudaError_t launch_gear_pair(const GearLayer& a, int mu1, int mu2, uint32_t ct1, uint32_t ct2, cudaStream_t s) {
    if (!gear_scan_fits(a) || gear_of(mu1) == gear_of(mu2)) return cudaErrorInvalidValue;
    return launch_gear_scan_any(a, mu1, mu2, ct1, ct2, s);
}

cudaError_t launch_gear_extract(const GearLayer& a, int64_t goal, plan_segment* seg, int cap, int32_t* status,
                                cudaStream_t s) {
    k_gear_extract<<<1, 32, 0, s>>>(a, goal, seg, cap, status);
    return cudaGetLastError();
}

}  // namespace nhp

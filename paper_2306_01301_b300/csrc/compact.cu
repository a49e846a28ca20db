// compact.cu -- the Compact graph (Section V.A, Fig. 12).
//
// Three vertices per cell: S (the straight maneuver type, which is also the
// transition state), L (left turns, forward and backward) and R (right
// turns), with ten edges: S -> L and S -> R at the transition cost ct, L -> S
// and R -> S free, and the six maneuver edges inside their types.  A turn
// layer walks its chains twice (the paper's two loops), entering from the
// cell's own turn state free or from S at ct, and stores what it carries into
// its turn state and, over the free edge back, into S; a straight layer
// moves within S.  Every cell of a layer's volumes is read once per step
// before its possible store and written only by its own chain, so the layer
// sees the values from before it.  Labels (maneuver << 13) | (entered from S
// << 12) | d, d <= n (a whole turn circle from S reaches the turn state of
// the same cell), so grids up to 2048.
//
// When the finite costs stay below TH, the turn layers run as maneuver
// scans of turn_scan.cuh over 32-chain tiles (the turn pairs of the cycle
// order, RB then RF and LB then the next cycle's LF, each on one turn type,
// fused into one launch) and the straight layers, which move within S with
// no transition cost, on the plain straight kernel; otherwise, and on grids
// the scan does not take, one thread walks each chain twice.
#include <algorithm>

#include "curve.cuh"
#include "plan_state.h"
#include "turn_scan.cuh"

namespace nhp {

struct CompactLayer {
    DevGrid g;
    const uint16_t* B;
    uint32_t *Vs, *Vl, *Vr;
    uint16_t *Ls, *Ll, *Lr;
    uint32_t ct;
    int32_t* err;  // the bounds-check build's error word (QueryDesc::err)
};

namespace {

constexpr uint32_t INF32 = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t sadd(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a + b;
    return s >= INF32 ? INF32 : (uint32_t)s;
}

__device__ __forceinline__ int type_of(int mu) { return (mu == LF || mu == LB) ? 1 : (mu == RF || mu == RB) ? 2 : 0; }

struct CWalk {
    uint32_t v = INF32;
    int qe = 0, vs = 0;
};

// What a step reads of its cell: obstacle cost, the value of the layer's
// vertex type and of S.  A layer stores into a cell only at that cell's own
// step of the second loop and never reads it afterwards, so every read sees
// the value from before the layer however early it is made: the walks read
// kAhead cells ahead.
struct CCell {
    uint16_t b;
    uint32_t uT, uS;
};
constexpr int kAhead = 8;

__device__ __forceinline__ CCell cread(const CompactLayer& a, int64_t c, int ty) {
    CCell x;
    x.b = a.B[c];
    x.uT = (ty == 1 ? a.Vl : ty == 2 ? a.Vr : a.Vs)[c];
    x.uS = a.Vs[c];
    return x;
}

__device__ __forceinline__ void cstep(CWalk& s, int64_t c, const CCell& x, int q, int n, int mu, uint32_t w,
                                      const CompactLayer& a) {
    const int ty = type_of(mu);
    uint32_t* Vt = ty == 1 ? a.Vl : ty == 2 ? a.Vr : a.Vs;
    uint16_t* Lt = ty == 1 ? a.Ll : ty == 2 ? a.Lr : a.Ls;
    const uint16_t b = x.b;
    const bool hard = b == HARD;
    const uint32_t uT = x.uT, uS = x.uS;  // before this layer
    if (q >= n && !hard) {
        const uint16_t lab = (uint16_t)((mu << 13) | (s.vs << 12) | (q - s.qe));
        if (s.v < uT) {
            Vt[c] = s.v;
            Lt[c] = lab;
        }
        if (ty != 0 && s.v < uS) {  // back to S over the free edge
            a.Vs[c] = s.v;
            a.Ls[c] = lab;
        }
    }
    const uint32_t tT = hard ? INF32 : uT;
    const uint32_t tS = (hard || ty == 0) ? INF32 : sadd(uS, a.ct);
    const int fromS = tS < tT;
    const uint32_t t = fromS ? tS : tT;
    if (t < s.v) {
        s.v = t;
        s.qe = q;
        s.vs = fromS;
    }
    s.v = sadd(s.v, hard ? INF32 : (uint32_t)(((uint64_t)w * b) >> 8));
}

__global__ void __launch_bounds__(256) kc_turn(const CompactLayer a, int mu) {
    const DevGrid& g = a.g;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t chain = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= nxy) return;
    const int xq = (int)(chain & g.mx), yq = (int)(chain >> g.lx);
    const int n = g.nt, ty = type_of(mu);
    CWalk s;
    for (int q0 = 0; q0 < 2 * n; q0 += kAhead) {  // 2n is a multiple of kAhead
        int64_t c[kAhead];
        CCell x[kAhead];
#pragma unroll
        for (int j = 0; j < kAhead; j++) {
            c[j] = turn_chain_cell(g, mu, xq, yq, q0 + j);
            x[j] = cread(a, c[j], ty);
        }
#pragma unroll
        for (int j = 0; j < kAhead; j++) cstep(s, c[j], x[j], q0 + j, n, mu, g.wA, a);
    }
}

__global__ void __launch_bounds__(256) kc_straight(const CompactLayer a, int mu) {
    const DevGrid& g = a.g;
    const int xq = blockIdx.x * blockDim.x + threadIdx.x;
    if (xq >= g.nx) return;
    const int T = blockIdx.y;
    const PlaneInfo pi = g.plane[T];
    const int n = g.nx, ty = type_of(mu);
    CWalk s;
    for (int q0 = 0; q0 < 2 * n; q0 += kAhead) {
        int64_t c[kAhead];
        CCell x[kAhead];
#pragma unroll
        for (int j = 0; j < kAhead; j++) {
            c[j] = line_cell(g, pi, mu, T, xq, q0 + j);
            x[j] = cread(a, c[j], ty);
        }
#pragma unroll
        for (int j = 0; j < kAhead; j++) cstep(s, c[j], x[j], q0 + j, n, mu, pi.wS, a);
    }
}

// ------------------------------------------------ turns on the sections scan
// A turn cell holds its turn state's value u and S's value s; entering costs
// min(u, s + ct) (the turn state on a tie) and a carried value stores into
// each of the two it beats, with the same label.
template <int K, int NTH>
struct CompactCells {
    uint32_t (&u)[K];           // the turn state's value, TH when unreached, 0 when hard
    uint32_t (&s)[K];           // S's value, the same way
    const uint32_t (*bp)[NTH];  // shared memory: B of cells 2j (low half) and 2j+1, by thread
    int tid;
    uint32_t ct;                // S -> turn state
    uint32_t oth;               // bit k: entering at cell k from S is strictly cheaper
    uint32_t wstep;
    __device__ __forceinline__ uint32_t bound(int k) const { return max(u[k], s[k]); }
    // which of the two took the value is read off at the write-back, against
    // the volumes, which still hold the values from before the layer
    __device__ __forceinline__ void store(int k, uint32_t v) {
        u[k] = min(u[k], v);
        s[k] = min(s[k], v);
    }
    __device__ __forceinline__ uint32_t ent(int k) const { return min(u[k], s[k] + ct); }
    __device__ __forceinline__ uint32_t e(int k) const {
        const uint32_t b = (bp[k >> 1][tid] >> ((k & 1) * 16)) & 0xFFFFu;
        return b == HARD ? TH : (wstep * b) >> 8;
    }
    __device__ __forceinline__ int tag(int k) const { return (int)(((oth >> k) & 1u) << 16); }
    __device__ __forceinline__ uint32_t label_bits(int pv, int q) const {
        return (uint32_t)((((pv >> 16) & 1) << 12) | (q - (pv & 0xFFFF)));
    }
};

template <int K, int SL>
struct CompactTurnSmem {
    int2 cell[K * SL];
    uint32_t bp[K / 2][32 * SL];
    TurnShared<K, SL, 2> sh;
};

// One tile: maneuver mu1, then mu2 (the same turn type, the other scan
// direction) when mu2 >= 0.
template <int K, int SL>
__global__ void __launch_bounds__(32 * SL, 1024 / (32 * SL) > 4 ? 4 : 1024 / (32 * SL))
kc_scan(const CompactLayer a, int mu1, int mu2) {
    extern __shared__ __align__(16) unsigned char compact_smem[];
    CompactTurnSmem<K, SL>& sm = *reinterpret_cast<CompactTurnSmem<K, SL>*>(compact_smem);
    const DevGrid& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, sec = tid >> 5;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t tile = blockIdx.x;
    const int x0 = (int)((tile * 32) & g.mx), y0 = (int)((tile * 32 >> g.lx) & g.mx);
    const int ty = type_of(mu1);
    const bool asc = mu1 == LF || mu1 == RB;  // heading up along the first scan
    uint32_t* Vt = ty == 1 ? a.Vl : a.Vr;
    uint16_t* Lt = ty == 1 ? a.Ll : a.Lr;
    if (lane < K) {
        const int t = sec * K + lane;
        const int4 b = __ldg(&g.beta4[t]);
        const int bx = ty == 1 ? b.x : b.z, by = ty == 1 ? b.y : b.w;
        sm.cell[t] = make_int2((int)(uint32_t)((((y0 + by) & g.mx) << g.lx) + (int64_t)t * nxy), (x0 + bx) & g.mx);
    }
    __syncwarp();
    uint32_t u[K], s[K];
    uint32_t sa = 0, bw = 0;
    bool live = false;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int2 c = sm.cell[sec * K + k];
        const uint32_t id = (uint32_t)c.x + (uint32_t)((c.y + lane) & g.mx);
        uint16_t b = HARD;
        uint32_t xt = TH, xs = TH;
        if (NHP_IN(id, nxy * g.nt, a.err, 36)) {
            b = __ldg(a.B + id);
            xt = min(__ldg(Vt + id), TH);
            xs = min(__ldg(a.Vs + id), TH);
        }
        const bool hard = b == HARD;
        u[k] = hard ? 0u : xt;
        s[k] = hard ? 0u : xs;
        if (k & 1) sm.bp[k >> 1][tid] = bw | ((uint32_t)b << 16);
        else bw = b;
        sa = min(sa + (hard ? TH : (g.wA * (uint32_t)b) >> 8), TH);
        live |= !hard && (xt < TH || xs < TH);
    }
    auto cheaper_from_s = [&]() {
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < K; k++) m |= (uint32_t)(s[k] + a.ct < u[k]) << k;
        return m;
    };
    // cells with a label from this scan: store where the value went down
    auto write_back = [&](uint32_t chg) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (chg & (1u << k)) {
                const int2 c = sm.cell[sec * K + k];
                const uint32_t id = (uint32_t)c.x + (uint32_t)((c.y + lane) & g.mx);
                if (!NHP_IN(id, nxy * g.nt, a.err, 37)) continue;
                const uint16_t lab = sm.sh.lab[k][tid];
                if (u[k] < min(Vt[id], TH)) { Vt[id] = u[k]; Lt[id] = lab; }
                if (s[k] < min(a.Vs[id], TH)) { a.Vs[id] = s[k]; a.Ls[id] = lab; }
            }
        }
    };
    uint32_t chg = 0, any = 0;
    {
        CompactCells<K, 32 * SL> cl{u, s, sm.bp, tid, a.ct, cheaper_from_s(), g.wA};
        if (asc) turn_scan<K, SL, 1, 2, true>(cl, chg, (uint32_t)mu1 << 13, sec, lane, 0, 0, 0, sa, live, sm.sh);
        else turn_scan<K, SL, 1, 2, false>(cl, chg, (uint32_t)mu1 << 13, sec, lane, 0, 0, 0, sa, live, sm.sh);
        if (chg) write_back(chg);  // labels are per thread: the second scan may reuse them
        any = chg;
    }
    if (mu2 < 0) return;
    live = live || any != 0;
    chg = 0;
    {
        CompactCells<K, 32 * SL> cl{u, s, sm.bp, tid, a.ct, cheaper_from_s(), g.wA};
        if (asc) turn_scan<K, SL, 1, 2, false>(cl, chg, (uint32_t)mu2 << 13, sec, lane, 0, 1, 1, sa, live, sm.sh);
        else turn_scan<K, SL, 1, 2, true>(cl, chg, (uint32_t)mu2 << 13, sec, lane, 0, 1, 1, sa, live, sm.sh);
        if (chg) write_back(chg);
    }
}

template <int K, int SL>
cudaError_t launch_kc_scan(const CompactLayer& a, int mu1, int mu2, cudaStream_t s) {
    const int bytes = (int)sizeof(CompactTurnSmem<K, SL>);
    cudaError_t e = cudaFuncSetAttribute(kc_scan<K, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    kc_scan<K, SL><<<(unsigned)((int64_t)a.g.nx * a.g.nx / 32), 32 * SL, bytes, s>>>(a, mu1, mu2);
    return cudaGetLastError();
}

cudaError_t launch_kc_scan_any(const CompactLayer& a, int mu1, int mu2, cudaStream_t s) {
    switch (a.g.nt) {
        case 128: return launch_kc_scan<16, 8>(a, mu1, mu2, s);
        case 256: return launch_kc_scan<16, 16>(a, mu1, mu2, s);
        default: return launch_kc_scan<16, 32>(a, mu1, mu2, s);
    }
}

__global__ void kc_init(CompactLayer a, int64_t nr, int64_t start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        a.Vs[i] = i == start ? 0u : INF32;
        a.Vl[i] = INF32;
        a.Vr[i] = INF32;
        a.Ls[i] = NONE;
        a.Ll[i] = NONE;
        a.Lr[i] = NONE;
    }
}

// Label walk from S(goal).  status: [0] segments or -1 / -3, [1] V_S(goal).
__global__ void kc_extract(const CompactLayer a, int64_t goal, plan_segment* seg, int cap, int32_t* status) {
    if (threadIdx.x != 0) return;
    status[1] = (int32_t)a.Vs[goal];
    if (a.Vs[goal] == INF32) { status[0] = -1; return; }
    int ty = 0, n = 0;
    int64_t x = goal;
    for (;;) {
        const uint16_t* Lt = ty == 1 ? a.Ll : ty == 2 ? a.Lr : a.Ls;
        const uint32_t* Vt = ty == 1 ? a.Vl : ty == 2 ? a.Vr : a.Vs;
        const uint16_t lab = Lt[x];
        if (lab == NONE) {
            status[0] = Vt[x] == 0 ? n : -3;
            return;
        }
        if (n >= (1 << 20)) { status[0] = -3; return; }
        const int mu = lab >> 13, fs = (lab >> 12) & 1, d = lab & 4095, T = type_of(mu);
        if (mu > 5 || d == 0 || (ty != 0 && T != ty)) { status[0] = -3; return; }
        const int64_t e = entry_cell(a.g, x, mu, d);
        if (n < cap) {
            plan_segment s;
            s.maneuver = mu;
            s.entry = pose_of(a.g, e);
            s.exit = pose_of(a.g, x);
            s.steps = d;
            s.cost = Vt[x];
            seg[n] = s;
        }
        n++;
        x = e;
        ty = fs ? 0 : T;
    }
}

// The scan path: whole 32-chain rows, 16 headings per warp, and finite
// costs below TH (each layer adds at most one segment: ct and at most
// max(Nx, N_theta) - 1 edges).
bool compact_scan_fits(const plan_s* p, int n_cycles) {
    if (p->nx < 32 || (p->nt != 128 && p->nt != 256 && p->nt != 512)) return false;
    const double e_max = std::floor((double)p->w_max * (double)obstacle_bound(p) / 256.0);
    const double layer = (double)p->costs.transition + (double)(std::max(p->nx, p->nt) - 1) * e_max;
    return 6.0 * n_cycles * layer < (double)TH;
}

CompactLayer layer_args(const plan_s* p) {
    CompactLayer a{};
    a.g = p->g;
    a.B = p->d_B;
    a.Vs = p->d_V;
    a.Vl = p->d_Vcl;
    a.Vr = p->d_Vcr;
    a.Ls = p->d_L;
    a.Ll = p->d_Lcl;
    a.Lr = p->d_Lcr;
    a.ct = p->costs.transition;
    a.err = p->d_status + 3;
    return a;
}

}  // namespace

void compact_release(plan_s* p) {
    p->dfree(p->d_Vcl, (size_t)p->nr * 4);
    p->dfree(p->d_Vcr, (size_t)p->nr * 4);
    p->dfree(p->d_Lcl, (size_t)p->nr * 2);
    p->dfree(p->d_Lcr, (size_t)p->nr * 2);
    p->dfree(p->d_qdc, sizeof(QueryDesc));
    p->d_Vcl = p->d_Vcr = nullptr;
    p->d_Lcl = p->d_Lcr = nullptr;
    p->d_qdc = nullptr;
    if (p->vol_kind == VOL_COMPACT) p->vol_kind = VOL_NONE;
}

}  // namespace nhp

using namespace nhp;

extern "C" {

int plan_set_compact_graph(plan_t* p, int enable) {
    if (!p) return PLAN_EINVAL;
    if (!enable) {
        compact_release(p);
        return PLAN_OK;
    }
    if (p->nx > 2048 || p->nt > 2048) return PLAN_EINVAL;
    if (!p->volumes) return PLAN_ESTATE;
    if (p->d_Vcl) return PLAN_OK;
    p->d_Vcl = (uint32_t*)p->dalloc((size_t)p->nr * 4);
    p->d_Vcr = (uint32_t*)p->dalloc((size_t)p->nr * 4);
    p->d_Lcl = (uint16_t*)p->dalloc((size_t)p->nr * 2);
    p->d_Lcr = (uint16_t*)p->dalloc((size_t)p->nr * 2);
    p->d_qdc = (QueryDesc*)p->dalloc(sizeof(QueryDesc));
    if (!p->d_Vcl || !p->d_Vcr || !p->d_Lcl || !p->d_Lcr || !p->d_qdc) {
        compact_release(p);
        return PLAN_ENOMEM;
    }
    return PLAN_OK;
}

int plan_sweep_compact(plan_t* p, plan_pose start, int n_cycles) {
    if (!p || n_cycles < 0 || n_cycles > 4096 || !pose_ok(p, start)) return PLAN_EINVAL;
    if (!p->d_Vcl || !p->rendered) return PLAN_ESTATE;
    if (pose_hard(p, start)) return PLAN_EINVAL;
    static const int order[6] = {LF, SF, RB, RF, SB, LB};  // Section XVI.A
    const CompactLayer a = layer_args(p);
    cudaStream_t s = p->stream;
    p->vol_kind = VOL_NONE;
    const int64_t blocks = std::min<int64_t>((p->nr + 255) / 256, 148 * 16);
    kc_init<<<(unsigned)blocks, 256, 0, s>>>(a, p->nr, cell_index(p, start));
    int rc = cuda_rc(cudaGetLastError());
    p->launches++;
    if (rc == PLAN_OK && compact_scan_fits(p, n_cycles)) {
        // Passes of the plain cycle schedule: a lone LF, then per cycle SF,
        // {RB, RF}, SB and {LB, next LF} (a lone LB at the end).  The
        // straights run on the plain kernel as passes 1 and 3 of a one-cycle
        // query on S with no transition cost.
        QueryDesc q = p->qd;
        for (int k = 0; k < 6; k++) q.g.ctm[k] = 0;
        q.n_cycles = 1;
        q.pass = -1;
        q.conv = nullptr;
        q.v.improved = nullptr;
        rc = cuda_rc(cudaMemcpyAsync(p->d_qdc, &q, sizeof(q), cudaMemcpyHostToDevice, s));
        if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(s));  // the host copy must outlive the copy
        Group gr{p->d_qdc, 1, p->lx, p->lt, p->max_runs > 0 ? p->max_runs : 1};
        gr.grid = p->straight_grid;
        for (int pass = 0; pass < pass_count(n_cycles) && rc == PLAN_OK; pass++) {
            if (pass_is_turn(pass)) {
                int m1, m2;
                turn_pass_maneuvers(pass, &m1, &m2);
                if (pass == 4 * n_cycles) m2 = -1;  // the last cycle's LB has no LF after it
                rc = cuda_rc(launch_kc_scan_any(a, m1, m2, s));
            } else {
                rc = cuda_rc(launch_straight(gr, (pass & 3) == 1 ? 1 : 3, p->straight_lines, s));
            }
            p->launches++;
        }
        if (rc == PLAN_OK) p->vol_kind = VOL_COMPACT;
        return rc;
    }
    for (int l = 0; l < 6 * n_cycles && rc == PLAN_OK; l++) {
        const int mu = order[l % 6];
        if (mu == SF || mu == SB)
            kc_straight<<<dim3((unsigned)((p->nx + 255) / 256), (unsigned)p->nt), 256, 0, s>>>(a, mu);
        else
            kc_turn<<<(unsigned)((p->nxy + 255) / 256), 256, 0, s>>>(a, mu);
        rc = cuda_rc(cudaGetLastError());
        p->launches++;
    }
    if (rc == PLAN_OK) p->vol_kind = VOL_COMPACT;
    return rc;
}

int plan_extract_compact(plan_t* p, plan_pose goal, plan_segment* out, int cap, int* n_out, uint32_t* cost) {
    if (!p || !n_out || !cost || cap < 0 || (cap > 0 && !out) || !pose_ok(p, goal)) return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    if (p->vol_kind != VOL_COMPACT) return PLAN_ESTATE;
    kc_extract<<<1, 32, 0, p->stream>>>(layer_args(p), cell_index(p, goal), p->d_seg, kDevSegCap, p->d_status);
    NHP_CK(cudaGetLastError());
    p->launches++;
    int32_t status[4] = {0, 0, 0, 0};  // [3]: the bounds-check build's error word
    NHP_CK(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    NHP_CK(cudaStreamSynchronize(p->stream));
    if (status[3] != 0) return check_failed(p, status[3]);
    if (status[0] == -1) return PLAN_EUNREACHABLE;
    if (status[0] < 0) return PLAN_EINTERNAL;
    *cost = (uint32_t)status[1];
    *n_out = status[0];
    if (status[0] > cap || status[0] > kDevSegCap) return PLAN_ERANGE;
    if (status[0] > 0) {
        NHP_CK(cudaMemcpyAsync(out, p->d_seg, sizeof(plan_segment) * status[0], cudaMemcpyDeviceToHost, p->stream));
        NHP_CK(cudaStreamSynchronize(p->stream));
        std::reverse(out, out + status[0]);
    }
    return PLAN_OK;
}

int plan_copy_compact_volumes(plan_t* p, uint32_t* VL, uint16_t* LL, uint32_t* VR, uint16_t* LR) {
    if (!p) return PLAN_EINVAL;
    if (!p->d_Vcl) return PLAN_ESTATE;
    const size_t n = (size_t)p->nr;
    if (VL) NHP_CK(cudaMemcpyAsync(VL, p->d_Vcl, n * 4, cudaMemcpyDeviceToHost, p->stream));
    if (LL) NHP_CK(cudaMemcpyAsync(LL, p->d_Lcl, n * 2, cudaMemcpyDeviceToHost, p->stream));
    if (VR) NHP_CK(cudaMemcpyAsync(VR, p->d_Vcr, n * 4, cudaMemcpyDeviceToHost, p->stream));
    if (LR) NHP_CK(cudaMemcpyAsync(LR, p->d_Lcr, n * 2, cudaMemcpyDeviceToHost, p->stream));
    return check_error_word(p);
}

}  // extern "C"

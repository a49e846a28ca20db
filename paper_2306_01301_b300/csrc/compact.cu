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
// the same cell), so grids up to 2048.  Feature path: one thread per chain.
#include <algorithm>

#include "curve.cuh"
#include "plan_state.h"

namespace nhp {

struct CompactLayer {
    DevGrid g;
    const uint16_t* B;
    uint32_t *Vs, *Vl, *Vr;
    uint16_t *Ls, *Ll, *Lr;
    uint32_t ct;
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
    return a;
}

}  // namespace

void compact_release(plan_s* p) {
    p->dfree(p->d_Vcl, (size_t)p->nr * 4);
    p->dfree(p->d_Vcr, (size_t)p->nr * 4);
    p->dfree(p->d_Lcl, (size_t)p->nr * 2);
    p->dfree(p->d_Lcr, (size_t)p->nr * 2);
    p->d_Vcl = p->d_Vcr = nullptr;
    p->d_Lcl = p->d_Lcr = nullptr;
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
    if (!p->d_Vcl || !p->d_Vcr || !p->d_Lcl || !p->d_Lcr) {
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
    int32_t status[2] = {0, 0};
    NHP_CK(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    NHP_CK(cudaStreamSynchronize(p->stream));
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
    NHP_CK(cudaStreamSynchronize(p->stream));
    return PLAN_OK;
}

}  // extern "C"

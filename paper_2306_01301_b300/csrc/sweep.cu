// sweep.cu -- maneuver-kernel sweeps over the value volume (Section VIII.B-C).
//
// One maneuver kernel considers, for every cell, starting from any transition
// state at its current value, entering the maneuver (transition cost ct),
// following any number of its edges (cost (w*B)>>8 per edge left) and
// returning to the transition state, storing the value when that is strictly
// better (Insert 1).  Along one maneuver curve this is the recurrence
//     v_{k+1} = min(v_k, u_k + ct) + e_k,    V'_k = min(V_k, v_k),
// a linear recurrence in the (min,+) semiring: a stretch of cells acts on the
// carried value as x -> min(x + a, b).  Composing such maps is associative,
// which lets a turn curve be cut into sections and scanned in parallel (the
// 'Sections' idea of Appendix D), exactly and in integers.
//
// Curves (Section V.C):
//   turn     thread (x', y') sweeps T; cell ((x' + beta_a(T)) & M,
//            (y' + beta_b(T)) & M, T) with (a, b) = (0, 3) LEFT, (2, 1) RIGHT
//            (eq. 18).  Cyclic: the paper runs two loops; here the carry into
//            the second loop is the first loop's composite map applied to
//            'nothing carried', and only the second loop stores.
//   straight thread (x', T) sweeps y'; cell (y', (x' + Bs(y')) & M) when
//            I(T) = 0, ((x' + Bs(y')) & M, y') when I(T) = 1 (eq. 23), y'
//            taken in the direction J(T) for forward, -J(T) for backward
//            (eq. 24).  y' = 0 is the wall cell, so one pass from there
//            suffices.
// Tie rule: a new entry replaces the carried one only when strictly cheaper,
// so among equally cheap entries the one furthest upstream is recorded.
//
// Value domain inside the kernels: u = min(V, TH) for non-hard cells and
// u = 0 for hard cells (a hard cell is never stored because v < 0 is
// impossible, and its entry is cancelled by its edge cost TH before it can
// reach another cell).
#include "internal.h"

namespace nhp {
namespace {

__device__ __forceinline__ uint32_t edge_cost(uint16_t b, uint32_t w) {
    return b == HARD ? TH : (w * (uint32_t)b) >> 8;
}

// Profiling only: add this warp's improved-cell count to the plan counter.
__device__ __forceinline__ void count_improved(unsigned long long* ctr, uint32_t n) {
    if (!ctr) return;
    const uint32_t mask = __activemask();
    uint32_t sum = n;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(mask, sum, off);
    if ((threadIdx.x & 31) == (__ffs(mask) - 1) && sum) atomicAdd(ctr, (unsigned long long)sum);
}

// ------------------------------------------------------------------- turns
// CTA = 32 chains x S sections; warp s holds headings [sK, sK+K) of its lane's
// chain in registers.  Scan-order positions: ascending r = T, descending
// r = NT-1-T; positions of the storing (second) loop are r + NT.

// Section-map arrays are [section][chain].  The carry scan reads them with
// lanes spread over (section, chain) = (l % S, l / S); a row pitch of
// 32 + 32/S words puts those 32 reads in 32 different banks.
template <int K, int S>
struct TurnSmem {
    static constexpr int P = 32 + 32 / S;
    int2 beta[K * S];
    uint32_t sa[S][P];
    uint32_t sb[S][P];
    int32_t sp[S][P];
};

// Compose an earlier stretch X with a later one Y (in place into Y):
// x -> min(x + A, B @ P).  X's entry positions precede Y's, so ties go to X.
__device__ __forceinline__ void combine(uint32_t xa, uint32_t xb, int xp, uint32_t& ya, uint32_t& yb,
                                        int& yp) {
    const uint32_t cand = xb + ya;  // xb <= 2TH + ct, ya <= TH: no wrap
    if (cand <= yb) { yb = cand; yp = xp; }
    ya = min(xa + ya, TH);
}

template <int K, int S, bool ASC>
__device__ __forceinline__ void turn_scan(uint32_t (&u)[K], const uint32_t (&e)[K], uint32_t (&lab)[(K + 1) / 2],
                                          uint32_t& chg, int mu, uint32_t ct, int sec, int lane,
                                          TurnSmem<K, S>& sm) {
    constexpr int NT = K * S;
    const int ss = ASC ? sec : S - 1 - sec;  // section index in scan order
    // 1) this section's map (first-loop positions in [0, NT)).
    uint32_t a = 0, b = 0xFFFFFFFFu;
    int pb = 0;
#pragma unroll
    for (int kk = 0; kk < K; kk++) {
        const int k = ASC ? kk : K - 1 - kk;
        const uint32_t t = u[k] + ct;
        if (t < b) { b = t; pb = ss * K + kk; }
        b += e[k];
        a = min(a + e[k], TH);
    }
    sm.sa[ss][lane] = a;
    sm.sb[ss][lane] = b;
    sm.sp[ss][lane] = pb;
    __syncthreads();
    // 2) carry into each section of the second loop: segmented warp scan
    //    over the S section maps of each chain (32/S chains per warp).
    {
        const int c = sec * (32 / S) + lane / S;
        const int s = lane % S;
        uint32_t A = sm.sa[s][c], B = sm.sb[s][c];
        int P = sm.sp[s][c];
#pragma unroll
        for (int off = 1; off < S; off <<= 1) {
            const uint32_t xa = __shfl_up_sync(0xFFFFFFFFu, A, off, S);
            const uint32_t xb = __shfl_up_sync(0xFFFFFFFFu, B, off, S);
            const int xp = __shfl_up_sync(0xFFFFFFFFu, P, off, S);
            if (s >= off) combine(xa, xb, xp, A, B, P);
        }
        // the whole first loop applied to 'nothing carried'
        const uint32_t bF = __shfl_sync(0xFFFFFFFFu, B, S - 1, S);
        const int pF = __shfl_sync(0xFFFFFFFFu, P, S - 1, S);
        // map of sections 0..s-1 of the second loop
        const uint32_t eA = __shfl_up_sync(0xFFFFFFFFu, A, 1, S);
        const uint32_t eB = __shfl_up_sync(0xFFFFFFFFu, B, 1, S);
        const int eP = __shfl_up_sync(0xFFFFFFFFu, P, 1, S);
        uint32_t cv = bF;
        int cp = pF;
        if (s > 0) {
            const uint32_t cand = bF + eA;  // first-loop entries are further upstream
            if (cand <= eB) { cv = cand; cp = pF; }
            else { cv = eB; cp = eP + NT; }
        }
        __syncwarp();
        sm.sb[s][c] = cv;
        sm.sp[s][c] = cp;
    }
    __syncthreads();
    // 3) second loop: store where strictly better.
    uint32_t v = sm.sb[ss][lane];
    int pv = sm.sp[ss][lane];
    const uint32_t mtag = (uint32_t)mu << 13;
#pragma unroll
    for (int kk = 0; kk < K; kk++) {
        const int k = ASC ? kk : K - 1 - kk;
        const int q = NT + ss * K + kk;
        const uint32_t uk = u[k];
        if (v < uk) {
            u[k] = v;
            const uint32_t l = mtag | (uint32_t)(q - pv);
            lab[k >> 1] = (k & 1) ? ((lab[k >> 1] & 0xFFFFu) | (l << 16)) : ((lab[k >> 1] & 0xFFFF0000u) | l);
            chg |= 1u << k;
        }
        const uint32_t t = uk + ct;
        if (t < v) { v = t; pv = q; }
        v += e[k];
    }
    __syncthreads();  // the shared summaries are reused by the next scan
}

template <int K, int S>
__global__ void __launch_bounds__(32 * S, 1)
k_turn(DevGrid g, Volumes vol, int family, int asc, int mu1, int mu2) {
    constexpr int NT = K * S;
    __shared__ TurnSmem<K, S> sm;
    const int tid = threadIdx.x, lane = tid & 31, sec = tid >> 5;
    for (int t = tid; t < NT; t += 32 * S) {
        const int4 b = g.beta4[t];
        sm.beta[t] = family ? make_int2(b.z, b.w) : make_int2(b.x, b.y);
    }
    __syncthreads();
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t chain = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = chain < nxy;
    const int xq = (int)(chain & g.mx), yq = (int)((chain >> g.lx) & g.mx);
    const uint32_t w = g.wA, ct = g.ct;

    uint32_t u[K], e[K], lab[(K + 1) / 2];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int T = sec * K + k;
        const int2 bb = sm.beta[T];
        const int64_t id = (int64_t)(((xq + bb.x) & g.mx) | (((yq + bb.y) & g.mx) << g.lx)) + (int64_t)T * nxy;
        uint32_t vv = 0xFFFFFFFFu;
        uint16_t ob = HARD;
        if (valid) {
            vv = __ldg(vol.V + id);
            ob = __ldg(vol.B + id);
        }
        e[k] = edge_cost(ob, w);
        u[k] = ob == HARD ? 0u : min(vv, TH);
    }
#pragma unroll
    for (int k = 0; k < (K + 1) / 2; k++) lab[k] = 0;
    uint32_t chg = 0;
    if (asc) turn_scan<K, S, true>(u, e, lab, chg, mu1, ct, sec, lane, sm);
    else turn_scan<K, S, false>(u, e, lab, chg, mu1, ct, sec, lane, sm);
    if (mu2 >= 0) {
        if (asc) turn_scan<K, S, false>(u, e, lab, chg, mu2, ct, sec, lane, sm);
        else turn_scan<K, S, true>(u, e, lab, chg, mu2, ct, sec, lane, sm);
    }
    if (vol.improved) count_improved(vol.improved, __popc(chg));
    if (!valid || chg == 0) return;
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (chg & (1u << k)) {
            const int T = sec * K + k;
            const int2 bb = sm.beta[T];
            const int64_t id =
                (int64_t)(((xq + bb.x) & g.mx) | (((yq + bb.y) & g.mx) << g.lx)) + (int64_t)T * nxy;
            vol.V[id] = u[k];
            vol.L[id] = (uint16_t)((k & 1) ? (lab[k >> 1] >> 16) : (lab[k >> 1] & 0xFFFFu));
        }
    }
}

template <int K, int S>
cudaError_t launch_turn_t(const DevGrid& g, Volumes v, int family, int asc, int mu1, int mu2, cudaStream_t s) {
    const int64_t chains = (int64_t)g.nx * g.nx;
    const unsigned blocks = (unsigned)((chains + 31) / 32);
    k_turn<K, S><<<blocks, 32 * S, 0, s>>>(g, v, family, asc, mu1, mu2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- straights
// One thread per line (x', T); a block owns `lines` neighbouring lines of one
// heading plane and walks them 16 steps at a time.  Each 16-step chunk of the
// block's lines is a sheared parallelogram of cells: Bs changes by at most 1
// per step (|slope| <= 1), so the chunk fits in a (lines + 15) x 16 tile.
//   shallow (I = 0): cell (line, step y') = row x' + Bs(y'), column y';
//                    tile rows = grid rows, tile columns = the 16 steps.
//   steep   (I = 1): cell = row y', column x' + Bs(y');
//                    tile rows = the 16 steps, tile columns = grid columns.
// Tiles are filled with 4-byte cp.async copies (whole row segments, so
// global reads coalesce in both cases), two stages deep: the next chunk is in
// flight while the current one is scanned.  Changed cells are marked in the
// tile (bit 31 of the value, the label in place of the obstacle value) and
// written back row segment by row segment.
constexpr int kSteps = 16;
constexpr int kMaxLines = 256;
constexpr int kSpan = kMaxLines + kSteps;           // tile extent across lines
constexpr int kVWords = kSpan * (kSteps + 1);       // >= kSteps * (kSpan + 1)
constexpr int kBHalves = kSpan * (kSteps + 2);      // >= kSteps * (kSpan + 4)
constexpr uint32_t kMark = 0x80000000u;             // changed; stored values are < TH

struct StraightStage {
    uint32_t v[kVWords];
    uint16_t b[kBHalves];
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct ChunkGeom {
    int y0;     // first step of the chunk (ascending y')
    int bmin;   // min of Bs over the chunk
    int span;   // lines + (max - min of Bs)
    int base;   // grid coordinate of tile index 0 across lines (masked)
};

__device__ __forceinline__ ChunkGeom chunk_geom(const int16_t* bs, int ch, int dir, int nx, int X0, int lines,
                                                int mx) {
    ChunkGeom c;
    c.y0 = dir > 0 ? ch * kSteps : nx - (ch + 1) * kSteps;
    const int b0 = bs[c.y0], b1 = bs[c.y0 + kSteps - 1];
    c.bmin = min(b0, b1);
    c.span = lines + max(b0, b1) - c.bmin;
    c.base = (X0 + c.bmin) & mx;
    return c;
}

// Issue the copies of one chunk into a stage.
__device__ __forceinline__ void straight_issue(StraightStage& st, const ChunkGeom& c, bool steep,
                                               const uint32_t* Vp, const uint16_t* Bp, int lx, int mx) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (!steep) {
        // rows r in [0, span), columns s in [0, 16): V words and B word pairs
        for (int k = tid; k < c.span * kSteps; k += nt) {
            const int r = k >> 4, s = k & 15;
            const int64_t row = (int64_t)((c.base + r) & mx) << lx;
            cp_async4(&st.v[r * (kSteps + 1) + s], Vp + row + c.y0 + s);
        }
        for (int k = tid; k < c.span * (kSteps / 2); k += nt) {
            const int r = k >> 3, s2 = (k & 7) * 2;
            const int64_t row = (int64_t)((c.base + r) & mx) << lx;
            cp_async4(&st.b[r * (kSteps + 2) + s2], Bp + row + c.y0 + s2);
        }
    } else {
        // step rows s in [0, 16), columns x in [0, span) starting at base
        for (int k = tid; k < kSteps * c.span; k += nt) {
            const int s = k / c.span, x = k - s * c.span;
            const int64_t row = (int64_t)(c.y0 + s) << lx;
            cp_async4(&st.v[s * (kSpan + 1) + x], Vp + row + ((c.base + x) & mx));
        }
        // B as aligned word pairs covering [base, base + span): halfword
        // index h of tile row s holds column (base & ~1) + h
        const int a = c.base & ~1;
        const int words = (c.span + 2) >> 1;
        for (int k = tid; k < kSteps * words; k += nt) {
            const int s = k / words, wd = k - s * words;
            const int64_t row = (int64_t)(c.y0 + s) << lx;
            cp_async4(&st.b[s * (kSpan + 4) + 2 * wd], Bp + row + ((a + 2 * wd) & mx));
        }
    }
}

__global__ void __launch_bounds__(kMaxLines, 3)
k_straight(DevGrid g, Volumes vol, int mu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StraightStage* stage = reinterpret_cast<StraightStage*>(smem_raw);
    const int T = blockIdx.y;
    const int lines = blockDim.x;  // min(Nx, 256)
    const int X0 = blockIdx.x * lines;
    const int t = threadIdx.x;
    const PlaneInfo pi = g.plane[T];
    const bool steep = pi.iflag != 0;
    const int dir = mu == SF ? pi.jsign : -pi.jsign;  // direction of y' along the sweep
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    uint32_t* Vp = vol.V + (int64_t)T * nxy;
    uint16_t* Lp = vol.L + (int64_t)T * nxy;
    const uint16_t* Bp = vol.B + (int64_t)T * nxy;
    const uint32_t w = pi.wS, ct = g.ct;
    const uint32_t mtag = (uint32_t)mu << 13;
    // Sweep order: dir > 0 visits y' = 0, 1, .., Nx-1 (q = y'); dir < 0
    // visits Nx-1, .., 1, 0 (q = Nx - y').  Starting at Nx-1 with nothing
    // carried equals starting at the wall cell y' = 0, which carries nothing.
    uint32_t v = 0xFFFFFFFFu;
    int pv = 0;
    uint32_t nimp = 0;
    const int nch = g.nx / kSteps;

    ChunkGeom geo0 = chunk_geom(bs, 0, dir, g.nx, X0, lines, g.mx), geo1 = geo0;
    straight_issue(stage[0], geo0, steep, Vp, Bp, g.lx, g.mx);
    cp_async_commit();
    if (nch > 1) {
        geo1 = chunk_geom(bs, 1, dir, g.nx, X0, lines, g.mx);
        straight_issue(stage[1], geo1, steep, Vp, Bp, g.lx, g.mx);
    }
    cp_async_commit();
    for (int ch = 0; ch < nch; ch++) {
        const int sb = ch & 1;
        StraightStage& st = stage[sb];
        const ChunkGeom c = sb ? geo1 : geo0;
        cp_async_wait1();
        __syncthreads();
        // ---- scan this thread's line over the chunk
        const int bofs = steep ? (c.base & 1) : 0;
#pragma unroll 4
        for (int kk = 0; kk < kSteps; kk++) {
            const int s = dir > 0 ? kk : kSteps - 1 - kk;
            const int y = c.y0 + s;
            const int q = dir > 0 ? y : g.nx - y;
            const int a = t + bs[y] - c.bmin;  // tile index across lines, in [0, span)
            const int vi = steep ? s * (kSpan + 1) + a : a * (kSteps + 1) + s;
            const int bi = steep ? s * (kSpan + 4) + a + bofs : a * (kSteps + 2) + s;
            const uint16_t ob = st.b[bi];
            const uint32_t e = edge_cost(ob, w);
            const uint32_t u = ob == HARD ? 0u : min(st.v[vi], TH);
            if (v < u) {
                st.v[vi] = v | kMark;
                st.b[bi] = (uint16_t)(mtag | (uint32_t)(q - pv));
            }
            const uint32_t tt = u + ct;
            if (tt < v) { v = tt; pv = q; }
            v += e;
        }
        __syncthreads();
        // ---- write back the marked cells, row segment by row segment
        if (!steep) {
            for (int k = t; k < c.span * kSteps; k += lines) {
                const int r = k >> 4, s = k & 15;
                const uint32_t x = st.v[r * (kSteps + 1) + s];
                if ((x >> 30) == 2u) {
                    const int64_t id = ((int64_t)((c.base + r) & g.mx) << g.lx) + c.y0 + s;
                    Vp[id] = x & ~kMark;
                    Lp[id] = st.b[r * (kSteps + 2) + s];
                    nimp++;
                }
            }
        } else {
            for (int k = t; k < kSteps * c.span; k += lines) {
                const int s = k / c.span, xx = k - s * c.span;
                const uint32_t x = st.v[s * (kSpan + 1) + xx];
                if ((x >> 30) == 2u) {
                    const int64_t id = ((int64_t)(c.y0 + s) << g.lx) + ((c.base + xx) & g.mx);
                    Vp[id] = x & ~kMark;
                    Lp[id] = st.b[s * (kSpan + 4) + xx + bofs];
                    nimp++;
                }
            }
        }
        __syncthreads();
        if (ch + 2 < nch) {
            const ChunkGeom nxt = chunk_geom(bs, ch + 2, dir, g.nx, X0, lines, g.mx);
            if (sb) geo1 = nxt;
            else geo0 = nxt;
            straight_issue(stage[sb], nxt, steep, Vp, Bp, g.lx, g.mx);
        }
        cp_async_commit();
    }
    cp_async_wait0();
    if (vol.improved) count_improved(vol.improved, nimp);
}

// Grids narrower than one 16-step chunk: the plain per-thread loop.
__global__ void k_straight_small(DevGrid g, Volumes vol, int mu) {
    const int T = blockIdx.y;
    const int xq = threadIdx.x;
    const PlaneInfo pi = g.plane[T];
    const int dir = mu == SF ? pi.jsign : -pi.jsign;
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    uint32_t* Vp = vol.V + (int64_t)T * nxy;
    uint16_t* Lp = vol.L + (int64_t)T * nxy;
    const uint16_t* Bp = vol.B + (int64_t)T * nxy;
    const uint32_t mtag = (uint32_t)mu << 13;
    uint32_t v = 0xFFFFFFFFu, nimp = 0;
    int pv = 0;
    for (int q = 0; q < g.nx; q++) {
        const int y = (dir * q) & g.mx;
        const int col = (xq + bs[y]) & g.mx;
        const uint32_t id = pi.iflag ? (uint32_t)(col | (y << g.lx)) : (uint32_t)(y | (col << g.lx));
        const uint16_t ob = Bp[id];
        const uint32_t e = edge_cost(ob, pi.wS);
        const uint32_t u = ob == HARD ? 0u : min(Vp[id], TH);
        if (v < u) {
            Vp[id] = v;
            Lp[id] = (uint16_t)(mtag | (uint32_t)(q - pv));
            nimp++;
        }
        const uint32_t tt = u + g.ct;
        if (tt < v) { v = tt; pv = q; }
        v += e;
    }
    if (vol.improved) count_improved(vol.improved, nimp);
}

__global__ void k_init(Volumes vol, int64_t n, int64_t start) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        vol.V[i] = i == start ? 0u : 0xFFFFFFFFu;
        vol.L[i] = NONE;
    }
}

}  // namespace

cudaError_t launch_turn(const DevGrid& g, Volumes v, int family, int asc, int mu1, int mu2, cudaStream_t s) {
    switch (g.nt) {
        case 4: return launch_turn_t<1, 4>(g, v, family, asc, mu1, mu2, s);
        case 8: return launch_turn_t<2, 4>(g, v, family, asc, mu1, mu2, s);
        case 16: return launch_turn_t<4, 4>(g, v, family, asc, mu1, mu2, s);
        case 32: return launch_turn_t<8, 4>(g, v, family, asc, mu1, mu2, s);
        case 64: return launch_turn_t<16, 4>(g, v, family, asc, mu1, mu2, s);
        case 128: return launch_turn_t<16, 8>(g, v, family, asc, mu1, mu2, s);
        case 256: return launch_turn_t<16, 16>(g, v, family, asc, mu1, mu2, s);
        case 512: return launch_turn_t<16, 32>(g, v, family, asc, mu1, mu2, s);
        case 1024: return launch_turn_t<32, 32>(g, v, family, asc, mu1, mu2, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_straight(const DevGrid& g, Volumes v, int mu, cudaStream_t s) {
    if (g.nx < kSteps) {
        k_straight_small<<<dim3(1, (unsigned)g.nt), g.nx, 0, s>>>(g, v, mu);
        return cudaGetLastError();
    }
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = 2 * sizeof(StraightStage);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(k_straight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const int tpb = g.nx < kMaxLines ? g.nx : kMaxLines;
    dim3 grid((unsigned)(g.nx / tpb), (unsigned)g.nt);
    k_straight<<<grid, tpb, smem, s>>>(g, v, mu);
    return cudaGetLastError();
}

cudaError_t launch_init(const DevGrid& g, Volumes v, int64_t start, cudaStream_t s) {
    const int64_t n = (int64_t)g.nx * g.nx * g.nt;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_init<<<(unsigned)blocks, 256, 0, s>>>(v, n, start);
    return cudaGetLastError();
}

}  // namespace nhp

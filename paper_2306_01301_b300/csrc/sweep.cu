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
#include <atomic>

#include <cooperative_groups.h>

#include "internal.h"
#include "turn_scan.cuh"

namespace nhp {
namespace {

__device__ __forceinline__ uint32_t edge_cost(uint16_t b, uint32_t w) {
    return b == HARD ? TH : (w * (uint32_t)b) >> 8;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Decode pass p of a query with N cycles (the schedule in internal.h).
struct PassInfo {
    bool active, turn;
    int family, asc, mu1, mu2;  // turns: curve family, first scan direction, maneuvers
    int mu;                     // straights
};
__device__ __forceinline__ PassInfo decode_pass(int p, int N) {
    PassInfo r{};
    r.active = p >= 0 && N > 0 && p <= 4 * N;
    r.turn = (p & 1) == 0;
    if (p == 0) { r.family = 0; r.asc = 1; r.mu1 = LF; r.mu2 = -1; }
    else if ((p & 3) == 2) { r.family = 1; r.asc = 1; r.mu1 = RB; r.mu2 = RF; }
    else if ((p & 3) == 0) { r.family = 0; r.asc = 0; r.mu1 = LB; r.mu2 = (p >> 2) < N ? LF : -1; }
    r.mu = (p & 3) == 1 ? SF : SB;
    return r;
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
// A block owns 32 chains (lanes: 32 neighbouring x' of one y', so every
// heading plane is read as one rotated 128-byte row segment) and SL sections
// of K headings each (warps).  With CL = 2 a thread-block cluster of two
// blocks shares the chains: block rank r holds headings [r*NT/2, (r+1)*NT/2)
// and the two halves exchange their composite section maps through
// distributed shared memory, so two independent 512-thread blocks fit on an
// SM and overlap each other's load and compute phases.
// Scan-order positions: ascending r = T, descending r = NT-1-T; positions of
// the storing (second) loop are r + NT.

template <int K, int SL, int CL>
struct TurnSmem {
    int2 cell[K * SL];   // per heading: (offset of the chain row in the volume, x shift)
    TurnShared<K, SL, 2> sh;
};

// Largest q with off[q] <= item (off[0] = 0, strictly increasing).
__device__ __forceinline__ int find_item(const int32_t* __restrict__ off, int nq, int64_t item) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)__ldg(off + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The plain plan's cells for turn_scan: entering costs the cell's value
// plus the maneuver's transition edges; labels are the step count alone.
template <int K>
struct PlainCells {
    uint32_t (&u)[K];
    const uint32_t (&ev)[K];
    uint32_t ct;
    __device__ __forceinline__ uint32_t bound(int k) const { return u[k]; }
    __device__ __forceinline__ void store(int k, uint32_t v) { u[k] = v; }
    __device__ __forceinline__ uint32_t ent(int k) const { return u[k] + ct; }
    __device__ __forceinline__ uint32_t e(int k) const { return ev[k]; }
    __device__ __forceinline__ int tag(int) const { return 0; }
    __device__ __forceinline__ uint32_t label_bits(int pv, int q) const { return (uint32_t)(q - pv); }
};

// One 32-chain tile of one query: load, scan (one or two maneuvers), store.
// `scans` counts the block's scans so far (it picks the set of section maps).
template <int K, int SL, int CL>
__device__ __forceinline__ void turn_tile(const QueryDesc& Q, const PassInfo& ps, int64_t tile, int rank,
                                          TurnSmem<K, SL, CL>& sm, int& scans, uint32_t ct_a, uint32_t ct_b,
                                          int pass_all) {
    constexpr int NTL = K * SL;  // headings held by this block
    const int tid = threadIdx.x, lane = tid & 31, sec = tid >> 5;
    const DevGrid g = Q.g;
    const Volumes vol = Q.v;
    const int family = ps.family, asc = ps.asc, mu1 = ps.mu1, mu2 = ps.mu2;
    const int T0 = rank * NTL;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t chain = tile * 32 + lane;
    const bool valid = chain < nxy;
    const int xq = (int)(chain & g.mx), yq = (int)((chain >> g.lx) & g.mx);
    // With Nx >= 32 all 32 chains of the block share y', so each heading's
    // chain row has one offset: precompute (row offset, x shift) per heading.
    // A warp reads only the entries of its own headings, so it writes them
    // itself and no block barrier is needed.
    const bool row_uniform = g.nx >= 32;
    if (lane < K) {
        const int t = sec * K + lane;
        const int4 b = g.beta4[T0 + t];
        const int bx = family ? b.z : b.x, by = family ? b.w : b.y;
        const int ybase = row_uniform ? (int)((tile * 32 >> g.lx) & g.mx) : 0;
        // volumes hold at most 2^32 cells, so 32-bit offsets suffice
        if (row_uniform)
            sm.cell[t] = make_int2((int)(uint32_t)((((ybase + by) & g.mx) << g.lx) + (int64_t)(T0 + t) * nxy), bx);
        else
            sm.cell[t] = make_int2((int)(uint32_t)((int64_t)(T0 + t) * nxy), (bx & g.mx) | ((by & g.mx) << 16));
    }
    __syncwarp();
    const uint32_t w = g.wA;
    auto cell_index = [&](int T) -> uint32_t {
        const int2 c = sm.cell[T];
        if (row_uniform) return (uint32_t)c.x + (uint32_t)((xq + c.y) & g.mx);
        const int bx = c.y & 0xFFFF, by = c.y >> 16;
        return (uint32_t)c.x + (uint32_t)(((xq + bx) & g.mx) | (((yq + by) & g.mx) << g.lx));
    };

    uint32_t u[K], e[K];
    uint32_t a = 0;     // summed edge costs of this thread's section
    bool live = false;  // the section holds a reached, non-hard cell
#pragma unroll
    for (int k = 0; k < K; k++) {
        const uint32_t id = cell_index(sec * K + k);
        uint32_t vv = 0xFFFFFFFFu;
        uint16_t ob = HARD;
        if (valid && NHP_IN(id, nxy * g.nt, Q.err, 1)) {
            vv = __ldg(vol.V + id);
            ob = __ldg(vol.B + id);
        }
        e[k] = edge_cost(ob, w);
        u[k] = ob == HARD ? 0u : min(vv, TH);
        a = min(a + e[k], TH);
        live |= vv < TH;  // a hard cell's value stays INF (never stored; the start is not hard)
    }
    uint32_t chg = 0;
    // the launch's costs (kernel parameters), else this query's own
    const uint32_t ct1 = ct_a != kCostPerQuery ? ct_a : __ldg(Q.g.ctm + mu1);
    int mb = scans & 1;
    PlainCells<K> c1{u, e, ct1};
    if (asc) turn_scan<K, SL, CL, 2, true>(c1, chg, label_tag(Q, mu1), sec, lane, rank, 0, mb, a, live, sm.sh);
    else turn_scan<K, SL, CL, 2, false>(c1, chg, label_tag(Q, mu1), sec, lane, rank, 0, mb, a, live, sm.sh);
    scans++;
    if (mu2 >= 0) {
        live = live || chg != 0;
        mb = scans & 1;
        const uint32_t ct2 = ct_b != kCostPerQuery ? ct_b : __ldg(Q.g.ctm + mu2);
        PlainCells<K> c2{u, e, ct2};
        if (asc) turn_scan<K, SL, CL, 2, false>(c2, chg, label_tag(Q, mu2), sec, lane, rank, 1, mb, a, live, sm.sh);
        else turn_scan<K, SL, CL, 2, true>(c2, chg, label_tag(Q, mu2), sec, lane, rank, 1, mb, a, live, sm.sh);
        scans++;
    }
    if (vol.improved) {
        count_improved(vol.improved, __popc(chg));
        if (__syncthreads_or(chg != 0) && threadIdx.x == 0) atomicAdd(vol.improved + 2, 1ull);
    }
    if (valid && chg) {
        uint32_t* conv = Q.conv;  // convergence record: this pass lowered a cell
        if (conv) conv[pass_all >= 0 ? pass_all : Q.pass] = 1u;
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (chg & (1u << k)) {
                const uint32_t id = cell_index(sec * K + k);
                if (NHP_IN(id, nxy * g.nt, Q.err, 2)) {
                    vol.V[id] = u[k];
                    vol.L[id] = sm.sh.lab[k][tid];
                }
            }
        }
    }
}

// Grid: CL blocks per work item.  Without item_off, item = query * tiles +
// tile; with it, items of different queries (any Nx, this N_theta) follow
// each other.  Blocks loop over items when the grid is smaller than the
// work (persistent launch); every block of a cluster visits the same items.
template <int K, int SL, int CL>
__global__ void __launch_bounds__(32 * SL, 1024 / (32 * SL) > 4 ? 4 : (1024 / (32 * SL) < 1 ? 1 : 1024 / (32 * SL)))
k_turn(const QueryDesc* __restrict__ qd, const int32_t* __restrict__ item_off, int nq, int64_t items,
       int tiles_per_q, int pass_all, uint32_t ct_a, uint32_t ct_b) {
    __shared__ TurnSmem<K, SL, CL> sm;
    const int rank = CL == 1 ? 0 : (int)(blockIdx.x % CL);
    const int64_t stride = gridDim.x / CL;
    int scans = 0;
    for (int64_t it = blockIdx.x / CL; it < items; it += stride) {
        int q;
        int64_t tile;
        if (item_off) {
            q = find_item(item_off, nq, it);
            tile = it - __ldg(item_off + q);
        } else {
            q = (int)(it / tiles_per_q);
            tile = it - (int64_t)q * tiles_per_q;
        }
        const QueryDesc& Q = qd[q];
        const PassInfo ps = decode_pass(pass_all >= 0 ? pass_all : Q.pass, Q.n_cycles);
        if (!ps.active || !ps.turn) continue;  // uniform over the block and the cluster
        turn_tile<K, SL, CL>(Q, ps, tile, rank, sm, scans, ct_a, ct_b, pass_all);
        // the partner blocks read this block's shared memory, and the next
        // item rewrites it: a cluster leaves the tile together.  Without a
        // cluster the next tile needs no barrier (own row entries, per-thread
        // labels, alternating section maps).
        if (CL > 1) cooperative_groups::this_cluster().sync();
    }
}

template <int K, int SL, int CL>
cudaError_t launch_turn_t(const Group& gr, int pass, cudaStream_t s) {
    // the pass's two transition costs when every query shares them
    uint32_t ca = kCostPerQuery, cb = kCostPerQuery;
    if (gr.ctm && pass >= 0 && pass_is_turn(pass)) {
        int m1, m2;
        turn_pass_maneuvers(pass, &m1, &m2);
        ca = gr.ctm[m1];
        cb = m2 >= 0 ? gr.ctm[m2] : 0u;
    }
    const int tiles = (int)turn_items(gr.lx);
    const int64_t items = gr.item_off ? gr.items : (int64_t)tiles * gr.nq;
    if (items <= 0) return cudaSuccess;
    const int64_t blocks = gr.grid > 0 && gr.grid < items ? gr.grid : items;
    if (CL == 1) {
        k_turn<K, SL, CL><<<(unsigned)blocks, 32 * SL, 0, s>>>(gr.d, gr.item_off, gr.nq, items, tiles, pass, ca, cb);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(blocks * CL));
    cfg.blockDim = dim3(32 * SL);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_turn<K, SL, CL>, gr.d, gr.item_off, gr.nq, items, tiles, pass, ca, cb);
}

template <int K, int SL, int CL>
int turn_occupancy() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_turn<K, SL, CL>, 32 * SL, 0) != cudaSuccess) return 0;
    return n;
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
// Tiles are filled with 16-byte cp.async copies (whole row segments, so
// global reads coalesce in both cases), two stages deep: the next chunk is in
// flight while the current one is scanned.  The two stages take 54 KB, so four
// 256-line blocks fit on an SM.  Changed cells are marked in the tile (bit 31
// of the value, the label in place of the obstacle value) and written back
// row segment by row segment.
constexpr int kSteps = 16;
constexpr int kMaxLines = 256;
constexpr int kSpan = kMaxLines + kSteps;  // tile extent across lines (>= lines + 15)
// Shallow tiles: rows = grid rows, 16 step columns, 16-byte aligned rows.
constexpr int kShV = 16;                   // word pitch: 4 chunks of 16 B, swizzled (shv)
constexpr int kShB = 16;                   // half pitch: 2 chunks of 16 B, swizzled (shb)
// Steep tiles: 16 step rows, columns = an aligned superset of the segment.
constexpr int kStV = kSpan + 8;            // word pitch   (segment + up to 3 lead + tail chunk)
constexpr int kStB = kSpan + 16;           // half pitch
constexpr int kVWords = (kSpan * kShV > kSteps * kStV) ? kSpan * kShV : kSteps * kStV;
constexpr int kBHalves = (kSpan * kShB > kSteps * kStB) ? kSpan * kShB : kSteps * kStB;
constexpr uint32_t kMark = 0x80000000u;    // changed; stored values are < TH

constexpr int kMaskWords = (kSpan + 31) / 32;

struct __align__(16) StraightStage {
    uint32_t v[kVWords];
    uint16_t b[kBHalves];
    uint32_t mask[kMaskWords];  // tile rows (shallow) or steps (steep, word 0) holding a changed cell
    int16_t bs[kSteps];         // Bs(y0 + s) - min over the chunk, s = 0..15
};


struct ChunkGeom {
    int y0;     // first step of the chunk (ascending y')
    int span;   // lines + (max - min of Bs over the chunk)
    int base;   // grid coordinate of tile index 0 across lines (masked)
};

__device__ __forceinline__ ChunkGeom chunk_geom(const int16_t* bs, int ch, int dir, int nx, int X0, int lines,
                                                int mx) {
    ChunkGeom c;
    c.y0 = dir > 0 ? ch * kSteps : nx - (ch + 1) * kSteps;
    const int b0 = bs[c.y0], b1 = bs[c.y0 + kSteps - 1];
    c.span = lines + max(b0, b1) - min(b0, b1);
    c.base = (X0 + min(b0, b1)) & mx;
    return c;
}

// Word / half index of tile element (step s, index a across lines).
// Shallow tiles keep whole 16-byte chunks (cp.async granules) but place
// chunk j of row r at j ^ (r >> 1) (V) or j ^ (r >> 2) (B), so a column read
// across 32 consecutive rows meets 8 row classes of banks, as an 80-byte /
// 48-byte padded pitch would, with no padding.
__device__ __forceinline__ int shv(int r, int s) { return r * kShV + ((((s >> 2) ^ (r >> 1)) & 3) << 2) + (s & 3); }
__device__ __forceinline__ int shb(int r, int s) { return r * kShB + ((((s >> 3) ^ (r >> 2)) & 1) << 3) + (s & 7); }

template <bool STEEP>
__device__ __forceinline__ int vidx(int s, int a, int base) {
    return STEEP ? s * kStV + a + (base & 3) : shv(a, s);
}
template <bool STEEP>
__device__ __forceinline__ int bidx(int s, int a, int base) {
    return STEEP ? s * kStB + a + (base & 7) : shb(a, s);
}

template <bool STEEP>
__device__ __forceinline__ void straight_issue(StraightStage& st, const ChunkGeom& c, const int16_t* bs,
                                               const uint32_t* Vp, const uint16_t* Bp, int lx, int mx,
                                               int32_t* err) {
    const int t = threadIdx.x, nt = blockDim.x;
    if (t < kSteps) st.bs[t] = (int16_t)(bs[c.y0 + t] - min(bs[c.y0], bs[c.y0 + kSteps - 1]));
    if (t < kMaskWords) st.mask[t] = 0;
    if (!STEEP) {
        // row r: 16 V words = 4 chunks (thread t copies chunk t & 3 of every
        // (nt/4)-th row), 16 B halves = 2 chunks (chunk t & 1 of every
        // (nt/2)-th row), all aligned
        const int jv = t & 3, jb = t & 1;
        for (int r = t >> 2; r < c.span; r += nt >> 2) {
            const uint32_t row = ((uint32_t)((c.base + r) & mx) << lx) + (uint32_t)c.y0;
            if (NHP_IN(row + 4 * jv + 3, (int64_t)1 << (2 * lx), err, 3) && NHP_IN(shv(r, 4 * jv) + 3, kVWords, err, 4))
                cp_async16(&st.v[shv(r, 4 * jv)], Vp + row + 4 * jv);
        }
        for (int r = t >> 1; r < c.span; r += nt >> 1) {
            const uint32_t row = ((uint32_t)((c.base + r) & mx) << lx) + (uint32_t)c.y0;
            if (NHP_IN(row + 8 * jb + 7, (int64_t)1 << (2 * lx), err, 3) && NHP_IN(shb(r, 8 * jb) + 7, kBHalves, err, 4))
                cp_async16(&st.b[shb(r, 8 * jb)], Bp + row + 8 * jb);
        }
    } else {
        // step row s: the aligned chunks covering columns [base, base + span)
        const int a4 = c.base & ~3, nv = ((c.base & 3) + c.span + 3) >> 2;
        const int a8 = c.base & ~7, nb = ((c.base & 7) + c.span + 7) >> 3;
        const int per = nv + nb;                   // chunks per step row (< blockDim for Nx >= 16)
        const int rpp = max(1, nt / per);          // step rows copied per pass of the block
        const int s0 = t / per, j = t - s0 * per;  // one division per thread and chunk
        if (s0 < rpp) {
            for (int s = s0; s < kSteps; s += rpp) {
                const uint32_t row = (uint32_t)(c.y0 + s) << lx;
                if (j < nv) {
                    if (NHP_IN(row + ((a4 + 4 * j) & mx) + 3, (int64_t)1 << (2 * lx), err, 3) &&
                        NHP_IN(s * kStV + 4 * j + 3, kVWords, err, 4))
                        cp_async16(&st.v[s * kStV + 4 * j], Vp + row + ((a4 + 4 * j) & mx));
                } else {
                    if (NHP_IN(row + ((a8 + 8 * (j - nv)) & mx) + 7, (int64_t)1 << (2 * lx), err, 3) &&
                        NHP_IN(s * kStB + 8 * (j - nv) + 7, kBHalves, err, 4))
                        cp_async16(&st.b[s * kStB + 8 * (j - nv)], Bp + row + ((a8 + 8 * (j - nv)) & mx));
                }
            }
        }
    }
}

template <bool STEEP, bool FWD>
__device__ __forceinline__ void straight_body(const DevGrid& g, const Volumes& vol, int mu, uint32_t mtag, int T,
                                              int lblock, StraightStage* stage, const PlaneInfo& pi,
                                              uint32_t* conv_p, int32_t* err) {
    const int lines = blockDim.x;  // min(Nx, 128 or 256)
    const int X0 = lblock * lines;
    const int t = threadIdx.x;
    constexpr int dir = FWD ? 1 : -1;  // direction of y' along the sweep
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    uint32_t* Vp = vol.V + (int64_t)T * nxy;
    uint16_t* Lp = vol.L + (int64_t)T * nxy;
    const uint16_t* Bp = vol.B + (int64_t)T * nxy;
    const uint32_t w = pi.wS, ct = mu == SF ? g.ctm[SF] : g.ctm[SB];
    // Sweep order: dir > 0 visits y' = 0, 1, .., Nx-1 (q = y'); dir < 0
    // visits Nx-1, .., 1, 0 (q = Nx - y').  Starting at Nx-1 with nothing
    // carried equals starting at the wall cell y' = 0, which carries nothing.
    uint32_t v = 0xFFFFFFFFu;
    int pv = 0;
    uint32_t nimp = 0;
    const int nch = g.nx / kSteps;

    ChunkGeom geo0 = chunk_geom(bs, 0, dir, g.nx, X0, lines, g.mx), geo1 = geo0;
    straight_issue<STEEP>(stage[0], geo0, bs, Vp, Bp, g.lx, g.mx, err);
    cp_async_commit();
    if (nch > 1) {
        geo1 = chunk_geom(bs, 1, dir, g.nx, X0, lines, g.mx);
        straight_issue<STEEP>(stage[1], geo1, bs, Vp, Bp, g.lx, g.mx, err);
    }
    cp_async_commit();
    for (int ch = 0; ch < nch; ch++) {
        const int sb = ch & 1;
        StraightStage& st = stage[sb];
        const ChunkGeom c = sb ? geo1 : geo0;
        cp_async_wait1();
        __syncthreads();
        const int qbase = FWD ? c.y0 : g.nx - c.y0;  // q = qbase + dir * s
        bool marked = false;
#pragma unroll
        for (int kk = 0; kk < kSteps; kk++) {
            const int s = FWD ? kk : kSteps - 1 - kk;
            const int a = t + st.bs[s];  // tile index across lines, in [0, span)
            const int vi = vidx<STEEP>(s, a, c.base), bi = bidx<STEEP>(s, a, c.base);
            if (!NHP_IN(vi, kVWords, err, 5) || !NHP_IN(bi, kBHalves, err, 5)) continue;
            const uint16_t ob = st.b[bi];
            const uint32_t e = edge_cost(ob, w);
            const uint32_t u = ob == HARD ? 0u : min(st.v[vi], TH);
            const int q = qbase + (FWD ? s : -s);
            if (v < u) {
                st.v[vi] = v | kMark;
                st.b[bi] = (uint16_t)(mtag | (uint32_t)(q - pv));
                marked = true;
                if (STEEP) atomicOr(&st.mask[0], 1u << s);
                else atomicOr(&st.mask[a >> 5], 1u << (a & 31));
            }
            const uint32_t tt = u + ct;
            if (tt < v) { v = tt; pv = q; }
            v += e;
        }
        // write back the marked cells (only when the block has any)
        if (__syncthreads_or(marked)) {
            if (conv_p && t == 0) *conv_p = 1u;
            if (!STEEP) {
                // the rows flagged in the mask, two per warp (16 lanes each)
                const int lane = t & 31, s = lane & 15, upper = lane >> 4;
                const bool two = lines >= 32;
                for (int i = t >> 5; i < kMaskWords; i += (lines + 31) >> 5) {
                    uint32_t m = st.mask[i];  // the same for the whole warp
                    while (m) {
                        int bit = __ffs(m) - 1;
                        m &= m - 1;
                        bool act = !upper;
                        if (two) {
                            if (upper) {
                                act = m != 0;
                                bit = act ? __ffs(m) - 1 : 0;
                            }
                            if (m) m &= m - 1;
                        }
                        if (act) {
                            const int r = i * 32 + bit;
                            const uint32_t x = st.v[shv(r, s)];
                            if ((x >> 30) == 2u) {
                                const uint32_t id = ((uint32_t)((c.base + r) & g.mx) << g.lx) + c.y0 + s;
                                if (NHP_IN(id, (int64_t)g.nx * g.nx, err, 6)) {
                                    Vp[id] = x & ~kMark;
                                    Lp[id] = st.b[shb(r, s)];
                                }
                                nimp++;
                            }
                        }
                    }
                }
            } else {
                const uint32_t steps = st.mask[0];
                for (int s = 0; s < kSteps; s++) {
                    if (!(steps & (1u << s))) continue;
                    for (int xx = t; xx < c.span; xx += lines) {
                        const uint32_t x = st.v[vidx<true>(s, xx, c.base)];
                        if ((x >> 30) == 2u) {
                            const uint32_t id = ((uint32_t)(c.y0 + s) << g.lx) + ((c.base + xx) & g.mx);
                            if (NHP_IN(id, (int64_t)g.nx * g.nx, err, 6)) {
                                Vp[id] = x & ~kMark;
                                Lp[id] = st.b[bidx<true>(s, xx, c.base)];
                            }
                            nimp++;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (ch + 2 < nch) {
            const ChunkGeom nxt = chunk_geom(bs, ch + 2, dir, g.nx, X0, lines, g.mx);
            if (sb) geo1 = nxt;
            else geo0 = nxt;
            straight_issue<STEEP>(stage[sb], nxt, bs, Vp, Bp, g.lx, g.mx, err);
        }
        cp_async_commit();
    }
    cp_async_wait0();
    if (vol.improved) count_improved(vol.improved + 1, nimp);
}

// ------------------------------------------- straights of the gear states
// A straight layer of the two gear states (gear.cu) on the staged tiles of
// the plain straight kernel: the same chunks of the own gear's values and
// B, plus the other gear's values in a third tile.  Entering a line at a
// cell costs the cheaper of its own gear's value and the other gear's value
// plus the penalty (own gear on a tie); a store must beat the own gear's
// value and records whether the segment was entered from the other gear
// (label bit 12).  Values at or above TH mean unreached (the host picks
// this kernel only when the finite costs stay below TH).
struct __align__(16) GearStage {
    StraightStage s;  // own gear's values, B (labels of marked cells), mask, shear
    uint32_t vo[kVWords];
};

// The other gear's chunk tile, copied like the own gear's values.
template <bool STEEP>
__device__ __forceinline__ void gear_issue_other(uint32_t* vo, const ChunkGeom& c, const uint32_t* Vop, int lx,
                                                 int mx, int32_t* err) {
    const int t = threadIdx.x, nt = blockDim.x;
    [[maybe_unused]] const int64_t plane = (int64_t)1 << (2 * lx);  // bounds-check build only
    if (!STEEP) {
        const int jv = t & 3;
        for (int r = t >> 2; r < c.span; r += nt >> 2) {
            const uint32_t row = ((uint32_t)((c.base + r) & mx) << lx) + (uint32_t)c.y0;
            if (NHP_IN(row + 4 * jv + 3, plane, err, 32) && NHP_IN(shv(r, 4 * jv) + 3, kVWords, err, 33))
                cp_async16(&vo[shv(r, 4 * jv)], Vop + row + 4 * jv);
        }
    } else {
        const int a4 = c.base & ~3, nv = ((c.base & 3) + c.span + 3) >> 2;
        const int rpp = max(1, nt / nv);
        const int s0 = t / nv, j = t - s0 * nv;
        if (s0 < rpp)
            for (int s = s0; s < kSteps; s += rpp) {
                const uint32_t gi = ((uint32_t)(c.y0 + s) << lx) + ((a4 + 4 * j) & mx);
                if (NHP_IN(gi + 3, plane, err, 32) && NHP_IN(s * kStV + 4 * j + 3, kVWords, err, 33))
                    cp_async16(&vo[s * kStV + 4 * j], Vop + gi);
            }
    }
}

template <bool STEEP, bool FWD>
__device__ __forceinline__ void gear_straight_body(const GearLayer& a, int mu, int T, int lblock, GearStage* stage) {
    const DevGrid& g = a.g;
    const int lines = blockDim.x;
    const int X0 = lblock * lines;
    const int t = threadIdx.x;
    constexpr int dir = FWD ? 1 : -1;
    const PlaneInfo pi = g.plane[T];
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int G = (mu == SB) ? 1 : 0;  // the backward straight belongs to the reverse gear
    uint32_t* Vp = (G ? a.Vr : a.Vf) + (int64_t)T * nxy;
    uint16_t* Lp = (G ? a.Lr : a.Lf) + (int64_t)T * nxy;
    const uint32_t* Vop = (G ? a.Vf : a.Vr) + (int64_t)T * nxy;
    const uint16_t* Bp = a.B + (int64_t)T * nxy;
    const uint32_t w = pi.wS, ct = a.cin + a.cout, pen = a.pen;
    const uint32_t mtag = (uint32_t)mu << 13;
    uint32_t v = 0xFFFFFFFFu;
    int pv = 0;
    uint32_t pvo = 0;  // the carried segment was entered from the other gear
    const int nch = g.nx / kSteps;
    ChunkGeom geo0 = chunk_geom(bs, 0, dir, g.nx, X0, lines, g.mx), geo1 = geo0;
    straight_issue<STEEP>(stage[0].s, geo0, bs, Vp, Bp, g.lx, g.mx, a.err);
    gear_issue_other<STEEP>(stage[0].vo, geo0, Vop, g.lx, g.mx, a.err);
    cp_async_commit();
    if (nch > 1) {
        geo1 = chunk_geom(bs, 1, dir, g.nx, X0, lines, g.mx);
        straight_issue<STEEP>(stage[1].s, geo1, bs, Vp, Bp, g.lx, g.mx, a.err);
        gear_issue_other<STEEP>(stage[1].vo, geo1, Vop, g.lx, g.mx, a.err);
    }
    cp_async_commit();
    for (int ch = 0; ch < nch; ch++) {
        const int sb = ch & 1;
        StraightStage& st = stage[sb].s;
        const uint32_t* vo = stage[sb].vo;
        const ChunkGeom c = sb ? geo1 : geo0;
        cp_async_wait1();
        __syncthreads();
        const int qbase = FWD ? c.y0 : g.nx - c.y0;
        bool marked = false;
#pragma unroll
        for (int kk = 0; kk < kSteps; kk++) {
            const int s = FWD ? kk : kSteps - 1 - kk;
            const int ai = t + st.bs[s];
            const int vi = vidx<STEEP>(s, ai, c.base), bi = bidx<STEEP>(s, ai, c.base);
            if (!NHP_IN(vi, kVWords, a.err, 34) || !NHP_IN(bi, kBHalves, a.err, 34)) continue;
            const uint16_t ob = st.b[bi];
            const bool hard = ob == HARD;
            const uint32_t e = edge_cost(ob, w);
            const uint32_t us = hard ? 0u : min(st.v[vi], TH);
            const uint32_t to = min(vo[vi], TH) + pen + ct, ts = us + ct;
            const int q = qbase + (FWD ? s : -s);
            if (v < us) {
                st.v[vi] = v | kMark;
                st.b[bi] = (uint16_t)(mtag | (pvo << 12) | (uint32_t)(q - pv));
                marked = true;
                if (STEEP) atomicOr(&st.mask[0], 1u << s);
                else atomicOr(&st.mask[ai >> 5], 1u << (ai & 31));
            }
            const bool o = !hard && to < ts;
            const uint32_t tt = o ? to : ts;
            if (tt < v) { v = tt; pv = q; pvo = o; }
            v += e;
        }
        if (__syncthreads_or(marked)) {
            if (!STEEP) {
                for (int r = t; r < c.span; r += lines) {
                    if (!(st.mask[r >> 5] & (1u << (r & 31)))) continue;
                    for (int s2 = 0; s2 < kSteps; s2++) {
                        const uint32_t x = st.v[shv(r, s2)];
                        if ((x >> 30) == 2u) {
                            const uint32_t id = ((uint32_t)((c.base + r) & g.mx) << g.lx) + c.y0 + s2;
                            if (!NHP_IN(id, nxy, a.err, 35)) continue;
                            Vp[id] = x & ~kMark;
                            Lp[id] = st.b[shb(r, s2)];
                        }
                    }
                }
            } else {
                const uint32_t steps = st.mask[0];
                for (int s2 = 0; s2 < kSteps; s2++) {
                    if (!(steps & (1u << s2))) continue;
                    for (int xx = t; xx < c.span; xx += lines) {
                        const uint32_t x = st.v[vidx<true>(s2, xx, c.base)];
                        if ((x >> 30) == 2u) {
                            const uint32_t id = ((uint32_t)(c.y0 + s2) << g.lx) + ((c.base + xx) & g.mx);
                            if (!NHP_IN(id, nxy, a.err, 35)) continue;
                            Vp[id] = x & ~kMark;
                            Lp[id] = st.b[bidx<true>(s2, xx, c.base)];
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (ch + 2 < nch) {
            const ChunkGeom nxt = chunk_geom(bs, ch + 2, dir, g.nx, X0, lines, g.mx);
            if (sb) geo1 = nxt;
            else geo0 = nxt;
            straight_issue<STEEP>(stage[sb].s, nxt, bs, Vp, Bp, g.lx, g.mx, a.err);
            gear_issue_other<STEEP>(stage[sb].vo, nxt, Vop, g.lx, g.mx, a.err);
        }
        cp_async_commit();
    }
    cp_async_wait0();
}

// One block per (heading plane, block of `lines` lines).
__global__ void __launch_bounds__(kMaxLines, 2) k_gear_straight_tiled(const GearLayer a, int mu) {
    extern __shared__ __align__(16) unsigned char gear_straight_smem[];
    GearStage* stage = reinterpret_cast<GearStage*>(gear_straight_smem);
    const int lines = blockDim.x;
    const int bpp = a.g.nx / lines;
    const int T = (int)(blockIdx.x / bpp), lblock = (int)(blockIdx.x - (unsigned)T * bpp);
    const PlaneInfo pi = a.g.plane[T];
    const bool fwd = (mu == SF ? pi.jsign : -pi.jsign) > 0;
    if (pi.iflag) {
        if (fwd) gear_straight_body<true, true>(a, mu, T, lblock, stage);
        else gear_straight_body<true, false>(a, mu, T, lblock, stage);
    } else {
        if (fwd) gear_straight_body<false, true>(a, mu, T, lblock, stage);
        else gear_straight_body<false, false>(a, mu, T, lblock, stage);
    }
}

// Grid: one block per (query, heading plane, line block) work item, the
// items of a query ordered plane by plane.  Without item_off every query has
// Nx = 2^lx; with it, queries of any Nx >= lines follow each other.  Blocks
// loop over items when the grid is smaller than the work.
__global__ void __launch_bounds__(kMaxLines, 4)
k_straight(const QueryDesc* __restrict__ qd, const int32_t* __restrict__ item_off, int nq, int64_t items,
           int items_per_q, int pass_all) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StraightStage* stage = reinterpret_cast<StraightStage*>(smem_raw);
    const int lines = blockDim.x;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        int q;
        int64_t rem;
        if (item_off) {
            q = find_item(item_off, nq, it);
            rem = it - __ldg(item_off + q);
        } else {
            q = (int)(it / items_per_q);
            rem = it - (int64_t)q * items_per_q;
        }
        const QueryDesc& Q = qd[q];
        const int p = pass_all >= 0 ? pass_all : Q.pass;
        const PassInfo ps = decode_pass(p, Q.n_cycles);
        if (!ps.active || ps.turn) continue;  // uniform over the block
        uint32_t* conv_p = Q.conv ? Q.conv + p : nullptr;
        const DevGrid g = Q.g;
        const Volumes vol = Q.v;
        const int mu = ps.mu;
        const uint32_t mtag = label_tag(Q, mu);
        const int bpp = g.nx / lines;  // line blocks per plane (powers of two)
        const int T = (int)(rem / bpp), lblock = (int)(rem - (int64_t)T * bpp);
        const PlaneInfo pi = g.plane[T];
        const bool fwd = (mu == SF ? pi.jsign : -pi.jsign) > 0;
        if (pi.iflag) {
            if (fwd) straight_body<true, true>(g, vol, mu, mtag, T, lblock, stage, pi, conv_p, Q.err);
            else straight_body<true, false>(g, vol, mu, mtag, T, lblock, stage, pi, conv_p, Q.err);
        } else {
            if (fwd) straight_body<false, true>(g, vol, mu, mtag, T, lblock, stage, pi, conv_p, Q.err);
            else straight_body<false, false>(g, vol, mu, mtag, T, lblock, stage, pi, conv_p, Q.err);
        }
        if (it + gridDim.x < items) __syncthreads();  // the stages are refilled by the next item
    }
}

// Grids narrower than one 16-step chunk: the plain per-thread loop.
__global__ void k_straight_small(const QueryDesc* __restrict__ qd, int pass_all) {
    const QueryDesc& Q = qd[blockIdx.x];
    const int p = pass_all >= 0 ? pass_all : Q.pass;
    const PassInfo ps = decode_pass(p, Q.n_cycles);
    if (!ps.active || ps.turn) return;
    const DevGrid g = Q.g;
    const Volumes vol = Q.v;
    const int mu = ps.mu;
    const int T = blockIdx.y;
    const int xq = threadIdx.x;
    const PlaneInfo pi = g.plane[T];
    const int dir = mu == SF ? pi.jsign : -pi.jsign;
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    const int64_t nxy = (int64_t)g.nx * g.nx;
    uint32_t* Vp = vol.V + (int64_t)T * nxy;
    uint16_t* Lp = vol.L + (int64_t)T * nxy;
    const uint16_t* Bp = vol.B + (int64_t)T * nxy;
    const uint32_t mtag = label_tag(Q, mu);
    uint32_t v = 0xFFFFFFFFu, nimp = 0;
    int pv = 0;
    for (int q = 0; q < g.nx; q++) {
        const int y = (dir * q) & g.mx;
        const int col = (xq + bs[y]) & g.mx;
        const uint32_t id = pi.iflag ? (uint32_t)(col | (y << g.lx)) : (uint32_t)(y | (col << g.lx));
        if (!NHP_IN(id, nxy, Q.err, 7)) continue;
        const uint16_t ob = Bp[id];
        const uint32_t e = edge_cost(ob, pi.wS);
        const uint32_t u = ob == HARD ? 0u : min(Vp[id], TH);
        if (v < u) {
            Vp[id] = v;
            Lp[id] = (uint16_t)(mtag | (uint32_t)(q - pv));
            nimp++;
        }
        const uint32_t tt = u + (mu == SF ? g.ctm[SF] : g.ctm[SB]);
        if (tt < v) { v = tt; pv = q; }
        v += e;
    }
    if (vol.improved) count_improved(vol.improved + 1, nimp);
    if (Q.conv && nimp) Q.conv[p] = 1u;
}

// Convergence gate of a launch group whose queries record convergence: a
// query whose last four passes lowered nothing gets pass -1 in its device
// descriptor, so the sweep kernel launched next skips its work items; with
// pass_all >= 0 the others get that pass.  Queries without records keep
// their pass.
__global__ void k_conv_gate(QueryDesc* __restrict__ qd, int nq, int pass_all) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    QueryDesc& Q = qd[i];
    const int p = pass_all >= 0 ? pass_all : Q.pass;
    Q.pass = pass_converged(Q.conv, p) ? -1 : p;
}

__global__ void k_init(const QueryDesc* __restrict__ qd) {
    const QueryDesc& Q = qd[blockIdx.y];
    const Volumes vol = Q.v;
    const int64_t n = (int64_t)Q.g.nx * Q.g.nx * Q.g.nt, start = Q.start;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (Q.conv && blockIdx.x == 0)
        for (int i = threadIdx.x; i <= 4 * Q.n_cycles; i += blockDim.x) Q.conv[i] = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        vol.V[i] = i == start ? 0u : 0xFFFFFFFFu;
        vol.L[i] = NONE;
    }
}

}  // namespace

// Shape of the 512-heading turn kernel: K headings per thread, SL sections
// (warps) per block, CL blocks per cluster, K * SL * CL = 512.  Measured on
// B300 at 512^3: one 1024-thread block per chain tile (no cluster) beats the
// 2-, 4- and 8-block clusters, whose barriers carry a memory fence, and a
// persistent variant that streamed the next tile through shared memory with
// cp.async while scanning the current one (the scans, not HBM, bound it).
#ifndef TURN512_K
#define TURN512_K 16
#define TURN512_SL 32
#define TURN512_CL 1
#endif

int turn_variants(int nt) { return nt >= 128 && nt <= 1024 ? 3 : 1; }

void turn_shape(int lt, int variant, int* K, int* SL, int* CL) {
    static const int shapes[11][3][3] = {
        {{0, 0, 0}}, {{0, 0, 0}},
        {{1, 4, 1}}, {{2, 4, 1}}, {{4, 4, 1}}, {{8, 4, 1}}, {{8, 8, 1}},
        {{16, 8, 1}, {8, 16, 1}, {16, 4, 2}},
        {{16, 16, 1}, {16, 8, 2}, {8, 32, 1}},
        {{TURN512_K, TURN512_SL, TURN512_CL}, {16, 16, 2}, {16, 8, 4}},
        {{16, 32, 2}, {16, 16, 4}, {16, 8, 8}},
    };
    const int v = lt >= 7 && lt <= 10 && variant > 0 && variant < 3 ? variant : 0;
    const int* sh = (lt >= 2 && lt <= 10) ? shapes[lt][v] : shapes[0][0];
    *K = sh[0];
    *SL = sh[1];
    *CL = sh[2];
}

// Kernel shapes per N_theta (K headings per thread, SL warps, CL blocks per
// cluster; K * SL * CL = N_theta).  Variant 0 is the default.
cudaError_t launch_turn(const Group& gr, int pass, int variant, cudaStream_t s) {
    const int v = variant < 0 ? 0 : variant;
    switch (1 << gr.lt) {
        case 4: return launch_turn_t<1, 4, 1>(gr, pass, s);
        case 8: return launch_turn_t<2, 4, 1>(gr, pass, s);
        case 16: return launch_turn_t<4, 4, 1>(gr, pass, s);
        case 32: return launch_turn_t<8, 4, 1>(gr, pass, s);
        case 64: return launch_turn_t<8, 8, 1>(gr, pass, s);
        case 128:
            return v == 1 ? launch_turn_t<8, 16, 1>(gr, pass, s)
                 : v == 2 ? launch_turn_t<16, 4, 2>(gr, pass, s)
                          : launch_turn_t<16, 8, 1>(gr, pass, s);
        case 256:
            return v == 1 ? launch_turn_t<16, 8, 2>(gr, pass, s)
                 : v == 2 ? launch_turn_t<8, 32, 1>(gr, pass, s)
                          : launch_turn_t<16, 16, 1>(gr, pass, s);
        case 512:
            return v == 1 ? launch_turn_t<16, 16, 2>(gr, pass, s)
                 : v == 2 ? launch_turn_t<16, 8, 4>(gr, pass, s)
                          : launch_turn_t<TURN512_K, TURN512_SL, TURN512_CL>(gr, pass, s);
        case 1024:
            return v == 1 ? launch_turn_t<16, 16, 4>(gr, pass, s)
                 : v == 2 ? launch_turn_t<16, 8, 8>(gr, pass, s)
                          : launch_turn_t<16, 32, 2>(gr, pass, s);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
// The attribute is per device; setting it twice (two host threads racing
// here) is harmless, the flags only save the call.
cudaError_t straight_attr() {
    static std::atomic<bool> attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(k_straight, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(StraightStage)));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_straight(const Group& gr, int pass, int lines, cudaStream_t s) {
    const int nx = 1 << gr.lx, nt = 1 << gr.lt;
    if (!gr.item_off && nx < kSteps) {
        k_straight_small<<<dim3((unsigned)gr.nq, (unsigned)nt), nx, 0, s>>>(gr.d, pass);
        return cudaGetLastError();
    }
    cudaError_t e = straight_attr();
    if (e != cudaSuccess) return e;
    int tpb = lines == 128 ? 128 : kMaxLines;
    if (gr.item_off) {
        if (lines != 128 && lines != kMaxLines) return cudaErrorInvalidValue;  // the caller sized the items
    } else if (nx < tpb) {
        tpb = nx;
    }
    const int ipq = (int)straight_items(gr.lx, gr.lt, tpb);
    const int64_t items = gr.item_off ? gr.items : (int64_t)ipq * gr.nq;
    if (items <= 0) return cudaSuccess;
    const int64_t blocks = gr.grid > 0 && gr.grid < items ? gr.grid : items;
    k_straight<<<(unsigned)blocks, tpb, 2 * sizeof(StraightStage), s>>>(gr.d, gr.item_off, gr.nq, items, ipq, pass);
    return cudaGetLastError();
}

int straight_blocks_per_sm(int lines) {
    if (straight_attr() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_straight, lines, 2 * sizeof(StraightStage)) !=
        cudaSuccess)
        return 0;
    return n;
}

int turn_blocks_per_sm(int lt, int variant) {
    const int v = variant < 0 ? 0 : variant;
    switch (1 << lt) {
        case 4: return turn_occupancy<1, 4, 1>();
        case 8: return turn_occupancy<2, 4, 1>();
        case 16: return turn_occupancy<4, 4, 1>();
        case 32: return turn_occupancy<8, 4, 1>();
        case 64: return turn_occupancy<8, 8, 1>();
        case 128: return v == 1 ? turn_occupancy<8, 16, 1>() : v == 2 ? turn_occupancy<16, 4, 2>()
                                                                      : turn_occupancy<16, 8, 1>();
        case 256: return v == 1 ? turn_occupancy<16, 8, 2>() : v == 2 ? turn_occupancy<8, 32, 1>()
                                                                      : turn_occupancy<16, 16, 1>();
        case 512: return v == 1 ? turn_occupancy<16, 16, 2>() : v == 2 ? turn_occupancy<16, 8, 4>()
                                                                       : turn_occupancy<TURN512_K, TURN512_SL, TURN512_CL>();
        case 1024: return v == 1 ? turn_occupancy<16, 16, 4>() : v == 2 ? turn_occupancy<16, 8, 8>()
                                                                        : turn_occupancy<16, 32, 2>();
        default: return 0;
    }
}

cudaError_t launch_gear_straight_tiled(const GearLayer& a, int mu, cudaStream_t s) {
    const int nx = a.g.nx;
    if (nx < kSteps) return cudaErrorInvalidValue;
    const int lines = nx < kMaxLines ? nx : kMaxLines;
    const int bytes = (int)(2 * sizeof(GearStage));
    cudaError_t e = cudaFuncSetAttribute(k_gear_straight_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)a.g.nt * (unsigned)(nx / lines);
    k_gear_straight_tiled<<<blocks, lines, bytes, s>>>(a, mu);
    return cudaGetLastError();
}

cudaError_t launch_conv_gate(QueryDesc* qd, int nq, int pass_all, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    k_conv_gate<<<(nq + 255) / 256, 256, 0, s>>>(qd, nq, pass_all);
    return cudaGetLastError();
}

cudaError_t launch_init(const Group& gr, cudaStream_t s) {
    const int64_t n = (int64_t)1 << (2 * gr.lx + gr.lt);
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (148 * 16 + gr.nq - 1) / gr.nq;
    if (blocks > cap) blocks = cap;
    k_init<<<dim3((unsigned)blocks, (unsigned)gr.nq), 256, 0, s>>>(gr.d);
    return cudaGetLastError();
}

}  // namespace nhp

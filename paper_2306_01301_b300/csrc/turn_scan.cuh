// turn_scan.cuh -- the segmented min-plus scan of one maneuver over a tile
// of turn chains (private; used by sweep.cu and gear.cu).
//
// A block owns 32 chains (lanes: 32 neighbouring x' of one y', so every
// heading plane is read as one rotated 128-byte row segment) and SL sections
// of K headings each (warps).  With CL = 2 a thread-block cluster of two
// blocks shares the chains: block rank r holds headings [r*NT/2, (r+1)*NT/2)
// and the two halves exchange their composite section maps through
// distributed shared memory, so two independent 512-thread blocks fit on an
// SM and overlap each other's load and compute phases.
// Scan-order positions: ascending r = T, descending r = NT-1-T; positions of
// the storing (second) loop are r + NT.
//
// What a cell contributes comes from a `Cells` policy with, for the
// thread's cell k of its section:
//   bound(k)        the value a carried segment must beat to store anything
//                   at the cell,
//   store(k, v)     store a carried value v < bound(k) (the policy updates
//                   the values it holds and notes what it stored),
//   ent(k)          the value of entering the maneuver at the cell (both
//                   transition edges included), read before any store of
//                   this scan,
//   e(k)            the edge cost of leaving the cell (TH when hard),
//   tag(k)          bits above the position (bit 16 up) that travel with an
//                   entry and reach its label,
//   label_bits(pv, q) the label's low 13 bits for a store at scan position
//                   q of a segment entered at pv (position and tag).
#pragma once
#include <cooperative_groups.h>

#include "internal.h"

namespace nhp {
namespace {

// Shared state of one turn scan: section maps, the cluster exchange slots
// (NSLOT of them, rotated so that a block never overwrites a slot its
// partners may still read) and the labels of improved cells.
template <int K, int SL, int NSLOT>
struct TurnShared {
    static constexpr int P = 32 + 32 / SL;  // pitch: the carry scan's reads hit 32 banks
    // two sets, used by alternate scans: a warp may start the next scan
    // while a slower one still reads the previous scan's carries
    uint32_t sa[2][SL][P];
    uint32_t sb[2][SL][P];
    int32_t sp[2][SL][P];
    uint32_t tot[NSLOT][3][32];             // per scan: this block's composite (A, B, P)
    uint16_t lab[K][32 * SL];               // labels of improved cells
};


// Compose an earlier stretch X with a later one Y (in place into Y):
// x -> min(x + A, B @ P).  X's entry positions precede Y's, so ties go to X.
__device__ __forceinline__ void combine(uint32_t xa, uint32_t xb, int xp, uint32_t& ya, uint32_t& yb,
                                        int& yp) {
    const uint32_t cand = xb + ya;  // xb <= 2TH + ct, ya <= TH: no wrap
    if (cand <= yb) { yb = cand; yp = xp; }
    ya = min(xa + ya, TH);
}

// One maneuver scan over the block's chains; `mtag` is the maneuver's bits of
// every label the scan writes.  `live`: this thread's section
// holds a reached, non-hard cell.  A warp whose sections hold none has no
// entries (its maps are "nothing produced") and, when nothing is carried in
// either, cannot improve any of its cells, so it skips those loops; the
// results are the same cell for cell.
template <int K, int SL, int CL, int NSLOT, bool ASC, class Cells>
__device__ __forceinline__ void turn_scan(Cells& cl, uint32_t& chg, uint32_t mtag, int sec, int lane, int rank,
                                          int slot, int mb, uint32_t a, bool live, TurnShared<K, SL, NSLOT>& sm) {
    constexpr int S = SL * CL, NT = K * S;
    const int sr = CL == 1 ? 0 : (ASC ? rank : CL - 1 - rank);  // this block's place in scan order
    const int sl = ASC ? sec : SL - 1 - sec;                     // section index in scan order, local
    const int ss = sr * SL + sl;                                 // ... global
    // 1) this section's map (first-loop positions in [0, NT)); its slope
    //    `a`, the section's summed edge costs, is the same in both directions.
    //    "Nothing produced" must stay within the composition bound (<= 2TH + ct).
    uint32_t b = TH;
    int pb = 0;
    if (__any_sync(0xFFFFFFFFu, live)) {
        b = 0xFFFFFFFFu;  // lowered to <= TH + ct by the first cell
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            const int k = ASC ? kk : K - 1 - kk;
            const uint32_t t = cl.ent(k);
            if (t < b) { b = t; pb = (ss * K + kk) | cl.tag(k); }
            b += cl.e(k);
        }
    }
    sm.sa[mb][sl][lane] = a;
    sm.sb[mb][sl][lane] = b;
    sm.sp[mb][sl][lane] = pb;
    __syncthreads();
    // 2) segmented warp scan over the SL local section maps of each chain
    //    (32/SL chains per warp), then the carry into each section of the
    //    second loop.
    {
        const int c = sec * (32 / SL) + lane / SL;
        const int s = lane % SL;
        uint32_t A = sm.sa[mb][s][c], B = sm.sb[mb][s][c];
        int P = sm.sp[mb][s][c];
#pragma unroll
        for (int off = 1; off < SL; off <<= 1) {
            const uint32_t xa = __shfl_up_sync(0xFFFFFFFFu, A, off, SL);
            const uint32_t xb = __shfl_up_sync(0xFFFFFFFFu, B, off, SL);
            const int xp = __shfl_up_sync(0xFFFFFFFFu, P, off, SL);
            if (s >= off) combine(xa, xb, xp, A, B, P);
        }
        // this block's whole stretch (inclusive map of its last section)
        const uint32_t tA = __shfl_sync(0xFFFFFFFFu, A, SL - 1, SL);
        const uint32_t tB = __shfl_sync(0xFFFFFFFFu, B, SL - 1, SL);
        const int tP = __shfl_sync(0xFFFFFFFFu, P, SL - 1, SL);
        // map of the local sections before s
        const uint32_t eA = __shfl_up_sync(0xFFFFFFFFu, A, 1, SL);
        const uint32_t eB = __shfl_up_sync(0xFFFFFFFFu, B, 1, SL);
        const int eP = __shfl_up_sync(0xFFFFFFFFu, P, 1, SL);
        uint32_t cv;  // carry into the first local section of the second loop
        int cp;
        if (CL == 1) {
            cv = tB;
            cp = tP;
        } else {
            if (s == 0) {
                sm.tot[slot][0][c] = tA;
                sm.tot[slot][1][c] = tB;
                sm.tot[slot][2][c] = tP;
            }
            cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
            cluster.sync();
            // composites of the blocks in scan order: j-th block holds scan
            // positions [j*NT/CL, (j+1)*NT/CL)
            uint32_t rA[CL], rB[CL];
            int rP[CL];
#pragma unroll
            for (int j = 0; j < CL; j++) {
                const int rk = ASC ? j : CL - 1 - j;  // cluster rank of scan-order block j
                const TurnShared<K, SL, NSLOT>* o = cluster.map_shared_rank(&sm, rk);
                rA[j] = o->tot[slot][0][c];
                rB[j] = o->tot[slot][1][c];
                rP[j] = o->tot[slot][2][c];
            }
            // the whole first loop applied to 'nothing carried'
            uint32_t fA = rA[0], fB = rB[0];
            int fP = rP[0];
#pragma unroll
            for (int j = 1; j < CL; j++) {
                uint32_t a2 = rA[j], b2 = rB[j];
                int p2 = rP[j];
                combine(fA, fB, fP, a2, b2, p2);
                fA = a2; fB = b2; fP = p2;
            }
            // then the second loop's blocks before this one
            cv = fB;
            cp = fP;
#pragma unroll
            for (int j = 0; j < CL - 1; j++) {
                if (j < sr) {
                    const uint32_t cand = cv + rA[j];
                    if (!(cand <= rB[j])) { cv = rB[j]; cp = rP[j] + NT; }
                    else cv = cand;
                }
            }
        }
        uint32_t iv = cv;
        int ip = cp;
        if (s > 0) {
            const uint32_t cand = cv + eA;  // earlier entries are further upstream
            if (cand <= eB) { iv = cand; ip = cp; }
            else { iv = eB; ip = eP + NT; }
        }
        __syncwarp();
        sm.sb[mb][s][c] = iv;
        sm.sp[mb][s][c] = ip;
    }
    __syncthreads();
    // 3) second loop: store where strictly better.
    const uint32_t v0 = sm.sb[mb][sl][lane];
    const int p0 = sm.sp[mb][sl][lane];
    // Lean pass: the carried value alone, and whether any cell improves.
    // Improvements are rare once the front has passed, so the pass that also
    // tracks entry positions and writes labels runs only in warps that need it.
    bool any = false;
    if (__any_sync(0xFFFFFFFFu, live || v0 < TH)) {
        uint32_t v = v0;
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            const int k = ASC ? kk : K - 1 - kk;
            any |= v < cl.bound(k);
            v = min(v, cl.ent(k)) + cl.e(k);
        }
    }
    if (__any_sync(0xFFFFFFFFu, any)) {
        uint32_t v = v0;
        int pv = p0;
        const int tid = sec * 32 + lane;
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            const int k = ASC ? kk : K - 1 - kk;
            const int q = NT + ss * K + kk;
            const uint32_t t = cl.ent(k);  // before this cell's store
            if (v < cl.bound(k)) {
                cl.store(k, v);
                sm.lab[k][tid] = (uint16_t)(mtag | cl.label_bits(pv, q));
                chg |= 1u << k;
            }
            if (t < v) { v = t; pv = q | cl.tag(k); }
            v += cl.e(k);
        }
    }
    // Without a cluster the next scan uses the other set of section maps,
    // and every warp passes this scan's two barriers before any warp can
    // reach the scan after next: no barrier here.  Cluster partners read
    // the exchange slots remotely, so clusters keep one.
    if (CL > 1) __syncthreads();
}

}  // namespace
}  // namespace nhp

// reach.cu -- maneuver-count reachability with bit vectors (Appendix C).
//
// With hard obstacles only and every maneuver edge free, the value of a pose
// is the fewest maneuvers that reach it, and one bit per pose says whether
// it is reachable within m maneuvers.  Bits are packed 32 poses per word
// along x (the volumes' own order), 0 = reachable as in Insert 2.  A cycle
// takes every maneuver from the previous cycle's reachability R_m: along a
// maneuver curve, v = (v & R_m) | H turns reachability on at reachable poses
// and off at hard ones (H = hard bit), and every pose the curve reaches is
// combined by AND into R_{m+1} (which starts as R_m).
//
// A 32-bit word carries 32 neighbouring curves (chains x' .. x'+31 of one
// row): the curves of a word meet the volume at a bit offset that changes
// with the heading (turns, eq. 18) or the step (straights, eq. 23), so a
// warp holds whole rows of words and realigns them with shuffles and funnel
// shifts -- every load and store is an aligned word, and no word is written
// by two threads.  Each curve is cut into sections (Appendix D, Inserts
// 6-8): a section's effect on what enters it is v -> (v | D) & S with D the
// OR of its hard bits and S what leaves it when nothing enters, these maps
// are rippled across the sections in shared memory (twice around for the
// cyclic turns, once for the straights, which start at the wall), and the
// sections are then swept with the rippled value coming in.  Straight lines
// of shallow planes (|tan theta| <= 1, eq. 19) run along x with one pose per
// row, so those planes are swept through bit-transposed copies, where they
// look like steep ones.
#include <algorithm>

#include "plan_state.h"

namespace nhp {
namespace {

__device__ __forceinline__ uint32_t rd(const uint32_t* p) { return __ldg(p); }

// Bits of the word of chains [32l, 32l+32) of a row whose cells start at bit
// offset s of the volume row held (one aligned word per lane) in `w`; the W
// lanes of a row form one shuffle group.
__device__ __forceinline__ uint32_t gather_bits(uint32_t w, int l, int s, int W) {
    const int q = s >> 5, r = s & 31;
    const uint32_t a = __shfl_sync(0xFFFFFFFFu, w, (l + q) & (W - 1), W);
    const uint32_t b = __shfl_sync(0xFFFFFFFFu, w, (l + q + 1) & (W - 1), W);
    return __funnelshift_r(a, b, r);
}

// The inverse: the aligned volume word l of the row, from the chain words
// (one per lane) whose cells start at bit offset s.
__device__ __forceinline__ uint32_t scatter_bits(uint32_t c, int l, int s, int W) {
    const int q = s >> 5, r = s & 31;
    const uint32_t c1 = __shfl_sync(0xFFFFFFFFu, c, (l - q) & (W - 1), W);
    const uint32_t c0 = __shfl_sync(0xFFFFFFFFu, c, (l - q - 1) & (W - 1), W);
    return __funnelshift_l(c0, c1, r);
}

__global__ void k_hard_bits(const uint16_t* __restrict__ B, uint32_t* __restrict__ H, int64_t words) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < words;
         g += (int64_t)gridDim.x * blockDim.x) {
        const uint4* p = reinterpret_cast<const uint4*>(B + g * 32);
        uint32_t bits = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint4 v = __ldg(p + c);
            const uint32_t h[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int b = c * 8 + k * 2;
                bits |= (uint32_t)((h[k] & 0xFFFFu) == HARD) << b;
                bits |= (uint32_t)((h[k] >> 16) == HARD) << (b + 1);
            }
        }
        H[g] = bits;
    }
}

__global__ void k_reach_init(uint32_t* __restrict__ R, int64_t words, int64_t start) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < words;
         g += (int64_t)gridDim.x * blockDim.x)
        R[g] = g == (start >> 5) ? ~(1u << (start & 31)) : 0xFFFFFFFFu;
}

// 32 x 32 bit matrix held one row per lane (bit c of lane r = entry (r, c)),
// transposed in place: five rounds, each swapping the two off-diagonal j x j
// blocks of every 2j x 2j block (j = 16, 8, 4, 2, 1) between lanes r and r ^ j.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int j = 16 >> i;
        // columns c with (c & j) == 0
        const uint32_t m = i == 0 ? 0x0000FFFFu : i == 1 ? 0x00FF00FFu : i == 2 ? 0x0F0F0F0Fu : i == 3 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

template <int G> struct WordVec;
template <> struct WordVec<2> { using T = uint2; };
template <> struct WordVec<4> { using T = uint4; };

__device__ __forceinline__ void unpack(const uint2& w, uint32_t* v) { v[0] = w.x; v[1] = w.y; }
__device__ __forceinline__ void unpack(const uint4& w, uint32_t* v) { v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w; }
__device__ __forceinline__ void pack(uint2& w, const uint32_t* v) { w.x = v[0]; w.y = v[1]; }
__device__ __forceinline__ void pack(uint4& w, const uint32_t* v) { w.x = v[0]; w.y = v[1]; w.z = v[2]; w.w = v[3]; }

// Transpose the 32 x 32 bit tiles of the listed planes: bit (row j, column
// i) goes to (row i, column j), ANDed into dst with `and_into`.  Each warp
// takes a G x G group of tiles (row blocks bj G.., words bi G..): every lane
// reads G consecutive words of each of its G source rows in one vector load
// and writes G consecutive words of each of its G destination rows in one
// vector store, so the plane moves in 16-byte (G = 4) pieces.
template <int G>
__global__ void __launch_bounds__(256) k_bit_transpose(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                       const int32_t* __restrict__ planes, int64_t ngroups, int lx,
                                                       int and_into) {
    using V = typename WordVec<G>::T;
    constexpr int LG = G == 4 ? 2 : 1;
    const int lane = threadIdx.x & 31, lw = lx - 5, W = 1 << lw, lb = lw - LG;
    const int64_t gi = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (gi >= ngroups) return;  // warp-uniform
    const int pi = (int)(gi >> (2 * lb));
    const int r = (int)(gi & ((1 << (2 * lb)) - 1)), bj = r >> lb, bi = r & ((1 << lb) - 1);
    const int64_t plane = (int64_t)__ldg(planes + pi) << (2 * lx - 5);
    uint32_t v[G][G];  // v[a][k]: source row block bj G + a, word bi G + k
#pragma unroll
    for (int a = 0; a < G; a++)
        unpack(*reinterpret_cast<const V*>(src + plane + (int64_t)((bj * G + a) * 32 + lane) * W + bi * G), v[a]);
#pragma unroll
    for (int k = 0; k < G; k++) {
        uint32_t o[G];  // destination row block bi G + k, words bj G + a
#pragma unroll
        for (int a = 0; a < G; a++) o[a] = transpose32(v[a][k], lane);
        V* at = reinterpret_cast<V*>(dst + plane + (int64_t)((bi * G + k) * 32 + lane) * W + bj * G);
        if (and_into) {
            uint32_t d[G];
            unpack(*at, d);
#pragma unroll
            for (int a = 0; a < G; a++) o[a] &= d[a];
        }
        V w;
        pack(w, o);
        *at = w;
    }
}

// The sections of one curve in ripple order, one per lane of an n-lane
// segment (p = the lane's position): section p maps what enters it to
// (v & A) | C.  Returns what enters section p when the ripple starts from
// all ones (unreachable) at section 0 -- for a cyclic curve after one full
// turn around the cycle, i.e. from F(all ones) with F all sections composed.
// The prefix compositions are a shuffle scan: the map of sections a..b
// followed by that of b+1..c is (v & A1 & A2) | (C1 & A2) | C2.
template <int N>
__device__ __forceinline__ uint32_t ripple(uint32_t A, uint32_t C, int p, int n, bool cyclic) {
#pragma unroll
    for (int o = 1; o < (N ? N : 32); o <<= 1) {
        if (!N && o >= n) break;
        const uint32_t A2 = __shfl_up_sync(0xFFFFFFFFu, A, o, N ? N : n);
        const uint32_t C2 = __shfl_up_sync(0xFFFFFFFFu, C, o, N ? N : n);
        if (p >= o) {
            C = (C2 & A) | C;
            A &= A2;
        }
    }
    const int w = N ? N : n;
    const uint32_t c0 = cyclic ? __shfl_sync(0xFFFFFFFFu, A | C, w - 1, w) : 0xFFFFFFFFu;
    const uint32_t Ap = __shfl_up_sync(0xFFFFFFFFu, A, 1, w), Cp = __shfl_up_sync(0xFFFFFFFFu, C, 1, w);
    return p == 0 ? c0 : ((c0 & Ap) | Cp);
}

// One turn family (LEFT: LF up, LB down; RIGHT: RB up, RF down).  Block: SEC
// warps = sections of K headings; a warp's lanes are G = 32 / W chain rows
// of W words.  Both maneuvers read R_m; what they reach goes to Rn by
// `mode`: 0 ANDed into it, 1 stored as R_m AND it (the first writer of a
// cycle, so that R_{m+1} needs no copy of R_m first), 2 stored as it is (a
// family running beside the others writes its own volume).
template <int K, int SEC>
__global__ void __launch_bounds__(32 * SEC, 1)
k_reach_turn(const DevGrid g, const uint32_t* __restrict__ Rm, uint32_t* __restrict__ Rn,
             const uint32_t* __restrict__ H, int family, int mode) {
    // [direction][chain word][section]: the section maps, then what enters
    // each section; the odd pitch keeps both access patterns conflict-free
    __shared__ uint32_t sA[2][32][SEC + 1], sC[2][32][SEC + 1];
    // per heading: the volume row of the block's first chain row << 16 | the
    // chains' bit offset; a warp fills and reads only its own K headings
    __shared__ uint32_t srow[K * SEC];
    const int W = 1 << (g.lx - 5), G = 32 / W;
    const int lane = threadIdx.x & 31, sec = threadIdx.x >> 5;
    const int r = lane / W, l = lane & (W - 1);
    if (lane < K) {
        const int T = sec * K + lane;
        const int4 b = __ldg(&g.beta4[T]);
        const int bx = family ? b.z : b.x, by = family ? b.w : b.y;
        srow[T] = ((uint32_t)((blockIdx.x * G + by) & g.mx) << 16) | (uint32_t)(bx & g.mx);
    }
    __syncwarp();
    // word of this lane's chain row and bit offset of the chain cells, heading
    // T (volumes here hold at most 2^22 words: 32-bit offsets)
    auto where = [&](int T, int& off) -> uint32_t {
        const uint32_t e = srow[T];
        off = (int)(e & 0xFFFFu);
        const uint32_t row = ((e >> 16) + (uint32_t)r) & (uint32_t)g.mx;
        return ((uint32_t)T << (2 * g.lx - 5)) + (row << (g.lx - 5)) + (uint32_t)l;
    };
    uint32_t vi[K], hb[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        int off;
        const uint32_t ix = where(sec * K + k, off);
        vi[k] = gather_bits(rd(Rm + ix), l, off, W);
        hb[k] = gather_bits(rd(H + ix), l, off, W);
    }
    // pass 1: the section's map in both directions, v -> (v | D) & S
    {
        uint32_t up = 0xFFFFFFFFu, down = 0xFFFFFFFFu, D = 0u;
#pragma unroll
        for (int k = 0; k < K; k++) {
            up = (up & vi[k]) | hb[k];
            down = (down & vi[K - 1 - k]) | hb[K - 1 - k];
            D |= hb[k];
        }
        sA[0][lane][sec] = up;
        sC[0][lane][sec] = D & up;
        sA[1][lane][sec] = down;
        sC[1][lane][sec] = D & down;
    }
    __syncthreads();
    // pass 2: thread t ripples chain word t / SEC at position t % SEC
    {
        const int w = threadIdx.x / SEC, p = threadIdx.x % SEC;
#pragma unroll 1  // both scans unrolled together need more than the 64 registers a thread has
        for (int dir = 0; dir < 2; dir++) {
            const int s = dir == 0 ? p : SEC - 1 - p;
            sA[dir][w][s] = ripple<SEC>(sA[dir][w][s], sC[dir][w][s], p, SEC, true);
        }
    }
    __syncthreads();
    // pass 3: sweep the section with what enters it, both directions
    uint32_t o[K];
    uint32_t v = sA[0][lane][sec];
#pragma unroll
    for (int k = 0; k < K; k++) {
        v = (v & vi[k]) | hb[k];
        o[k] = ~v;  // reachable (0 bits) collected as 1s
    }
    v = sA[1][lane][sec];
#pragma unroll
    for (int k = K - 1; k >= 0; k--) {
        v = (v & vi[k]) | hb[k];
        o[k] |= ~v;
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        int off;
        const uint32_t ix = where(sec * K + k, off);
        const uint32_t word = scatter_bits(~o[k], l, off, W);
        if (mode == 2) Rn[ix] = word;
        else if (mode == 1) Rn[ix] = rd(Rm + ix) & word;
        else Rn[ix] &= word;
    }
}

// Straight lines of one plane per block (steep planes in place, shallow
// planes through their transposed copies); results stored (steep into Rn,
// shallow into OT), not combined: lines x' packed 32 per word,
// steps y' along the view's rows, row y' shifted by Bs(y') (eq. 23).  A
// warp's lanes are 32 / W sections of W words; SEC sections of K steps.  SF
// and SB walk the line in opposite directions; what either reaches counts.
template <int K>
__global__ void __launch_bounds__(512, 2) k_reach_straight(const DevGrid g, const uint32_t* __restrict__ Rm,
                                 const uint32_t* __restrict__ H, const uint32_t* __restrict__ RmT,
                                 const uint32_t* __restrict__ HT, uint32_t* __restrict__ Rn,
                                 uint32_t* __restrict__ OT) {
    extern __shared__ uint32_t smem[];
    const int T = blockIdx.x;
    const PlaneInfo pi = g.plane[T];
    const bool steep = pi.iflag != 0;
    const int W = 1 << (g.lx - 5), SPW = 32 / W;  // sections per warp
    const int SEC = g.nx / K, P = SEC + 1;
    // [direction][word][section] maps, then what enters each section
    uint32_t* sA = smem;
    uint32_t* sC = sA + 2 * W * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sec = warp * SPW + lane / W, l = lane & (W - 1);
    const int64_t nplane = (int64_t)W << g.lx;
    const uint32_t* src = steep ? Rm : RmT;
    const uint32_t* hsrc = steep ? H : HT;
    const int16_t* bs = g.bshear + (int64_t)T * g.nx;
    uint32_t vi[K], hb[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int y = sec * K + k;  // step y' = row of the view
        const int off = bs[y] & g.mx;
        const int64_t ix = (int64_t)T * nplane + (int64_t)y * W + l;
        vi[k] = gather_bits(rd(src + ix), l, off, W);
        hb[k] = gather_bits(rd(hsrc + ix), l, off, W);
    }
    {
        uint32_t up = 0xFFFFFFFFu, down = 0xFFFFFFFFu, D = 0u;
#pragma unroll
        for (int k = 0; k < K; k++) {
            up = (up & vi[k]) | hb[k];
            down = (down & vi[K - 1 - k]) | hb[K - 1 - k];
            D |= hb[k];
        }
        sA[l * P + sec] = up;
        sC[l * P + sec] = D & up;
        sA[(W + l) * P + sec] = down;
        sC[(W + l) * P + sec] = D & down;
    }
    __syncthreads();
    // one ripple: a line starts at the wall, so nothing enters the first section
    {
        const int w = threadIdx.x / SEC, p = threadIdx.x % SEC;
#pragma unroll
        for (int dir = 0; dir < 2; dir++) {
            const int at = (dir * W + w) * P + (dir == 0 ? p : SEC - 1 - p);
            sA[at] = ripple<0>(sA[at], sC[at], p, SEC, false);
        }
    }
    __syncthreads();
    // forward sweep into shared memory (this thread's slots), then the
    // backward sweep, each word stored as soon as both directions have it
    // (a third register array would push the kernel past two blocks per SM)
    uint32_t* sF = sC + 2 * W * P;  // [k][thread]
    const int nth = blockDim.x;
    uint32_t v = sA[l * P + sec];
#pragma unroll
    for (int k = 0; k < K; k++) {
        v = (v & vi[k]) | hb[k];
        sF[k * nth + threadIdx.x] = v;
    }
    v = sA[(W + l) * P + sec];
#pragma unroll
    for (int k = K - 1; k >= 0; k--) {
        v = (v & vi[k]) | hb[k];
        const int y = sec * K + k;
        const int64_t ix = (int64_t)T * nplane + (int64_t)y * W + l;
        const uint32_t word = scatter_bits(sF[k * nth + threadIdx.x] & v, l, bs[y] & g.mx, W);
        if (steep) Rn[ix] = word;
        else OT[ix] = word;
    }
}

// R_{m+1} &= (second turn family) & (straights), 16 bytes per thread.
__global__ void k_reach_combine(uint4* __restrict__ Rn, const uint4* __restrict__ X1, const uint4* __restrict__ X2,
                                int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 a = Rn[i], b = __ldg(X1 + i), c = __ldg(X2 + i);
        Rn[i] = make_uint4(a.x & b.x & c.x, a.y & b.y & c.y, a.z & b.z & c.z, a.w & b.w & c.w);
    }
}

// Fewest maneuvers per pose from R_0 .. R_N (255 beyond N).
__global__ void k_reach_counts(const uint32_t* __restrict__ R, int n, int64_t words, uint8_t* __restrict__ count) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < words;
         g += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[8];
#pragma unroll
        for (int i = 0; i < 8; i++) c[i] = 0xFFFFFFFFu;
        uint32_t seen = 0;
        for (int m = 0; m <= n; m++) {
            const uint32_t fresh = ~R[(int64_t)m * words + g] & ~seen;
            seen |= fresh;
            for (uint32_t f = fresh; f; f &= f - 1) {
                const int b = __ffs(f) - 1;
                c[b >> 2] = (c[b >> 2] & ~(0xFFu << (8 * (b & 3)))) | ((uint32_t)m << (8 * (b & 3)));
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(count + g * 32);
        dst[0] = make_uint4(c[0], c[1], c[2], c[3]);
        dst[1] = make_uint4(c[4], c[5], c[6], c[7]);
    }
}

}  // namespace


cudaError_t launch_hard_bits(const uint16_t* B, uint32_t* H, int64_t nr, cudaStream_t s) {
    const int64_t words = nr / 32;
    const int64_t blocks = std::min<int64_t>((words + 255) / 256, 148 * 16);
    k_hard_bits<<<(unsigned)blocks, 256, 0, s>>>(B, H, words);
    return cudaGetLastError();
}

cudaError_t launch_reach_init(uint32_t* R, int64_t nr, int64_t start, cudaStream_t s) {
    const int64_t words = nr / 32;
    const int64_t blocks = std::min<int64_t>((words + 255) / 256, 148 * 16);
    k_reach_init<<<(unsigned)blocks, 256, 0, s>>>(R, words, start);
    return cudaGetLastError();
}

cudaError_t launch_bit_transpose(const uint32_t* src, uint32_t* dst, const int32_t* planes, int nplanes, int lx,
                                 bool and_into, cudaStream_t s) {
    if (nplanes == 0) return cudaSuccess;
    const int W = 1 << (lx - 5);
    const int G = W >= 4 ? 4 : 2;  // W is a power of two, at least 2
    const int64_t ngroups = (int64_t)nplanes * (W / G) * (W / G);
    const unsigned blocks = (unsigned)((ngroups + 7) / 8);
    if (G == 4) k_bit_transpose<4><<<blocks, 256, 0, s>>>(src, dst, planes, ngroups, lx, and_into ? 1 : 0);
    else k_bit_transpose<2><<<blocks, 256, 0, s>>>(src, dst, planes, ngroups, lx, and_into ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_reach_turn(const DevGrid& g, const uint32_t* Rm, uint32_t* Rn, const uint32_t* H, int family,
                              int mode, cudaStream_t s) {
    const int W = 1 << (g.lx - 5), G = 32 / W;
    const unsigned blocks = (unsigned)(g.nx / G);
    switch (g.lt) {  // K = 16 headings per section
        case 5: k_reach_turn<16, 2><<<blocks, 32 * 2, 0, s>>>(g, Rm, Rn, H, family, mode); break;
        case 6: k_reach_turn<16, 4><<<blocks, 32 * 4, 0, s>>>(g, Rm, Rn, H, family, mode); break;
        case 7: k_reach_turn<16, 8><<<blocks, 32 * 8, 0, s>>>(g, Rm, Rn, H, family, mode); break;
        case 8: k_reach_turn<16, 16><<<blocks, 32 * 16, 0, s>>>(g, Rm, Rn, H, family, mode); break;
        case 9: k_reach_turn<16, 32><<<blocks, 32 * 32, 0, s>>>(g, Rm, Rn, H, family, mode); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reach_straight(const DevGrid& g, const uint32_t* Rm, const uint32_t* H, const uint32_t* RmT,
                                  const uint32_t* HT, uint32_t* Rn, uint32_t* OT, cudaStream_t s) {
    // K steps per section such that the (section, word) lanes fill whole
    // warps and one block: Nx = 64 -> 4, 128 .. 512 -> 16, 1024 -> 32
    const int K = g.nx == 64 ? 4 : 16;
    const int W = 1 << (g.lx - 5);
    const int SEC = g.nx / K;
    const int threads = SEC * W;
    if (g.nx < 64 || g.nx > 512 || threads % 32 != 0 || threads > 512) return cudaErrorInvalidValue;
    // section maps and carries (4 W (SEC + 1) words) + the forward sweep (K words per thread)
    const size_t smem = (4 * (size_t)(SEC + 1) * W + (size_t)K * threads) * sizeof(uint32_t);
    if (K == 4) k_reach_straight<4><<<(unsigned)g.nt, threads, smem, s>>>(g, Rm, H, RmT, HT, Rn, OT);
    else k_reach_straight<16><<<(unsigned)g.nt, threads, smem, s>>>(g, Rm, H, RmT, HT, Rn, OT);
    return cudaGetLastError();
}

cudaError_t launch_reach_combine(uint32_t* Rn, const uint32_t* X1, const uint32_t* X2, int64_t nr, cudaStream_t s) {
    const int64_t n4 = nr / 128;  // 32 poses per word, 4 words per thread (Nx >= 64)
    const int64_t blocks = std::min<int64_t>((n4 + 255) / 256, 148 * 8);
    k_reach_combine<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<uint4*>(Rn), reinterpret_cast<const uint4*>(X1),
                                                      reinterpret_cast<const uint4*>(X2), n4);
    return cudaGetLastError();
}

cudaError_t launch_reach_counts(const uint32_t* R, int n, int64_t nr, uint8_t* count, cudaStream_t s) {
    const int64_t words = nr / 32;
    const int64_t blocks = std::min<int64_t>((words + 255) / 256, 148 * 16);
    k_reach_counts<<<(unsigned)blocks, 256, 0, s>>>(R, n, words, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host
namespace {

int reach_alloc(plan_s* p, int n_cycles) {
    const size_t vol = (size_t)(p->nr / 8);
    if (!p->d_hb) {
        p->d_hb = (uint32_t*)p->dalloc(vol);
        p->d_hbt = (uint32_t*)p->dalloc(vol);
        p->d_rt = (uint32_t*)p->dalloc(vol);
        p->d_ot = (uint32_t*)p->dalloc(vol);
        p->d_x1 = (uint32_t*)p->dalloc(vol);
        p->d_x2 = (uint32_t*)p->dalloc(vol);
        p->d_shallow = (int32_t*)p->dalloc(sizeof(int32_t) * (size_t)p->nt);
        if (!p->d_hb || !p->d_hbt || !p->d_rt || !p->d_ot || !p->d_x1 || !p->d_x2 || !p->d_shallow) {
            // give back what was taken: the next call starts from nothing
            p->dfree(p->d_hb, vol);
            p->dfree(p->d_hbt, vol);
            p->dfree(p->d_rt, vol);
            p->dfree(p->d_ot, vol);
            p->dfree(p->d_x1, vol);
            p->dfree(p->d_x2, vol);
            p->dfree(p->d_shallow, sizeof(int32_t) * (size_t)p->nt);
            p->d_hb = p->d_hbt = p->d_rt = p->d_ot = p->d_x1 = p->d_x2 = nullptr;
            p->d_shallow = nullptr;
            return PLAN_ENOMEM;
        }
        std::vector<int32_t> sh;
        for (int T = 0; T < p->nt; T++)
            if (p->planes[T].iflag == 0) sh.push_back(T);
        p->n_shallow = (int)sh.size();
        p->shallow = sh;
        if (!sh.empty())
            NHP_CK(cudaMemcpyAsync(p->d_shallow, p->shallow.data(), sizeof(int32_t) * sh.size(),
                                   cudaMemcpyHostToDevice, p->stream));
    }
    for (auto& st : p->reach_side)
        if (!st) NHP_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto& e : p->reach_ev)
        if (!e) NHP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (n_cycles + 1 > p->reach_cap) {
        p->dfree(p->d_reach, vol * (size_t)p->reach_cap);
        p->d_reach = (uint32_t*)p->dalloc(vol * (size_t)(n_cycles + 1));
        p->reach_cap = p->d_reach ? n_cycles + 1 : 0;
        if (!p->d_reach) return PLAN_ENOMEM;
    }
    return PLAN_OK;
}

}  // namespace
}  // namespace nhp

using namespace nhp;

extern "C" {

int plan_reach_sweep(plan_t* p, plan_pose start, int n_cycles) {
    if (!p || n_cycles < 0 || n_cycles > 254 || !pose_ok(p, start)) return PLAN_EINVAL;
    if (p->nx < 64 || p->nx > 512 || p->nt < 32 || p->nt > 512) return PLAN_EINVAL;
    if (!p->rendered) return PLAN_ESTATE;
    if (pose_hard(p, start)) return PLAN_EINVAL;
    int rc = reach_alloc(p, n_cycles);
    if (rc != PLAN_OK) return rc;
    cudaStream_t s = p->stream;
    const DevGrid& g = p->g;
    const int64_t words = p->nr / 32;
    NHP_CK(launch_hard_bits(p->d_B, p->d_hb, p->nr, s));
    NHP_CK(launch_bit_transpose(p->d_hb, p->d_hbt, p->d_shallow, p->n_shallow, p->lx, false, s));
    NHP_CK(launch_reach_init(p->d_reach, p->nr, cell_index(p, start), s));
    p->launches += 3;
    // A cycle's maneuvers all read R_m, so they run side by side: the first
    // turn family writes R_{m+1} = R_m AND its result on the plan's stream,
    // the second family its own volume on one side stream, the straights
    // (shallow planes through their transposes) theirs on the other; then
    // R_{m+1} &= both.
    cudaStream_t a1 = p->reach_side[0], a2 = p->reach_side[1];
    for (int m = 0; m < n_cycles; m++) {
        const uint32_t* Rm = p->d_reach + (size_t)m * words;
        uint32_t* Rn = p->d_reach + (size_t)(m + 1) * words;
        NHP_CK(cudaEventRecord(p->reach_ev[0], s));
        NHP_CK(cudaStreamWaitEvent(a1, p->reach_ev[0], 0));
        NHP_CK(cudaStreamWaitEvent(a2, p->reach_ev[0], 0));
        NHP_CK(launch_bit_transpose(Rm, p->d_rt, p->d_shallow, p->n_shallow, p->lx, false, a1));
        NHP_CK(launch_reach_straight(g, Rm, p->d_hb, p->d_rt, p->d_hbt, p->d_x2, p->d_ot, a1));
        NHP_CK(launch_bit_transpose(p->d_ot, p->d_x2, p->d_shallow, p->n_shallow, p->lx, false, a1));
        NHP_CK(launch_reach_turn(g, Rm, p->d_x1, p->d_hb, 1, 2, a2));
        NHP_CK(launch_reach_turn(g, Rm, Rn, p->d_hb, 0, 1, s));
        NHP_CK(cudaEventRecord(p->reach_ev[1], a1));
        NHP_CK(cudaEventRecord(p->reach_ev[2], a2));
        NHP_CK(cudaStreamWaitEvent(s, p->reach_ev[1], 0));
        NHP_CK(cudaStreamWaitEvent(s, p->reach_ev[2], 0));
        NHP_CK(launch_reach_combine(Rn, p->d_x1, p->d_x2, p->nr, s));
        p->launches += 6;
    }
    p->reach_n = n_cycles;
    p->reach_ready = true;
    return PLAN_OK;
}

int plan_reach_extract(plan_t* p, plan_pose goal, plan_segment* out, int cap, int* n_out, int* maneuvers) {
    if (!p || !n_out || !maneuvers || cap < 0 || (cap > 0 && !out) || !pose_ok(p, goal)) return PLAN_EINVAL;
    *n_out = 0;
    *maneuvers = -1;
    if (!p->reach_ready) return PLAN_ESTATE;
    const int64_t words = p->nr / 32;
    NHP_CK(launch_reach_extract(p->g, p->d_reach, p->reach_n, words, p->d_hb, cell_index(p, goal), p->d_seg,
                                kDevSegCap, p->d_status, p->stream));
    p->launches++;
    int32_t status[2] = {0, 0};
    NHP_CK(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    NHP_CK(cudaStreamSynchronize(p->stream));
    if (status[0] == -1) return PLAN_EUNREACHABLE;
    if (status[0] < 0) return PLAN_EINTERNAL;
    *maneuvers = status[1];
    *n_out = status[0];
    if (status[0] > cap || status[0] > kDevSegCap) return PLAN_ERANGE;
    if (status[0] > 0) {
        NHP_CK(cudaMemcpyAsync(out, p->d_seg, sizeof(plan_segment) * status[0], cudaMemcpyDeviceToHost, p->stream));
        NHP_CK(cudaStreamSynchronize(p->stream));
        std::reverse(out, out + status[0]);  // the back-track runs goal -> start
    }
    return PLAN_OK;
}

int plan_reach_counts(plan_t* p, uint8_t* counts) {
    if (!p || !counts) return PLAN_EINVAL;
    if (!p->reach_ready) return PLAN_ESTATE;
    uint8_t* d = (uint8_t*)p->dalloc((size_t)p->nr);
    if (!d) return PLAN_ENOMEM;
    int rc = cuda_rc(launch_reach_counts(p->d_reach, p->reach_n, p->nr, d, p->stream));
    p->launches++;
    if (rc == PLAN_OK) rc = cuda_rc(cudaMemcpyAsync(counts, d, (size_t)p->nr, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    p->dfree(d, (size_t)p->nr);
    return rc;
}

}  // extern "C"

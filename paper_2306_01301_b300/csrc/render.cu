// render.cu -- configuration-space obstacle rendering (Section VI).
//
// B(i, j, T) is the maximum of the obstacle image over the vehicle footprint
// placed at pose (i, j, T), with the one-cell hard walls at i = 0 and j = 0
// inserted first (Section V.C) and all coordinates taken modulo Nx.  Because
// HARD = 0xFFFF is the largest uint16, a plain maximum also marks every pose
// whose footprint touches a hard cell.
//
// The footprint of heading T is stored as maximal row runs (dy, [lo, hi]).
// A row maximum over any run costs two lookups in a per-row sparse table
// S_k[y][x] = max(img[y][x .. x + 2^k - 1]) (cyclic in x): the paper's
// separable dilation idea (cost independent of the run length), but exact
// for the rotated rectangle's rasterisation.
#include "internal.h"

namespace nhp {
namespace {

// level 0: the image with the walls inserted
__global__ void k_table_level0(const QueryDesc* __restrict__ qd) {
    const QueryDesc& Q = qd[blockIdx.y];
    const uint16_t* img = Q.img;
    uint16_t* t0 = Q.table;
    const int lx = Q.g.lx;
    const int n = 1 << lx;
    const int64_t total = (int64_t)n * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k & (n - 1)), y = (int)(k >> lx);
        t0[k] = (x == 0 || y == 0) ? HARD : img[k];
    }
}

// level k from level k-1: window 2^k = two windows of 2^(k-1)
__global__ void k_table_level(const QueryDesc* __restrict__ qd, int k) {
    const QueryDesc& Q = qd[blockIdx.y];
    const int lx = Q.g.lx, half = 1 << (k - 1);
    const int64_t nxy = (int64_t)1 << (2 * lx);
    const uint16_t* prev = Q.table + (k - 1) * nxy;
    uint16_t* cur = Q.table + k * nxy;
    const int n = 1 << lx;
    const int64_t total = (int64_t)n * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k & (n - 1));
        const int64_t row = k - x;
        const uint16_t a = prev[k], b = prev[row + ((x + half) & (n - 1))];
        cur[k] = a > b ? a : b;
    }
}

// One thread per pose cell of heading blockIdx.y; the heading's runs are
// staged in shared memory.
__global__ void __launch_bounds__(256) k_render(const QueryDesc* __restrict__ qd) {
    extern __shared__ Run runs[];
    const QueryDesc& Q = qd[blockIdx.z];
    const DevGrid g = Q.g;
    const uint16_t* __restrict__ table = Q.table;
    uint16_t* __restrict__ B = Q.v.B;
    const int T = blockIdx.y;
    const int r0 = g.run_off[T], nr = g.run_off[T + 1] - r0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) runs[r] = g.runs[r0 + r];
    __syncthreads();
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nxy) return;
    const int i = (int)(cell & g.mx), j = (int)(cell >> g.lx);
    uint16_t m = 0;
    // HARD is the largest value: once every lane of the warp has met a hard
    // cell, no later run can change the result.
    for (int r0 = 0; r0 < nr; r0 += 4) {
#pragma unroll
        for (int r = r0; r < r0 + 4; r++) {
            if (r < nr) {
                const Run ru = runs[r];
                const int64_t ro = (int64_t)ru.lvl * nxy + ((int64_t)((j + ru.dy) & g.mx) << g.lx);
                if (!NHP_IN(ro, (int64_t)(g.lx + 1) * nxy, Q.err, 10)) continue;
                const uint16_t* row = table + ro;
                const uint16_t a = __ldg(row + ((i + ru.lo) & g.mx));
                const uint16_t b = __ldg(row + ((i + ru.hi2) & g.mx));
                m = max(m, max(a, b));
            }
        }
        if (__all_sync(__activemask(), m == HARD)) break;
    }
    if (NHP_IN((int64_t)T * nxy + cell, nxy * g.nt, Q.err, 11)) B[(int64_t)T * nxy + cell] = m;
}

// ----------------------------------------------------------- bit-parallel
// The hard test alone: bit x of word row Hk[y] is 1 when any of the cells
// x .. x + 2^k - 1 of image row y (cyclic) is hard or a wall.  One 32-bit
// word covers 32 neighbouring poses, so one thread tests 32 poses per
// footprint run with two funnel-shifted word pairs.

// bits [p, p+32) of a cyclic row of nw words
__device__ __forceinline__ uint32_t row_window(const uint32_t* row, int p, int nw_mask) {
    const int w0 = p >> 5, sh = p & 31;
    const uint32_t lo = __ldg(row + (w0 & nw_mask)), hi = __ldg(row + ((w0 + 1) & nw_mask));
    return __funnelshift_r(lo, hi, sh);
}

__global__ void k_bits_level0(const QueryDesc* __restrict__ qd) {
    const QueryDesc& Q = qd[blockIdx.y];
    const uint16_t* __restrict__ img = Q.img;
    uint32_t* __restrict__ h0 = Q.bits;
    const int lx = Q.g.lx;
    const int n = 1 << lx, nw = n >> 5;
    const int64_t total = (int64_t)n * nw;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / nw), w = (int)(k % nw);
        const uint16_t* r = img + (int64_t)y * n + 32 * w;
        uint32_t bits = 0;
#pragma unroll 8
        for (int t = 0; t < 32; t++) {
            const int x = 32 * w + t;
            if (x == 0 || y == 0 || r[t] == HARD) bits |= 1u << t;
        }
        h0[k] = bits;
    }
}

__global__ void k_bits_level(const QueryDesc* __restrict__ qd, int lvl) {
    const QueryDesc& Q = qd[blockIdx.y];
    const int lx = Q.g.lx, half = 1 << (lvl - 1);
    const int64_t words = (int64_t)(1 << lx) * ((1 << lx) >> 5);
    const uint32_t* __restrict__ prev = Q.bits + (lvl - 1) * words;
    uint32_t* __restrict__ cur = Q.bits + lvl * words;
    const int n = 1 << lx, nw = n >> 5;
    const int64_t total = (int64_t)n * nw;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / nw), w = (int)(k % nw);
        const uint32_t* row = prev + (int64_t)y * nw;
        cur[k] = row[w] | row_window(row, 32 * w + half, nw - 1);
    }
}

// A footprint row run decoded for one heading: the table level's word
// offset, the row shift, and the word offset and bit shift of its two
// windows (both starts taken modulo Nx).
struct RunW {
    int32_t base, dy, q1, s1, q2, s2;
};

// One thread per (32-pose word, row j) of heading blockIdx.y.  Writes HARD
// where the footprint meets a hard cell; elsewhere `free_value` (256 for a
// hard-only image, 0 as a placeholder when a soft pass follows).  With at
// most 32 words per row (Nx <= 1024) the words of a row are neighbouring
// lanes: a window's two words are this lane's load and the next lane's
// (a shuffle within the row's segment of lanes), and everything about a run
// but the lane's own word index is the same for the whole warp.
__global__ void __launch_bounds__(256) k_render_bits(const QueryDesc* __restrict__ qd, uint16_t free_value) {
    extern __shared__ RunW rw[];
    const QueryDesc& Q = qd[blockIdx.z];
    const DevGrid g = Q.g;
    const uint32_t* __restrict__ bits = Q.bits;
    uint16_t* __restrict__ B = Q.v.B;
    const int T = blockIdx.y;
    const int r0 = g.run_off[T], nr = g.run_off[T + 1] - r0;
    const int nw = g.nx >> 5;
    const int64_t plane_words = (int64_t)g.nx * nw;  // words of one table level (<= 2^19)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const Run ru = g.runs[r0 + r];
        const int lo = ru.lo & g.mx, hi = ru.hi2 & g.mx;
        rw[r] = RunW{(int32_t)(ru.lvl * plane_words), ru.dy, lo >> 5, lo & 31, hi >> 5, hi & 31};
    }
    __syncthreads();
    const int64_t words = (int64_t)g.nx * nw;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= words) return;  // whole warps: words is a multiple of 32
    const int j = (int)(k / nw), w = (int)(k % nw);
    uint32_t hard = 0;
    if (nw <= 32) {
        const int nm = nw - 1, next = (w + 1) & nm;
        for (int r = 0; r < nr; r++) {
            if ((r & 7) == 0 && __all_sync(0xFFFFFFFFu, hard == 0xFFFFFFFFu)) break;
            const RunW ru = rw[r];
            const int64_t ro = ru.base + (int64_t)((j + ru.dy) & g.mx) * nw;
            if (!NHP_IN(ro, (int64_t)(g.lx + 1) * plane_words, Q.err, 12)) continue;
            const uint32_t* row = bits + ro;
            const uint32_t a1 = __ldg(row + ((w + ru.q1) & nm));
            const uint32_t b1 = __shfl_sync(0xFFFFFFFFu, a1, next, nw);
            const uint32_t a2 = __ldg(row + ((w + ru.q2) & nm));
            const uint32_t b2 = __shfl_sync(0xFFFFFFFFu, a2, next, nw);
            hard |= __funnelshift_r(a1, b1, ru.s1) | __funnelshift_r(a2, b2, ru.s2);
        }
    } else {
        for (int r = 0; r < nr && hard != 0xFFFFFFFFu; r++) {
            const RunW ru = rw[r];
            const uint32_t* row = bits + ru.base + (int64_t)((j + ru.dy) & g.mx) * nw;
            hard |= row_window(row, 32 * (w + ru.q1) + ru.s1, nw - 1) |
                    row_window(row, 32 * (w + ru.q2) + ru.s2, nw - 1);
        }
    }
    if (!NHP_IN((int64_t)T * g.nx * g.nx + (int64_t)j * g.nx + 32 * w + 31, (int64_t)g.nx * g.nx * g.nt, Q.err, 13))
        return;
    uint4* out = (uint4*)(B + (int64_t)T * g.nx * g.nx + (int64_t)j * g.nx + 32 * w);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t v[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int t = 8 * q + 2 * h;
            const uint32_t a = (hard >> t) & 1u ? HARD : free_value;
            const uint32_t b = (hard >> (t + 1)) & 1u ? HARD : free_value;
            v[h] = a | (b << 16);
        }
        out[q] = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// Soft values for the poses the bit pass left non-hard.
__global__ void __launch_bounds__(256) k_render_soft(const QueryDesc* __restrict__ qd) {
    extern __shared__ Run runs[];
    const QueryDesc& Q = qd[blockIdx.z];
    const DevGrid g = Q.g;
    const uint16_t* __restrict__ table = Q.table;
    uint16_t* __restrict__ B = Q.v.B;
    const int T = blockIdx.y;
    const int r0 = g.run_off[T], nr = g.run_off[T + 1] - r0;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) runs[r] = g.runs[r0 + r];
    __syncthreads();
    const int64_t nxy = (int64_t)g.nx * g.nx;
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nxy) return;
    uint16_t* dst = B + (int64_t)T * nxy + cell;
    const bool hard = *dst == HARD;
    if (__all_sync(__activemask(), hard)) return;
    const int i = (int)(cell & g.mx), j = (int)(cell >> g.lx);
    uint16_t m = 0;
    for (int r = 0; r < nr; r++) {
        const Run ru = runs[r];
        const int64_t ro = (int64_t)ru.lvl * nxy + ((int64_t)((j + ru.dy) & g.mx) << g.lx);
        if (!NHP_IN(ro, (int64_t)(g.lx + 1) * nxy, Q.err, 14)) continue;
        const uint16_t* row = table + ro;
        m = max(m, max(__ldg(row + ((i + ru.lo) & g.mx)), __ldg(row + ((i + ru.hi2) & g.mx))));
    }
    if (!hard) *dst = m;
}

}  // namespace

// Footprints with many row runs need more than the default 48 KB of dynamic
// shared memory for a heading's runs: raise the kernel's limit (up to what
// the device allows) when a launch needs it.
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0, most = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&most, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)most) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_sparse_table(const Group& gr, cudaStream_t s) {
    const int64_t nxy = (int64_t)1 << (2 * gr.lx);
    int64_t blocks = (nxy + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    const dim3 grid((unsigned)blocks, (unsigned)gr.nq);
    k_table_level0<<<grid, 256, 0, s>>>(gr.d);
    for (int k = 1; k <= gr.lx; k++) k_table_level<<<grid, 256, 0, s>>>(gr.d, k);
    return cudaGetLastError();
}

cudaError_t launch_render_table(const Group& gr, cudaStream_t s) {
    const int64_t nxy = (int64_t)1 << (2 * gr.lx);
    dim3 grid((unsigned)((nxy + 255) / 256), (unsigned)(1 << gr.lt), (unsigned)gr.nq);
    const size_t bytes = (size_t)gr.max_runs * sizeof(Run);
    const cudaError_t e = allow_smem(k_render, bytes);
    if (e != cudaSuccess) return e;
    k_render<<<grid, 256, bytes, s>>>(gr.d);
    return cudaGetLastError();
}

cudaError_t launch_render(const Group& gr, bool soft, cudaStream_t s, int* launches) {
    const int nx = 1 << gr.lx, nt = 1 << gr.lt;
    int n = 0;
    cudaError_t e = cudaSuccess;
    if (soft || nx < 32) {
        e = launch_sparse_table(gr, s);
        n += gr.lx + 1;
    }
    if (e == cudaSuccess && nx >= 32) {
        // bit-parallel hard test; soft maxima only for the non-hard poses
        const int64_t words = (int64_t)nx * (nx >> 5);
        int64_t blocks = (words + 255) / 256;
        if (blocks > 148 * 8) blocks = 148 * 8;
        const dim3 lg((unsigned)blocks, (unsigned)gr.nq);
        k_bits_level0<<<lg, 256, 0, s>>>(gr.d);
        for (int k = 1; k <= gr.lx; k++) k_bits_level<<<lg, 256, 0, s>>>(gr.d, k);
        const dim3 grid((unsigned)((words + 255) / 256), (unsigned)nt, (unsigned)gr.nq);
        const size_t wbytes = (size_t)gr.max_runs * sizeof(RunW), rbytes = (size_t)gr.max_runs * sizeof(Run);
        e = allow_smem(k_render_bits, wbytes);
        if (e == cudaSuccess) e = soft ? allow_smem(k_render_soft, rbytes) : cudaSuccess;
        if (e != cudaSuccess) return e;
        k_render_bits<<<grid, 256, wbytes, s>>>(gr.d, soft ? 0 : 256);
        n += gr.lx + 2;
        if (soft) {
            const dim3 g2((unsigned)(((int64_t)nx * nx + 255) / 256), (unsigned)nt, (unsigned)gr.nq);
            k_render_soft<<<g2, 256, rbytes, s>>>(gr.d);
            n += 1;
        }
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        e = launch_render_table(gr, s);
        n += 1;
    }
    if (launches) *launches = n;
    return e;
}

}  // namespace nhp

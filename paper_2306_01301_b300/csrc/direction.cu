// direction.cu -- direction penalties (Section XVI, Fig. 19: stay in the
// right-hand lane, do not drive against a lane's direction).
//
// A field gives each cell a preferred heading (or none).  A pose whose
// reference cell has one and whose own heading differs from it by more than
// a tolerance (circular distance in heading steps) has its obstacle value B
// scaled by a Q8 penalty after rendering: moving there costs more per step,
// as if the vehicle had to crawl.  Hard poses stay hard; scaled values are
// capped just below HARD.  One elementwise pass over B, eight poses (16
// bytes) per thread along x, the field read through L2.
#include <algorithm>

#include "internal.h"

namespace nhp {
namespace {

__device__ __forceinline__ uint16_t penalised(uint16_t b, uint16_t h, int T, int mt, int nt, int tol, uint32_t pen) {
    if (b == HARD || h == NO_DIRECTION) return b;
    int d = (T - (int)h) & mt;
    d = min(d, nt - d);
    if (d <= tol) return b;
    return (uint16_t)min((uint32_t)b * pen >> 8, (uint32_t)HARD - 1u);
}

// Nx >= 8: a thread takes 8 consecutive poses of one row of one heading.
__global__ void __launch_bounds__(256) k_direction8(uint16_t* __restrict__ B, const uint16_t* __restrict__ field,
                                                    int lx, int lt, int tol, uint32_t pen, int64_t groups) {
    const int mt = (1 << lt) - 1, nt = 1 << lt;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < groups;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = gi * 8;
        const int T = (int)(c0 >> (2 * lx));
        const int64_t xy = c0 & (((int64_t)1 << (2 * lx)) - 1);
        uint4 bv = reinterpret_cast<uint4*>(B)[gi];
        const uint4 hv = __ldg(reinterpret_cast<const uint4*>(field) + (xy >> 3));
        uint32_t* bw = reinterpret_cast<uint32_t*>(&bv);
        const uint32_t* hw = reinterpret_cast<const uint32_t*>(&hv);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint16_t lo = penalised((uint16_t)(bw[k] & 0xFFFFu), (uint16_t)(hw[k] & 0xFFFFu), T, mt, nt, tol, pen);
            const uint16_t hi = penalised((uint16_t)(bw[k] >> 16), (uint16_t)(hw[k] >> 16), T, mt, nt, tol, pen);
            bw[k] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        reinterpret_cast<uint4*>(B)[gi] = bv;
    }
}

__global__ void k_direction1(uint16_t* __restrict__ B, const uint16_t* __restrict__ field, int lx, int lt, int tol,
                             uint32_t pen, int64_t cells) {
    const int mt = (1 << lt) - 1, nt = 1 << lt;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int T = (int)(c >> (2 * lx));
        B[c] = penalised(B[c], field[c & (((int64_t)1 << (2 * lx)) - 1)], T, mt, nt, tol, pen);
    }
}

}  // namespace

cudaError_t launch_direction(uint16_t* B, const uint16_t* field, int lx, int lt, int tol, uint32_t pen,
                             cudaStream_t s) {
    const int64_t cells = (int64_t)1 << (2 * lx + lt);
    if (lx >= 3) {
        const int64_t groups = cells / 8;
        const unsigned blocks = (unsigned)std::min<int64_t>((groups + 255) / 256, 148 * 16);
        k_direction8<<<blocks, 256, 0, s>>>(B, field, lx, lt, tol, pen, groups);
    } else {
        k_direction1<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(B, field, lx, lt, tol, pen, cells);
    }
    return cudaGetLastError();
}

}  // namespace nhp

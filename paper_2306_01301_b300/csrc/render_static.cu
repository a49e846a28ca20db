// render_static.cu -- obstacle rendering without any allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// rendering: code that runs after a process has handed all device memory to
// another owner (a serving runtime with a fixed memory plan, a real-time
// control loop that forbids allocation after start-up, a host framework whose
// allocator must not be re-entered from a callback).  This entry point renders
// the obstacle volume into a caller-provided device buffer and keeps its own
// scratch -- the per-row sparse table and the footprint run list -- in one
// file-scope device array of fixed size.
//
// The array lives in every GPU that loads this library until the process
// exits.  Host code must not use the array's name as a device address (in
// host code it is only a stand-in); the device address is fetched once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

using namespace nhp;

namespace {

constexpr int kMaxNxLog2 = 9;           // Nx <= 512
constexpr int kMaxNtLog2 = 10;          // N_theta <= 1024
constexpr int kMaxRuns = 1 << 16;       // footprint rows over all headings
constexpr size_t kTableBytes = (size_t)(kMaxNxLog2 + 1) << (2 * kMaxNxLog2) << 1;  // 10 levels of 512^2 uint16
constexpr size_t kRunBytes = sizeof(Run) * kMaxRuns;
constexpr size_t kOffBytes = sizeof(int32_t) * ((1 << kMaxNtLog2) + 1);
constexpr size_t kOffPad = (kOffBytes + 255) & ~size_t(255);
constexpr size_t kDescBytes = 512;  // room for the kernel descriptor
constexpr size_t kScratchBytes = kTableBytes + kRunBytes + kOffPad + kDescBytes;

static __device__ __align__(256) unsigned char g_render_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Host staging for the run list and the kernel descriptor (static, so the
// call allocates nothing; cudaMemcpyAsync from pageable memory returns once
// the source may be reused).
Run g_host_runs[kMaxRuns];
int32_t g_host_off[(1 << kMaxNtLog2) + 1];
QueryDesc g_host_desc;
static_assert(sizeof(QueryDesc) <= kDescBytes, "descriptor slot too small");

int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PLAN_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_render_scratch) != cudaSuccess || !p) return PLAN_ECUDA;
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return PLAN_OK;
}

// Footprint runs of every heading (same covering rule as plan_create: the
// closed rectangle about the rear axle at the eq. 16 pose, cell centres,
// 1e-9 tolerance, the origin cell always covered).
int build_runs_static(int lx, int lt, const plan_footprint* f, double R, uint32_t flags, int* max_runs) {
    const double kPi = 3.14159265358979323846;
    const int nx = 1 << lx, nt = 1 << lt;
    const bool half = (flags & PLAN_FLAG_HALF_SHIFT) != 0;
    const int ext = std::max(f->front, f->rear);
    const int lim = (int)ceil(sqrt((double)ext * ext + (double)f->half_width * f->half_width)) + 2;
    int psi2[1 << kMaxNtLog2];
    for (int T = 0; T < nt; T++) {
        const long z = lround(2.0 * (R * sin((2.0 * kPi) * (double)T / (double)nt)));
        psi2[T] = half ? (int)(z & 1) : 0;
    }
    char row[2 * 2900 + 8];
    if (2 * lim + 1 > (int)sizeof(row)) return PLAN_EINVAL;
    int n = 0;
    *max_runs = 0;
    g_host_off[0] = 0;
    const double eps = 1e-9;
    for (int T = 0; T < nt; T++) {
        const double th = (2.0 * kPi) * (double)T / (double)nt;
        const double c = cos(th), s = sin(th);
        const double px0 = 0.5 * psi2[T], py0 = 0.5 * psi2[(T + nt / 4) % nt];
        const int first = n;
        for (int dy = -lim; dy <= lim; dy++) {
            for (int dx = -lim; dx <= lim; dx++) {
                bool in = dx == 0 && dy == 0;
                if (!in) {
                    const double ax = (double)dx - px0, ay = (double)dy - py0;
                    const double xv = c * ax + s * ay, yv = -s * ax + c * ay;
                    in = xv >= -(double)f->rear - eps && xv <= (double)f->front + eps &&
                         yv >= -(double)f->half_width - eps && yv <= (double)f->half_width + eps;
                }
                row[dx + lim] = in;
            }
            for (int a = 0; a <= 2 * lim;) {
                if (!row[a]) { a++; continue; }
                int b = a;
                while (b + 1 <= 2 * lim && row[b + 1]) b++;
                if (n >= kMaxRuns) return PLAN_ERANGE;
                const int lo = a - lim, hi = b - lim, w = hi - lo + 1;
                Run r;
                r.dy = (int16_t)dy;
                r.lo = (int16_t)lo;
                if (w >= nx) {
                    r.lvl = (int16_t)lx;
                    r.hi2 = (int16_t)lo;
                } else {
                    int lvl = 0;
                    while ((2 << lvl) <= w) lvl++;
                    r.lvl = (int16_t)lvl;
                    r.hi2 = (int16_t)(hi - (1 << lvl) + 1);
                }
                g_host_runs[n++] = r;
                a = b + 1;
            }
        }
        g_host_off[T + 1] = n;
        *max_runs = std::max(*max_runs, n - first);
    }
    return PLAN_OK;
}

}  // namespace

extern "C" int plan_render_cspace_static(const uint16_t* image_dev, int nx_log2, int ntheta_log2,
                                         const plan_footprint* footprint, double turn_radius_cells,
                                         uint32_t flags, uint16_t* B_dev, void* cuda_stream) {
    if (!image_dev || !B_dev || !footprint) return PLAN_EINVAL;
    if (nx_log2 < 2 || ntheta_log2 < 2 || ntheta_log2 > kMaxNtLog2) return PLAN_EINVAL;
    if (nx_log2 > kMaxNxLog2) return PLAN_ERANGE;  // scratch holds at most 512 x 512 cells per level
    if (!(turn_radius_cells > 0) || turn_radius_cells > 1e6) return PLAN_EINVAL;
    if (footprint->front < 0 || footprint->rear < 0 || footprint->half_width < 0 || footprint->front > 2000 ||
        footprint->rear > 2000 || footprint->half_width > 2000)
        return PLAN_EINVAL;
    unsigned char* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PLAN_OK) return rc;
    // the host staging buffers are shared: one caller at a time on the host
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    int max_runs = 0;
    rc = build_runs_static(nx_log2, ntheta_log2, footprint, turn_radius_cells, flags, &max_runs);
    if (rc != PLAN_OK) return rc;
    const int nt = 1 << ntheta_log2;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint16_t* table = (uint16_t*)scratch;
    Run* runs = (Run*)(scratch + kTableBytes);
    int32_t* off = (int32_t*)(scratch + kTableBytes + kRunBytes);
    // every scratch byte the kernels read is rewritten here or by the sparse
    // table kernels before it is read; nothing needs clearing
    if (cudaMemcpyAsync(runs, g_host_runs, sizeof(Run) * std::max(1, g_host_off[nt]), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(off, g_host_off, sizeof(int32_t) * (nt + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PLAN_ECUDA;
    QueryDesc* desc = (QueryDesc*)(scratch + kTableBytes + kRunBytes + kOffPad);
    QueryDesc& q = g_host_desc;
    q = QueryDesc{};
    q.g.lx = nx_log2;
    q.g.lt = ntheta_log2;
    q.g.nx = 1 << nx_log2;
    q.g.nt = nt;
    q.g.mx = q.g.nx - 1;
    q.g.mt = nt - 1;
    q.g.run_off = off;
    q.g.runs = runs;
    q.v.B = B_dev;
    q.img = image_dev;
    q.table = table;
    q.max_runs = std::max(1, max_runs);
    if (cudaMemcpyAsync(desc, &q, sizeof(QueryDesc), cudaMemcpyHostToDevice, s) != cudaSuccess) return PLAN_ECUDA;
    const Group gr{desc, 1, nx_log2, ntheta_log2, q.max_runs};
    if (launch_sparse_table(gr, s) != cudaSuccess) return PLAN_ECUDA;
    if (launch_render_table(gr, s) != cudaSuccess) return PLAN_ECUDA;
    return PLAN_OK;
}

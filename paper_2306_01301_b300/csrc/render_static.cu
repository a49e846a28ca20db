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

#include "footprint.h"
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

// Footprint runs of every heading into the static staging arrays: the same
// shift table and rasterisation as plan_create (footprint.h).
int build_runs_static(int lx, int lt, const plan_footprint* f, double R, uint32_t flags, int* max_runs) {
    const int nt = 1 << lt;
    static int psi2[1 << kMaxNtLog2];
    static char row[2 * 2900 + 8];
    if (reach_width(*f) > (int)sizeof(row)) return PLAN_EINVAL;
    shift_tables(R, nt, (flags & PLAN_FLAG_HALF_SHIFT) != 0, nullptr, psi2);
    int n = 0, first = 0;
    *max_runs = 0;
    g_host_off[0] = 0;
    const bool fits = footprint_rows(
        lx, nt, *f, psi2, row, [](int, int) { return true; },
        [&](const Run& r) {
            if (n >= kMaxRuns) return false;
            g_host_runs[n++] = r;
            return true;
        },
        [&](int T) {
            g_host_off[T + 1] = n;
            *max_runs = std::max(*max_runs, n - first);
            first = n;
            return true;
        });
    return fits ? PLAN_OK : PLAN_ERANGE;
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

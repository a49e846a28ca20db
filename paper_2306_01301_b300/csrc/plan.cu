// plan.cu -- host side of the nhplan C ABI: geometry tables, footprint runs,
// device memory, the maneuver-cycle schedule and plan extraction.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <cstdio>
#include <vector>

#include "footprint.h"
#include "plan_state.h"

using namespace nhp;

namespace {

constexpr double kPi = 3.14159265358979323846;

void* default_alloc(size_t bytes, void*, void*) {
    void* p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
void default_free(void* p, size_t, void*, void*) { cudaFree(p); }

size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

}  // namespace


namespace {

// ------------------------------------------------------------ geometry tables
// Section V.C.  Heading T stands for theta = 2 pi T / N_theta.
//   eq. 11-13: alpha = R sin(theta); with the half-cell option
//              zeta(alpha) = round(2 alpha)/2, beta = floor(zeta), Psi = zeta -
//              beta; without it beta = round(alpha), Psi = 0.
//   eq. 19:    I = 0 iff |tan theta| <= 1, decided on the integer heading
//              (angular distance m*2pi/N to the nearest multiple of pi is at
//              most pi/4 iff 8m <= N).
//   eq. 20-22: K = tan (I = 0) or cot (I = 1); B(y', T) = round(y' K).
//   eq. 24:    J = sign(cos) (I = 0) or sign(sin) (I = 1).
//   Section V.D edge lengths: turn 2 pi R / N_theta, straight
//              1/max(|cos|,|sin|), scaled by the integer step units and rounded.
void build_tables(plan_s* p, std::vector<int>& beta, std::vector<int>& psi2) {
    const int nt = p->nt, nx = p->nx;
    const bool half = (p->costs.flags & PLAN_FLAG_HALF_SHIFT) != 0;
    beta.assign(nt, 0);
    psi2.assign(nt, 0);
    p->planes.assign(nt, PlaneInfo{});
    p->bshear.assign((size_t)nt * nx, 0);
    uint32_t wmax = 0;
    shift_tables(p->R, nt, half, beta.data(), psi2.data());
    for (int T = 0; T < nt; T++) {
        const double th = (2.0 * kPi) * (double)T / (double)nt;
        const double s = sin(th), c = cos(th);
        const int halfN = nt / 2;
        const int r = T % halfN;
        const int m = std::min(r, halfN - r);
        PlaneInfo& pi = p->planes[T];
        pi.iflag = 8 * m <= nt ? 0 : 1;
        if (pi.iflag == 0) {
            const int d0 = std::min(T, nt - T);
            pi.jsign = 4 * d0 < nt ? 1 : -1;
        } else {
            pi.jsign = 2 * T < nt ? 1 : -1;
        }
        const double K = pi.iflag == 0 ? s / c : c / s;
        for (int y = 0; y < nx; y++) p->bshear[(size_t)T * nx + y] = (int16_t)lround((double)y * K);
        pi.wS = (uint32_t)lround((double)p->costs.step_straight * (1.0 / fmax(fabs(c), fabs(s))));
        wmax = std::max(wmax, pi.wS);
    }
    p->wA = (uint32_t)lround((double)p->costs.step_scale * (2.0 * kPi) * p->R / (double)nt);
    p->w_max = std::max(wmax, p->wA);
    p->beta4.resize(nt);
    const int q = nt / 4;
    for (int T = 0; T < nt; T++)
        p->beta4[T] = make_int4(beta[T], beta[(T + 3 * q) % nt], beta[(T + 2 * q) % nt], beta[(T + q) % nt]);
}

// Footprint runs and cells of every heading (footprint.h).
void build_runs(plan_s* p, const std::vector<int>& psi2) {
    const int nt = p->nt;
    p->run_off.assign(nt + 1, 0);
    p->runs.clear();
    p->fp_off.assign(nt + 1, 0);
    p->fp_dx.clear();
    p->fp_dy.clear();
    p->max_runs = 0;
    std::vector<char> row(reach_width(p->fp));
    int first = 0;
    footprint_rows(
        p->lx, nt, p->fp, psi2.data(), row.data(),
        [&](int dx, int dy) {
            p->fp_dx.push_back(dx);
            p->fp_dy.push_back(dy);
            return true;
        },
        [&](const Run& r) {
            p->runs.push_back(r);
            return true;
        },
        [&](int T) {
            p->run_off[T + 1] = (int32_t)p->runs.size();
            p->fp_off[T + 1] = (int32_t)p->fp_dx.size();
            p->max_runs = std::max(p->max_runs, (int)p->runs.size() - first);
            first = (int)p->runs.size();
            return true;
        });
}

int check_image(const uint16_t* img, int64_t n, uint32_t* max_soft) {
    uint32_t m = 256;
    for (int64_t k = 0; k < n; k++) {
        const uint16_t v = img[k];
        if (v == PLAN_HARD) continue;
        if (v < 256) return PLAN_EINVAL;
        if (v > m) m = v;
    }
    *max_soft = m;
    return PLAN_OK;
}

}  // namespace

namespace nhp {

bool pose_ok(const plan_s* p, plan_pose q) {
    return q.x >= 0 && q.y >= 0 && q.theta >= 0 && q.x < p->nx && q.y < p->nx && q.theta < p->nt;
}

int64_t cell_index(const plan_s* p, plan_pose q) {
    return (int64_t)q.x + ((int64_t)q.y << p->lx) + ((int64_t)q.theta << (2 * p->lx));
}

// Is pose q hard?  Same definition as the render kernel, evaluated on the
// host copy of the image for one pose.
bool pose_hard(const plan_s* p, plan_pose q) {
    const int M = p->nx - 1;
    for (int k = p->fp_off[q.theta]; k < p->fp_off[q.theta + 1]; k++) {
        const int x = (q.x + p->fp_dx[k]) & M, y = (q.y + p->fp_dy[k]) & M;
        if (x == 0 || y == 0 || p->img[(size_t)y * p->nx + x] == PLAN_HARD) return true;
    }
    return false;
}

namespace {
thread_local char g_last_error[256];
}

int cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorName(e));
    return PLAN_ECUDA;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PLAN_OK : cuda_fail(e, "CUDA runtime call"); }

const char* last_error_text() { return g_last_error; }

void record_check_failure(int site) {
    snprintf(g_last_error, sizeof(g_last_error), "bounds check failed at site %d", site);
}

uint64_t max_transition(const plan_s* p) {
    uint64_t m = 0;
    for (int k = 0; k < 6; k++) m = std::max<uint64_t>(m, (uint64_t)p->cin[k] + p->cout[k]);
    return m;
}

void set_transition(plan_s* p, const uint32_t* cin, const uint32_t* cout) {
    for (int k = 0; k < 6; k++) {
        p->cin[k] = cin[k];
        p->cout[k] = cout[k];
        p->g.ctm[k] = p->qd.g.ctm[k] = cin[k] + cout[k];
        p->g.cout[k] = p->qd.g.cout[k] = cout[k];
    }
}

uint64_t obstacle_bound(const plan_s* p) {
    return p->d_dir ? std::min<uint64_t>((uint64_t)p->img_max_soft * p->dir_pen >> 8, HARD - 1u)
                    : p->img_max_soft;
}

int range_check_layers(const plan_s* p, int layers) {
    // Every finite value is a sum over at most one segment per layer of ct
    // plus at most max(Nx, N_theta) - 1 edges; it must stay below the
    // kernels' TH.
    const uint64_t b_max = obstacle_bound(p);
    const double e_max = (double)(((uint64_t)p->w_max * b_max) >> 8);
    const double bound =
        (double)layers * ((double)max_transition(p) + (double)(std::max(p->nx, p->nt) - 1) * e_max);
    return bound >= (double)TH ? PLAN_ERANGE : PLAN_OK;
}

int range_check(const plan_s* p, int n_cycles) { return range_check_layers(p, 6 * n_cycles); }

int check_sweep(const plan_s* p, plan_pose start, int n_cycles) {
    if (n_cycles < 1 || n_cycles > 4096 || !pose_ok(p, start) || pose_hard(p, start)) return PLAN_EINVAL;
    return range_check(p, n_cycles);
}

int check_error_word(plan_s* p) {
    int32_t err = 0;
    int rc = cuda_rc(cudaMemcpyAsync(&err, p->d_status + 3, 4, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    return rc == PLAN_OK && err != 0 ? check_failed(p, err) : rc;
}

int check_failed(plan_s* p, int32_t site) {
    record_check_failure(site);
    cudaMemsetAsync(p->d_status + 3, 0, 4, p->stream);
    return PLAN_EINTERNAL;
}

int upload_desc(plan_s* p) {
    return cuda_rc(cudaMemcpyAsync(p->d_qd, &p->qd, sizeof(QueryDesc), cudaMemcpyHostToDevice, p->stream));
}

}  // namespace nhp

namespace {

// goals, then one GoalBest per goal, then the result
size_t goal_buffer_bytes(int n) { return (size_t)n * (sizeof(plan_goal) + sizeof(GoalBest)) + sizeof(GoalBest); }

void release(plan_s* p) {
    p->dfree(p->d_blob, p->blob_bytes);
    p->dfree(p->d_img, (size_t)p->nxy * 2);
    p->dfree(p->d_table, p->table_bytes);
    p->dfree(p->d_bits, p->bits_bytes);
    p->dfree(p->d_V, (size_t)p->nr * 4);
    p->dfree(p->d_L, (size_t)p->nr * 2);
    p->dfree(p->d_B, (size_t)p->nr * 2);
    p->dfree(p->d_seg, sizeof(plan_segment) * kDevSegCap);
    p->dfree(p->d_status, 16);
    p->dfree(p->d_goals, goal_buffer_bytes(p->goal_cap));
    p->dfree(p->d_dir, (size_t)p->nxy * 2);
    p->dfree(p->d_Vr, (size_t)p->nr * 4);
    p->dfree(p->d_Lr, (size_t)p->nr * 2);
    curv4_release(p);
    compact_release(p);
    p->dfree(p->d_cnt, 32);
    p->dfree(p->d_qd, sizeof(QueryDesc));
    const size_t bits = (size_t)(p->nr / 8);
    p->dfree(p->d_hb, bits);
    p->dfree(p->d_hbt, bits);
    p->dfree(p->d_rt, bits);
    p->dfree(p->d_ot, bits);
    p->dfree(p->d_x1, bits);
    p->dfree(p->d_x2, bits);
    for (auto& st : p->reach_side)
        if (st) cudaStreamDestroy(st);
    for (auto& e : p->reach_ev)
        if (e) cudaEventDestroy(e);
    p->dfree(p->d_shallow, sizeof(int32_t) * (size_t)p->nt);
    p->dfree(p->d_reach, bits * (size_t)p->reach_cap);
    for (auto& m : p->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto e : p->spare) cudaEventDestroy(e);
    p->marks.clear();
    p->spare.clear();
}

enum { K_TURN = 0, K_STRAIGHT = 1, K_RENDER = 2, K_INIT = 3 };

cudaEvent_t take_event(plan_s* p) {
    if (!p->spare.empty()) {
        cudaEvent_t e = p->spare.back();
        p->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket one pass with an event pair when profiling; returns the start mark.
int mark_begin(plan_s* p, int kind) {
    if (!p->prof) return -1;
    plan_s::Mark m{kind, take_event(p), take_event(p)};
    if (!m.a || !m.b) return -1;
    cudaEventRecord(m.a, p->stream);
    p->marks.push_back(m);
    return (int)p->marks.size() - 1;
}
void mark_end(plan_s* p, int idx) {
    if (idx >= 0) cudaEventRecord(p->marks[idx].b, p->stream);
}

}  // namespace

namespace nhp {

int create_plan(const plan_grid* grid, const plan_footprint* footprint, double turn_radius_cells,
                const plan_costs* costs, const plan_allocator* allocator, void* cuda_stream, bool volumes,
                plan_s** out) {
    if (!out) return PLAN_EINVAL;
    *out = nullptr;
    if (!grid || !footprint || !costs || !grid->image) return PLAN_EINVAL;
    if (grid->nx_log2 < 2 || grid->nx_log2 > 12 || grid->ntheta_log2 < 2 || grid->ntheta_log2 > 10 ||
        2 * grid->nx_log2 + grid->ntheta_log2 > 32)  // at most 2^32 pose cells
        return PLAN_EINVAL;
    if (!(turn_radius_cells > 0) || turn_radius_cells > 1e6) return PLAN_EINVAL;
    if (footprint->front < 0 || footprint->rear < 0 || footprint->half_width < 0 || footprint->front > 2000 ||
        footprint->rear > 2000 || footprint->half_width > 2000)
        return PLAN_EINVAL;
    if (costs->transition >= (1u << 28) || costs->step_straight == 0 || costs->step_scale == 0)
        return PLAN_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free)) return PLAN_EINVAL;

    plan_s* p = new (std::nothrow) plan_s();
    if (!p) return PLAN_ENOMEM;
    p->lx = grid->nx_log2;
    p->lt = grid->ntheta_log2;
    p->nx = 1 << p->lx;
    p->nt = 1 << p->lt;
    p->nxy = (int64_t)p->nx * p->nx;
    p->nr = p->nxy * p->nt;
    p->R = turn_radius_cells;
    p->costs = *costs;
    p->fp = *footprint;
    p->stream = (cudaStream_t)cuda_stream;
    if (allocator) p->alloc = *allocator;
    else p->alloc = plan_allocator{default_alloc, default_free, nullptr};

    int rc = check_image(grid->image, p->nxy, &p->img_max_soft);
    if (rc != PLAN_OK) { delete p; return rc; }
    p->img.assign(grid->image, grid->image + p->nxy);

    std::vector<int> beta, psi2;
    build_tables(p, beta, psi2);
    if (p->wA == 0 || p->w_max > 0xFFFF) { delete p; return PLAN_EINVAL; }
    build_runs(p, psi2);

    // table blob: beta4 | planes | bshear | run_off | runs
    const size_t o_beta = 0;
    const size_t o_plane = o_beta + round16(sizeof(int4) * p->nt);
    const size_t o_bsh = o_plane + round16(sizeof(PlaneInfo) * p->nt);
    const size_t o_roff = o_bsh + round16(sizeof(int16_t) * p->bshear.size());
    const size_t o_runs = o_roff + round16(sizeof(int32_t) * p->run_off.size());
    p->blob_bytes = o_runs + round16(sizeof(Run) * std::max<size_t>(1, p->runs.size()));
    p->blob.assign(p->blob_bytes, 0);
    memcpy(p->blob.data() + o_beta, p->beta4.data(), sizeof(int4) * p->nt);
    memcpy(p->blob.data() + o_plane, p->planes.data(), sizeof(PlaneInfo) * p->nt);
    memcpy(p->blob.data() + o_bsh, p->bshear.data(), sizeof(int16_t) * p->bshear.size());
    memcpy(p->blob.data() + o_roff, p->run_off.data(), sizeof(int32_t) * p->run_off.size());
    if (!p->runs.empty()) memcpy(p->blob.data() + o_runs, p->runs.data(), sizeof(Run) * p->runs.size());

    p->table_bytes = (size_t)(p->lx + 1) * p->nxy * 2;
    p->bits_bytes = p->nx >= 32 ? (size_t)(p->lx + 1) * p->nxy / 8 : 0;
    p->d_blob = (unsigned char*)p->dalloc(p->blob_bytes);
    p->d_img = (uint16_t*)p->dalloc((size_t)p->nxy * 2);
    p->d_table = (uint16_t*)p->dalloc(p->table_bytes);
    p->volumes = volumes;
    if (volumes) {
        p->d_V = (uint32_t*)p->dalloc((size_t)p->nr * 4);
        p->d_L = (uint16_t*)p->dalloc((size_t)p->nr * 2);
    }
    p->d_B = (uint16_t*)p->dalloc((size_t)p->nr * 2);
    p->d_seg = (plan_segment*)p->dalloc(sizeof(plan_segment) * kDevSegCap);
    p->d_status = (int*)p->dalloc(16);
    p->d_cnt = (unsigned long long*)p->dalloc(32);
    p->d_qd = (QueryDesc*)p->dalloc(sizeof(QueryDesc));
    if (p->bits_bytes) p->d_bits = (uint32_t*)p->dalloc(p->bits_bytes);
    if ((p->bits_bytes && !p->d_bits) || !p->d_cnt || !p->d_qd ||
        !p->d_blob || !p->d_img || !p->d_table || (volumes && (!p->d_V || !p->d_L)) || !p->d_B || !p->d_seg ||
        !p->d_status) {
        release(p);
        delete p;
        return PLAN_ENOMEM;
    }
    rc = cuda_rc(cudaMemcpyAsync(p->d_blob, p->blob.data(), p->blob_bytes, cudaMemcpyHostToDevice, p->stream));
    if (rc == PLAN_OK)
        rc = cuda_rc(cudaMemcpyAsync(p->d_img, p->img.data(), (size_t)p->nxy * 2, cudaMemcpyHostToDevice, p->stream));
    if (rc != PLAN_OK) {
        release(p);
        delete p;
        return rc;
    }
    DevGrid& g = p->g;
    g.lx = p->lx; g.lt = p->lt; g.nx = p->nx; g.nt = p->nt; g.mx = p->nx - 1; g.mt = p->nt - 1;
    g.wA = p->wA;
    for (int k = 0; k < 6; k++) {
        p->cin[k] = g.ctm[k] = p->costs.transition;
        p->cout[k] = g.cout[k] = 0;
    }
    g.beta4 = (const int4*)(p->d_blob + o_beta);
    g.plane = (const PlaneInfo*)(p->d_blob + o_plane);
    g.bshear = (const int16_t*)(p->d_blob + o_bsh);
    g.run_off = (const int32_t*)(p->d_blob + o_roff);
    g.runs = (const Run*)(p->d_blob + o_runs);
    QueryDesc& q = p->qd;
    q.g = g;
    q.v = Volumes{p->d_V, p->d_L, p->d_B, nullptr};
    q.start = 0;
    q.goal = 0;
    q.n_cycles = 0;
    q.pass = -1;
    q.img = p->d_img;
    q.bits = p->d_bits;
    q.table = p->d_table;
    q.seg = p->d_seg;
    q.status = p->d_status;
    q.err = p->d_status + 3;  // the bounds-check build's error word (zero)
    q.seg_cap = kDevSegCap;
    q.max_runs = std::max(1, p->max_runs);
    rc = cuda_rc(cudaMemsetAsync(p->d_status, 0, 16, p->stream));
    if (rc == PLAN_OK) rc = upload_desc(p);
    if (rc != PLAN_OK) {
        release(p);
        delete p;
        return rc;
    }
    *out = p;
    return PLAN_OK;
}

}  // namespace nhp

namespace {

int sweep_impl(plan_s* p, plan_pose start, int n_cycles, const uint32_t* entry) {
    if (!p || n_cycles < 0 || n_cycles > 4096 || !pose_ok(p, start)) return PLAN_EINVAL;
    if (!p->volumes) return PLAN_ESTATE;
    if (!p->rendered) return PLAN_ESTATE;
    if (pose_hard(p, start)) return PLAN_EINVAL;
    bool seeded = false;
    StartEntry se{};
    if (entry) {
        for (int m = 0; m < 6; m++) {
            if (entry[m] > p->cin[m]) return PLAN_EINVAL;
            se.e[m] = entry[m];
            seeded |= entry[m] < p->cin[m];
        }
    }
    if (range_check_layers(p, 6 * n_cycles + (seeded ? 1 : 0)) != PLAN_OK) return PLAN_ERANGE;
    p->qd.start = cell_index(p, start);
    p->qd.n_cycles = n_cycles;
    p->qd.v.improved = p->prof_count ? p->d_cnt : nullptr;
    p->vol_kind = VOL_NONE;
    int rc = upload_desc(p);
    if (rc != PLAN_OK) return rc;
    const Group gr = p->group();
    cudaStream_t s = p->stream;
    int mk = mark_begin(p, K_INIT);
    rc = cuda_rc(launch_init(gr, s));
    p->launches++;
    if (rc == PLAN_OK && seeded) {  // the start layer (Section XII)
        rc = cuda_rc(launch_seed(p->d_qd, se, s));
        p->launches++;
    }
    mark_end(p, mk);
    // Passes 0 .. 4N of the cycle schedule (internal.h): the consecutive
    // turns on one curve family, {RB, RF} and {LB of cycle c, LF of cycle
    // c+1}, share a pass, so N cycles (6N maneuver layers) take 4N + 1.
    const int np = pass_count(n_cycles);
    for (int pass = 0; pass < np && rc == PLAN_OK; pass++) {
        const bool turn = pass_is_turn(pass);
        const int m = mark_begin(p, turn ? K_TURN : K_STRAIGHT);
        Group g2 = gr;
        g2.grid = turn ? p->turn_grid : p->straight_grid;
        rc = cuda_rc(turn ? launch_turn(g2, pass, p->turn_variant, s) : launch_straight(g2, pass, p->straight_lines, s));
        mark_end(p, m);
        p->launches++;
    }
    if (rc == PLAN_OK) p->vol_kind = VOL_PLAIN;
    return rc;
}

int device_check_failed(plan_s* p, int32_t site) { return check_failed(p, site); }

// Status of the label walk just launched: segment count, V(goal); copies the
// segments in driving order.  Synchronises.
int finish_extract(plan_s* p, plan_segment* out, int cap, int* n_out, uint32_t* cost) {
    int32_t status[4] = {0, 0, 0, 0};
    int rc = cuda_rc(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    if (status[3] != 0) return device_check_failed(p, status[3]);
    if (status[0] == -1) return PLAN_EUNREACHABLE;
    if (status[0] < 0) return PLAN_EINTERNAL;
    *cost = (uint32_t)(status[1] & 0xFFFF) | ((uint32_t)status[2] << 16);
    *n_out = status[0];
    if (status[0] > cap || status[0] > kDevSegCap) return PLAN_ERANGE;
    if (status[0] > 0) {
        rc = cuda_rc(cudaMemcpyAsync(out, p->d_seg, sizeof(plan_segment) * status[0], cudaMemcpyDeviceToHost,
                                     p->stream));
        if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
        if (rc != PLAN_OK) return rc;
        std::reverse(out, out + status[0]);  // the walk runs goal -> start
    }
    return PLAN_OK;
}

}  // namespace

extern "C" {

int plan_create(const plan_grid* grid, const plan_footprint* footprint, double turn_radius_cells,
                const plan_costs* costs, const plan_allocator* allocator, void* cuda_stream, plan_t** out) {
    return nhp::create_plan(grid, footprint, turn_radius_cells, costs, allocator, cuda_stream, true, out);
}

int plan_set_image(plan_t* p, const uint16_t* image) {
    if (!p || !image) return PLAN_EINVAL;
    uint32_t m;
    int rc = check_image(image, p->nxy, &m);
    if (rc != PLAN_OK) return rc;
    // the previous upload may still read the host copy: finish it first
    rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    p->img_max_soft = m;
    p->img.assign(image, image + p->nxy);
    p->rendered = false;
    return cuda_rc(cudaMemcpyAsync(p->d_img, p->img.data(), (size_t)p->nxy * 2, cudaMemcpyHostToDevice, p->stream));
}

int plan_render_cspace(plan_t* p) {
    if (!p) return PLAN_EINVAL;
    const int mk = mark_begin(p, K_RENDER);
    int n = 0;
    int rc = cuda_rc(launch_render(p->group(), p->img_max_soft > 256, p->stream, &n));
    p->launches += n;
    if (rc == PLAN_OK && p->d_dir) {
        rc = cuda_rc(launch_direction(p->d_B, p->d_dir, p->lx, p->lt, p->dir_tol, p->dir_pen, p->stream));
        p->launches++;
    }
    mark_end(p, mk);
    if (rc == PLAN_OK) p->rendered = true;
    return rc;
}

int plan_sweep(plan_t* p, plan_pose start, int n_cycles) { return sweep_impl(p, start, n_cycles, nullptr); }

int plan_set_gear_penalty(plan_t* p, uint32_t penalty) {
    if (!p) return PLAN_EINVAL;
    if (penalty == PLAN_GEAR_OFF) {
        p->dfree(p->d_Vr, (size_t)p->nr * 4);
        p->dfree(p->d_Lr, (size_t)p->nr * 2);
        p->d_Vr = nullptr;
        p->d_Lr = nullptr;
        p->gear_on = false;
        if (p->vol_kind == VOL_GEAR) p->vol_kind = VOL_NONE;
        return PLAN_OK;
    }
    if (penalty >= (1u << 28) || p->nx > 2048 || p->nt > 2048) return PLAN_EINVAL;
    if (!p->volumes) return PLAN_ESTATE;
    if (!p->d_Vr) {
        p->d_Vr = (uint32_t*)p->dalloc((size_t)p->nr * 4);
        p->d_Lr = (uint16_t*)p->dalloc((size_t)p->nr * 2);
        if (!p->d_Vr || !p->d_Lr) {
            p->dfree(p->d_Vr, (size_t)p->nr * 4);
            p->dfree(p->d_Lr, (size_t)p->nr * 2);
            p->d_Vr = nullptr;
            p->d_Lr = nullptr;
            return PLAN_ENOMEM;
        }
    }
    p->gear_pen = penalty;
    p->gear_on = true;
    if (p->vol_kind == VOL_GEAR) p->vol_kind = VOL_NONE;  // swept with another penalty
    return PLAN_OK;
}

int plan_sweep_gear(plan_t* p, plan_pose start, int start_gear, int n_cycles) {
    if (!p || n_cycles < 0 || n_cycles > 4096 || start_gear < 0 || start_gear > 2 || !pose_ok(p, start))
        return PLAN_EINVAL;
    if (!p->gear_on || !p->rendered) return PLAN_ESTATE;
    if (pose_hard(p, start)) return PLAN_EINVAL;
    GearLayer a{};
    a.g = p->g;
    a.B = p->d_B;
    a.Vf = p->d_V;
    a.Vr = p->d_Vr;
    a.Lf = p->d_L;
    a.Lr = p->d_Lr;
    a.pen = p->gear_pen;
    a.err = p->d_status + 3;
    // every layer adds at most one segment and one gear change
    a.scan = range_check_layers(p, 6 * n_cycles) == PLAN_OK &&
             (double)6 * n_cycles * (double)p->gear_pen + (double)6 * n_cycles * 65536.0 < (double)(1u << 29);
    cudaStream_t s = p->stream;
    p->vol_kind = VOL_NONE;
    int rc = cuda_rc(launch_gear_init(p->d_V, p->d_Vr, p->d_L, p->d_Lr, p->nr, cell_index(p, start), start_gear, s));
    p->launches++;
    // Maneuver ids are the cycle order.  Where the grid allows, RB, RF and
    // LB, next cycle's LF run as fused pairs (the same layers in the same
    // order, each pair one launch).
    const bool fuse = gear_pair_fused(a);
    for (int l = 0; l < 6 * n_cycles && rc == PLAN_OK; l++) {
        const int mu = l % 6;
        const int mu2 = mu == RB ? RF : (mu == LB && l + 1 < 6 * n_cycles ? LF : -1);
        if (fuse && mu2 >= 0) {
            rc = cuda_rc(launch_gear_pair(a, mu, mu2, p->cin[mu] + p->cout[mu], p->cin[mu2] + p->cout[mu2], s));
            l++;
        } else {
            a.cin = p->cin[mu];
            a.cout = p->cout[mu];
            rc = cuda_rc(launch_gear_layer(a, mu, s));
        }
        p->launches++;
    }
    if (rc == PLAN_OK) p->vol_kind = VOL_GEAR;
    return rc;
}

int plan_extract_gear(plan_t* p, plan_pose goal, plan_segment* out, int cap, int* n_out, uint32_t* cost,
                      int* end_gear) {
    if (!p || !n_out || !cost || !end_gear || cap < 0 || (cap > 0 && !out) || !pose_ok(p, goal)) return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    *end_gear = -1;
    if (p->vol_kind != VOL_GEAR) return PLAN_ESTATE;
    GearLayer a{};
    a.g = p->g;
    a.Vf = p->d_V;
    a.Vr = p->d_Vr;
    a.Lf = p->d_L;
    a.Lr = p->d_Lr;
    int rc = cuda_rc(launch_gear_extract(a, cell_index(p, goal), p->d_seg, kDevSegCap, p->d_status, p->stream));
    p->launches++;
    int32_t status[4] = {0, 0, 0, 0};  // [3]: the bounds-check build's error word
    if (rc == PLAN_OK)
        rc = cuda_rc(cudaMemcpyAsync(status, p->d_status, sizeof(status), cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    if (status[3] != 0) return check_failed(p, status[3]);
    if (status[0] == -1) return PLAN_EUNREACHABLE;
    if (status[0] < 0) return PLAN_EINTERNAL;
    *cost = (uint32_t)status[1];
    *end_gear = status[2];
    *n_out = status[0];
    if (status[0] > cap || status[0] > kDevSegCap) return PLAN_ERANGE;
    if (status[0] > 0) {
        rc = cuda_rc(cudaMemcpyAsync(out, p->d_seg, sizeof(plan_segment) * status[0], cudaMemcpyDeviceToHost,
                                     p->stream));
        if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
        if (rc != PLAN_OK) return rc;
        std::reverse(out, out + status[0]);
    }
    return PLAN_OK;
}

int plan_copy_reverse_volumes(plan_t* p, uint32_t* V, uint16_t* L) {
    if (!p) return PLAN_EINVAL;
    if (!p->gear_on) return PLAN_ESTATE;
    int rc = PLAN_OK;
    if (V) rc = cuda_rc(cudaMemcpyAsync(V, p->d_Vr, (size_t)p->nr * 4, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK && L)
        rc = cuda_rc(cudaMemcpyAsync(L, p->d_Lr, (size_t)p->nr * 2, cudaMemcpyDeviceToHost, p->stream));
    return rc == PLAN_OK ? check_error_word(p) : rc;
}

int plan_set_direction_field(plan_t* p, const uint16_t* heading, int tolerance, uint32_t penalty_q8) {
    if (!p) return PLAN_EINVAL;
    if (!heading) {
        p->dfree(p->d_dir, (size_t)p->nxy * 2);
        p->d_dir = nullptr;
        p->rendered = false;  // B still holds the penalties
        return PLAN_OK;
    }
    if (tolerance < 0 || tolerance > p->nt / 2 || penalty_q8 < 256 || penalty_q8 > 65535) return PLAN_EINVAL;
    for (int64_t i = 0; i < p->nxy; i++)
        if (heading[i] != PLAN_NO_DIRECTION && heading[i] >= p->nt) return PLAN_EINVAL;
    if (!p->d_dir) {
        p->d_dir = (uint16_t*)p->dalloc((size_t)p->nxy * 2);
        if (!p->d_dir) return PLAN_ENOMEM;
    }
    const int rc = cuda_rc(cudaMemcpyAsync(p->d_dir, heading, (size_t)p->nxy * 2, cudaMemcpyHostToDevice, p->stream));
    if (rc != PLAN_OK) return rc;
    p->dir_tol = tolerance;
    p->dir_pen = penalty_q8;
    p->rendered = false;  // B must be rendered again with the field
    return PLAN_OK;
}

int plan_set_transition_costs(plan_t* p, const uint32_t cost_in[6], const uint32_t cost_out[6]) {
    if (!p || !cost_in || !cost_out) return PLAN_EINVAL;
    for (int k = 0; k < 6; k++)
        if ((uint64_t)cost_in[k] + cost_out[k] >= (1u << 28)) return PLAN_EINVAL;
    set_transition(p, cost_in, cost_out);
    return PLAN_OK;
}

int plan_sweep_state(plan_t* p, plan_pose start, const uint32_t entry[6], int n_cycles) {
    if (!entry) return PLAN_EINVAL;
    return sweep_impl(p, start, n_cycles, entry);
}

int plan_extract(plan_t* p, plan_pose goal, plan_segment* out, int cap, int* n_out, uint32_t* cost) {
    if (!p || !n_out || !cost || cap < 0 || (cap > 0 && !out) || !pose_ok(p, goal)) return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    if (p->vol_kind != VOL_PLAIN) return PLAN_ESTATE;
    p->qd.goal = cell_index(p, goal);
    int rc = upload_desc(p);
    if (rc == PLAN_OK) rc = cuda_rc(launch_extract(p->group(), p->stream));
    p->launches++;
    if (rc != PLAN_OK) return rc;
    return finish_extract(p, out, cap, n_out, cost);
}

int plan_extract_goal_set(plan_t* p, const plan_goal* goals, int n_goals, plan_segment* out, int cap, int* n_out,
                          uint32_t* cost, plan_pose* best, uint64_t* score) {
    if (!p || !goals || n_goals < 1 || n_goals > PLAN_MAX_GOALS || !n_out || !cost || !best || !score || cap < 0 ||
        (cap > 0 && !out))
        return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    *score = ~0ull;
    for (int i = 0; i < n_goals; i++) {
        const plan_goal& q = goals[i];
        if (!pose_ok(p, q.pose) || q.radius_xy < 0 || q.radius_xy > 255 || q.radius_theta < 0 ||
            q.radius_theta > 255 || 2 * q.radius_theta >= p->nt)
            return PLAN_EINVAL;
    }
    if (!p->volumes || p->vol_kind != VOL_PLAIN) return PLAN_ESTATE;
    if (n_goals > p->goal_cap) {
        p->dfree(p->d_goals, goal_buffer_bytes(p->goal_cap));
        p->d_goals = (unsigned char*)p->dalloc(goal_buffer_bytes(n_goals));
        p->goal_cap = p->d_goals ? n_goals : 0;
        if (!p->d_goals) return PLAN_ENOMEM;
    }
    plan_goal* d_goal = reinterpret_cast<plan_goal*>(p->d_goals);
    GoalBest* d_per = reinterpret_cast<GoalBest*>(p->d_goals + (size_t)p->goal_cap * sizeof(plan_goal));
    GoalBest* d_res = d_per + p->goal_cap;
    p->qd.goal = cell_index(p, goals[0].pose);  // replaced on the device by the chosen pose
    int rc = upload_desc(p);
    if (rc == PLAN_OK)
        rc = cuda_rc(cudaMemcpyAsync(d_goal, goals, sizeof(plan_goal) * n_goals, cudaMemcpyHostToDevice, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(launch_goal_search(p->d_qd, d_goal, n_goals, d_per, d_res, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(launch_extract(p->group(), p->stream));
    p->launches += 3;
    GoalBest res{};
    if (rc == PLAN_OK) rc = cuda_rc(cudaMemcpyAsync(&res, d_res, sizeof(res), cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    if (res.cell < 0) return PLAN_EUNREACHABLE;
    best->x = (int32_t)(res.cell & (p->nx - 1));
    best->y = (int32_t)((res.cell >> p->lx) & (p->nx - 1));
    best->theta = (int32_t)(res.cell >> (2 * p->lx));
    *score = res.score;
    return finish_extract(p, out, cap, n_out, cost);
}

int plan_set_kernel_shapes(plan_t* p, int turn_variant, int turn_grid, int straight_lines, int straight_grid) {
    if (!p || turn_variant < -1 || turn_variant >= turn_variants(p->nt) || turn_grid < 0 || straight_grid < 0 ||
        (straight_lines != 0 && straight_lines != 128 && straight_lines != 256))
        return PLAN_EINVAL;
    p->turn_variant = turn_variant;
    p->turn_grid = turn_grid;
    p->straight_lines = straight_lines;
    p->straight_grid = straight_grid;
    return PLAN_OK;
}

int plan_autotune(plan_t* p, plan_pose start, plan_tune_entry* out, int cap, int* n_out) {
    if (!p || cap < 0 || (cap > 0 && !out) || !pose_ok(p, start)) return PLAN_EINVAL;
    if (!p->volumes) return PLAN_ESTATE;
    if (!p->rendered) return PLAN_ESTATE;
    if (pose_hard(p, start)) return PLAN_EINVAL;
    if (n_out) *n_out = 0;
    p->vol_kind = VOL_NONE;  // the timed passes leave V and L in between
    // Start the sweeps (init, passes 0 and 1), then time every turn shape on
    // pass 2 (RB, RF) and every straight shape on pass 3 (SB).  Repeating a
    // pass changes the values; the next plan_sweep initialises again.
    p->qd.start = cell_index(p, start);
    p->qd.n_cycles = 1;
    p->qd.v.improved = nullptr;
    int rc = upload_desc(p);
    if (rc != PLAN_OK) return rc;
    const Group gr = p->group();
    cudaStream_t s = p->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NHP_CK(cudaEventCreate(&e0));
    if (const cudaError_t ee = cudaEventCreate(&e1); ee != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ee, "cudaEventCreate");
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t err = launch_init(gr, s);
    if (err == cudaSuccess) err = launch_turn(gr, 0, -1, s);
    if (err == cudaSuccess) err = launch_straight(gr, 1, 0, s);
    int n = 0;
    float best_t = 1e30f, best_s = 1e30f;
    auto timed = [&](auto launch) -> float {
        if (launch() != cudaSuccess) return -1.f;  // warm-up
        float best = 1e30f;
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, s);
            if (launch() != cudaSuccess) return -1.f;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    const int nv = turn_variants(p->nt);
    for (int v = 0; v < nv && err == cudaSuccess; v++) {
        int K, SL, CL;
        turn_shape(p->lt, v, &K, &SL, &CL);
        for (int pers = 0; pers < 2 && err == cudaSuccess; pers++) {
            const int occ = pers ? turn_blocks_per_sm(p->lt, v) : 0;
            const int grid = pers ? std::max(1, occ * sms / CL) : 0;
            if (pers && occ == 0) continue;
            Group g2 = gr;
            g2.grid = grid;
            const float ms = timed([&] { return launch_turn(g2, 2, v, s); });
            if (ms < 0) { err = cudaGetLastError(); break; }
            if (n < cap) out[n] = plan_tune_entry{0, v, grid, ms};
            n++;
            if (ms < best_t) { best_t = ms; p->turn_variant = v; p->turn_grid = grid; }
        }
    }
    const int widths[2] = {128, 256};
    for (int wi = 0; wi < 2 && err == cudaSuccess; wi++) {
        const int w = widths[wi];
        if (p->nx < w && !(wi == 0 && p->nx < 128)) continue;
        for (int pers = 0; pers < 2 && err == cudaSuccess; pers++) {
            const int occ = pers ? straight_blocks_per_sm(w) : 0;
            if (pers && (occ == 0 || p->nx < 16)) continue;
            Group g2 = gr;
            g2.grid = pers ? occ * sms : 0;
            const float ms = timed([&] { return launch_straight(g2, 3, w, s); });
            if (ms < 0) { err = cudaGetLastError(); break; }
            if (n < cap) out[n] = plan_tune_entry{1, w, g2.grid, ms};
            n++;
            if (ms < best_s) { best_s = ms; p->straight_lines = w; p->straight_grid = g2.grid; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "plan_autotune");
    if (n_out) *n_out = n;
    return n > cap ? PLAN_ERANGE : PLAN_OK;
}

int plan_copy_volumes(plan_t* p, uint32_t* V, uint16_t* L, uint16_t* B) {
    if (!p) return PLAN_EINVAL;
    int rc = PLAN_OK;
    if (V) rc = cuda_rc(cudaMemcpyAsync(V, p->d_V, (size_t)p->nr * 4, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK && L) rc = cuda_rc(cudaMemcpyAsync(L, p->d_L, (size_t)p->nr * 2, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK && B) rc = cuda_rc(cudaMemcpyAsync(B, p->d_B, (size_t)p->nr * 2, cudaMemcpyDeviceToHost, p->stream));
    int32_t err = 0;
    if (rc == PLAN_OK) rc = cuda_rc(cudaMemcpyAsync(&err, p->d_status + 3, 4, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc == PLAN_OK && err != 0) rc = device_check_failed(p, err);
    return rc;
}

int plan_device_volumes(plan_t* p, uint32_t** V, uint16_t** L, uint16_t** B) {
    if (!p) return PLAN_EINVAL;
    if (V) *V = p->d_V;
    if (L) *L = p->d_L;
    if (B) *B = p->d_B;
    return PLAN_OK;
}

int plan_profile(plan_t* p, int enable) {
    if (!p || enable < PLAN_PROFILE_OFF || enable > PLAN_PROFILE_TIMING) return PLAN_EINVAL;
    int rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    for (auto& m : p->marks) { p->spare.push_back(m.a); p->spare.push_back(m.b); }
    p->marks.clear();
    p->acc = plan_profile_stats{};
    p->prof = enable != PLAN_PROFILE_OFF;
    p->prof_count = enable == PLAN_PROFILE_ALL;
    return cuda_rc(cudaMemsetAsync(p->d_cnt, 0, 32, p->stream));
}

int plan_profile_read(plan_t* p, plan_profile_stats* out) {
    if (!p || !out) return PLAN_EINVAL;
    unsigned long long cnt[4] = {0, 0, 0, 0};
    int rc = cuda_rc(cudaMemcpyAsync(cnt, p->d_cnt, 32, cudaMemcpyDeviceToHost, p->stream));
    if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(p->stream));
    if (rc != PLAN_OK) return rc;
    for (auto& m : p->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) != cudaSuccess) return PLAN_ECUDA;
        switch (m.kind) {
            case K_TURN: p->acc.turn_passes++; p->acc.turn_ms += ms; break;
            case K_STRAIGHT: p->acc.straight_passes++; p->acc.straight_ms += ms; break;
            case K_RENDER: p->acc.render_passes++; p->acc.render_ms += ms; break;
            default: p->acc.init_passes++; p->acc.init_ms += ms; break;
        }
        p->spare.push_back(m.a);
        p->spare.push_back(m.b);
    }
    p->marks.clear();
    p->acc.turn_improved = cnt[0];
    p->acc.straight_improved = cnt[1];
    p->acc.turn_tiles_improved = cnt[2];
    *out = p->acc;
    return PLAN_OK;
}

int plan_kernel_launches(plan_t* p, int64_t* count) {
    if (!p || !count) return PLAN_EINVAL;
    *count = p->launches;
    return PLAN_OK;
}

int plan_destroy(plan_t* p) {
    if (!p) return PLAN_EINVAL;
    cudaStreamSynchronize(p->stream);
    release(p);
    delete p;
    return PLAN_OK;
}

const char* plan_last_error(void) { return nhp::last_error_text(); }

const char* plan_strerror(int code) {
    switch (code) {
        case PLAN_OK: return "ok";
        case PLAN_EINVAL: return "invalid argument";
        case PLAN_ENOMEM: return "device allocation failed";
        case PLAN_ECUDA: return "CUDA runtime error";
        case PLAN_ETIMEOUT: return "device wait timed out";
        case PLAN_EUNREACHABLE: return "goal unreachable";
        case PLAN_ERANGE: return "capacity or cost range exceeded";
        case PLAN_EINTERNAL: return "internal consistency check failed";
        case PLAN_ESTATE: return "call out of order";
        case PLAN_ECANCELED: return "request cancelled";
        default: return "unknown error";
    }
}

// Section VII: soft obstacle costs from the distance to the nearest obstacle.
// Exact squared Euclidean distance transform by two passes of the 1-D lower
// envelope of parabolas (Felzenszwalb & Huttenlocher), the linear-time family
// of methods the paper points to (Meijster et al.).
int plan_soft_image(int nx, const uint8_t* occ, int radius, int soft_max, uint16_t* image) {
    if (nx <= 0 || nx > 65536 || !occ || !image || radius < 0 || radius > 255 || soft_max < 0 || soft_max > 65000)
        return PLAN_EINVAL;
    const int64_t n = (int64_t)nx * nx;
    const int64_t big = 4ll * nx * nx + 1;  // larger than any in-image squared distance
    std::vector<int64_t> d2(n), f(nx), out(nx);
    std::vector<int> vpos(nx);
    std::vector<double> z(nx + 1);
    auto dt1 = [&](int64_t* line, int64_t stride) {
        for (int q = 0; q < nx; q++) f[q] = line[q * stride];
        int k = 0;
        vpos[0] = 0;
        z[0] = -1e300;
        z[1] = 1e300;
        for (int q = 1; q < nx; q++) {
            double sv;
            for (;;) {  // z[0] = -inf, so this stops at k = 0 at the latest
                const int r = vpos[k];
                sv = ((double)(f[q] + (int64_t)q * q) - (double)(f[r] + (int64_t)r * r)) / (2.0 * (q - r));
                if (sv > z[k]) break;
                k--;
            }
            k++;
            vpos[k] = q;
            z[k] = sv;
            z[k + 1] = 1e300;
        }
        k = 0;
        for (int q = 0; q < nx; q++) {
            while (z[k + 1] < q) k++;
            const int64_t dq = q - vpos[k];
            out[q] = dq * dq + f[vpos[k]];
        }
        for (int q = 0; q < nx; q++) line[q * stride] = std::min(out[q], big);
    };
    for (int64_t k = 0; k < n; k++) d2[k] = occ[k] ? 0 : big;
    for (int x = 0; x < nx; x++) dt1(d2.data() + x, nx);           // columns
    for (int y = 0; y < nx; y++) dt1(d2.data() + (int64_t)y * nx, 1);  // rows
    const int64_t r2 = (int64_t)radius * radius;
    for (int64_t k = 0; k < n; k++) {
        if (occ[k]) { image[k] = PLAN_HARD; continue; }
        const int64_t pen = d2[k] < r2 ? (int64_t)soft_max * (r2 - d2[k]) / r2 : 0;
        image[k] = (uint16_t)(256 + pen);
    }
    return PLAN_OK;
}

}  // extern "C"

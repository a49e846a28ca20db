// batch.cu -- many planning queries per launch, replayed as one CUDA graph.
//
// A batch borrows a set of plans (one per query: its own image, footprint,
// turn radius, costs and volumes) and runs the whole hot path for all of
// them: rendering, initialisation, the 4N + 1 fused sweep passes and the
// label walk.  Queries are dealt into lanes by heading count and straight
// kernel width; each sweep pass of a lane is ONE launch over every query of
// the lane that still has that pass (queries sorted by N, so the active ones
// are a prefix), its blocks walking the concatenated work items of queries
// of different sizes.  Lanes are independent chains of launches; a CUDA
// graph captures them as parallel branches, so uneven queries share the GPU
// without host round trips.  Before the first capture an autotuner times the
// candidate kernel shapes of each lane on the lane's own data and keeps the
// fastest: the turn kernel's heading grouping (headings per thread, warps per
// block, blocks per cluster), the straight kernel's line-block width, and
// for each whether the grid is one block per work item or persistent (a
// multiple of the SM count, blocks looping over items).  All shapes give the
// same bits.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "plan_state.h"

using namespace nhp;

namespace {

constexpr int kTuneReps = 3;

struct Lane {
    int lt = 0;
    int nx_key = 0;        // the Nx shared by all queries (< 256), or 256: any Nx >= 256
    int lx_max = 0;
    bool uniform = true;   // one Nx: launches index queries directly
    bool same_costs = true;  // every member has the same transition costs
    std::vector<int> members;  // query indices in launch order (N descending)
    std::vector<int> n_of;     // N of each member, same order
    plan_batch_lane_info info{};
    size_t desc_off = 0;       // offsets into the descriptor mirror
    size_t turn_item_off = 0;
    size_t str_item_off[2] = {0, 0};  // straight items for 128 / 256 lines
    std::vector<int32_t> turn_items, str_items[2];
    cudaStream_t stream = nullptr;  // nullptr: the batch stream
    cudaEvent_t done = nullptr;
};

struct RenderGroup {
    int lx = 0, lt = 0, max_runs = 1;
    std::vector<int> members;
    size_t desc_off = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct plan_batch_s {
    std::vector<plan_s*> plans;
    uint32_t flags = 0;
    cudaStream_t user_stream = nullptr;  // the caller's stream (ordering only)
    cudaStream_t stream = nullptr;       // the batch's own stream
    std::vector<cudaStream_t> plan_streams;
    plan_allocator alloc{};
    int sms = 148;
    std::vector<Lane> lanes;
    std::vector<RenderGroup> rgroups;
    std::vector<plan_query> q;  // queries of the current run
    std::vector<int> key;       // N of every query + render flag: what the graph was built for
    std::vector<int> seg_cap;
    std::vector<size_t> seg_base;
    // descriptor mirror: pinned host staging, copied to the device by the run
    unsigned char* h_stage = nullptr;
    unsigned char* d_stage = nullptr;
    size_t stage_bytes = 0, stage_cap = 0;
    // results: per query int32[4] status, then the segment arrays
    unsigned char* h_res = nullptr;
    unsigned char* d_res = nullptr;
    size_t res_bytes = 0, res_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr, enter = nullptr;
    bool tuned = false;
    bool in_flight = false;
    int64_t launches_per_run = 0, launches = 0;

    void* dalloc(size_t bytes) { return alloc.alloc(bytes, (void*)stream, alloc.ctx); }
    void dfree(void* p, size_t bytes) {
        if (p) alloc.free(p, bytes, (void*)stream, alloc.ctx);
    }
};

namespace {

void* batch_default_alloc(size_t bytes, void*, void*) {
    void* p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
void batch_default_free(void* p, size_t, void*, void*) { cudaFree(p); }

void drop_graph(plan_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
}

void release(plan_batch_s* b) {
    drop_graph(b);
    for (auto& L : b->lanes) {
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.done) cudaEventDestroy(L.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->enter) cudaEventDestroy(b->enter);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->h_res) cudaFreeHost(b->h_res);
    b->dfree(b->d_stage, b->stage_cap);
    b->dfree(b->d_res, b->res_cap);
    if (b->stream) cudaStreamDestroy(b->stream);
}

// Lane of a plan shape: turn kernels are compiled per N_theta, straight
// kernels need Nx >= the block's lines (128 or 256) to mix sizes.
int lane_key_nx(int nx) { return nx >= 256 ? 256 : nx; }

Group lane_group(const plan_batch_s* b, const Lane& L, int nact) {
    Group g{};
    g.d = (const QueryDesc*)(b->d_stage + L.desc_off);
    g.nq = nact;
    g.lx = L.lx_max;
    g.lt = L.lt;
    g.max_runs = 1;
    if (L.same_costs) g.ctm = b->plans[L.members[0]]->g.ctm;
    return g;
}

// Number of members whose pass `p` exists (members are sorted by N, descending).
int active_count(const Lane& L, int p) {
    int n = 0;
    while (n < (int)L.n_of.size() && p < pass_count(L.n_of[n])) n++;
    return n;
}

cudaError_t lane_turn(const plan_batch_s* b, const Lane& L, int pass, int nact, int variant, int grid,
                      cudaStream_t s) {
    Group g = lane_group(b, L, nact);
    if (!L.uniform) {
        g.item_off = (const int32_t*)(b->d_stage + L.turn_item_off);
        g.items = L.turn_items[nact];
    }
    g.grid = grid;
    return launch_turn(g, pass, variant, s);
}

cudaError_t lane_straight(const plan_batch_s* b, const Lane& L, int pass, int nact, int lines, int grid,
                          cudaStream_t s) {
    Group g = lane_group(b, L, nact);
    if (!L.uniform) {
        const int k = lines == 128 ? 0 : 1;
        g.item_off = (const int32_t*)(b->d_stage + L.str_item_off[k]);
        g.items = L.str_items[k][nact];
    }
    g.grid = grid;
    return launch_straight(g, pass, lines, s);
}

int persistent_grid(const plan_batch_s* b, int per_sm, int cl) {
    return per_sm > 0 ? std::max(1, per_sm * b->sms / cl) : 0;
}

int turn_cluster(int lt, int variant) {
    int K, SL, CL;
    turn_shape(lt, variant, &K, &SL, &CL);
    return CL;
}

// Build the descriptor mirror for the current queries: lanes, render
// groups, result slots.  Returns PLAN_* codes.
int build_layout(plan_batch_s* b) {
    const int n = (int)b->plans.size();
    // result slots: the label walk yields at most one segment per maneuver layer
    b->seg_cap.assign(n, 0);
    b->seg_base.assign(n, 0);
    size_t res = align_up((size_t)n * 16, 256);
    for (int i = 0; i < n; i++) {
        b->seg_cap[i] = std::max(1, 6 * b->q[i].n_cycles);
        b->seg_base[i] = res;
        res += align_up(sizeof(plan_segment) * b->seg_cap[i], 16);
    }
    if (res > b->res_cap) {
        b->dfree(b->d_res, b->res_cap);
        if (b->h_res) cudaFreeHost(b->h_res);
        b->h_res = nullptr;
        b->d_res = (unsigned char*)b->dalloc(res);
        b->res_cap = b->d_res ? res : 0;
        if (!b->d_res) return PLAN_ENOMEM;
        if (cudaMallocHost((void**)&b->h_res, res) != cudaSuccess) return PLAN_ENOMEM;
    }
    b->res_bytes = res;

    // lane order: N descending, then query index (deterministic)
    size_t off = 0;
    for (auto& L : b->lanes) {
        std::sort(L.members.begin(), L.members.end(), [&](int x, int y) {
            const int nx_ = b->q[x].n_cycles, ny_ = b->q[y].n_cycles;
            return nx_ != ny_ ? nx_ > ny_ : x < y;
        });
        L.n_of.clear();
        for (int m : L.members) L.n_of.push_back(b->q[m].n_cycles);
        const int nq = (int)L.members.size();
        L.desc_off = off;
        off = align_up(off + sizeof(QueryDesc) * nq, 256);
        L.turn_items.assign(nq + 1, 0);
        L.str_items[0].assign(nq + 1, 0);
        L.str_items[1].assign(nq + 1, 0);
        for (int k = 0; k < nq; k++) {
            const plan_s* p = b->plans[L.members[k]];
            L.turn_items[k + 1] = L.turn_items[k] + (int32_t)turn_items(p->lx);
            if (p->nx >= 128) L.str_items[0][k + 1] = L.str_items[0][k] + (int32_t)straight_items(p->lx, p->lt, 128);
            if (p->nx >= 256) L.str_items[1][k + 1] = L.str_items[1][k] + (int32_t)straight_items(p->lx, p->lt, 256);
        }
        L.turn_item_off = off;
        off = align_up(off + sizeof(int32_t) * (nq + 1), 256);
        L.str_item_off[0] = off;
        off = align_up(off + sizeof(int32_t) * (nq + 1), 256);
        L.str_item_off[1] = off;
        off = align_up(off + sizeof(int32_t) * (nq + 1), 256);
    }
    for (auto& R : b->rgroups) {
        R.desc_off = off;
        off = align_up(off + sizeof(QueryDesc) * R.members.size(), 256);
    }
    if (off > b->stage_cap) {
        b->dfree(b->d_stage, b->stage_cap);
        if (b->h_stage) cudaFreeHost(b->h_stage);
        b->h_stage = nullptr;
        b->d_stage = (unsigned char*)b->dalloc(off);
        b->stage_cap = b->d_stage ? off : 0;
        if (!b->d_stage) return PLAN_ENOMEM;
        if (cudaMallocHost((void**)&b->h_stage, off) != cudaSuccess) return PLAN_ENOMEM;
    }
    b->stage_bytes = off;
    return PLAN_OK;
}

QueryDesc query_desc(const plan_batch_s* b, int i) {
    const plan_s* p = b->plans[i];
    QueryDesc d = p->qd;
    d.v.improved = nullptr;
    d.start = cell_index(p, b->q[i].start);
    d.goal = cell_index(p, b->q[i].goal);
    d.n_cycles = b->q[i].n_cycles;
    d.pass = -1;
    d.status = (int32_t*)(b->d_res + (size_t)i * 16);
    d.seg = (plan_segment*)(b->d_res + b->seg_base[i]);
    d.seg_cap = b->seg_cap[i];
    return d;
}

// Fill the pinned staging buffer (descriptors and item offsets).
void fill_stage(plan_batch_s* b) {
    for (auto& L : b->lanes) {
        QueryDesc* d = (QueryDesc*)(b->h_stage + L.desc_off);
        for (size_t k = 0; k < L.members.size(); k++) d[k] = query_desc(b, L.members[k]);
        memcpy(b->h_stage + L.turn_item_off, L.turn_items.data(), sizeof(int32_t) * L.turn_items.size());
        memcpy(b->h_stage + L.str_item_off[0], L.str_items[0].data(), sizeof(int32_t) * L.str_items[0].size());
        memcpy(b->h_stage + L.str_item_off[1], L.str_items[1].data(), sizeof(int32_t) * L.str_items[1].size());
    }
    for (auto& R : b->rgroups) {
        QueryDesc* d = (QueryDesc*)(b->h_stage + R.desc_off);
        for (size_t k = 0; k < R.members.size(); k++) d[k] = query_desc(b, R.members[k]);
    }
}

int enqueue_render(plan_batch_s* b, cudaStream_t s, int64_t* launches) {
    for (auto& R : b->rgroups) {
        Group g{};
        g.d = (const QueryDesc*)(b->d_stage + R.desc_off);
        g.nq = (int)R.members.size();
        g.lx = R.lx;
        g.lt = R.lt;
        g.max_runs = R.max_runs;
        bool soft = false;
        for (int m : R.members) soft = soft || b->plans[m]->img_max_soft > 256;
        int n = 0;
        NHP_CK(launch_render(g, soft, s, &n));
        *launches += n;
    }
    // direction penalties of the plans that have a field, as plan_render_cspace applies them
    for (const plan_s* p : b->plans)
        if (p->d_dir) {
            NHP_CK(launch_direction(p->d_B, p->d_dir, p->lx, p->lt, p->dir_tol, p->dir_pen, s));
            (*launches)++;
        }
    return PLAN_OK;
}

// One lane: init, all passes, label walk.  Work of the lane goes to stream s.
int enqueue_lane(plan_batch_s* b, Lane& L, cudaStream_t s, int64_t* launches) {
    const int nq = (int)L.members.size();
    if (nq == 0) return PLAN_OK;
    Group g = lane_group(b, L, nq);
    NHP_CK(launch_init(g, s));
    (*launches)++;
    const int np = pass_count(L.n_of[0]);
    for (int p = 0; p < np; p++) {
        const int nact = active_count(L, p);
        if (nact == 0) break;
        cudaError_t e = pass_is_turn(p)
                            ? lane_turn(b, L, p, nact, L.info.turn_variant, L.info.turn_grid, s)
                            : lane_straight(b, L, p, nact, L.info.straight_lines, L.info.straight_grid, s);
        NHP_CK(e);
        (*launches)++;
    }
    NHP_CK(launch_extract(g, s));
    (*launches)++;
    return PLAN_OK;
}

// The whole run on b->stream: staging upload, render, lanes (forked onto the
// lane streams), results download.
int enqueue_run(plan_batch_s* b, bool render, int64_t* launches) {
    cudaStream_t s = b->stream;
    NHP_CK(cudaMemcpyAsync(b->d_stage, b->h_stage, b->stage_bytes, cudaMemcpyHostToDevice, s));
    int rc = PLAN_OK;
    if (render) rc = enqueue_render(b, s, launches);
    if (rc != PLAN_OK) return rc;
    const bool fork = b->lanes.size() > 1;
    if (fork) NHP_CK(cudaEventRecord(b->fork, s));
    for (auto& L : b->lanes) {
        cudaStream_t ls = fork ? L.stream : s;
        if (fork) NHP_CK(cudaStreamWaitEvent(ls, b->fork, 0));
        rc = enqueue_lane(b, L, ls, launches);
        if (rc != PLAN_OK) return rc;
        if (fork) NHP_CK(cudaEventRecord(L.done, ls));
    }
    if (fork)
        for (auto& L : b->lanes) NHP_CK(cudaStreamWaitEvent(s, L.done, 0));
    NHP_CK(cudaMemcpyAsync(b->h_res, b->d_res, b->res_bytes, cudaMemcpyDeviceToHost, s));
    return PLAN_OK;
}

// Time `launch` (already warmed up) kTuneReps times on stream s; min ms.
template <class F>
float time_min(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F launch) {
    float best = 1e30f;
    for (int r = 0; r < kTuneReps; r++) {
        cudaEventRecord(e0, s);
        if (launch() != cudaSuccess) return -1.f;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    return best;
}

// Autotune one lane on its own data: start the sweeps (init, passes 0 and
// 1), then time every turn shape on pass 2 (RB, RF) and every straight
// shape on pass 3 (SB).  Repeating a pass changes the values, which does not
// matter: the real run initialises again.
int tune_lane(plan_batch_s* b, Lane& L) {
    const int nq = (int)L.members.size();
    cudaStream_t s = b->stream;
    Lane& li = L;
    plan_batch_lane_info& I = li.info;
    I.turn_variant = 0;
    I.turn_grid = 0;
    I.straight_lines = L.nx_key >= 256 ? 256 : (L.nx_key >= 128 ? 128 : L.nx_key);
    I.straight_grid = 0;
    if (!(b->flags & PLAN_BATCH_NO_TUNE)) {
        cudaEvent_t e0, e1;
        NHP_CK(cudaEventCreate(&e0));
        if (const cudaError_t ee = cudaEventCreate(&e1); ee != cudaSuccess) {
            cudaEventDestroy(e0);
            return cuda_fail(ee, "cudaEventCreate");
        }
        int rc = PLAN_OK;
        Group g = lane_group(b, L, nq);
        cudaError_t e = launch_init(g, s);
        if (e == cudaSuccess) e = lane_turn(b, L, 0, nq, 0, 0, s);
        if (e == cudaSuccess) e = lane_straight(b, L, 1, nq, I.straight_lines, 0, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tuning: first passes");
        float best = 1e30f;
        I.n_candidates = 0;
        const int nv = turn_variants(1 << L.lt);
        for (int v = 0; v < nv && rc == PLAN_OK; v++) {
            for (int pers = 0; pers < 2 && rc == PLAN_OK; pers++) {
                const int grid = pers ? persistent_grid(b, turn_blocks_per_sm(L.lt, v), turn_cluster(L.lt, v)) : 0;
                if (pers && grid == 0) continue;
                auto f = [&]() { return lane_turn(b, L, 2, nq, v, grid, s); };
                if (const cudaError_t ef = f(); ef != cudaSuccess) { rc = cuda_fail(ef, "tuning: candidate launch"); break; }
                const float ms = time_min(s, e0, e1, f);
                if (ms < 0) { rc = cuda_fail(cudaGetLastError(), "tuning: timing"); break; }
                I.n_candidates++;
                if (ms < best) { best = ms; I.turn_variant = v; I.turn_grid = grid; I.turn_ms = ms; }
            }
        }
        best = 1e30f;
        std::vector<int> widths;
        if (L.nx_key >= 256) widths = {128, 256};
        else widths = {I.straight_lines};
        for (int w : widths) {
            for (int pers = 0; pers < 2 && rc == PLAN_OK; pers++) {
                if (L.nx_key < 16 && pers) continue;  // the narrow-grid kernel has one shape
                const int grid = pers ? persistent_grid(b, straight_blocks_per_sm(w), 1) : 0;
                if (pers && grid == 0) continue;
                auto f = [&]() { return lane_straight(b, L, 3, nq, w, grid, s); };
                if (const cudaError_t ef = f(); ef != cudaSuccess) { rc = cuda_fail(ef, "tuning: candidate launch"); break; }
                const float ms = time_min(s, e0, e1, f);
                if (ms < 0) { rc = cuda_fail(cudaGetLastError(), "tuning: timing"); break; }
                I.n_candidates++;
                if (ms < best) { best = ms; I.straight_lines = w; I.straight_grid = grid; I.straight_ms = ms; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != PLAN_OK) return rc;
        NHP_CK(cudaStreamSynchronize(s));
    } else {
        // no timing; still set the kernels' attributes before any capture
        if (L.nx_key >= 16 && straight_blocks_per_sm(I.straight_lines == 128 ? 128 : 256) == 0)
            return cuda_fail(cudaGetLastError(), "straight kernel attributes");
    }
    turn_shape(L.lt, I.turn_variant, &I.turn_k, &I.turn_sections, &I.turn_cluster);
    I.n_queries = nq;
    I.ntheta_log2 = L.lt;
    I.nx_min = 1 << 30;
    I.nx_max = 0;
    for (int m : L.members) {
        I.nx_min = std::min(I.nx_min, b->plans[m]->nx);
        I.nx_max = std::max(I.nx_max, b->plans[m]->nx);
    }
    return PLAN_OK;
}

// Streams, events and the SM count; the plans' pending uploads finish first.
int batch_init(plan_batch_s* b) {
    int dev = 0;
    NHP_CK(cudaGetDevice(&dev));
    NHP_CK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    for (auto st : b->plan_streams) NHP_CK(cudaStreamSynchronize(st));
    // the batch works on a stream of its own (a capturable one: the caller's
    // may be the legacy default stream) ordered after the caller's stream
    NHP_CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    NHP_CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    NHP_CK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
    NHP_CK(cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming));
    if (b->lanes.size() > 1)
        for (auto& L : b->lanes) {
            NHP_CK(cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
            NHP_CK(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
        }
    return PLAN_OK;
}

}  // namespace

extern "C" {

int plan_batch_create(plan_t* const* plans, int n, uint32_t flags, const plan_allocator* allocator,
                      void* cuda_stream, plan_batch_t** out) {
    if (!out) return PLAN_EINVAL;
    *out = nullptr;
    if (!plans || n <= 0 || n > (1 << 20)) return PLAN_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free)) return PLAN_EINVAL;
    for (int i = 0; i < n; i++) {
        if (!plans[i]) return PLAN_EINVAL;
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return PLAN_EINVAL;  // each query needs its own volumes
    }
    plan_batch_s* b = new (std::nothrow) plan_batch_s();
    if (!b) return PLAN_ENOMEM;
    b->plans.assign(plans, plans + n);
    b->flags = flags;
    b->user_stream = (cudaStream_t)cuda_stream;
    b->alloc = allocator ? *allocator : plan_allocator{batch_default_alloc, batch_default_free, nullptr};
    for (int i = 0; i < n; i++) {
        const plan_s* p = b->plans[i];
        if (std::find(b->plan_streams.begin(), b->plan_streams.end(), p->stream) == b->plan_streams.end())
            b->plan_streams.push_back(p->stream);
        const int key = lane_key_nx(p->nx);
        Lane* L = nullptr;
        for (auto& l : b->lanes)
            if (l.lt == p->lt && l.nx_key == key) L = &l;
        if (!L) {
            b->lanes.emplace_back();
            L = &b->lanes.back();
            L->lt = p->lt;
            L->nx_key = key;
        }
        L->members.push_back(i);
        L->lx_max = std::max(L->lx_max, p->lx);
        RenderGroup* R = nullptr;
        for (auto& r : b->rgroups)
            if (r.lx == p->lx && r.lt == p->lt) R = &r;
        if (!R) {
            b->rgroups.emplace_back();
            R = &b->rgroups.back();
            R->lx = p->lx;
            R->lt = p->lt;
        }
        R->members.push_back(i);
        R->max_runs = std::max(R->max_runs, std::max(1, p->max_runs));
    }
    for (auto& L : b->lanes)
        for (int m : L.members) {
            const plan_s* a = b->plans[m];
            const plan_s* z = b->plans[L.members[0]];
            if (a->lx != z->lx) L.uniform = false;
            for (int k = 0; k < 6; k++)
                if (a->g.ctm[k] != z->g.ctm[k]) L.same_costs = false;
        }
    const int rc = batch_init(b);
    if (rc != PLAN_OK) {
        release(b);
        delete b;
        return rc;
    }
    *out = b;
    return PLAN_OK;
}

int plan_batch_run(plan_batch_t* b, const plan_query* queries, int render) {
    if (!b || !queries) return PLAN_EINVAL;
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; i++) {
        const plan_s* p = b->plans[i];
        const plan_query& q = queries[i];
        if (q.n_cycles < 1 || q.n_cycles > 4096 || !pose_ok(p, q.start) || !pose_ok(p, q.goal)) return PLAN_EINVAL;
        if (pose_hard(p, q.start)) return PLAN_EINVAL;
        if (range_check(p, q.n_cycles) != PLAN_OK) return PLAN_ERANGE;
        if (!render && !p->rendered) return PLAN_ESTATE;
    }
    // the previous run may still read the staging buffer
    if (b->in_flight) NHP_CK(cudaEventSynchronize(b->done));
    b->in_flight = false;
    // the batch's stream follows the caller's stream and the plans' streams
    NHP_CK(cudaEventRecord(b->enter, b->user_stream));
    NHP_CK(cudaStreamWaitEvent(b->stream, b->enter, 0));
    for (auto st : b->plan_streams) {
        if (st == b->user_stream) continue;
        NHP_CK(cudaEventRecord(b->enter, st));
        NHP_CK(cudaStreamWaitEvent(b->stream, b->enter, 0));
    }
    b->q.assign(queries, queries + n);
    std::vector<int> key;
    key.reserve(n + 1);
    for (int i = 0; i < n; i++) key.push_back(queries[i].n_cycles);
    key.push_back(render ? 1 : 0);
    // launch parameters a captured graph holds: transition costs, direction fields
    for (const plan_s* p : b->plans) {
        for (int k = 0; k < 6; k++) key.push_back((int)p->g.ctm[k]);
        key.push_back(p->d_dir ? 1 : 0);
        key.push_back(p->dir_tol);
        key.push_back((int)p->dir_pen);
        key.push_back((int)((uintptr_t)p->d_dir & 0x7FFFFFFF));
    }
    const bool use_graph = !(b->flags & PLAN_BATCH_NO_GRAPH);
    int rc = PLAN_OK;
    if (key != b->key || !use_graph) {
        drop_graph(b);
        rc = build_layout(b);
        if (rc != PLAN_OK) return rc;
    }
    fill_stage(b);
    if (!b->tuned) {
        // first run: upload, render if asked, then tune every lane in place
        cudaStream_t s = b->stream;
        NHP_CK(cudaMemcpyAsync(b->d_stage, b->h_stage, b->stage_bytes, cudaMemcpyHostToDevice, s));
        int64_t dummy = 0;
        if (render && (rc = enqueue_render(b, s, &dummy)) != PLAN_OK) return rc;
        for (auto& L : b->lanes)
            if ((rc = tune_lane(b, L)) != PLAN_OK) return rc;
        NHP_CK(cudaStreamSynchronize(s));
        b->tuned = true;
    }
    int64_t nl = 0;
    if (use_graph) {
        if (!b->exec) {
            cudaGraph_t g = nullptr;
            NHP_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_run(b, render != 0, &nl);
            const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (rc != PLAN_OK || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return rc != PLAN_OK ? rc : cuda_fail(ce, "cudaStreamEndCapture");
            }
            b->graph = g;
            if (const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0); ie != cudaSuccess) {
                drop_graph(b);
                return cuda_fail(ie, "cudaGraphInstantiate");
            }
            b->key = key;
            b->launches_per_run = nl;
        }
        NHP_CK(cudaGraphLaunch(b->exec, b->stream));
        b->launches += b->launches_per_run;
    } else {
        rc = enqueue_run(b, render != 0, &nl);
        if (rc != PLAN_OK) return rc;
        b->launches_per_run = nl;
        b->launches += nl;
    }
    if (render)
        for (auto* p : b->plans) p->rendered = true;
    for (auto* p : b->plans) p->vol_kind = VOL_PLAIN;
    NHP_CK(cudaEventRecord(b->done, b->stream));
    b->in_flight = true;
    // later work on the caller's and the plans' streams sees the results
    NHP_CK(cudaStreamWaitEvent(b->user_stream, b->done, 0));
    for (auto st : b->plan_streams)
        if (st != b->user_stream) NHP_CK(cudaStreamWaitEvent(st, b->done, 0));
    return PLAN_OK;
}

int plan_batch_sync(plan_batch_t* b) {
    if (!b) return PLAN_EINVAL;
    if (b->in_flight) NHP_CK(cudaEventSynchronize(b->done));
    return PLAN_OK;
}

int plan_batch_result(plan_batch_t* b, int i, plan_segment* out, int cap, int* n_out, uint32_t* cost) {
    if (!b || !n_out || !cost || cap < 0 || (cap > 0 && !out) || i < 0 || i >= (int)b->plans.size())
        return PLAN_EINVAL;
    *n_out = 0;
    *cost = PLAN_INF;
    if (b->q.empty()) return PLAN_ESTATE;
    int rc = plan_batch_sync(b);
    if (rc != PLAN_OK) return rc;
    const int32_t* st = (const int32_t*)(b->h_res + (size_t)i * 16);
    if (st[0] == -1) return PLAN_EUNREACHABLE;
    if (st[0] < 0) return PLAN_EINTERNAL;
    *cost = (uint32_t)(st[1] & 0xFFFF) | ((uint32_t)st[2] << 16);
    *n_out = st[0];
    if (st[0] > b->seg_cap[i]) return PLAN_EINTERNAL;  // more segments than maneuver layers
    if (st[0] > cap) return PLAN_ERANGE;
    const plan_segment* seg = (const plan_segment*)(b->h_res + b->seg_base[i]);
    for (int k = 0; k < st[0]; k++) out[k] = seg[st[0] - 1 - k];  // the walk runs goal -> start
    return PLAN_OK;
}

int plan_batch_lanes(plan_batch_t* b, int* n_lanes) {
    if (!b || !n_lanes) return PLAN_EINVAL;
    *n_lanes = (int)b->lanes.size();
    return PLAN_OK;
}

int plan_batch_lane(plan_batch_t* b, int lane, plan_batch_lane_info* out) {
    if (!b || !out || lane < 0 || lane >= (int)b->lanes.size()) return PLAN_EINVAL;
    if (!b->tuned) return PLAN_ESTATE;
    *out = b->lanes[lane].info;
    return PLAN_OK;
}

int plan_batch_kernel_launches(plan_batch_t* b, int64_t* per_run, int64_t* total) {
    if (!b) return PLAN_EINVAL;
    if (per_run) *per_run = b->launches_per_run;
    if (total) *total = b->launches;
    return PLAN_OK;
}

int plan_batch_destroy(plan_batch_t* b) {
    if (!b) return PLAN_EINVAL;
    if (b->in_flight) cudaEventSynchronize(b->done);
    release(b);
    delete b;
    return PLAN_OK;
}

}  // extern "C"

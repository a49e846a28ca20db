// server.cu -- a planning server: cached scenes, HBM-budget admission and
// continuous batching of the sweep passes.
//
// Scenes (occupancy image + vehicle + costs) are rendered once into their
// obstacle volumes and stay on the device.  A request names a scene, a start
// and goal pose and N; it needs its own value and label volumes (6 bytes per
// pose cell), carved from one device arena whose size is the server's memory
// budget (the scenes are carved from it too).  A native scheduler thread runs
// the GPU in steps: each step initialises newly admitted requests, advances
// every other request by one sweep pass -- one launch per lane (same
// N_theta, compatible Nx) and pass kind, each request at its own pass of the
// cycle schedule -- and walks the labels of the requests whose last pass ran
// in this step, writing their plans straight into mapped host memory.
// Requests that arrive while others are on the GPU join at the next step as
// soon as the arena has room for their volumes, so their work overlaps on
// the device.  Every request runs exactly the kernels and passes it would run
// alone, so its result does not depend on what else is in flight.
//
// For comparison the server also has a one-at-a-time mode: requests are
// taken in arrival order and each is planned with the single-plan launch
// sequence (init, 4N + 1 passes, label walk, synchronise) before the next
// starts.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan_state.h"

using namespace nhp;

namespace {

constexpr int kDepth = 2;            // steps queued on the GPU ahead of the host
constexpr int kSlots = kDepth + 1;   // descriptor / result slots in rotation
constexpr size_t kAlign = 256;
// Default descriptor (arena) and result (mapped host) bytes of every slot,
// reserved at creation: room for about 140 requests in one step.
constexpr size_t kDescMin = (size_t)64 << 10;
constexpr size_t kResMin = (size_t)64 << 10;
constexpr int kMaxScenes = 4096;
constexpr int kTracks = 3;           // 0: big, 1: heavy, 2: light requests
constexpr int kLight = kTracks - 1;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit suballocator over one device block, with coalescing.
class Arena {
  public:
    void init(unsigned char* base, size_t bytes) {
        base_ = base;
        size_ = bytes;
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    unsigned char* alloc(size_t bytes) {
        std::lock_guard<std::mutex> lk(mu_);
        bytes = align_up(std::max<size_t>(bytes, 1), kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            live_[off] = bytes;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return base_ + off;
        }
        return nullptr;
    }
    void release(void* p) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        const size_t off = (size_t)((unsigned char*)p - base_);
        auto lv = live_.find(off);
        if (lv == live_.end()) return;
        size_t o = off, n = lv->second;
        live_.erase(lv);
        used_ -= n;
        auto nx = free_.lower_bound(o);
        if (nx != free_.end() && nx->first == o + n) {
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == o) {
                o = pv->first;
                n += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = n;
    }
    size_t used() {
        std::lock_guard<std::mutex> lk(mu_);
        return used_;
    }
    size_t peak() {
        std::lock_guard<std::mutex> lk(mu_);
        return peak_;
    }
    size_t size() const { return size_; }

  private:
    std::mutex mu_;
    unsigned char* base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
    std::unordered_map<size_t, size_t> live_;
};

void* arena_alloc(size_t bytes, void*, void* ctx) { return ((Arena*)ctx)->alloc(bytes); }
void arena_free(void* p, size_t, void*, void* ctx) { ((Arena*)ctx)->release(p); }

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    int scene = 0;
    plan_pose start{}, goal{};
    int n_cycles = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int pass = -1;            // next pass; -1 = not initialised yet
    unsigned char* mem = nullptr;
    size_t mem_bytes = 0;
    bool finishing = false;   // its label walk is on the GPU
    bool done = false;
    int status = PLAN_OK;
    uint32_t cost = PLAN_INF;
    std::vector<plan_segment> segs;
    int res_off = 0;          // offset of its result in the step's result area
    int track = kLight;
    std::atomic<bool> cancel{false};  // set by plan_server_cancel
};
using ReqPtr = std::shared_ptr<Request>;

struct Slot {
    unsigned char* h_desc = nullptr;  // pinned staging
    unsigned char* d_desc = nullptr;  // device copy
    size_t desc_cap = 0;
    unsigned char* h_res = nullptr;   // mapped pinned: written by the label walk
    unsigned char* d_res = nullptr;   // its device address
    size_t res_cap = 0;
};

struct Step {
    cudaEvent_t ev = nullptr;
    int slot = 0;
    std::vector<ReqPtr> finishing;
    // requests taken out of the schedule in this step (cancelled, or whose
    // step could not get descriptor space): their memory is released and
    // their status set once the work queued before them has finished
    std::vector<std::pair<ReqPtr, int>> dropped;
};

// A sequence of steps on its own stream.  Requests are classed by size:
// big (at least big_cells pose cells, track 0), heavy (at least heavy_cells,
// track 1) and light (track 2).  Within the big and the heavy class at most
// max_heavy requests run at once, in arrival order; light requests are not
// limited.  Each track advances at its own pace on a stream of its own, light
// kernels at the highest stream priority and big ones at the lowest, so a
// request is slowed only by the work of its own and of smaller classes.
struct Track {
    cudaStream_t stream = nullptr;
    std::vector<ReqPtr> active;  // admitted, not finished
    std::deque<Step> steps;      // on the GPU
    Slot slots[kSlots];
    uint64_t step_count = 0;
    bool has_work() const {
        for (auto& r : active)
            if (!r->finishing) return true;
        return false;
    }
};

// One launch of a step: requests of one lane and pass kind.
struct LaunchSet {
    int lt = 0, nx_key = 0;
    bool turn = false;
    std::vector<ReqPtr> reqs;
};

}  // namespace

struct plan_server_s {
    plan_server_config cfg{};
    plan_allocator alloc{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    unsigned char* arena_base = nullptr;
    Arena arena;
    std::mutex mu;                    // guards everything below
    std::condition_variable cv_in, cv_done;
    // scenes: slots are written once (under mu) before their index is handed
    // out, so the scheduler reads them without locking
    plan_s* scenes[kMaxScenes] = {};
    int n_scenes = 0;
    std::deque<ReqPtr> incoming;      // submitted, not yet seen by the scheduler
    std::unordered_map<uint64_t, ReqPtr> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = PLAN_OK;
    plan_server_stats stats{};
    // scheduler-thread state
    std::deque<ReqPtr> pending;       // arrival order, waiting for memory / a slot
    Track tracks[kTracks];
    std::vector<cudaEvent_t> spare_events;
    std::thread worker;

    bool conv() const { return (cfg.flags & PLAN_SERVE_STOP_AT_CONVERGENCE) != 0; }
    int inflight() const {
        int n = 0;
        for (auto& t : tracks) n += (int)t.active.size();
        return n;
    }
    bool busy() const {
        for (auto& t : tracks)
            if (!t.active.empty() || !t.steps.empty()) return true;
        return false;
    }
};

namespace {

// A request's arena block: V, L and (with PLAN_SERVE_STOP_AT_CONVERGENCE)
// one convergence word per pass.
size_t l_offset(const plan_s* sc) { return align_up((size_t)sc->nr * 4, kAlign); }
size_t conv_offset(const plan_s* sc) { return align_up(l_offset(sc) + (size_t)sc->nr * 2, kAlign); }
size_t request_bytes(const plan_s* sc, int n_cycles, bool conv) {
    return conv ? conv_offset(sc) + 4 * ((size_t)4 * n_cycles + 1) : l_offset(sc) + (size_t)sc->nr * 2;
}

int lane_nx_key(int nx) { return nx >= 256 ? 256 : nx; }

QueryDesc request_desc(const plan_s* sc, const Request& r, bool conv) {
    QueryDesc d = sc->qd;
    d.v.V = (uint32_t*)r.mem;
    d.v.L = (uint16_t*)(r.mem + l_offset(sc));
    d.conv = conv ? (uint32_t*)(r.mem + conv_offset(sc)) : nullptr;
    d.v.improved = nullptr;
    d.start = cell_index(sc, r.start);
    d.goal = cell_index(sc, r.goal);
    d.n_cycles = r.n_cycles;
    d.pass = r.pass;
    d.seg = nullptr;
    d.status = nullptr;
    d.seg_cap = 0;
    return d;
}

size_t result_bytes(const Request& r) { return 16 + sizeof(plan_segment) * 6 * (size_t)r.n_cycles; }

void free_slot(Slot& s, plan_server_s* v) {
    if (s.h_desc) cudaFreeHost(s.h_desc);
    if (s.h_res) cudaFreeHost(s.h_res);
    v->arena.release(s.d_desc);
    s = Slot{};
}

// Fresh buffers for one slot; false (and nothing held) when any allocation fails.
bool alloc_slot(plan_server_s* v, Slot& s, size_t desc, size_t res) {
    s = Slot{};
    s.d_desc = v->arena.alloc(desc);
    bool ok = s.d_desc != nullptr;
    ok = ok && cudaHostAlloc((void**)&s.h_desc, desc, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaHostAlloc((void**)&s.h_res, res, cudaHostAllocMapped) == cudaSuccess;
    ok = ok && cudaHostGetDevicePointer((void**)&s.d_res, s.h_res, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();  // a failed host allocation is not a sticky error
        free_slot(s, v);
        return false;
    }
    s.desc_cap = desc;
    s.res_cap = res;
    return true;
}

void retire(plan_server_s* v, Track& tr, Step& st);

// Grow every slot of the track to hold `desc` descriptor and `res` result
// bytes.  The new buffers are taken before the old ones are given back, so a
// failed growth changes nothing and returns false; the track's steps in
// flight (which use the old buffers) are waited for only once the new ones
// exist.  A CUDA error while waiting is returned through *rc.
bool grow_slots(plan_server_s* v, Track& tr, size_t desc, size_t res, int* rc) {
    desc = align_up(desc, 4096);
    res = align_up(res, 4096);
    Slot fresh[kSlots];
    for (int i = 0; i < kSlots; i++) {
        if (!alloc_slot(v, fresh[i], std::max(desc, tr.slots[i].desc_cap), std::max(res, tr.slots[i].res_cap))) {
            for (int j = 0; j < i; j++) free_slot(fresh[j], v);
            return false;
        }
    }
    if (cudaStreamSynchronize(tr.stream) != cudaSuccess) {
        for (auto& f : fresh) free_slot(f, v);
        *rc = cuda_fail(cudaGetLastError(), "server track synchronise");
        return false;
    }
    while (!tr.steps.empty()) {
        retire(v, tr, tr.steps.front());
        tr.steps.pop_front();
    }
    for (int i = 0; i < kSlots; i++) {
        free_slot(tr.slots[i], v);
        tr.slots[i] = fresh[i];
    }
    return true;
}

cudaEvent_t take_event(plan_server_s* v) {
    if (!v->spare_events.empty()) {
        cudaEvent_t e = v->spare_events.back();
        v->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// Store the results of a finished step and free the requests' volumes.
void retire(plan_server_s* v, Track& tr, Step& st) {
    const double t = now_s();
    Slot& sl = tr.slots[st.slot];
    std::lock_guard<std::mutex> lk(v->mu);
    for (auto& r : st.finishing) {
        const int32_t* h = (const int32_t*)(sl.h_res + r->res_off);
        const plan_segment* seg = (const plan_segment*)(sl.h_res + r->res_off + 16);
        if (h[0] == -1) {
            r->status = PLAN_EUNREACHABLE;
        } else if (h[0] < 0 || h[0] > 6 * r->n_cycles) {
            r->status = PLAN_EINTERNAL;
        } else {
            r->status = PLAN_OK;
            r->cost = (uint32_t)(h[1] & 0xFFFF) | ((uint32_t)h[2] << 16);
            r->segs.resize(h[0]);
            for (int k = 0; k < h[0]; k++) r->segs[k] = seg[h[0] - 1 - k];  // walk runs goal -> start
        }
        v->arena.release(r->mem);
        r->mem = nullptr;
        r->t_done = t;
        r->done = true;
        v->stats.completed++;
    }
    for (auto& d : st.dropped) {
        const ReqPtr& r = d.first;
        v->arena.release(r->mem);
        r->mem = nullptr;
        r->status = d.second;
        r->t_done = t;
        r->done = true;
        if (d.second == PLAN_ECANCELED) v->stats.cancelled++;
        else v->stats.rejected++;
    }
    v->spare_events.push_back(st.ev);
    v->cv_done.notify_all();
}

// End a request that holds no memory and has nothing on the GPU.
void finish_now(plan_server_s* v, const ReqPtr& r, int status) {
    std::lock_guard<std::mutex> lk(v->mu);
    r->status = status;
    r->done = true;
    r->t_done = now_s();
    if (status == PLAN_ECANCELED) v->stats.cancelled++;
    else v->stats.rejected++;
    v->cv_done.notify_all();
}

void fail_all(plan_server_s* v, int code) {
    std::lock_guard<std::mutex> lk(v->mu);
    v->fatal = code;
    auto fin = [&](ReqPtr& r) {
        if (r->done) return;
        r->status = code;
        r->done = true;
        r->t_done = now_s();
    };
    for (auto& r : v->pending) fin(r);
    for (auto& r : v->incoming) fin(r);
    for (auto& tr : v->tracks) {
        for (auto& r : tr.active) fin(r);
        for (auto& st : tr.steps)
            for (auto& r : st.finishing) fin(r);
    }
    v->cv_done.notify_all();
}

// Track of a request: 0 big, 1 heavy, kLight light.
int track_of(const plan_server_s* v, const plan_s* sc) {
    if (v->cfg.big_cells > 0 && sc->nr >= v->cfg.big_cells) return 0;
    if (v->cfg.heavy_cells > 0 && sc->nr >= v->cfg.heavy_cells) return 1;
    return kLight;
}

// Admit pending requests in arrival order while memory and slots allow.  A
// big or heavy request waiting for a slot of its class lets later requests
// of other classes pass; a request waiting for memory stops admission (no
// overtaking for memory, so large requests cannot starve).
void admit(plan_server_s* v) {
    int running[kTracks];
    for (int k = 0; k < kTracks; k++) running[k] = (int)v->tracks[k].active.size();
    for (auto it = v->pending.begin(); it != v->pending.end();) {
        ReqPtr r = *it;
        if (r->cancel.load()) {
            it = v->pending.erase(it);
            finish_now(v, r, PLAN_ECANCELED);
            continue;
        }
        if (v->cfg.max_inflight > 0 && v->inflight() >= v->cfg.max_inflight) break;
        const plan_s* sc = v->scenes[r->scene];
        const int k = track_of(v, sc);
        if (k != kLight && v->cfg.max_heavy > 0 && running[k] >= v->cfg.max_heavy) {
            ++it;
            continue;
        }
        r->mem_bytes = request_bytes(sc, r->n_cycles, v->conv());
        r->mem = v->arena.alloc(r->mem_bytes);
        if (!r->mem) break;
        r->t_admit = now_s();
        r->pass = -1;
        r->track = k;
        running[k]++;
        it = v->pending.erase(it);
        v->tracks[k].active.push_back(r);
        std::lock_guard<std::mutex> lk(v->mu);
        v->stats.admitted++;
        v->stats.peak_inflight = std::max<int64_t>(v->stats.peak_inflight, (int64_t)v->inflight());
    }
}

// Descriptor layout of one step for the first n requests of `reqs` (none
// of them finishing): requests not yet initialised get init and pass 0,
// every request one pass (one launch per lane and pass kind), and requests
// whose last pass this is a label walk.
struct StepPlan {
    std::vector<ReqPtr> init, fin;
    std::vector<LaunchSet> sets;
    std::vector<size_t> o_set, o_items;
    size_t o_init = 0, o_fin = 0, desc = 0, res = 0;
};

StepPlan plan_step(const plan_server_s* v, const std::vector<ReqPtr>& reqs, size_t n) {
    StepPlan P;
    for (size_t i = 0; i < n; i++) {
        const ReqPtr& r = reqs[i];
        if (r->pass < 0) P.init.push_back(r);
        const int pass = r->pass < 0 ? 0 : r->pass;
        const plan_s* sc = v->scenes[r->scene];
        const bool turn = pass_is_turn(pass);
        const int key = lane_nx_key(sc->nx);
        LaunchSet* ls = nullptr;
        for (auto& st : P.sets)
            if (st.lt == sc->lt && st.nx_key == key && st.turn == turn) ls = &st;
        if (!ls) {
            P.sets.emplace_back();
            ls = &P.sets.back();
            ls->lt = sc->lt;
            ls->nx_key = key;
            ls->turn = turn;
        }
        ls->reqs.push_back(r);
        if (pass + 1 == pass_count(r->n_cycles)) P.fin.push_back(r);
    }
    size_t off = 0;
    P.o_init = off;
    off = align_up(off + sizeof(QueryDesc) * P.init.size(), kAlign);
    P.o_set.resize(P.sets.size());
    P.o_items.resize(P.sets.size());
    for (size_t k = 0; k < P.sets.size(); k++) {
        P.o_set[k] = off;
        off = align_up(off + sizeof(QueryDesc) * P.sets[k].reqs.size(), kAlign);
        P.o_items[k] = off;
        off = align_up(off + sizeof(int32_t) * (P.sets[k].reqs.size() + 1), kAlign);
    }
    P.o_fin = off;
    off = align_up(off + sizeof(QueryDesc) * P.fin.size(), kAlign);
    P.desc = off;
    for (auto& r : P.fin) P.res = align_up(P.res + result_bytes(*r), 16);
    return P;
}

// Build and enqueue one continuous-batching step of a track.
int launch_step(plan_server_s* v, Track& tr) {
    Step st;
    std::vector<ReqPtr> sched;
    for (auto& r : tr.active) {
        if (r->finishing) continue;
        if (r->cancel.load()) {  // no further passes; memory back once its queued work is done
            st.dropped.emplace_back(r, PLAN_ECANCELED);
            r->finishing = true;
            continue;
        }
        sched.push_back(r);
    }
    size_t n = sched.size();
    StepPlan P = plan_step(v, sched, n);
    bool partial = false;
    if (n > 0 && (P.desc > tr.slots[0].desc_cap || P.res > tr.slots[0].res_cap)) {
        int rc = PLAN_OK;
        if (!grow_slots(v, tr, P.desc, P.res, &rc)) {
            if (rc != PLAN_OK) return rc;
            // no room to grow: advance the requests that fit, the rest wait
            while (n > 0 && (P.desc > tr.slots[0].desc_cap || P.res > tr.slots[0].res_cap)) P = plan_step(v, sched, --n);
            partial = true;
            if (n == 0) {  // even the oldest request alone never fits
                st.dropped.emplace_back(sched[0], PLAN_ENOMEM);
                sched[0]->finishing = true;
            }
        }
    }
    if (n == 0 && st.dropped.empty()) return PLAN_OK;
    for (size_t i = 0; i < n; i++)
        if (sched[i]->pass < 0) sched[i]->pass = 0;
    size_t res = 0;
    for (auto& r : P.fin) {
        r->res_off = (int)res;
        res = align_up(res + result_bytes(*r), 16);
    }
    const int si = (int)(tr.step_count % kSlots);
    Slot& sl = tr.slots[si];
    unsigned char* h = sl.h_desc;
    cudaStream_t s = tr.stream;
    const bool conv = v->conv();
    int64_t launches = 0;
    for (size_t k = 0; k < P.init.size(); k++) {
        QueryDesc d = request_desc(v->scenes[P.init[k]->scene], *P.init[k], conv);
        memcpy(h + P.o_init + k * sizeof(QueryDesc), &d, sizeof d);
    }
    std::vector<int64_t> items(P.sets.size(), 0);
    for (size_t k = 0; k < P.sets.size(); k++) {
        int32_t* it = (int32_t*)(h + P.o_items[k]);
        it[0] = 0;
        for (size_t j = 0; j < P.sets[k].reqs.size(); j++) {
            const Request& r = *P.sets[k].reqs[j];
            const plan_s* sc = v->scenes[r.scene];
            QueryDesc d = request_desc(sc, r, conv);
            memcpy(h + P.o_set[k] + j * sizeof(QueryDesc), &d, sizeof d);
            const int64_t ni = P.sets[k].turn ? turn_items(sc->lx)
                                              : (sc->nx >= 256 ? straight_items(sc->lx, sc->lt, 256) : 0);
            it[j + 1] = (int32_t)(it[j] + ni);
        }
        items[k] = it[P.sets[k].reqs.size()];
    }
    for (size_t k = 0; k < P.fin.size(); k++) {
        const Request& r = *P.fin[k];
        QueryDesc d = request_desc(v->scenes[r.scene], r, conv);
        d.status = (int32_t*)(sl.d_res + r.res_off);
        d.seg = (plan_segment*)(sl.d_res + r.res_off + 16);
        d.seg_cap = 6 * r.n_cycles;
        memcpy(h + P.o_fin + k * sizeof(QueryDesc), &d, sizeof d);
    }
    if (P.desc) NHP_CK(cudaMemcpyAsync(sl.d_desc, h, P.desc, cudaMemcpyHostToDevice, s));
    if (!P.init.empty()) {
        Group g{};
        g.d = (const QueryDesc*)(sl.d_desc + P.o_init);
        g.nq = (int)P.init.size();
        for (auto& r : P.init) {
            g.lx = std::max(g.lx, v->scenes[r->scene]->lx);
            g.lt = std::max(g.lt, v->scenes[r->scene]->lt);
        }
        NHP_CK(launch_init(g, s));
        launches++;
    }
    for (size_t k = 0; k < P.sets.size(); k++) {
        const LaunchSet& ls = P.sets[k];
        const plan_s* sc0 = v->scenes[ls.reqs[0]->scene];
        bool uniform = true;
        for (auto& r : ls.reqs) uniform = uniform && v->scenes[r->scene]->lx == sc0->lx;
        Group g{};
        g.d = (const QueryDesc*)(sl.d_desc + P.o_set[k]);
        g.nq = (int)ls.reqs.size();
        g.lx = sc0->lx;
        g.lt = ls.lt;
        g.max_runs = 1;
        if (!uniform) {
            g.item_off = (const int32_t*)(sl.d_desc + P.o_items[k]);
            g.items = items[k];
        }
        // pass -1: every request at its own pass (QueryDesc::pass); with
        // convergence records, converged requests first drop out of it
        if (conv) {
            NHP_CK(launch_conv_gate((QueryDesc*)(sl.d_desc + P.o_set[k]), g.nq, -1, s));
            launches++;
        }
        const int lines = ls.nx_key >= 256 ? 256 : (ls.nx_key >= 128 ? 128 : ls.nx_key);
        NHP_CK(ls.turn ? launch_turn(g, -1, -1, s) : launch_straight(g, -1, lines, s));
        launches++;
    }
    if (!P.fin.empty()) {
        Group g{};
        g.d = (const QueryDesc*)(sl.d_desc + P.o_fin);
        g.nq = (int)P.fin.size();
        NHP_CK(launch_extract(g, s));
        launches++;
    }
    st.ev = take_event(v);
    st.slot = si;
    st.finishing = P.fin;
    if (!st.ev) return PLAN_ECUDA;
    NHP_CK(cudaEventRecord(st.ev, s));
    tr.steps.push_back(std::move(st));
    tr.step_count++;
    for (size_t i = 0; i < n; i++) {
        Request& r = *sched[i];
        r.pass++;
        if (r.pass == pass_count(r.n_cycles)) r.finishing = true;
    }
    tr.active.erase(std::remove_if(tr.active.begin(), tr.active.end(), [](const ReqPtr& r) { return r->finishing; }),
                    tr.active.end());
    std::lock_guard<std::mutex> lk(v->mu);
    v->stats.steps++;
    v->stats.launches += launches;
    if (partial) v->stats.partial_steps++;
    return PLAN_OK;
}

// One-at-a-time: the single-plan launch sequence for the oldest request.
int run_one(plan_server_s* v) {
    ReqPtr r = v->pending.front();
    v->pending.pop_front();
    if (r->cancel.load()) {
        finish_now(v, r, PLAN_ECANCELED);
        return PLAN_OK;
    }
    const plan_s* sc = v->scenes[r->scene];
    const bool conv = v->conv();
    r->mem_bytes = request_bytes(sc, r->n_cycles, conv);
    r->mem = v->arena.alloc(r->mem_bytes);
    if (!r->mem) {  // nothing else holds memory: the request can never fit
        finish_now(v, r, PLAN_ENOMEM);
        return PLAN_OK;
    }
    r->t_admit = now_s();
    Track& tr = v->tracks[kLight];
    if (sizeof(QueryDesc) > tr.slots[0].desc_cap || result_bytes(*r) > tr.slots[0].res_cap) {
        int rc = PLAN_OK;
        if (!grow_slots(v, tr, sizeof(QueryDesc), result_bytes(*r), &rc)) {
            v->arena.release(r->mem);
            r->mem = nullptr;
            if (rc != PLAN_OK) return rc;
            finish_now(v, r, PLAN_ENOMEM);
            return PLAN_OK;
        }
    }
    Slot& sl = tr.slots[0];
    cudaStream_t s = tr.stream;
    QueryDesc d = request_desc(sc, *r, conv);
    d.pass = -1;
    d.status = (int32_t*)sl.d_res;
    d.seg = (plan_segment*)(sl.d_res + 16);
    d.seg_cap = 6 * r->n_cycles;
    memcpy(sl.h_desc, &d, sizeof d);
    NHP_CK(cudaMemcpyAsync(sl.d_desc, sl.h_desc, sizeof d, cudaMemcpyHostToDevice, s));
    Group g{};
    g.d = (const QueryDesc*)sl.d_desc;
    g.nq = 1;
    g.lx = sc->lx;
    g.lt = sc->lt;
    g.max_runs = 1;
    g.ctm = sc->g.ctm;
    int64_t launches = 0;
    NHP_CK(launch_init(g, s));
    launches++;
    const int np = pass_count(r->n_cycles);
    for (int p = 0; p < np; p++) {
        // with convergence records the descriptor carries the pass, -1 once converged
        const int pl = conv ? -1 : p;
        if (conv) {
            NHP_CK(launch_conv_gate((QueryDesc*)sl.d_desc, 1, p, s));
            launches++;
        }
        NHP_CK(pass_is_turn(p) ? launch_turn(g, pl, -1, s) : launch_straight(g, pl, 0, s));
        launches++;
    }
    NHP_CK(launch_extract(g, s));
    launches++;
    NHP_CK(cudaStreamSynchronize(s));
    Step st;
    st.slot = 0;
    st.ev = take_event(v);
    r->res_off = 0;
    st.finishing.push_back(r);
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stats.admitted++;
        v->stats.steps++;
        v->stats.launches += launches;
        v->stats.peak_inflight = std::max<int64_t>(v->stats.peak_inflight, 1);
    }
    retire(v, tr, st);
    return PLAN_OK;
}

// Retire the finished steps at the front of every track; true if any.
bool retire_done(plan_server_s* v) {
    bool any = false;
    for (auto& tr : v->tracks)
        while (!tr.steps.empty() && cudaEventQuery(tr.steps.front().ev) == cudaSuccess) {
            retire(v, tr, tr.steps.front());
            tr.steps.pop_front();
            any = true;
        }
    return any;
}

void worker_main(plan_server_s* v) {
    if (cudaSetDevice(v->device) != cudaSuccess) {
        fail_all(v, cuda_fail(cudaGetLastError(), "server thread: cudaSetDevice"));
        return;
    }
    const bool serial = v->cfg.mode == PLAN_SERVE_ONE_AT_A_TIME;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(v->mu);
            while (!v->incoming.empty()) {
                v->pending.push_back(v->incoming.front());
                v->incoming.pop_front();
            }
            const bool idle = v->pending.empty() && !v->busy();
            if (idle && v->stop) return;
            if (idle) {
                v->cv_in.wait(lk, [&] { return v->stop || !v->incoming.empty(); });
                continue;
            }
        }
        int rc = PLAN_OK;
        if (serial) {
            if (!v->pending.empty()) rc = run_one(v);
        } else {
            // retire what the GPU finished, admit, then keep each track
            // kDepth steps ahead
            retire_done(v);
            admit(v);
            bool launched = false;
            for (auto& tr : v->tracks) {
                if (rc == PLAN_OK && tr.has_work() && (int)tr.steps.size() < kDepth) {
                    rc = launch_step(v, tr);
                    launched = true;
                }
            }
            bool on_gpu = false;
            for (auto& tr : v->tracks) on_gpu = on_gpu || !tr.steps.empty();
            if (rc == PLAN_OK && !launched && on_gpu) {
                // poll (a step takes microseconds to milliseconds); new
                // requests are picked up between polls
                if (!retire_done(v)) std::this_thread::yield();
            } else if (rc == PLAN_OK && !launched && !on_gpu && !v->pending.empty() && !v->busy()) {
                // nothing on the GPU and the head request still does not fit
                ReqPtr r = v->pending.front();
                v->pending.pop_front();
                finish_now(v, r, r->cancel.load() ? PLAN_ECANCELED : PLAN_ENOMEM);
            }
        }
        if (rc != PLAN_OK) {
            fail_all(v, rc);
            return;
        }
    }
}

void server_release(plan_server_s* v) {
    if (v->stream) cudaStreamSynchronize(v->stream);
    for (auto& tr : v->tracks)
        if (tr.stream) cudaStreamSynchronize(tr.stream);
    for (int i = 0; i < v->n_scenes; i++) plan_destroy(v->scenes[i]);  // arena blocks
    v->n_scenes = 0;
    for (auto& tr : v->tracks) {
        for (auto& s : tr.slots) free_slot(s, v);
        for (auto& st : tr.steps)
            if (st.ev) cudaEventDestroy(st.ev);
        if (tr.stream) cudaStreamDestroy(tr.stream);
        tr.stream = nullptr;
    }
    for (auto e : v->spare_events) cudaEventDestroy(e);
    if (v->arena_base) v->alloc.free(v->arena_base, v->arena.size(), (void*)v->stream, v->alloc.ctx);
    if (v->stream) cudaStreamDestroy(v->stream);
}

void* server_default_alloc(size_t bytes, void*, void*) {
    void* p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
void server_default_free(void* p, size_t, void*, void*) { cudaFree(p); }

}  // namespace

extern "C" {

int plan_server_create(const plan_server_config* cfg, const plan_allocator* allocator, void* cuda_stream,
                       plan_server_t** out) {
    if (!out) return PLAN_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->budget_bytes < ((size_t)1 << 20) || cfg->max_inflight < 0 || cfg->max_heavy < 0 ||
        cfg->heavy_cells < 0 || cfg->big_cells < 0 || (cfg->flags & ~PLAN_SERVE_STOP_AT_CONVERGENCE) != 0 ||
        (cfg->slot_bytes != 0 && (cfg->slot_bytes < 4096 || cfg->slot_bytes > ((int64_t)1 << 30))) ||
        (cfg->mode != PLAN_SERVE_CONTINUOUS && cfg->mode != PLAN_SERVE_ONE_AT_A_TIME))
        return PLAN_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free)) return PLAN_EINVAL;
    plan_server_s* v = new (std::nothrow) plan_server_s();
    if (!v) return PLAN_ENOMEM;
    v->cfg = *cfg;
    v->alloc = allocator ? *allocator : plan_allocator{server_default_alloc, server_default_free, nullptr};
    v->user_stream = (cudaStream_t)cuda_stream;
    int rc = PLAN_OK;
    if (cudaGetDevice(&v->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "server stream");
    // light requests' kernels take precedence: the block scheduler then
    // starts their blocks ahead of a heavy pass's waiting blocks
    int prio_low = 0, prio_high = 0;
    if (rc == PLAN_OK && cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "stream priorities");
    for (int k = 0; k < kTracks && rc == PLAN_OK; k++) {
        // priorities: numerically lower is higher; spread big .. light over the range
        const int prio = prio_low + (prio_high - prio_low) * k / (kTracks - 1);
        if (cudaStreamCreateWithPriority(&v->tracks[k].stream, cudaStreamNonBlocking, prio) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "server track stream");
    }
    if (rc == PLAN_OK) {
        v->arena_base = (unsigned char*)v->alloc.alloc(cfg->budget_bytes, (void*)v->stream, v->alloc.ctx);
        if (!v->arena_base) rc = PLAN_ENOMEM;
        else v->arena.init(v->arena_base, cfg->budget_bytes);
    }
    // every track's launch descriptors, before any scene or request
    for (int k = 0; k < kTracks && rc == PLAN_OK; k++)
        for (auto& sl : v->tracks[k].slots)
            if (rc == PLAN_OK && !alloc_slot(v, sl, cfg->slot_bytes ? (size_t)cfg->slot_bytes : kDescMin, kResMin))
                rc = PLAN_ENOMEM;
    if (rc == PLAN_OK) v->stats.reserved_bytes = (int64_t)v->arena.used();
    if (rc == PLAN_OK && v->user_stream) {
        // the arena may still be in use by the caller's stream's earlier work
        if (cudaStreamSynchronize(v->user_stream) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "caller stream");
    }
    if (rc != PLAN_OK) {
        server_release(v);
        delete v;
        return rc;
    }
    v->worker = std::thread(worker_main, v);
    *out = v;
    return PLAN_OK;
}

int plan_server_add_scene(plan_server_t* v, const plan_grid* grid, const plan_footprint* footprint,
                          double turn_radius_cells, const plan_costs* costs, int32_t* scene_id) {
    if (!v || !scene_id) return PLAN_EINVAL;
    *scene_id = -1;
    cudaStream_t s = nullptr;
    NHP_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const plan_allocator al{arena_alloc, arena_free, &v->arena};
    plan_s* p = nullptr;
    int rc = create_plan(grid, footprint, turn_radius_cells, costs, &al, (void*)s, false, &p);
    if (rc == PLAN_OK) {
        p->stream = s;
        rc = plan_render_cspace(p);
        if (rc == PLAN_OK) rc = cuda_rc(cudaStreamSynchronize(s));
    }
    if (p) p->stream = v->stream;  // nothing else runs on the scene's own stream
    cudaStreamDestroy(s);
    if (rc != PLAN_OK) {
        if (p) plan_destroy(p);
        return rc;
    }
    std::lock_guard<std::mutex> lk(v->mu);
    if (v->n_scenes >= kMaxScenes) {
        plan_destroy(p);
        return PLAN_ERANGE;
    }
    v->scenes[v->n_scenes] = p;
    *scene_id = (int32_t)v->n_scenes++;
    v->stats.scenes = v->n_scenes;
    v->stats.scene_bytes = (int64_t)v->arena.used() - v->stats.reserved_bytes;
    return PLAN_OK;
}

int plan_server_submit(plan_server_t* v, int32_t scene_id, plan_pose start, plan_pose goal, int32_t n_cycles,
                       uint64_t* ticket) {
    if (!v || !ticket) return PLAN_EINVAL;
    *ticket = 0;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(v->mu);
    if (v->fatal != PLAN_OK) return v->fatal;
    if (v->stop) return PLAN_ESTATE;
    if (scene_id < 0 || scene_id >= v->n_scenes) return PLAN_EINVAL;
    const plan_s* sc = v->scenes[scene_id];
    int rc = check_sweep(sc, start, n_cycles);
    if (rc != PLAN_OK) return rc;
    if (!pose_ok(sc, goal)) return PLAN_EINVAL;
    // scenes stay for the server's lifetime: the rest is all a request can get
    const size_t held = (size_t)(v->stats.scene_bytes + v->stats.reserved_bytes);
    if (request_bytes(sc, n_cycles, v->conv()) > v->arena.size() - held) return PLAN_ENOMEM;
    auto r = std::make_shared<Request>();
    r->ticket = v->next_ticket++;
    r->scene = scene_id;
    r->start = start;
    r->goal = goal;
    r->n_cycles = n_cycles;
    r->t_submit = t;
    v->tickets[r->ticket] = r;
    v->incoming.push_back(r);
    v->stats.submitted++;
    *ticket = r->ticket;
    v->cv_in.notify_one();
    return PLAN_OK;
}

int plan_server_wait(plan_server_t* v, uint64_t ticket, double timeout_s, plan_request_info* info,
                     plan_segment* out, int cap, int* n_out) {
    if (!v || !info || cap < 0 || (cap > 0 && !out)) return PLAN_EINVAL;
    std::unique_lock<std::mutex> lk(v->mu);
    auto it = v->tickets.find(ticket);
    if (it == v->tickets.end()) return PLAN_EINVAL;
    ReqPtr r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) v->cv_done.wait(lk, ready);
    else if (!v->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return PLAN_ETIMEOUT;
    v->tickets.erase(it);
    memset(info, 0, sizeof *info);
    info->status = r->status;
    info->cost = r->cost;
    info->n_segments = (int32_t)r->segs.size();
    info->scene = r->scene;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
    if (n_out) *n_out = (int)r->segs.size();
    const int n = std::min(cap, (int)r->segs.size());
    for (int k = 0; k < n; k++) out[k] = r->segs[k];
    return (int)r->segs.size() > cap && r->status == PLAN_OK ? PLAN_ERANGE : PLAN_OK;
}

int plan_server_cancel(plan_server_t* v, uint64_t ticket) {
    if (!v) return PLAN_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->tickets.find(ticket);
    if (it == v->tickets.end()) return PLAN_EINVAL;
    if (!it->second->done) it->second->cancel.store(true);
    v->cv_in.notify_one();
    return PLAN_OK;
}

int plan_server_stats_read(plan_server_t* v, plan_server_stats* out) {
    if (!v || !out) return PLAN_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    *out = v->stats;
    out->arena_bytes = (int64_t)v->arena.size();
    out->peak_bytes = (int64_t)v->arena.peak();
    return PLAN_OK;
}

int plan_server_destroy(plan_server_t* v) {
    if (!v) return PLAN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
        v->cv_in.notify_all();
    }
    if (v->worker.joinable()) v->worker.join();  // finishes every submitted request first
    server_release(v);
    delete v;
    return PLAN_OK;
}

}  // extern "C"

// Serving: a request loop that super-resolves projections as an acquisition produces them
// (Sec. 3.2: each rotation angle's frames are reconstructed while the scan goes on).
//
// Continuous batching.  A worker thread owns a private stream and a pool of slots; a slot is a
// plan (workspace + device-resident SCG state) of one geometry class.  Requests queue in
// arrival order and are admitted into free slots; a slot is created when a request's class has
// none free and the slot's workspace fits the HBM budget (free device memory minus a reserve,
// or an explicit budget).  Every tick runs a few fused-pass launches over the tiles of all live
// slots at once (one SCG iteration each per launch), so requests that arrive while others are on
// the GPU join the next launch; a finished projection is copied out and its slot freed.  Each
// projection keeps its own state and fixed-order reductions: the result is the same alone and in
// the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "misr.h"
#include "misr_internal.h"

using namespace misr;
using namespace misr_host;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// owned copy of a descriptor (its shift and PSF arrays included)
struct DescCopy {
    misr_desc d{};
    std::vector<float> shifts, psf;
    DescCopy() = default;
    // a copy points its descriptor at its own shift and PSF vectors
    DescCopy(const DescCopy &o) : d(o.d), shifts(o.shifts), psf(o.psf) { repoint(); }
    DescCopy &operator=(const DescCopy &o) {
        d = o.d;
        shifts = o.shifts;
        psf = o.psf;
        repoint();
        return *this;
    }
    void repoint() {
        d.shifts = shifts.empty() ? nullptr : shifts.data();
        d.psf = psf.empty() ? nullptr : psf.data();
    }
    void set(const misr_desc &src) {
        d = src;
        shifts.assign(src.shifts, src.shifts + 2 * src.K);
        psf.assign(src.psf, src.psf + src.psf_size * src.psf_size);
        d.shifts = shifts.data();
        d.psf = psf.data();
    }
    bool same_class(const DescCopy &o) const {
        const misr_desc &a = d, &b = o.d;
        return a.lr_h == b.lr_h && a.lr_w == b.lr_w && a.K == b.K && a.factor == b.factor &&
               a.psf_size == b.psf_size && a.lambda == b.lambda && a.btv_alpha == b.btv_alpha &&
               a.btv_w == b.btv_w && a.eps == b.eps && a.iters == b.iters && a.x0_mode == b.x0_mode &&
               a.in_dtype == b.in_dtype && a.flat_field == b.flat_field && a.iterate_dtype == b.iterate_dtype &&
               a.tile_shape == b.tile_shape && a.data_norm == b.data_norm && a.decimation == b.decimation &&
               (a.data_norm != MISR_NORM_L1 || a.data_eps == b.data_eps) &&
               shifts == o.shifts && psf == o.psf;
    }
};

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Request {
    uint64_t ticket = 0;
    DescCopy desc;
    const void *y = nullptr;
    float *x = nullptr;
    ReqState state = RQ_QUEUED;
    misr_status status = MISR_OK;
    bool cancel = false;            // cancelled while running: finish at the end of the tick
    misr_stats stats{};
    double t_submit = 0, t_start = 0, t_end = 0;
    int slot = -1;
};

struct Slot {
    misr_plan_t plan = nullptr;
    DescCopy desc;
    bool busy = false;
    uint64_t ticket = 0;
    int passes = 0;        // fused passes run since admission (counted as their ticks are read)
    int queued = 0;        // SCG passes queued since admission: at the plan's iteration count the
                           // solve ends within them, and the slot gets no more
    int2 *items = nullptr;  // device tile and group lists of this slot alone (for its init pass)
    int n_list = 0;         // tiles in that list (the groups follow)
    PassSegs segs;
    bool fork = true;       // its own stream must wait for the server stream (its admission) first
};

// device bytes of one slot: its plan's workspace (the layout misr_plan_create allocates) plus
// the slot's own tile and group list
size_t plan_bytes_estimate(const misr_desc &d) {
    const size_t H = (size_t)d.factor * d.lr_h, W = (size_t)d.factor * d.lr_w;
    const size_t tiles = ((H + 15) / 16) * ((W + 31) / 32);   // a bound on any shape's tiles
    return plan_bytes(d) + tiles * sizeof(int2) + (1 << 16);
}

}  // namespace

struct misr_server_s {
    misr_server_cfg cfg{};
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::atomic<uint64_t> wakes{0};   // submits and the stop: what an idle worker's poll watches
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    // worker-owned state
    std::vector<Slot> slots;
    size_t slot_bytes = 0;
    cudaStream_t stream = nullptr;
    DevProblem *dprobs = nullptr;   // one record per slot (capacity cfg.max_slots)
    int2 *ditems = nullptr;         // tile list of the live slots, then their group list
    int live_tiles = 0, live_groups = 0;
    PassSegs live_segs;
    unsigned int *work = nullptr;   // the fused pass's tile counter
    size_t ditems_cap = 0;
    // page-locked states, one per slot, for two ticks: the worker queues tick t + 1 before it
    // reads tick t's states, so that the GPU does not wait for the host between ticks
    ScgState *st_host = nullptr;    // [2][cfg.max_slots]
    // device copies of the states of slots on their own streams, taken on those streams after
    // each tick's last pass: the next tick's passes then follow on the slot's stream at once,
    // without waiting for the state's copy to the host on the server stream
    ScgState *st_snap = nullptr;    // [2][cfg.max_slots]
    cudaEvent_t tick_done[2] = {nullptr, nullptr};
    cudaStream_t fin_stream = nullptr;   // copies of finished images, beside the next tick
    std::vector<int2> h_items;
    std::vector<int> live_idx;   // the slots in those lists
    bool items_dirty = true;
    misr_status worker_error = MISR_OK;
    uint64_t passes_launched = 0;
    // Slots whose problem runs in launches of its own (launch_alone) take their SCG passes on a
    // stream per slot index, forked from `stream` after the slot's admission and joined back
    // before each tick's states are read: independent problems' launches then overlap, the next
    // one filling the SMs the last items of the previous one leave idle.  Created on first use.
    std::vector<cudaStream_t> slot_streams;   // [cfg.max_slots]
    std::vector<cudaEvent_t> slot_joins;      // [cfg.max_slots]
    cudaEvent_t fork = nullptr;
};

namespace {

// a short wait inside a polling loop
inline void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
    for (int k = 0; k < 64; ++k) __builtin_ia32_pause();
#else
    std::this_thread::yield();
#endif
}

misr_status grow_items(misr_server_t s, size_t need) {
    if (need <= s->ditems_cap) return MISR_OK;
    size_t cap = std::max<size_t>(need, 2 * s->ditems_cap);
    if (s->ditems) {
        CK(cudaStreamSynchronize(s->stream));
        cudaFree(s->ditems);
        s->ditems = nullptr;
    }
    cudaError_t e = cudaMalloc(&s->ditems, cap * sizeof(int2));
    if (e != cudaSuccess) { cudaGetLastError(); s->ditems_cap = 0; return fail(MISR_ENOMEM, "work items: %s", cudaGetErrorString(e)); }
    s->ditems_cap = cap;
    return MISR_OK;
}

// Can a new slot for `d` be created?  (slot count, explicit budget, free device memory)
bool can_create(misr_server_t s, const misr_desc &d) {
    int held = 0;   // slots holding a plan (an evicted slot keeps its index, empty)
    for (const Slot &sl : s->slots) held += sl.plan != nullptr;
    if (held >= s->cfg.max_slots) return false;
    const size_t need = plan_bytes_estimate(d);
    if (s->cfg.hbm_budget_bytes > 0) return s->slot_bytes + need <= s->cfg.hbm_budget_bytes;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return false; }
    return free_b > need + s->cfg.hbm_reserve_bytes;
}

// Free one idle slot of another class (when memory or the slot count blocks a request).  The
// slot is emptied under the server lock (misr_server_counters reads the table); its plan is
// destroyed after the lock is released.
bool evict_idle(misr_server_t s, const DescCopy &want) {
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot &sl = s->slots[i];
        if (!sl.busy && sl.plan && !sl.desc.same_class(want)) {
            cudaStreamSynchronize(s->stream);
            if (s->slot_streams[i]) cudaStreamSynchronize(s->slot_streams[i]);
            misr_plan_t p = sl.plan;
            int2 *items = sl.items;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->slot_bytes -= plan_bytes_estimate(sl.desc.d);
                sl.plan = nullptr;   // the index stays (records are per index), empty
                sl.items = nullptr;
            }
            misr_plan_destroy(p);
            cudaFree(items);
            return true;
        }
    }
    return false;
}

// Make a slot of `d`'s class (creating its plan and its own tile and group lists), freeing
// idle slots of other classes when memory or the slot count is short.  Worker thread only.
// The plan and the lists are made without the server lock, so that submit and poll are not
// held up by the allocations and copies; the slot is entered in the table under the lock.
// Returns the slot index, -1 when no room can be made now, or -2 with *status set when the
// descriptor cannot be served at all.
int make_slot(misr_server_t s, const DescCopy &want, misr_status *status) {
    const misr_desc &d = want.d;
    bool ok = can_create(s, d);
    while (!ok && evict_idle(s, want)) ok = can_create(s, d);
    if (!ok) return -1;
    int idx = -1;   // reuse an empty index first
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].plan) { idx = (int)i; break; }
    const bool grow = idx < 0;
    if (grow) {
        if ((int)s->slots.size() >= s->cfg.max_slots) return -1;
        idx = (int)s->slots.size();
    }
    misr_plan_t p = nullptr;
    const misr_status pc = misr_plan_create(&d, &p);
    if (pc != MISR_OK) {
        cudaGetLastError();
        if (pc == MISR_ENOMEM || pc == MISR_ECUDA) return -1;
        *status = pc;
        return -2;
    }
    std::vector<int2> t, gl;
    PassSegs segs;
    build_pass_lists({&p->hp}, {idx}, t, gl, segs);
    const int n_list = (int)t.size();
    t.insert(t.end(), gl.begin(), gl.end());
    int2 *items = nullptr;
    const bool ok2 = cudaMalloc(&items, sizeof(int2) * t.size()) == cudaSuccess &&
                     cudaMemcpy(items, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                     cudaMemcpy(&s->dprobs[idx], &p->hp, sizeof(DevProblem), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok2) {
        cudaGetLastError();
        misr_plan_destroy(p);
        if (items) cudaFree(items);
        return -1;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (grow) s->slots.emplace_back();   // capacity reserved at creation: no reallocation
    Slot &sl = s->slots[idx];
    sl.plan = p;
    sl.items = items;
    sl.n_list = n_list;
    sl.segs = std::move(segs);
    sl.desc = want;
    s->slot_bytes += plan_bytes_estimate(d);
    return idx;
}

// Assign queued requests to slots; returns the slots admitted this tick.  The queue is read and
// every decision recorded under the server lock; slots are made without it.
std::vector<int> admit(misr_server_t s) {
    std::vector<int> started;
    std::vector<std::pair<uint64_t, DescCopy>> queued;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (uint64_t t : s->queue) queued.push_back({t, s->reqs[t].desc});
    }
    std::vector<char> taken(s->slots.size() + queued.size(), 0);   // slots given out this tick
    for (auto &q : queued) {
        int use = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (s->slots[i].plan && !s->slots[i].busy && !taken[i] && s->slots[i].desc.same_class(q.second)) {
                use = (int)i;
                break;
            }
        misr_status bad = MISR_OK;
        if (use < 0) {
            use = make_slot(s, q.second, &bad);
            if (use >= 0 && (size_t)use >= taken.size()) taken.resize(use + 1, 0);
        }
        bool any_busy = false;
        for (auto &sl : s->slots) any_busy |= sl.busy;
        std::lock_guard<std::mutex> lock(s->mu);
        auto qit = std::find(s->queue.begin(), s->queue.end(), q.first);
        if (qit == s->queue.end()) continue;   // cancelled meanwhile (a slot made for it stays idle)
        Request &rq = s->reqs[q.first];
        if (use < 0) {
            if (use == -1 && any_busy) continue;   // stays queued until a running projection frees room
            rq.state = RQ_FAILED;
            rq.status = use == -2 ? bad
                                  : fail(MISR_ENOMEM, "a %dx%d x%d projection does not fit the server's HBM budget",
                                         rq.desc.d.lr_h, rq.desc.d.lr_w, rq.desc.d.factor);
            rq.t_end = now_s();
            s->queue.erase(qit);
            s->cv_done.notify_all();
            continue;
        }
        taken[use] = 1;
        Slot &sl = s->slots[use];
        sl.busy = true;
        sl.ticket = rq.ticket;
        sl.passes = 0;
        sl.queued = 0;
        sl.fork = true;
        rq.state = RQ_RUNNING;
        rq.slot = use;
        rq.t_start = now_s();
        started.push_back(use);
        s->queue.erase(qit);
        s->items_dirty = true;
    }
    return started;
}

void finish(misr_server_t s, int idx, const ScgState &h, misr_status st_code) {
    Slot &sl = s->slots[idx];
    std::lock_guard<std::mutex> lock(s->mu);
    Request &rq = s->reqs[sl.ticket];
    rq.stats.iters_done = h.iter;
    rq.stats.accepted = h.accepted;
    rq.stats.status = st_code;
    rq.stats.reserved = 0;
    rq.stats.J_final = h.E;
    rq.stats.rnorm2 = h.rn2;
    rq.stats.lambda_scg = h.lam;
    rq.status = st_code;
    rq.state = st_code == MISR_OK ? RQ_DONE : RQ_FAILED;
    rq.t_end = now_s();
    sl.busy = false;
    s->items_dirty = true;
}

// One tick as queued: the slots (and their tickets) whose states it copies to st_host[buf].
struct TickRecord {
    std::vector<std::pair<int, uint64_t>> live;   // (slot, ticket) whose states the tick copies
    std::vector<char> ran;                         // per entry of live: the tick ran passes on it
    int buf = 0;
};

void fail_queue(misr_server_t s, misr_status r) {
    std::lock_guard<std::mutex> lock(s->mu);
    s->worker_error = r;
    for (uint64_t t : s->queue) {
        Request &rq = s->reqs[t];
        rq.state = RQ_FAILED;
        rq.status = r;
        rq.t_end = now_s();
    }
    s->queue.clear();
    s->cv_done.notify_all();
}

// Completions of a queued tick, once its states have landed: finished slots copy their image
// out on the second stream (the passes queued after them skip finished problems), cancelled
// ones are released.  A slot whose ticket changed since the tick was queued is not this
// tick's to judge.
misr_status complete_tick(misr_server_t s, const TickRecord &tk, misr_status r) {
    const ScgState *sth = s->st_host + (size_t)tk.buf * s->cfg.max_slots;
    std::vector<char> cancelled(s->slots.size(), 0);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (auto &lt : tk.live)
            if (s->slots[lt.first].busy && s->slots[lt.first].ticket == lt.second)
                cancelled[lt.first] = s->reqs[lt.second].cancel;
    }
    std::vector<int> done;
    for (size_t e = 0; e < tk.live.size(); ++e) {
        const auto &lt = tk.live[e];
        const int i = lt.first;
        Slot &sl = s->slots[i];
        if (!sl.busy || sl.ticket != lt.second) continue;
        if (tk.ran[e]) sl.passes += std::max(1, s->cfg.passes_per_tick);
        if (r != MISR_OK || sth[i].done || cancelled[i]) done.push_back(i);
        else if (sl.queued >= sl.plan->d.iters && sl.passes >= sl.queued) {   // not done at its count:
            sl.queued = sl.passes - sl.plan->d.iters;                         // queue passes again
            s->items_dirty = true;
        }
    }
    std::vector<misr_status> codes(done.size(), r);
    bool copies = false;
    for (size_t d = 0; d < done.size(); ++d) {
        const int idx = done[d];
        Slot &sl = s->slots[idx];
        misr_status &code = codes[d];
        if (code == MISR_OK && cancelled[idx]) code = MISR_ECANCELED;
        if (code == MISR_OK && sth[idx].status != DEV_OK) code = MISR_ETIMEOUT;
        if (code == MISR_OK) {
            const Request *rq;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                rq = &s->reqs[sl.ticket];
            }
            code = launch_finalize_raw(s->dprobs, idx, sl.plan->n, rq->x, s->fin_stream);
            copies = true;
        }
    }
    if (copies && cudaStreamSynchronize(s->fin_stream) != cudaSuccess) {
        const misr_status e = fail(MISR_ECUDA, "server copy stream failed");
        for (auto &c : codes)
            if (c == MISR_OK) c = e;
        r = e;
    }
    for (size_t d = 0; d < done.size(); ++d) finish(s, done[d], sth[done[d]], codes[d]);
    if (!done.empty()) s->cv_done.notify_all();
    return r;
}

void worker_main(misr_server_t s) {
    cudaSetDevice(s->device);
    const int k_passes = std::max(1, s->cfg.passes_per_tick);
    TickRecord pending;          // the tick queued last, whose states are not read yet
    bool have_pending = false;
    int buf = 0;
    for (;;) {
        if (!have_pending) {
            // idle: poll for a new request for idle_spin_us (no wake-up when one comes), then sleep
            bool idle = true;
            for (auto &sl : s->slots) idle &= !sl.busy;
            if (idle && s->cfg.idle_spin_us > 0) {
                const uint64_t w0 = s->wakes.load(std::memory_order_acquire);
                bool seen = false;
                {
                    std::lock_guard<std::mutex> lock(s->mu);
                    seen = s->stop || !s->queue.empty();
                }
                const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(s->cfg.idle_spin_us);
                while (!seen && s->wakes.load(std::memory_order_acquire) == w0 && std::chrono::steady_clock::now() < until)
                    cpu_relax();
            }
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] {
                if (s->stop || !s->queue.empty()) return true;
                for (auto &sl : s->slots)
                    if (sl.busy) return true;
                return false;
            });
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->stop) break;
        }
        // 1. admission: prepare + initial pass of each newly admitted projection (queued
        // behind the pending tick, whose passes skip finished problems)
        std::vector<int> started = admit(s);
        misr_status r = MISR_OK;
        for (int idx : started) {
            Slot &sl = s->slots[idx];
            const Request *rq;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                rq = &s->reqs[sl.ticket];
            }
            misr_plan_t p = sl.plan;
            if (r == MISR_OK)
                r = launch_prepare_raw(s->dprobs, idx, p->hp, p->d, rq->y, rq->x, p->d.x0_mode, 1 | 2 | 4, s->stream);
            if (r == MISR_OK) r = launch_pass_raw(s->dprobs, sl.items, sl.segs, sl.items + sl.n_list, p->hp.n_groups,
                                                  s->work, MODE_INIT, 0.0, 0.0, s->stream);
        }
        // 2. the live slots' tile and group lists (uploaded in stream order, after the
        // pending tick's passes have read the old ones)
        if (r == MISR_OK && s->items_dirty) {
            s->h_items.clear();
            std::vector<int2> gl;
            std::vector<const DevProblem *> rp;
            std::vector<int> idx;
            for (size_t i = 0; i < s->slots.size(); ++i)
                if (s->slots[i].busy && s->slots[i].queued < s->slots[i].plan->d.iters &&
                    !launch_alone(s->slots[i].plan->hp)) {
                    rp.push_back(&s->slots[i].plan->hp);
                    idx.push_back((int)i);
                }
            build_pass_lists(rp, idx, s->h_items, gl, s->live_segs);
            s->live_idx = idx;
            s->live_tiles = (int)s->h_items.size();
            s->live_groups = (int)gl.size();
            s->h_items.insert(s->h_items.end(), gl.begin(), gl.end());
            r = grow_items(s, std::max<size_t>(s->h_items.size(), 1));
            if (r == MISR_OK && !s->h_items.empty() &&
                cudaMemcpyAsync(s->ditems, s->h_items.data(), sizeof(int2) * s->h_items.size(), cudaMemcpyHostToDevice,
                                s->stream) != cudaSuccess)
                r = fail(MISR_ECUDA, "tile list upload failed");
            s->items_dirty = false;
        }
        // 3. k SCG iterations of every live projection, then their states into this tick's
        // half of st_host
        const int nt = s->live_tiles;
        std::vector<int> own;       // busy slots that run on their own streams
        std::vector<int> observe;   // busy slots with no pass queued or in flight (their count is
                                    // reached, or 0): a state read only, to see them finish
        bool live = s->live_segs.total() > 0;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            const Slot &sl = s->slots[i];
            if (!sl.busy) continue;
            if (sl.queued < sl.plan->d.iters) {
                if (launch_alone(sl.plan->hp)) {
                    own.push_back((int)i);
                    live = true;
                }
            } else if (sl.passes >= sl.queued) {
                observe.push_back((int)i);
                live = true;
            }
        }
        TickRecord tk;
        tk.buf = buf;
        if (live) {
            if (!own.empty()) {
                if (!s->fork && cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess)
                    r = fail(MISR_ECUDA, "server fork event failed");
                for (int i : own) {
                    if (r == MISR_OK && !s->slot_streams[i] &&
                        cudaStreamCreateWithFlags(&s->slot_streams[i], cudaStreamNonBlocking) != cudaSuccess)
                        r = fail(MISR_ECUDA, "slot stream failed");
                    if (r == MISR_OK && !s->slot_joins[i] &&
                        cudaEventCreateWithFlags(&s->slot_joins[i], cudaEventDisableTiming) != cudaSuccess)
                        r = fail(MISR_ECUDA, "slot event failed");
                }
                // a slot admitted since its last tick waits for its prepare and initial pass on
                // the server stream; the others' streams are already ordered behind those
                bool any_fork = false;
                for (int i : own) any_fork |= s->slots[i].fork;
                if (r == MISR_OK && any_fork && cudaEventRecord(s->fork, s->stream) != cudaSuccess)
                    r = fail(MISR_ECUDA, "fork failed");
                for (int i : own)
                    if (r == MISR_OK && s->slots[i].fork) {
                        if (cudaStreamWaitEvent(s->slot_streams[i], s->fork, 0) != cudaSuccess)
                            r = fail(MISR_ECUDA, "fork wait failed");
                        s->slots[i].fork = false;
                    }
            }
            for (int it = 0; it < k_passes && r == MISR_OK; ++it) {
                if (s->live_segs.total() > 0) {
                    r = launch_pass_raw(s->dprobs, s->ditems, s->live_segs, s->ditems + nt, s->live_groups, s->work,
                                        MODE_ITER, 0.0, 0.0, s->stream);
                    ++s->passes_launched;
                }
                for (size_t q = 0; q < own.size() && r == MISR_OK; ++q) {   // each on the slot's plan's counter
                    Slot &sl = s->slots[own[q]];
                    r = launch_pass_raw(s->dprobs, sl.items, sl.segs, sl.items + sl.n_list, sl.plan->hp.n_groups,
                                        sl.plan->work, MODE_ITER, 0.0, 0.0, s->slot_streams[own[q]]);
                    ++s->passes_launched;
                }
            }
            for (int i : own) {   // the state as this tick left it, then join before it is read
                if (r == MISR_OK && cudaMemcpyAsync(s->st_snap + (size_t)buf * s->cfg.max_slots + i,
                                                    s->slots[i].plan->hp.st, sizeof(ScgState),
                                                    cudaMemcpyDeviceToDevice, s->slot_streams[i]) != cudaSuccess)
                    r = fail(MISR_ECUDA, "state snapshot failed");
                if (r == MISR_OK && cudaEventRecord(s->slot_joins[i], s->slot_streams[i]) != cudaSuccess)
                    r = fail(MISR_ECUDA, "join failed");
                if (r == MISR_OK && cudaStreamWaitEvent(s->stream, s->slot_joins[i], 0) != cudaSuccess)
                    r = fail(MISR_ECUDA, "join wait failed");
            }
            // the states of the slots this tick ran passes on; a slot whose passes now reach its
            // iteration count gets no more (its last tick decides it)
            std::vector<int> ran = own;
            if (s->live_segs.total() > 0) ran.insert(ran.end(), s->live_idx.begin(), s->live_idx.end());
            const size_t n_ran = ran.size();
            ran.insert(ran.end(), observe.begin(), observe.end());
            ScgState *sth = s->st_host + (size_t)buf * s->cfg.max_slots;
            for (size_t q = 0; q < ran.size(); ++q) {
                const int i = ran[q];
                Slot &sl = s->slots[i];
                if (r != MISR_OK || !sl.busy) continue;
                // own slots' states from their snapshots (their streams may run on into the next
                // tick); the others' (and observed slots', with no pass in flight) directly
                const ScgState *src = q < own.size() ? s->st_snap + (size_t)buf * s->cfg.max_slots + i : sl.plan->hp.st;
                if (cudaMemcpyAsync(&sth[i], src, sizeof(ScgState), cudaMemcpyDeviceToHost, s->stream) !=
                    cudaSuccess)
                    r = fail(MISR_ECUDA, "state copy failed");
                tk.live.push_back({i, sl.ticket});
                tk.ran.push_back(q < n_ran ? 1 : 0);
                if (q >= n_ran) continue;   // observed only
                sl.queued += k_passes;
                if (sl.queued >= sl.plan->d.iters && !launch_alone(sl.plan->hp)) s->items_dirty = true;
            }
            if (r == MISR_OK && cudaEventRecord(s->tick_done[buf], s->stream) != cudaSuccess)
                r = fail(MISR_ECUDA, "tick event failed");
        }
        // 4. the previous tick's completions, while this one runs
        if (have_pending) {
            if (r == MISR_OK && cudaEventSynchronize(s->tick_done[pending.buf]) != cudaSuccess)
                r = fail(MISR_ECUDA, "server stream failed");
            r = complete_tick(s, pending, r);
            have_pending = false;
        }
        if (r == MISR_OK && live) {
            pending = std::move(tk);
            have_pending = true;
            buf ^= 1;
        } else if (r != MISR_OK && live) {
            cudaStreamSynchronize(s->stream);
            complete_tick(s, tk, r);
        }
        if (r != MISR_OK) {   // the stream is unusable: fail what runs and what is queued, stop serving
            cudaStreamSynchronize(s->stream);
            for (cudaStream_t st : s->slot_streams)
                if (st) cudaStreamSynchronize(st);
            cudaGetLastError();
            const ScgState none{};
            for (size_t i = 0; i < s->slots.size(); ++i)
                if (s->slots[i].busy) finish(s, (int)i, none, r);
            fail_queue(s, r);
            break;
        }
    }
    // stopping: let the last queued tick finish before the slots are torn down
    if (have_pending) {
        cudaStreamSynchronize(s->stream);
        complete_tick(s, pending, MISR_OK);
    }
}

}  // namespace

extern "C" misr_status misr_server_create(const misr_server_cfg *cfg, misr_server_t *out) {
    if (!out || !cfg) return fail(MISR_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 4096) return fail(MISR_EINVAL, "max_slots must be in [1, 4096]");
    if (cfg->passes_per_tick < 0 || cfg->passes_per_tick > 1000) return fail(MISR_EINVAL, "passes_per_tick must be in [0, 1000]");
    if (cfg->idle_spin_us < 0 || cfg->idle_spin_us > 1000000) return fail(MISR_EINVAL, "idle_spin_us must be in [0, 1e6]");
    misr_server_t s = new (std::nothrow) misr_server_s();
    if (!s) return fail(MISR_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    if (s->cfg.passes_per_tick == 0) s->cfg.passes_per_tick = 4;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->dprobs, sizeof(DevProblem) * cfg->max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->work, 256);
    if (e == cudaSuccess) e = cudaMemset(s->work, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->st_host, 2 * sizeof(ScgState) * cfg->max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->st_snap, 2 * sizeof(ScgState) * cfg->max_slots);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fin_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->tick_done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        misr_status r = fail(MISR_ENOMEM, "server setup: %s", cudaGetErrorString(e));
        for (auto &ev : s->tick_done)
            if (ev) cudaEventDestroy(ev);
        if (s->fin_stream) cudaStreamDestroy(s->fin_stream);
        if (s->st_host) cudaFreeHost(s->st_host);
        if (s->st_snap) cudaFree(s->st_snap);
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->dprobs) cudaFree(s->dprobs);
        if (s->work) cudaFree(s->work);
        delete s;
        return r;
    }
    s->slots.reserve(cfg->max_slots);
    s->slot_streams.assign(cfg->max_slots, nullptr);
    s->slot_joins.assign(cfg->max_slots, nullptr);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return MISR_OK;
}

extern "C" misr_status misr_server_destroy(misr_server_t s) {
    if (!s) return MISR_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->wakes.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    DeviceGuard g(s->device);
    cudaStreamSynchronize(s->stream);
    for (cudaStream_t st : s->slot_streams)
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (cudaEvent_t ev : s->slot_joins)
        if (ev) cudaEventDestroy(ev);
    if (s->fork) cudaEventDestroy(s->fork);
    for (auto &sl : s->slots) {
        if (sl.plan) misr_plan_destroy(sl.plan);
        if (sl.items) cudaFree(sl.items);
    }
    if (s->ditems) cudaFree(s->ditems);
    if (s->dprobs) cudaFree(s->dprobs);
    if (s->work) cudaFree(s->work);
    if (s->st_host) cudaFreeHost(s->st_host);
    if (s->st_snap) cudaFree(s->st_snap);
    for (auto &ev : s->tick_done)
        if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(s->fin_stream);
    cudaStreamDestroy(s->fin_stream);
    cudaStreamDestroy(s->stream);
    delete s;
    return MISR_OK;
}

extern "C" misr_status misr_submit(misr_server_t s, const misr_desc *desc, const void *y_dev, float *x_dev,
                                   uint64_t *ticket) {
    if (!s || !desc || !y_dev || !x_dev || !ticket) return fail(MISR_EINVAL, "NULL argument");
    const misr_status chk = check_desc(*desc);
    if (chk != MISR_OK) return chk;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->worker_error != MISR_OK) return fail(s->worker_error, "the server stopped after an error");
    const uint64_t t = s->next_ticket++;
    Request &rq = s->reqs[t];
    rq.ticket = t;
    rq.desc.set(*desc);
    rq.y = y_dev;
    rq.x = x_dev;
    rq.t_submit = now_s();
    s->queue.push_back(t);
    *ticket = t;
    s->wakes.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_all();
    return MISR_OK;
}

extern "C" misr_status misr_poll(misr_server_t s, uint64_t ticket, misr_stats *stats, double *times) {
    if (!s) return fail(MISR_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MISR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    const Request &rq = it->second;
    if (rq.state == RQ_QUEUED || rq.state == RQ_RUNNING) return MISR_EAGAIN;
    if (stats) *stats = rq.stats;
    if (times) { times[0] = rq.t_submit; times[1] = rq.t_start; times[2] = rq.t_end; }
    const misr_status st = rq.status;
    s->reqs.erase(it);
    if (st != MISR_OK) return fail(st, "request %llu failed", (unsigned long long)ticket);
    return MISR_OK;
}

extern "C" misr_status misr_cancel(misr_server_t s, uint64_t ticket) {
    if (!s) return fail(MISR_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MISR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request &rq = it->second;
    if (rq.state == RQ_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
        rq.state = RQ_FAILED;
        rq.status = MISR_ECANCELED;
        rq.t_end = now_s();
        s->cv_done.notify_all();
    } else if (rq.state == RQ_RUNNING) {
        rq.cancel = true;   // the worker finishes it after its current tick
    }
    return MISR_OK;
}

extern "C" misr_status misr_server_wait(misr_server_t s, uint64_t ticket, double timeout_s) {
    if (!s) return fail(MISR_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto done = [&] {
        auto it = s->reqs.find(ticket);
        return it == s->reqs.end() || (it->second.state != RQ_QUEUED && it->second.state != RQ_RUNNING) ||
               s->worker_error != MISR_OK;
    };
    if (s->reqs.find(ticket) == s->reqs.end()) return fail(MISR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done))
        return fail(MISR_ETIMEOUT, "ticket %llu not finished within %.3f s", (unsigned long long)ticket, timeout_s);
    auto it = s->reqs.find(ticket);
    if (it != s->reqs.end() && (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING))
        return fail(s->worker_error, "the server stopped after an error");
    return MISR_OK;
}

extern "C" misr_status misr_server_counters(misr_server_t s, int64_t *out) {
    if (!s || !out) return fail(MISR_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t live = 0, slots = 0;
    for (auto &sl : s->slots) { live += sl.busy; slots += sl.plan != nullptr; }
    out[0] = (int64_t)s->queue.size();
    out[1] = live;
    out[2] = slots;
    out[3] = (int64_t)s->slot_bytes;
    out[4] = (int64_t)s->passes_launched;
    return MISR_OK;
}

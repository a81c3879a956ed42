// server.cu -- the served form of the hot path.
//
// Views arrive one at a time, as a scanning microscope emits them (Section 3:
// the stage delivers views at up to 5 Hz per microscope).  A worker thread
// groups the views waiting in the queue into a micro-batch, runs the batched
// path on it and keeps the per-view results until the caller polls them.
// While one micro-batch runs, new arrivals accumulate, so the batch size
// adapts to the arrival rate.  Two micro-batches alternate: the next is
// staged and enqueued behind the running one before the running one's
// results are collected, so the device does not idle while the host gathers
// views and splits results.
//
// Memory budget.  The two slots' batches hold device buffers that only grow
// (a slot keeps its high-water buffers for the next micro-batch).  A
// micro-batch is admitted only if the bytes its slot will hold -- per buffer
// group the larger of what it holds and what the views need, planned with the
// batch's own sizing code -- plus the bytes the other slot holds stay within
// the budget.  When even the oldest view does not fit, the worker first waits
// for the other slot's run to end, then frees the idle slot's buffers.  A
// batch whose buffers must grow after a run (candidate overflow) may grow only
// within what the other slot leaves; beyond that its views fail with
// ET_ERR_OOM.
#include "runtime.h"

#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace et {

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    uint64_t tag;
    std::vector<int32_t> xyz;
    int64_t n;
    int64_t t_submit;
};

struct Done {
    et_result r;
    std::vector<et_track> tracks;
    std::vector<int32_t> members;
};

struct ServerRT {
    Ctx *ctx;
    et_params p;
    uint64_t budget;
    int max_views;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> pending;
    std::deque<Done> done;
    std::unordered_map<uint64_t, Done> polled;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
    size_t max_pending = 1 << 20;
    // sizing of candidate micro-batches (host only): one for the worker, one
    // for submit's check that a view fits the budget on its own
    BatchRT *planner = nullptr, *submit_planner = nullptr;
    std::mutex submit_mu;
    // accounting (under mu)
    uint64_t held_now = 0, held_peak = 0;
    int64_t n_done = 0, n_batches = 0, n_busy = 0;

    // Two micro-batches alternate: while one runs on the device, the worker
    // gathers and enqueues the next (same stream, so the device runs them back
    // to back) and then collects the first.  Each slot keeps its own host
    // staging buffers, valid until its results are fetched.
    struct Slot {
        BatchRT *batch = nullptr;
        std::vector<Pending> take;
        int32_t *xyz = nullptr;   // page-locked staging of the views' grains
        size_t xyz_cap = 0;       // in int32 elements
        std::vector<int64_t> off;
        int64_t t_admit = 0;
        et_status status = ET_OK;
        bool busy = false;
    };
    Slot slots[2];

    ServerRT(Ctx *c, const et_params &pp, uint64_t b, int mv) : ctx(c), p(pp), budget(b), max_views(mv) {}

    et_status start() {
        cudaSetDevice(ctx->device);
        cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "server stream");
        for (auto &sl : slots) sl.batch = new BatchRT(ctx, p);
        planner = new BatchRT(ctx, p);
        submit_planner = new BatchRT(ctx, p);
        worker = std::thread([this] { run(); });
        return ET_OK;
    }

    // Device bytes a batch of one view of n grains holds.
    uint64_t single_view_bytes(int64_t n) {
        std::lock_guard<std::mutex> g(submit_mu);
        size_t sz[BatchRT::NGROUP];
        submit_planner->plan_shape(1, n, n, (double)n * (double)n, sz);
        uint64_t t = 0;
        for (size_t v : sz) t += v;
        return t;
    }

    void account() {
        const uint64_t h = slots[0].batch->held_bytes() + slots[1].batch->held_bytes();
        std::lock_guard<std::mutex> g(mu);
        held_now = h;
        held_peak = std::max(held_peak, h);
    }

    ~ServerRT() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv_work.notify_all();
        if (worker.joinable()) worker.join();
        for (auto &sl : slots) {
            delete sl.batch;
            if (sl.xyz) cudaFreeHost(sl.xyz);
        }
        delete planner;
        delete submit_planner;
        if (stream) cudaStreamDestroy(stream);
    }

    // Moves pending views into sl.take while the slot's planned device bytes
    // plus the other slot's held bytes fit the budget; waits for arrivals
    // only if `wait` (nothing else is in flight).  False: stop.
    bool gather(Slot &sl, const Slot &other, bool wait) {
        sl.take.clear();
        const uint64_t other_held = other.batch->held_bytes();
        const uint64_t avail = budget > other_held ? budget - other_held : 0;
        std::unique_lock<std::mutex> g(mu);
        if (wait) cv_work.wait(g, [this] { return stop || !pending.empty(); });
        if (stop && pending.empty()) return false;
        long long n = 0, mx = 0;
        double s2 = 0;
        size_t sz[BatchRT::NGROUP];
        while (!pending.empty() && (int)sl.take.size() < max_views) {
            const long long vn = pending.front().n;
            planner->plan_shape((int)sl.take.size() + 1, n + vn, std::max(mx, vn), s2 + (double)vn * vn, sz);
            if (sl.batch->footprint_with(sz) > avail) break;
            n += vn;
            mx = std::max(mx, vn);
            s2 += (double)vn * vn;
            sl.take.push_back(std::move(pending.front()));
            pending.pop_front();
        }
        return true;
    }

    void reject_oldest() {
        std::lock_guard<std::mutex> g(mu);
        if (pending.empty()) return;
        Done d;
        memset(&d.r, 0, sizeof d.r);
        d.r.tag = pending.front().tag;
        d.r.status = ET_ERR_OOM;
        d.r.n_grains = pending.front().n;
        d.r.t_submit_ns = pending.front().t_submit;
        d.r.t_admit_ns = d.r.t_done_ns = now_ns();
        pending.pop_front();
        done.push_back(std::move(d));
        ++n_done;
        cv_done.notify_all();
    }

    bool has_pending() {
        std::lock_guard<std::mutex> g(mu);
        return !pending.empty();
    }

    void launch(Slot &sl) {
        sl.t_admit = now_ns();
        sl.off.assign(1, 0);
        for (auto &v : sl.take) sl.off.push_back(sl.off.back() + v.n);
        const size_t need = (size_t)std::max<int64_t>(3 * sl.off.back(), 3);
        sl.status = ET_OK;
        if (need > sl.xyz_cap) {   // grows rarely; the slot's previous run is fetched already
            if (sl.xyz) cudaFreeHost(sl.xyz);
            sl.xyz = nullptr;
            sl.xyz_cap = 0;
            const size_t cap = need + need / 2;
            if (cudaHostAlloc((void **)&sl.xyz, cap * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                sl.xyz = nullptr;
                sl.status = fail(ET_ERR_OOM, "page-locked staging of %zu grains", need / 3);
            } else {
                sl.xyz_cap = cap;
            }
        }
        if (sl.status == ET_OK) {
            size_t o = 0;
            for (auto &v : sl.take) {
                if (!v.xyz.empty()) memcpy(sl.xyz + o, v.xyz.data(), v.xyz.size() * sizeof(int32_t));
                o += v.xyz.size();
            }
            const uint64_t other_held = slots[&sl == &slots[0] ? 1 : 0].batch->held_bytes();
            sl.batch->byte_limit = budget > other_held ? budget - other_held : 1;
            sl.status = sl.batch->load(sl.xyz, sl.off.data(), (int)sl.take.size(), false, stream);
        }
        if (sl.status == ET_OK) sl.status = sl.batch->find(stream, false);
        sl.busy = true;
        account();
    }

    void complete(Slot &sl, std::vector<int64_t> &vtrk, std::vector<et_track> &trk, std::vector<int32_t> &mem) {
        et_status s = sl.status;
        int64_t nt = 0, nm = 0;
        vtrk.assign(sl.take.size() + 1, 0);
        {   // a re-run after an overflow may grow the slot only within what the other leaves
            const uint64_t other_held = slots[&sl == &slots[0] ? 1 : 0].batch->held_bytes();
            sl.batch->byte_limit = budget > other_held ? budget - other_held : 1;
        }
        if (s == ET_OK) {
            s = sl.batch->fetch(vtrk.data(), nullptr, 0, &nt, nullptr, 0, &nm);
            if (s == ET_ERR_CAPACITY || s == ET_OK) {
                trk.resize((size_t)std::max<int64_t>(nt, 1));
                mem.resize((size_t)std::max<int64_t>(nm, 1));
                s = sl.batch->fetch(vtrk.data(), trk.data(), nt, &nt, mem.data(), nm, &nm);
            }
        }
        const int64_t t_done = now_ns();
        std::vector<Done> out(sl.take.size());
        for (size_t v = 0; v < sl.take.size(); ++v) {
            Done &d = out[v];
            memset(&d.r, 0, sizeof d.r);
            d.r.tag = sl.take[v].tag;
            d.r.status = s;
            d.r.n_grains = sl.take[v].n;
            d.r.t_submit_ns = sl.take[v].t_submit;
            d.r.t_admit_ns = sl.t_admit;
            d.r.t_done_ns = t_done;
            if (s == ET_OK) {
                const int64_t t0 = vtrk[v], t1 = vtrk[v + 1];
                d.tracks.assign(trk.begin() + t0, trk.begin() + t1);
                int64_t m0 = t1 > t0 ? trk[t0].member_offset : 0;
                int64_t m1 = t1 > t0 ? trk[t1 - 1].member_offset + trk[t1 - 1].nhits : 0;
                d.members.assign(mem.begin() + m0, mem.begin() + m1);
                for (auto &t : d.tracks) {
                    t.member_offset -= m0;
                    t.view = 0;
                }
                d.r.n_tracks = (int32_t)(t1 - t0);
                d.r.n_members = m1 - m0;
            }
        }
        {
            std::lock_guard<std::mutex> g(mu);
            for (auto &d : out) done.push_back(std::move(d));
            n_done += (int64_t)out.size();
            ++n_batches;
        }
        cv_done.notify_all();
        sl.take.clear();
        sl.busy = false;
        account();
    }

    void run() {
        cudaSetDevice(ctx->device);
        std::vector<int64_t> vtrk;
        std::vector<et_track> trk;
        std::vector<int32_t> mem;
        int cur = 0;
        for (;;) {
            Slot &sl = slots[cur], &other = slots[cur ^ 1];
            // wait for arrivals only when nothing is in flight
            const bool live = gather(sl, other, !other.busy);
            if (sl.take.empty() && has_pending()) {
                // the oldest view does not fit beside the other slot: end the
                // other slot's run, then free idle buffers, and try again
                if (other.busy) complete(other, vtrk, trk, mem);
                else if (other.batch->held_bytes() > 0) other.batch->release_groups();
                else if (sl.batch->held_bytes() > 0) sl.batch->release_groups();
                else reject_oldest();   // does not fit even alone (submit checks the same plan)
                account();
                continue;
            }
            if (!sl.take.empty()) launch(sl);
            if (other.busy) complete(other, vtrk, trk, mem);
            if (!live && !sl.busy && !other.busy) return;
            cur ^= 1;
        }
    }
};

}  // namespace et

using namespace et;

struct et_server : public ServerRT {
    using ServerRT::ServerRT;
};

extern "C" {

et_status et_server_create(et_ctx *ctx, const et_params *params, uint64_t mem_budget_bytes, int32_t max_batch_views,
                           et_server **out) {
    try {
        if (!ctx || !out) return fail(ET_ERR_INVALID_ARG, "ctx/out is NULL");
        *out = nullptr;
        et_status s = check_params(params);
        if (s != ET_OK) return s;
        if (max_batch_views <= 0) max_batch_views = 256;
        if (mem_budget_bytes == 0) return fail(ET_ERR_INVALID_ARG, "memory budget is 0");
        et_server *sv = new et_server((Ctx *)ctx, *params, mem_budget_bytes, max_batch_views);
        s = sv->start();
        if (s != ET_OK) {
            delete sv;
            return s;
        }
        *out = sv;
        return ET_OK;
    } catch (...) {
        return fail(ET_ERR_OOM, "server creation failed");
    }
}

et_status et_server_submit(et_server *s, const int32_t *xyz, int64_t n, uint64_t tag) {
    if (!s || (n > 0 && !xyz) || n < 0) return fail(ET_ERR_INVALID_ARG, "bad submit arguments");
    if (n > (1 << 21) - 1) return fail(ET_ERR_INVALID_ARG, "view of %lld grains too large", (long long)n);
    if (s->single_view_bytes(n) > s->budget) {
        std::lock_guard<std::mutex> g(s->mu);
        ++s->n_busy;
        return fail(ET_ERR_BUSY, "view exceeds the memory budget on its own");
    }
    Pending pv;
    pv.tag = tag;
    pv.n = n;
    pv.t_submit = now_ns();
    try {
        pv.xyz.assign(xyz, xyz + 3 * n);
    } catch (...) {
        return fail(ET_ERR_OOM, "host copy of the view");
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->pending.size() >= s->max_pending) {
            ++s->n_busy;
            return fail(ET_ERR_BUSY, "pending queue full");
        }
        s->pending.push_back(std::move(pv));
    }
    s->cv_work.notify_one();
    return ET_OK;
}

et_status et_server_poll(et_server *s, et_result *out, int32_t max, int32_t *n_done, int32_t timeout_us) {
    if (!s || !n_done || (max > 0 && !out)) return fail(ET_ERR_INVALID_ARG, "bad poll arguments");
    *n_done = 0;
    std::unique_lock<std::mutex> g(s->mu);
    s->polled.clear();
    if (s->done.empty() && timeout_us > 0)
        s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), [s] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        Done d = std::move(s->done.front());
        s->done.pop_front();
        out[k++] = d.r;
        s->polled.emplace(d.r.tag, std::move(d));
    }
    *n_done = k;
    return ET_OK;
}

et_status et_server_fetch(et_server *s, uint64_t tag, et_track *tracks, int64_t cap, int64_t *n_tracks,
                          int32_t *members, int64_t member_cap, int64_t *n_members) {
    if (!s) return fail(ET_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->polled.find(tag);
    if (it == s->polled.end()) return fail(ET_ERR_INVALID_ARG, "tag not among the last poll's results");
    const Done &d = it->second;
    if (d.r.status != ET_OK) return d.r.status;
    const int64_t nt = (int64_t)d.tracks.size(), nm = (int64_t)d.members.size();
    if (n_tracks) *n_tracks = nt;
    if (n_members) *n_members = nm;
    if ((nt > 0 && (!tracks || cap < nt)) || (nm > 0 && (!members || member_cap < nm)))
        return fail(ET_ERR_CAPACITY, "need %lld tracks / %lld members", (long long)nt, (long long)nm);
    if (nt) memcpy(tracks, d.tracks.data(), sizeof(et_track) * nt);
    if (nm) memcpy(members, d.members.data(), sizeof(int32_t) * nm);
    return ET_OK;
}

et_status et_server_set_max_pending(et_server *s, int64_t max_pending) {
    if (!s || max_pending < 1) return fail(ET_ERR_INVALID_ARG, "server is NULL or max_pending < 1");
    std::lock_guard<std::mutex> g(s->mu);
    s->max_pending = (size_t)max_pending;
    return ET_OK;
}

et_status et_server_get_stats(et_server *s, et_server_stats *out) {
    if (!s || !out) return fail(ET_ERR_INVALID_ARG, "server/out is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->budget_bytes = s->budget;
    out->device_bytes = s->held_now;
    out->peak_device_bytes = s->held_peak;
    out->views_done = s->n_done;
    out->batches = s->n_batches;
    out->busy_rejections = s->n_busy;
    out->pending = (int64_t)s->pending.size();
    return ET_OK;
}

et_status et_server_destroy(et_server *s) {
    if (!s) return fail(ET_ERR_INVALID_ARG, "server is NULL");
    delete s;
    return ET_OK;
}

}  // extern "C"

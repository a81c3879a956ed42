// server.cu -- the served form of the hot path.
//
// Views arrive one at a time, as a scanning microscope emits them (Section 3:
// the stage delivers views at up to 5 Hz per microscope).  A worker thread
// groups the views waiting in the queue into a micro-batch whose estimated
// device memory fits the budget, runs the batched path on it and keeps the
// per-view results until the caller polls them.  While one micro-batch runs,
// new arrivals accumulate, so the batch size adapts to the arrival rate.  Two
// micro-batches alternate: the next is staged and enqueued behind the running
// one before the running one's results are collected, so the device does not
// idle while the host gathers views and splits results.
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

// Device bytes a view of n grains needs inside a batch (same formulas as the
// batch's own sizing; seeds are not stored, they size the candidates).
static uint64_t view_bytes(const et_params &p, int64_t n) {
    const double vol = (double)p.extent[0] * p.extent[1] * p.extent[2];
    const double shell = 4.0 / 3.0 * M_PI * (std::pow((double)p.seed_max, 3) - std::pow((double)p.seed_min, 3));
    const double seeds = 1.3 * 0.5 * (double)n * (double)n * std::min(1.0, shell / vol) + 4096;
    const double cand = std::max(65536.0 / 64, seeds / 16);
    return (uint64_t)(n * 160.0 + cand * (48.0 + 24 * 4.0) + (1 << 20));
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
        worker = std::thread([this] { run(); });
        return ET_OK;
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
        if (stream) cudaStreamDestroy(stream);
    }

    // Moves pending views into sl.take within the memory budget; waits for
    // arrivals only if `wait` (nothing else is in flight).  False: stop.
    bool gather(Slot &sl, bool wait) {
        sl.take.clear();
        std::unique_lock<std::mutex> g(mu);
        if (wait) cv_work.wait(g, [this] { return stop || !pending.empty(); });
        if (stop && pending.empty()) return false;
        uint64_t bytes = 0;
        while (!pending.empty() && (int)sl.take.size() < max_views) {
            uint64_t vb = view_bytes(p, pending.front().n);
            if (!sl.take.empty() && bytes + vb > budget) break;
            bytes += vb;
            sl.take.push_back(std::move(pending.front()));
            pending.pop_front();
        }
        return true;
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
            sl.status = sl.batch->load(sl.xyz, sl.off.data(), (int)sl.take.size(), false, stream);
        }
        if (sl.status == ET_OK) sl.status = sl.batch->find(stream, false);
        sl.busy = true;
    }

    void complete(Slot &sl, std::vector<int64_t> &vtrk, std::vector<et_track> &trk, std::vector<int32_t> &mem) {
        et_status s = sl.status;
        int64_t nt = 0, nm = 0;
        vtrk.assign(sl.take.size() + 1, 0);
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
        }
        cv_done.notify_all();
        sl.take.clear();
        sl.busy = false;
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
            const bool live = gather(sl, !other.busy);
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
    if (view_bytes(s->p, n) > s->budget) return fail(ET_ERR_BUSY, "view exceeds the memory budget on its own");
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
        if (s->pending.size() >= s->max_pending) return fail(ET_ERR_BUSY, "pending queue full");
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

et_status et_server_destroy(et_server *s) {
    if (!s) return fail(ET_ERR_INVALID_ARG, "server is NULL");
    delete s;
    return ET_OK;
}

}  // extern "C"

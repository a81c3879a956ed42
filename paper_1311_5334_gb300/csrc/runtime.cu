// runtime.cu -- host runtime behind the C ABI of include/et.h: contexts,
// batches (a view is a batch of one), device buffers with capacity growth,
// the launch sequence of the hot path and its CUDA-graph replay.
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

namespace et {

cudaError_t launch_merge_coop(const Batch &b, const Work &w, int grid, cudaStream_t st);
void launch_output(const Batch &b, const Work &w, Out &o, long long acc_cap, long long out_member_cap,
                   void *temp, cudaStream_t st);

static thread_local std::string g_last_error;

et_status fail(et_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

et_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(ET_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(ET_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char *last_error() { return g_last_error.c_str(); }

int bits_for(unsigned long long maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}


// ---------------------------------------------------------------- context

void *Ctx::dalloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (alloc) return alloc(bytes, user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Ctx::dfree(void *p) {
    if (!p) return;
    if (free_fn) free_fn(p, user);
    else cudaFree(p);
}

// ---------------------------------------------------------------- groups

bool Group::reserve(Ctx *ctx, size_t need) {
    if (need <= bytes && base) return true;
    release(ctx);
    base = (char *)ctx->dalloc(need);
    if (!base) return false;
    bytes = need;
    ++generation;
    return true;
}

void Group::release(Ctx *ctx) {
    if (base) ctx->dfree(base);
    base = nullptr;
    bytes = 0;
}


// ---------------------------------------------------------------- parameters

et_status check_params(const et_params *p) {
    if (!p) return fail(ET_ERR_INVALID_ARG, "params is NULL");
    for (int k = 0; k < 3; ++k)
        if (p->extent[k] <= 0 || p->extent[k] > (1 << 21))
            return fail(ET_ERR_INVALID_ARG, "extent[%d] = %d outside (0, 2^21]", k, p->extent[k]);
    if (p->seed_max < 1 || p->seed_min < 0 || p->seed_min > p->seed_max)
        return fail(ET_ERR_INVALID_ARG, "seed window [%d, %d) invalid", p->seed_min, p->seed_max);
    if (p->tube_r < 0 || p->tube_r > (1 << 20)) return fail(ET_ERR_INVALID_ARG, "tube_r = %d", p->tube_r);
    if (p->min_hits < 1) return fail(ET_ERR_INVALID_ARG, "min_hits = %d < 1", p->min_hits);
    if (p->flags & ~(ET_FLAG_SINGLE_PASS | ET_FLAG_ANGLE_CUT))
        return fail(ET_ERR_INVALID_ARG, "flags = %u: unknown variant bits", p->flags);
    if (p->flags & ET_FLAG_ANGLE_CUT) {
        if (p->cut_base < 0 || p->cut_base > (1 << 21) || p->cut_slope < 0 || p->cut_slope > (1 << 20) ||
            p->cut_tan_max < 0 || p->cut_tan_max > 1024)
            return fail(ET_ERR_INVALID_ARG, "angle cut (%d, %d, %d) outside the limits", p->cut_base,
                        p->cut_slope, p->cut_tan_max);
    }
    if (p->reserved != 0) return fail(ET_ERR_INVALID_ARG, "reserved field must be 0");
    {   // r^2 |w|^2 of a seed (|w_e| < seed_max) must stay below 2^63
        const double rr = (double)p->tube_r * (double)p->tube_r * 3.0 * (double)p->seed_max * (double)p->seed_max;
        if (rr >= 9.2e18)
            return fail(ET_ERR_PRECONDITION, "3 tube_r^2 seed_max^2 = %.3g >= 2^63: the tube bound leaves int64", rr);
    }
    for (int a = 0; a < 3; ++a)
        for (int c = a + 1; c < 3; ++c) {
            long long v = ((long long)p->extent[a] + p->extent[c]) * (long long)p->seed_max;
            if (v >= (1ll << 31))
                return fail(ET_ERR_PRECONDITION,
                            "(extent[%d] + extent[%d]) * seed_max = %lld >= 2^31: cross products leave int32", a,
                            c, v);
        }
    return ET_OK;
}

// ---------------------------------------------------------------- batch

BatchRT::BatchRT(Ctx *c, const et_params &pp) : ctx(c), p(pp) {
    memset(&tune, 0, sizeof tune);
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
}

BatchRT::~BatchRT() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (done) cudaEventDestroy(done);
    for (cudaEvent_t &e : ev)
        if (e) cudaEventDestroy(e);
    for (Group *g : {&g_small, &g_grain, &g_cells, &g_cand, &g_members, &g_out, &g_rec, &g_temp})
        g->release(ctx);
}

// Cells of one batch's cell table (views x cells per view): the kernels index
// it with 32-bit signed arithmetic.
static constexpr double kMaxCells = 2147483647.0;

void BatchRT::choose_cells() {
    for (int k = 0; k < 3; ++k) cs[k] = tune.cell[k];
    if (cs[0] <= 0 || cs[1] <= 0 || cs[2] <= 0) {
        // s0: the edge of a cube holding 0.35 grains at the mean density of the
        // batch; cells are short along the x rows and s0 * 1.1 across them, the
        // region where timed sweeps find the fastest tube walk
        double vol = (double)p.extent[0] * p.extent[1] * p.extent[2];
        double nmean = V > 0 ? (double)N / V : 1.0;
        double rho = std::max(nmean, 1.0) / vol;
        double s = std::cbrt(0.35 / rho);
        s = std::min(std::max(s, 64.0), 4096.0);
        static const double f[3] = {0.22, 1.1, 1.1};
        for (int k = 0; k < 3; ++k)
            if (tune.cell[k] <= 0) cs[k] = std::max(16, (int)std::lround(s * f[k]));
    }
    for (int k = 0; k < 3; ++k) {
        cs[k] = std::max(1, std::min(cs[k], p.extent[k]));
        nc[k] = (p.extent[k] + cs[k] - 1) / cs[k];
    }
    ncell = (long long)nc[0] * nc[1] * nc[2];
    // the second list swaps the x and y cell edges, so its rows (along y) are
    // as short as the first list's rows (along x)
    dual = tune.row_lists != 1;   // 0 (automatic) uses both lists
    csy[0] = std::max(1, std::min(cs[1], p.extent[0]));
    csy[1] = std::max(1, std::min(cs[0], p.extent[1]));
    csy[2] = cs[2];
    for (int k = 0; k < 3; ++k) ncy[k] = (p.extent[k] + csy[k] - 1) / csy[k];
    ncelly = dual ? (long long)ncy[0] * ncy[1] * ncy[2] : 1;
}

// Autotuner: time the whole path for candidate cell shapes around the
// density-based default s0 (about 0.35 grains per cell), each with one and
// with both cell lists, then the seed generator's work-ticket size (origins
// per ticket) for the fastest shape, and keep the fastest combination.
et_status BatchRT::autotune(cudaStream_t st, int max_trials, et_tuning *chosen, float *best_ms) {
    if (!loaded) return fail(ET_ERR_NOT_READY, "no grains loaded");
    if (!st) st = ctx->stream;
    const double vol = (double)p.extent[0] * p.extent[1] * p.extent[2];
    const double nmean = V > 0 ? std::max(1.0, (double)N / V) : 1.0;
    const double s0 = std::cbrt(0.35 * vol / nmean);
    // (x, y, z) factors of s0; rows run along x, so x cells may be short
    static const double cand[][3] = {{0.22, 1.1, 1.1}, {0.33, 1.3, 1.3}, {0.16, 1.1, 1.1}, {0.27, 0.95, 0.95},
                                     {0.22, 1.3, 1.3}, {0.33, 1.1, 1.1}, {0.5, 1.6, 1.3}, {1.0, 1.0, 1.0},
                                     {0.16, 1.22, 1.22}, {0.16, 1.35, 1.1}, {0.18, 1.6, 1.6}};
    const int ncand = (int)(sizeof cand / sizeof cand[0]);
    if (max_trials <= 0 || max_trials > ncand) max_trials = ncand;
    const et_tuning saved = tune;
    const bool saved_prof = profile;
    profile = true;
    float best = 3.0e38f;
    et_tuning best_t = tune;
    // best of two timed runs of the path under tuning t (a negative time: skipped)
    auto trial = [&](const et_tuning &t, float &ms_out) -> et_status {
        ms_out = -1.0f;
        tune = t;
        choose_cells();
        if ((double)V * (double)std::max(ncell, ncelly) >= kMaxCells) return ET_OK;
        et_status s = reserve();
        if (s != ET_OK) return s;
        float t_best = 3.0e38f;
        for (int rep = 0; rep < 2; ++rep) {
            s = enqueue(st, false);
            if (s != ET_OK) return s;
            cudaEventRecord(done, st);
            run_stream = st;
            ran = true;
            profiled_run = true;
            s = settle(false);
            if (s != ET_OK) return s;
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev[0], ev[NSTAGE]) == cudaSuccess) t_best = std::min(t_best, ms);
        }
        ms_out = t_best;
        return ET_OK;
    };
    for (int k = 0; k < 2 * max_trials; ++k) {   // every shape with one and with both cell lists
        et_tuning t = saved;
        for (int a = 0; a < 3; ++a)
            t.cell[a] = std::max(16, std::min(p.extent[a], (int)std::lround(s0 * cand[k / 2][a])));
        t.row_lists = 1 + (k & 1);
        float ms = 0;
        et_status s = trial(t, ms);
        if (s != ET_OK) {
            tune = saved;
            profile = saved_prof;
            return s;
        }
        if (ms >= 0.0f && ms < best) {
            best = ms;
            best_t = t;
        }
    }
    if (saved.ticket_origins == 0) {   // origins per work ticket, for the fastest shape
        const et_tuning shape = best_t;
        for (int o : {1, 2, 4}) {
            et_tuning t = shape;
            t.ticket_origins = o;
            float ms = 0;
            et_status s = trial(t, ms);
            if (s != ET_OK) {
                tune = saved;
                profile = saved_prof;
                return s;
            }
            if (ms >= 0.0f && ms < best) {
                best = ms;
                best_t = t;
            }
        }
    }
    profile = saved_prof;
    if (best_t.ticket_origins == 0) best_t.ticket_origins = 2;   // the automatic choice, made explicit
    tune = best_t;
    choose_cells();
    et_status s = reserve();
    if (s != ET_OK) return s;
    if (chosen) *chosen = best_t;
    if (best_ms) *best_ms = best;
    ran = false;
    return ET_OK;
}

void BatchRT::estimate_caps() {
    const double vol = (double)p.extent[0] * p.extent[1] * p.extent[2];
    const double shell = 4.0 / 3.0 * M_PI *
                         (std::pow((double)p.seed_max, 3) - std::pow((double)p.seed_min, 3));
    const double frac = std::min(1.0, shell / vol);
    const double s = 0.5 * sum_n2 * frac;
    const u64 seeds = (u64)(1.3 * s) + 4096;   // seeds are not stored: they size the candidates
    want_cand = std::max(want_cand, std::max<u64>(65536, seeds / 16));
    want_members = std::max(want_members, want_cand * 24);
}

// Device arrays of one batch, carved out of eight groups (one allocation
// each).  Carving with a null base only measures.
struct DevPtrs {
    Ctl *ctl = nullptr;
    long long *goff = nullptr, *view_trk = nullptr;
    int *xyz_in = nullptr;
    u64 *keys[2] = {nullptr, nullptr};
    u32 *vals[2] = {nullptr, nullptr};
    int4 *gr = nullptr, *gc = nullptr, *gcy = nullptr;
    u64 *gp = nullptr, *gpy = nullptr;
    u64 *best[2] = {nullptr, nullptr};
    int *owner = nullptr;
    u32 *cell_count = nullptr, *cell_start = nullptr, *cell_count_y = nullptr, *cell_start_y = nullptr;
    int *c_lo = nullptr, *c_hi = nullptr;
    u32 *c_cnt = nullptr, *c_nfree = nullptr;
    u64 *c_key = nullptr, *c_moff = nullptr;
    unsigned char *c_state = nullptr;
    int *clist[2] = {nullptr, nullptr};
    int *members = nullptr;
    int *acc = nullptr, *trk_view = nullptr, *out_members = nullptr;
    u64 *sort_k[2] = {nullptr, nullptr};
    u32 *sort_v[2] = {nullptr, nullptr};
    u64 *trk_moff = nullptr;
    et_track *tracks = nullptr;
    int *rec_lo = nullptr, *rec_hi = nullptr, *rec_cnt = nullptr;
    void *temp = nullptr;
};

// Carves group k (0 small, 1 grains, 2 cells, 3 candidates, 4 members,
// 5 outputs, 6 seed records, 7 temporary) out of c; returns its size.
size_t BatchRT::lay_group(int k, char *base, DevPtrs &P) const {
    Carver c{0, base};
    const size_t n = (size_t)std::max<long long>(N, 1);
    const size_t cells = (size_t)V * (size_t)ncell, cellsy = (size_t)V * (size_t)ncelly;
    switch (k) {
    case 0:   // control block, goff, per-view track offsets
        P.ctl = c.take<Ctl>(1);
        P.goff = c.take<long long>(V + 1);
        P.view_trk = c.take<long long>(V + 1);
        break;
    case 1:
        P.xyz_in = c.take<int>(3 * n);
        P.keys[0] = c.take<u64>(n);
        P.keys[1] = c.take<u64>(n);
        P.vals[0] = c.take<u32>(n);
        P.vals[1] = c.take<u32>(n);
        P.gr = c.take<int4>(n);
        // the two cell orders back to back (the y-row list at offset n), so a
        // walk addresses either through one array
        P.gc = c.take<int4>(2 * n);
        P.gcy = P.gc ? P.gc + n : nullptr;
        P.gp = c.take<u64>(2 * n);
        P.gpy = P.gp ? P.gp + n : nullptr;
        P.best[0] = c.take<u64>(n);
        P.best[1] = c.take<u64>(n);
        P.owner = c.take<int>(n);
        break;
    case 2:
        P.cell_count = c.take<u32>(cells);
        P.cell_start = c.take<u32>(cells + 1);
        P.cell_count_y = c.take<u32>(cellsy);
        P.cell_start_y = c.take<u32>(cellsy + 1);
        break;
    case 3: {
        const size_t cc = want_cand;
        P.c_lo = c.take<int>(cc);
        P.c_hi = c.take<int>(cc);
        P.c_cnt = c.take<u32>(cc);
        P.c_key = c.take<u64>(cc);
        P.c_moff = c.take<u64>(cc + 1);
        P.c_state = c.take<unsigned char>(cc);
        P.c_nfree = c.take<u32>(cc);
        P.clist[0] = c.take<int>(cc);
        P.clist[1] = c.take<int>(cc);
        break;
    }
    case 4:
        P.members = c.take<int>(want_members);
        break;
    case 5: {
        const size_t cc = want_cand, sk = std::max<size_t>(cc, n);
        P.acc = c.take<int>(cc);
        P.sort_k[0] = c.take<u64>(sk);
        P.sort_k[1] = c.take<u64>(sk);
        P.sort_v[0] = c.take<u32>(sk);
        P.sort_v[1] = c.take<u32>(sk);
        P.trk_view = c.take<int>(cc);
        P.trk_moff = c.take<u64>(cc + 1);
        P.tracks = c.take<et_track>(cc);
        P.out_members = c.take<int>(n);
        break;
    }
    case 6:
        if (want_rec) {
            P.rec_lo = c.take<int>(want_rec);
            P.rec_hi = c.take<int>(want_rec);
            P.rec_cnt = c.take<int>(want_rec);
        }
        break;
    default: {
        size_t t = 0;
        t = std::max(t, radix_temp_bytes((long long)n));
        t = std::max(t, radix_temp_bytes((long long)std::max<size_t>(want_cand, n)));
        t = std::max(t, scan_temp_bytes((long long)std::max(cells, cellsy) + 1));
        t = std::max(t, scan_temp_bytes((long long)n + 1));
        t = std::max(t, scan_temp_bytes((long long)want_cand + 1));
        t = std::max(t, scan_temp_bytes((long long)V + 1));
        P.temp = c.take<char>(t);
        break;
    }
    }
    return c.off;
}

Group *BatchRT::group(int k) {
    Group *g[NGROUP] = {&g_small, &g_grain, &g_cells, &g_cand, &g_members, &g_out, &g_rec, &g_temp};
    return g[k];
}

void BatchRT::plan_groups(size_t sizes[NGROUP]) const {
    DevPtrs P;
    for (int k = 0; k < NGROUP; ++k) sizes[k] = lay_group(k, nullptr, P);
}

size_t BatchRT::held_bytes() const {
    size_t t = 0;
    for (const Group *g : {&g_small, &g_grain, &g_cells, &g_cand, &g_members, &g_out, &g_rec, &g_temp}) t += g->bytes;
    return t;
}

size_t BatchRT::footprint_with(const size_t sizes[NGROUP]) const {
    const Group *g[NGROUP] = {&g_small, &g_grain, &g_cells, &g_cand, &g_members, &g_out, &g_rec, &g_temp};
    size_t t = 0;
    for (int k = 0; k < NGROUP; ++k) t += std::max(g[k]->bytes, sizes[k]);
    return t;
}

void BatchRT::release_groups() {
    for (int k = 0; k < NGROUP; ++k) group(k)->release(ctx);
}

et_status BatchRT::reserve() {
    size_t sizes[NGROUP];
    plan_groups(sizes);
    if (byte_limit && footprint_with(sizes) > byte_limit)
        return fail(ET_ERR_OOM, "device memory of %zu bytes would exceed the limit of %zu bytes",
                    footprint_with(sizes), byte_limit);
    static const char *what[NGROUP] = {"control block", "grain buffers", "cell tables", "candidates",
                                       "members", "outputs", "seed records", "temp"};
    DevPtrs P;
    for (int k = 0; k < NGROUP; ++k) {
        Group *g = group(k);
        if (sizes[k] == 0) continue;
        if (!g->reserve(ctx, sizes[k])) return fail(ET_ERR_OOM, "%s (%zu bytes)", what[k], sizes[k]);
        lay_group(k, g->base, P);
    }
    ctl = P.ctl;
    goff = P.goff;
    view_trk = P.view_trk;
    xyz_in = P.xyz_in;
    keys[0] = P.keys[0];
    keys[1] = P.keys[1];
    vals[0] = P.vals[0];
    vals[1] = P.vals[1];
    gr = P.gr;
    gc = P.gc;
    gcy = P.gcy;
    gp = P.gp;
    gpy = P.gpy;
    best[0] = P.best[0];
    best[1] = P.best[1];
    owner = P.owner;
    cell_count = P.cell_count;
    cell_start = P.cell_start;
    cell_count_y = P.cell_count_y;
    cell_start_y = P.cell_start_y;
    c_lo = P.c_lo;
    c_hi = P.c_hi;
    c_cnt = P.c_cnt;
    c_key = P.c_key;
    c_moff = P.c_moff;
    c_state = P.c_state;
    c_nfree = P.c_nfree;
    clist[0] = P.clist[0];
    clist[1] = P.clist[1];
    cap_cand = want_cand;
    members = P.members;
    cap_members = g_members.bytes / sizeof(int);
    acc = P.acc;
    sort_k[0] = P.sort_k[0];
    sort_k[1] = P.sort_k[1];
    sort_v[0] = P.sort_v[0];
    sort_v[1] = P.sort_v[1];
    trk_view = P.trk_view;
    trk_moff = P.trk_moff;
    tracks = P.tracks;
    out_members = P.out_members;
    if (want_rec) {
        rec_lo = P.rec_lo;
        rec_hi = P.rec_hi;
        rec_cnt = P.rec_cnt;
        cap_rec = want_rec;
    }
    temp = g_temp.base;
    return ET_OK;
}

// Sizes of the device groups a batch of the given shape would hold, without
// allocating (the served loop's admission).
void BatchRT::plan_shape(int nv, long long n, long long mx, double s2, size_t sizes[NGROUP]) {
    V = nv;
    N = n;
    maxN = mx;
    sum_n2 = s2;
    want_cand = want_members = want_rec = 0;
    choose_cells();
    estimate_caps();
    plan_groups(sizes);
}

unsigned long long BatchRT::layout_generation() const {
    unsigned long long g = 0;
    for (const Group *x : {&g_small, &g_grain, &g_cells, &g_cand, &g_members, &g_out, &g_rec, &g_temp})
        g = g * 1315423911ull + x->generation;
    return g;
}

// Everything a captured launch sequence bakes into its kernel arguments and
// launch shapes: buffer layouts, batch shape, cell grids, capacities.  A
// captured graph is replayed only while this is unchanged.
unsigned long long BatchRT::graph_signature() const {
    unsigned long long h = layout_generation();
    auto mix = [&h](unsigned long long v) { h = (h ^ v) * 0x100000001b3ull + 0x9e3779b97f4a7c15ull; };
    mix((unsigned long long)N);
    mix((unsigned long long)V);
    mix((unsigned long long)maxN);
    for (int k = 0; k < 3; ++k) {
        mix((unsigned long long)cs[k]);
        mix((unsigned long long)nc[k]);
        mix((unsigned long long)csy[k]);
        mix((unsigned long long)ncy[k]);
    }
    mix((unsigned long long)ncell);
    mix((unsigned long long)ncelly);
    mix(dual ? 1ull : 0ull);
    mix(cap_cand);
    mix(cap_members);
    mix(cap_rec);
    mix((unsigned long long)tune.wait_polls);
    mix((unsigned long long)tune.ticket_origins);
    mix((unsigned long long)tune.assoc_window);
    return h;
}

et_status BatchRT::load(const int32_t *xyz, const int64_t *offsets, int nv, bool on_device, cudaStream_t st) {
    if (nv < 0 || !offsets) return fail(ET_ERR_INVALID_ARG, "bad view list");
    if (offsets[0] != 0) return fail(ET_ERR_INVALID_ARG, "offsets[0] must be 0");
    long long mx = 0;
    for (int v = 0; v < nv; ++v) {
        long long n = offsets[v + 1] - offsets[v];
        if (n < 0) return fail(ET_ERR_INVALID_ARG, "offsets must be non-decreasing");
        if (n > (1 << 21) - 1) return fail(ET_ERR_INVALID_ARG, "view %d has %lld grains (max 2^21-1)", v, n);
        mx = std::max(mx, n);
    }
    const long long total = offsets[nv];
    if (total > 0 && !xyz) return fail(ET_ERR_INVALID_ARG, "xyz is NULL");
    if (total >= (1ll << 31) - 1) return fail(ET_ERR_INVALID_ARG, "batch of %lld grains too large", total);
    // canonical key: view | x | y | z
    int cb[3];
    for (int k = 0; k < 3; ++k) cb[k] = bits_for((unsigned long long)(p.extent[k] - 1));
    int vb = bits_for((unsigned long long)std::max(nv - 1, 0));
    if (cb[0] + cb[1] + cb[2] + vb > 64) return fail(ET_ERR_INVALID_ARG, "too many views for the key width");
    V = nv;
    N = total;
    maxN = mx;
    goff_h.assign(offsets, offsets + nv + 1);
    sum_n2 = 0;
    for (int v = 0; v < nv; ++v) sum_n2 += (double)(offsets[v + 1] - offsets[v]) * (double)(offsets[v + 1] - offsets[v]);
    for (int k = 0; k < 3; ++k) cbits[k] = cb[k];
    choose_cells();
    if ((double)V * (double)std::max(ncell, ncelly) >= kMaxCells)
        return fail(ET_ERR_INVALID_ARG, "cell table of %.3g cells too large (limit 2^31 - 1)",
                    (double)V * (double)std::max(ncell, ncelly));
    estimate_caps();
    et_status s = reserve();
    if (s != ET_OK) return s;
    cudaError_t e = cudaMemcpyAsync(goff, goff_h.data(), sizeof(long long) * (V + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && N > 0)
        e = cudaMemcpyAsync(xyz_in, xyz, sizeof(int) * 3 * (size_t)N,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "grain upload");
    loaded = true;
    ran = false;
    return ET_OK;
}

Batch BatchRT::dev_batch() const {
    Batch b;
    memset(&b, 0, sizeof b);
    b.V = V;
    b.N = (int)N;
    b.goff = goff;
    for (int k = 0; k < 3; ++k) {
        b.ext[k] = p.extent[k];
        b.cs[k] = cs[k];
        b.nc[k] = nc[k];
        b.ics[k] = 1.0f / (float)cs[k];
        b.cbits[k] = cbits[k];
    }
    b.smin = p.seed_min;
    b.smax = p.seed_max;
    b.r = p.tube_r;
    b.H = p.min_hits;
    b.smin2 = (long long)p.seed_min * p.seed_min;
    b.smax2 = (long long)p.seed_max * p.seed_max;
    b.r2 = (long long)p.tube_r * p.tube_r;
    b.flags = p.flags;
    b.spin_limit = tune.wait_polls > 0 ? (long long)tune.wait_polls : 0;
    b.gen_origins = tune.ticket_origins > 0 ? tune.ticket_origins : 2;
    const bool cut = (p.flags & ET_FLAG_ANGLE_CUT) != 0;
    b.cut_base = cut ? p.cut_base : 0;
    b.cut_slope = cut ? p.cut_slope : 0;
    b.cut_tmax = cut ? p.cut_tan_max : 0;
    b.ncell = (int)ncell;
    for (int k = 0; k < 3; ++k) {
        b.csy[k] = csy[k];
        b.ncy[k] = ncy[k];
        b.icsy[k] = 1.0f / (float)csy[k];
    }
    b.ncelly = (int)ncelly;
    b.dual = dual ? 1 : 0;
    b.gcy = gcy;
    b.gpy = gpy;
    b.cell_start_y = cell_start_y;
    b.vshift = cbits[0] + cbits[1] + cbits[2];
    b.rbits = std::max(1, bits_for((unsigned long long)maxN));
    b.xyz_in = xyz_in;
    b.gr = gr;
    b.gc = gc;
    b.gp = gp;
    b.cell_start = cell_start;
    b.ctl = ctl;
    return b;
}

Work BatchRT::dev_work() const {
    Work w;
    memset(&w, 0, sizeof w);
    w.c_lo = c_lo;
    w.c_hi = c_hi;
    w.c_cnt = c_cnt;
    w.c_key = c_key;
    w.c_moff = c_moff;
    w.c_state = c_state;
    w.c_nfree = c_nfree;
    w.cand_cap = cap_cand;
    w.members = members;
    w.member_cap = cap_members;
    w.best[0] = best[0];
    w.best[1] = best[1];
    w.owner = owner;
    w.clist[0] = clist[0];
    w.clist[1] = clist[1];
    w.rec_lo = rec_lo;
    w.rec_hi = rec_hi;
    w.rec_cnt = rec_cnt;
    w.rec_cap = cap_rec;
    return w;
}

Out BatchRT::dev_out() const {
    Out o;
    memset(&o, 0, sizeof o);
    o.acc = acc;
    o.acc_cap = cap_cand;
    o.sort_k[0] = sort_k[0];
    o.sort_k[1] = sort_k[1];
    o.sort_v[0] = sort_v[0];
    o.sort_v[1] = sort_v[1];
    o.trk_view = trk_view;
    o.trk_moff = trk_moff;
    o.view_trk = view_trk;
    o.tracks = tracks;
    o.out_members = out_members;
    o.out_member_cap = (u64)std::max<long long>(N, 1);
    return o;
}

et_status BatchRT::enqueue(cudaStream_t st, bool record) {
    const Batch b = dev_batch();
    const Work w = dev_work();
    Out o = dev_out();
    const long long n = N;
    const size_t cells = (size_t)V * (size_t)ncell;
    mark(0, st);
    cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
    if (n > 0) {
        cudaMemsetAsync(cell_count, 0, sizeof(u32) * cells, st);
        launch_canonical_keys(b, keys[0], vals[0], st);
        const int kb = b.vshift + bits_for((unsigned long long)std::max(V - 1, 0));
        int c1 = radix_sort_pairs(keys[0], vals[0], keys[1], vals[1], n, kb, temp, st, &ctl->error, ERRB_TIMEOUT,
                                  ctl->bar, b.spin_limit);
        u32 *sv = vals[c1], *cell_of = vals[c1 ^ 1];
        launch_canonical_order(b, keys[c1], sv, cell_of, cell_count, st);
        // cell list by counting sort: starts from the counts, then the counts
        // are zeroed and serve as per-cell cursors of the scatter
        exclusive_scan_u32(cell_count, cell_start, (long long)cells, temp, st, &ctl->error, ERRB_TIMEOUT, ctl->bar,
                           b.spin_limit);
        cudaMemsetAsync(cell_count, 0, sizeof(u32) * cells, st);
        launch_cell_scatter(b, cell_of, cell_start, cell_count, 0, st);
        if (dual) {   // second cell list (rows along y) from the same canonical order
            const size_t cellsy = (size_t)V * (size_t)ncelly;
            cudaMemsetAsync(cell_count_y, 0, sizeof(u32) * cellsy, st);
            launch_y_cells(b, cell_of, cell_count_y, st);
            exclusive_scan_u32(cell_count_y, cell_start_y, (long long)cellsy, temp, st, &ctl->error, ERRB_TIMEOUT,
                               ctl->bar, b.spin_limit);
            cudaMemsetAsync(cell_count_y, 0, sizeof(u32) * cellsy, st);
            launch_cell_scatter(b, cell_of, cell_start_y, cell_count_y, 1, st);
        }
        mark(1, st);   // seeds are generated inside the tube-count kernel: stage 1 stays empty
        mark(2, st);
        launch_tube_count(b, w, record ? 1 : 0, st);
        mark(3, st);
        const bool sp = (p.flags & ET_FLAG_SINGLE_PASS) != 0;
        launch_cand_keys(b, w, sp ? nullptr : o.sort_k[0], sp ? nullptr : o.sort_v[0], st);
        exclusive_scan_u64_dev(c_moff, c_moff, (long long)cap_cand, &ctl->n_cand, temp, &ctl->n_members, st,
                               &ctl->error, ERRB_TIMEOUT, ctl->bar, b.spin_limit);
        launch_member_fill(b, w, st);
        cudaMemsetAsync(best[0], 0xFF, sizeof(u64) * n, st);
        cudaMemsetAsync(best[1], 0xFF, sizeof(u64) * n, st);
        cudaMemsetAsync(owner, 0xFF, sizeof(int) * n, st);
        mark(4, st);
        if (p.flags & ET_FLAG_SINGLE_PASS) {
            launch_single_pass(b, w, st);
        } else {
            Work wm = w;
            wm.corder = launch_cand_order(b, w, o, temp, st);
            wm.window = tune.assoc_window > 0 ? (u64)tune.assoc_window : 0;
            cudaError_t e = launch_merge_coop(b, wm, ctx->merge_grid, st);
            if (e != cudaSuccess) return cuda_fail(e, "merge launch");
        }
        mark(5, st);
        launch_output(b, w, o, (long long)cap_cand, std::max<long long>(n, 1), temp, st);
        mark(6, st);
    } else {
        cudaMemsetAsync(view_trk, 0, sizeof(long long) * (V + 1), st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return ET_OK;
}

et_status BatchRT::find(cudaStream_t st, bool use_graph) {
    if (!loaded) return fail(ET_ERR_NOT_READY, "no grains loaded");
    if (!st) st = ctx->stream;
    et_status s;
    if (use_graph && N > 0) {
        const unsigned long long key = graph_signature() ^ (profile ? 0x8000000000000000ull : 0ull);
        if (!gexec || key != graph_key) {
            if (gexec) {
                cudaGraphExecDestroy(gexec);
                gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "begin capture");
            s = enqueue(st, false);
            e = cudaStreamEndCapture(st, &g);
            if (s != ET_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            graph_key = key;
        }
        cudaError_t e = cudaGraphLaunch(gexec, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    } else {
        s = enqueue(st, false);
        if (s != ET_OK) return s;
    }
    cudaError_t e = cudaEventRecord(done, st);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    run_stream = st;
    ran = true;
    profiled_run = profile;
    return ET_OK;
}

et_status BatchRT::read_ctl(Ctl &h) {
    cudaError_t e = cudaEventSynchronize(done);
    if (e != cudaSuccess) return cuda_fail(e, "wait for the view");
    e = cudaMemcpy(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read control block");
    return ET_OK;
}

// Waits; on internal overflow grows the buffers and runs again (synchronously).
et_status BatchRT::settle(bool record) {
    if (!ran) return fail(ET_ERR_NOT_READY, "et_track_find was not called");
    for (int attempt = 0;; ++attempt) {
        et_status s = read_ctl(hctl);
        if (s != ET_OK) return s;
        if (hctl.error & ERRB_OUT_OF_RANGE) return fail(ET_ERR_OUT_OF_RANGE, "a grain lies outside [0, extent)");
        if (hctl.error & ERRB_DUPLICATE) return fail(ET_ERR_DUPLICATE_GRAIN, "two grains share coordinates");
        if (hctl.error & ERRB_TIMEOUT) return fail(ET_ERR_TIMEOUT, "device-side wait timed out (merge barrier or sort look-back)");
        if (!(hctl.error & ERRB_OVF_MASK)) return ET_OK;
        if (attempt >= 6) return fail(ET_ERR_CAPACITY, "internal buffers kept overflowing");
        if (hctl.error & ERRB_OVF_CAND) {
            want_cand = std::max<u64>(want_cand, hctl.n_cand + 1024);
            want_members = std::max<u64>(want_members, want_cand * 24);
        }
        if (hctl.error & ERRB_OVF_MEMBERS) want_members = std::max<u64>(want_members, hctl.n_members + 1024);
        if (hctl.error & ERRB_OVF_RECORD) want_rec = std::max<u64>(want_rec, hctl.n_seeds);
        s = reserve();
        if (s != ET_OK) return s;
        s = enqueue(ctx->stream, record);
        if (s != ET_OK) return s;
        cudaError_t e = cudaEventRecord(done, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
        run_stream = ctx->stream;
    }
}

et_status BatchRT::fetch(int64_t *view_off, et_track *out, int64_t cap, int64_t *n_tracks, int32_t *mem,
                         int64_t mcap, int64_t *n_members) {
    et_status s = settle(false);
    if (s != ET_OK) return s;
    const int64_t nt = (int64_t)hctl.n_acc, nm = (int64_t)hctl.n_out_members;
    if (n_tracks) *n_tracks = nt;
    if (n_members) *n_members = nm;
    if ((nt > 0 && (!out || cap < nt)) || (nm > 0 && (!mem || mcap < nm)))
        return fail(ET_ERR_CAPACITY, "need %lld tracks / %lld members", (long long)nt, (long long)nm);
    cudaError_t e = cudaSuccess;
    if (nt > 0) e = cudaMemcpy(out, tracks, sizeof(et_track) * nt, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nm > 0) e = cudaMemcpy(mem, out_members, sizeof(int) * nm, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && view_off) {
        std::vector<long long> tmp(V + 1);
        e = cudaMemcpy(tmp.data(), view_trk, sizeof(long long) * (V + 1), cudaMemcpyDeviceToHost);
        for (int v = 0; v <= V; ++v) view_off[v] = tmp[v];
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy results");
    return ET_OK;
}

et_status BatchRT::seed_counts(int32_t *si, int32_t *sj, int32_t *cnt, int64_t cap, int64_t *n_seeds) {
    et_status s = settle(false);
    if (s != ET_OK) return s;
    const u64 ns = hctl.n_seeds;
    if (n_seeds) *n_seeds = (int64_t)ns;
    if (ns > 0 && (!si || !sj || !cnt || (u64)cap < ns))
        return fail(ET_ERR_CAPACITY, "need %llu seed records", (unsigned long long)ns);
    want_rec = std::max<u64>(want_rec, ns + 1);
    s = reserve();
    if (s != ET_OK) return s;
    s = enqueue(ctx->stream, true);
    if (s != ET_OK) return s;
    cudaEventRecord(done, ctx->stream);
    run_stream = ctx->stream;
    s = settle(true);
    if (s != ET_OK) return s;
    cudaError_t e = cudaSuccess;
    if (ns > 0) {
        e = cudaMemcpy(si, rec_lo, sizeof(int) * ns, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sj, rec_hi, sizeof(int) * ns, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cnt, rec_cnt, sizeof(int) * ns, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy seed records");
    return ET_OK;
}

void BatchRT::mark(int stage, cudaStream_t st) {
    if (!profile) return;
    if (!ev[stage]) cudaEventCreate(&ev[stage]);
    // inside stream capture a plain record only expresses a dependency; an
    // external record becomes an event node that fires on every replay
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[stage], st, cudaEventRecordExternal);
    else cudaEventRecord(ev[stage], st);
}

// Number of kernels in one run of the path: capture the launch sequence into
// a graph that is never executed and count its kernel nodes.
int BatchRT::count_kernels() {
    const unsigned long long key = graph_signature();
    if (kernel_launches >= 0 && key == launches_key) return kernel_launches;
    if (!loaded || N == 0) return 0;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -1;
    const bool prof = profile;
    profile = false;
    cudaGraph_t g = nullptr;
    int count = -1;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        et_status s = enqueue(st, false);
        cudaStreamEndCapture(st, &g);
        if (s == ET_OK && g) {
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(g, nodes.data(), &nn);
            count = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++count;
            }
        }
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    profile = prof;
    cudaStreamDestroy(st);
    kernel_launches = count;
    launches_key = key;
    return count;
}

void BatchRT::stats(et_stats *o) {
    memset(o, 0, sizeof *o);
    o->n_grains = N;
    o->n_seeds = (int64_t)hctl.n_seeds;
    o->n_tests = (int64_t)hctl.n_tests;
    o->n_hits = (int64_t)hctl.n_hits;
    o->n_candidates = (int64_t)hctl.n_cand;
    o->n_members = (int64_t)hctl.n_members;
    o->n_tracks = (int64_t)hctl.n_acc;
    o->n_track_members = (int64_t)hctl.n_out_members;
    o->n_pair_tests = (int64_t)hctl.n_pair_tests;
    o->merge_rounds = (int32_t)hctl.rounds;
    for (int k = 0; k < 3; ++k) o->cell[k] = cs[k];
    o->kernel_launches = count_kernels();
    o->profiled = 0;
    if (profiled_run && ran) {
        cudaEventSynchronize(done);
        bool ok = true;
        for (int k = 0; k < NSTAGE; ++k) {
            float ms = 0;
            if (!ev[k] || !ev[k + 1] || cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) ok = false;
            o->stage_ms[k] = ms;
        }
        cudaGetLastError();
        o->profiled = ok ? 1 : 0;
    }
}

}  // namespace et

// ==================================================================== C ABI

using namespace et;

extern "C" {

int32_t et_abi_version(void) { return ET_ABI_VERSION; }

const char *et_last_error(void) { return last_error(); }

const char *et_status_string(et_status s) {
    switch (s) {
    case ET_OK: return "ok";
    case ET_ERR_INVALID_ARG: return "invalid argument";
    case ET_ERR_OUT_OF_RANGE: return "coordinate out of range";
    case ET_ERR_DUPLICATE_GRAIN: return "duplicate grain";
    case ET_ERR_PRECONDITION: return "parameters break the int32 cross-product bound";
    case ET_ERR_CAPACITY: return "buffer too small";
    case ET_ERR_OOM: return "out of device memory";
    case ET_ERR_BUSY: return "busy";
    case ET_ERR_TIMEOUT: return "device wait timed out";
    case ET_ERR_CUDA: return "CUDA error";
    case ET_ERR_NOT_READY: return "not ready";
    default: return "unknown status";
    }
}

et_status et_ctx_create(int device, et_ctx **out) {
    GUARD_BEGIN
    if (!out) return fail(ET_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(ET_ERR_CUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    if (device < 0 || device >= n) return fail(ET_ERR_INVALID_ARG, "device %d of %d", device, n);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    et_ctx *c = new et_ctx();
    c->device = device;
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "stream create");
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    c->merge_grid = merge_grid_blocks(device);
    init_scan_sort();
    *out = c;
    return ET_OK;
    GUARD_END
}

et_status et_ctx_destroy(et_ctx *ctx) {
    if (!ctx) return fail(ET_ERR_INVALID_ARG, "ctx is NULL");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ET_OK;
}

et_status et_ctx_set_allocator(et_ctx *ctx, et_alloc_fn alloc, et_free_fn free_fn, void *user) {
    if (!ctx) return fail(ET_ERR_INVALID_ARG, "ctx is NULL");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(ET_ERR_INVALID_ARG, "give both hooks or none");
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    return ET_OK;
}

et_status et_ctx_info(et_ctx *ctx, int32_t *sm_count, int32_t *cc_major, int32_t *cc_minor) {
    if (!ctx) return fail(ET_ERR_INVALID_ARG, "ctx is NULL");
    if (sm_count) *sm_count = ctx->sms;
    if (cc_major) *cc_major = ctx->cc_major;
    if (cc_minor) *cc_minor = ctx->cc_minor;
    return ET_OK;
}

et_status et_batch_create(et_ctx *ctx, const et_params *params, et_batch **out) {
    GUARD_BEGIN
    if (!ctx || !out) return fail(ET_ERR_INVALID_ARG, "ctx/out is NULL");
    *out = nullptr;
    et_status s = check_params(params);
    if (s != ET_OK) return s;
    cudaSetDevice(ctx->device);
    *out = new et_batch(ctx, *params);
    return ET_OK;
    GUARD_END
}

et_status et_batch_destroy(et_batch *b) {
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    if (b->ran) cudaEventSynchronize(b->done);
    delete b;
    return ET_OK;
}

et_status et_batch_load(et_batch *b, const int32_t *xyz, const int64_t *offsets, int32_t n_views,
                        int32_t on_device, void *stream) {
    GUARD_BEGIN
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : b->ctx->stream;
    if (b->ran) cudaEventSynchronize(b->done);   // buffers may be reused
    return b->load(xyz, offsets, n_views, on_device != 0, st);
    GUARD_END
}

et_status et_batch_set_tuning(et_batch *b, const et_tuning *t) {
    if (!b || !t) return fail(ET_ERR_INVALID_ARG, "batch/tuning is NULL");
    for (int k = 0; k < 3; ++k)
        if (t->cell[k] < 0) return fail(ET_ERR_INVALID_ARG, "cell[%d] < 0", k);
    if (t->assoc_window < 0) return fail(ET_ERR_INVALID_ARG, "assoc_window < 0");
    if (t->wait_polls < 0) return fail(ET_ERR_INVALID_ARG, "wait_polls < 0");
    if (t->ticket_origins != 0 && t->ticket_origins != 1 && t->ticket_origins != 2 && t->ticket_origins != 4)
        return fail(ET_ERR_INVALID_ARG, "ticket_origins = %d: 0, 1, 2 or 4", t->ticket_origins);
    b->tune = *t;
    b->loaded = false;   // the cell grid changes: reload required
    return ET_OK;
}

et_status et_batch_autotune(et_batch *b, void *stream, int32_t max_trials, et_tuning *chosen, float *best_ms) {
    GUARD_BEGIN
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    return b->autotune((cudaStream_t)stream, max_trials, chosen, best_ms);
    GUARD_END
}

et_status et_batch_find(et_batch *b, void *stream, int32_t use_graph) {
    GUARD_BEGIN
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    return b->find((cudaStream_t)stream, use_graph != 0);
    GUARD_END
}

et_status et_batch_fetch(et_batch *b, int64_t *view_track_offsets, et_track *tracks, int64_t cap,
                         int64_t *n_tracks, int32_t *members, int64_t member_cap, int64_t *n_members) {
    GUARD_BEGIN
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    return b->fetch(view_track_offsets, tracks, cap, n_tracks, members, member_cap, n_members);
    GUARD_END
}

et_status et_batch_sync(et_batch *b) {
    GUARD_BEGIN
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    return b->settle(false);
    GUARD_END
}

et_status et_batch_stats(et_batch *b, et_stats *out) {
    GUARD_BEGIN
    if (!b || !out) return fail(ET_ERR_INVALID_ARG, "batch/out is NULL");
    cudaSetDevice(b->ctx->device);
    b->stats(out);
    return ET_OK;
    GUARD_END
}

et_status et_batch_set_profiling(et_batch *b, int32_t on) {
    if (!b) return fail(ET_ERR_INVALID_ARG, "batch is NULL");
    b->profile = on != 0;
    return ET_OK;
}

// ---- views: batches of one

et_status et_view_create(et_ctx *ctx, const int32_t *xyz, int64_t n, const et_params *params, et_view **out) {
    if (n < 0) return fail(ET_ERR_INVALID_ARG, "n < 0");
    et_status s = et_batch_create(ctx, params, out);
    if (s != ET_OK) return s;
    int64_t off[2] = {0, n};
    s = et_batch_load(*out, xyz, off, 1, 0, nullptr);
    if (s == ET_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);   // the caller may free xyz on return
        if (e != cudaSuccess) s = cuda_fail(e, "grain upload");
    }
    if (s != ET_OK) {
        et_batch_destroy(*out);
        *out = nullptr;
    }
    return s;
}

et_status et_view_create_device(et_ctx *ctx, const int32_t *d_xyz, int64_t n, const et_params *params,
                                et_view **out) {
    if (n < 0) return fail(ET_ERR_INVALID_ARG, "n < 0");
    et_status s = et_batch_create(ctx, params, out);
    if (s != ET_OK) return s;
    int64_t off[2] = {0, n};
    s = et_batch_load(*out, d_xyz, off, 1, 1, nullptr);
    if (s != ET_OK) {
        et_batch_destroy(*out);
        *out = nullptr;
    }
    return s;
}

et_status et_view_load(et_view *view, const int32_t *xyz, int64_t n, void *stream) {
    if (n < 0) return fail(ET_ERR_INVALID_ARG, "n < 0");
    int64_t off[2] = {0, n};
    return et_batch_load(view, xyz, off, 1, 0, stream);
}

et_status et_view_destroy(et_view *view) { return et_batch_destroy(view); }

et_status et_track_find(et_view *view, void *stream) { return et_batch_find(view, stream, 0); }

et_status et_track_fetch(et_view *view, et_track *tracks, int64_t cap, int64_t *n_tracks, int32_t *members,
                         int64_t member_cap, int64_t *n_members) {
    return et_batch_fetch(view, nullptr, tracks, cap, n_tracks, members, member_cap, n_members);
}

et_status et_view_seed_counts(et_view *view, int32_t *seed_i, int32_t *seed_j, int32_t *count, int64_t cap,
                              int64_t *n_seeds) {
    GUARD_BEGIN
    if (!view) return fail(ET_ERR_INVALID_ARG, "view is NULL");
    cudaSetDevice(view->ctx->device);
    return view->seed_counts(seed_i, seed_j, count, cap, n_seeds);
    GUARD_END
}

}  // extern "C"

// runtime.h -- host-side objects behind the C ABI (include/et.h).
#pragma once
#include <vector>

#include "common.cuh"
#include "et.h"

namespace et {

et_status fail(et_status s, const char *fmt, ...);
et_status cuda_fail(cudaError_t e, const char *what);
et_status check_params(const et_params *p);
int bits_for(unsigned long long maxval);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carves consecutive 256-byte aligned slices out of one allocation.
struct Carver {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count) {
        size_t o = off;
        off = align_up(off + count * sizeof(T), 256);
        return base ? (T *)(base + o) : nullptr;
    }
};


struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 0, cc_major = 0, cc_minor = 0;
    int merge_grid = 0;
    et_alloc_fn alloc = nullptr;
    et_free_fn free_fn = nullptr;
    void *user = nullptr;
    void *dalloc(size_t bytes);
    void dfree(void *p);
};

// One device allocation that is carved into arrays; reallocated only to grow.
struct Group {
    char *base = nullptr;
    size_t bytes = 0;
    unsigned long long generation = 0;
    bool reserve(Ctx *ctx, size_t need);
    void release(Ctx *ctx);
};

struct DevPtrs;

// A batch of views sharing one et_params (a view is a batch of one).
struct BatchRT {
    static constexpr int NGROUP = 8;
    Ctx *ctx;
    et_params p;
    et_tuning tune;
    // shape
    int V = 0;
    long long N = 0, maxN = 0;
    double sum_n2 = 0;   // sum over views of (grains)^2: sizes the candidate buffers
    std::vector<long long> goff_h;
    int cs[3] = {1, 1, 1}, nc[3] = {1, 1, 1}, cbits[3] = {0, 0, 0};
    long long ncell = 1;
    int csy[3] = {1, 1, 1}, ncy[3] = {1, 1, 1};   // second cell list (rows along y)
    long long ncelly = 1;
    bool dual = false;
    // requested capacities
    u64 want_cand = 0, want_members = 0, want_rec = 0;
    // granted capacities
    u64 cap_cand = 0, cap_members = 0, cap_rec = 0;
    // device bytes the groups may hold together after a reserve (0: no limit);
    // a reserve beyond it fails with ET_ERR_OOM
    size_t byte_limit = 0;
    // device memory
    Group g_small, g_grain, g_cells, g_cand, g_members, g_out, g_rec, g_temp;
    Ctl *ctl = nullptr;
    long long *goff = nullptr, *view_trk = nullptr;
    int *xyz_in = nullptr;
    u64 *keys[2] = {nullptr, nullptr};
    u32 *vals[2] = {nullptr, nullptr};
    int4 *gr = nullptr, *gc = nullptr;
    u64 *gp = nullptr, *gpy = nullptr;
    u64 *best[2] = {nullptr, nullptr};
    int *owner = nullptr;
    int *clist[2] = {nullptr, nullptr};
    u32 *cell_count = nullptr, *cell_start = nullptr;
    u32 *cell_count_y = nullptr, *cell_start_y = nullptr;
    int4 *gcy = nullptr;
    int *c_lo = nullptr, *c_hi = nullptr;
    u32 *c_cnt = nullptr, *c_nfree = nullptr;
    u64 *c_key = nullptr, *c_moff = nullptr;
    unsigned char *c_state = nullptr;
    int *members = nullptr;
    int *acc = nullptr, *trk_view = nullptr, *out_members = nullptr;
    u64 *sort_k[2] = {nullptr, nullptr};
    u32 *sort_v[2] = {nullptr, nullptr};
    u64 *trk_moff = nullptr;
    et_track *tracks = nullptr;
    int *rec_lo = nullptr, *rec_hi = nullptr, *rec_cnt = nullptr;
    void *temp = nullptr;
    // run state
    cudaEvent_t done = nullptr;
    cudaStream_t run_stream = nullptr;
    bool loaded = false, ran = false;
    Ctl hctl{};
    cudaGraphExec_t gexec = nullptr;
    unsigned long long graph_key = 0;
    // profiling
    static constexpr int NSTAGE = 6;
    bool profile = false, profiled_run = false;
    cudaEvent_t ev[NSTAGE + 1] = {};
    int kernel_launches = -1;
    unsigned long long launches_key = 0;

    BatchRT(Ctx *c, const et_params &pp);
    ~BatchRT();
    void choose_cells();
    et_status autotune(cudaStream_t st, int max_trials, et_tuning *chosen, float *best_ms);
    void estimate_caps();
    size_t lay_group(int k, char *base, DevPtrs &P) const;
    Group *group(int k);
    void plan_groups(size_t sizes[NGROUP]) const;
    size_t held_bytes() const;
    size_t footprint_with(const size_t sizes[NGROUP]) const;
    void release_groups();
    void plan_shape(int nv, long long n, long long mx, double s2, size_t sizes[NGROUP]);
    et_status reserve();
    unsigned long long layout_generation() const;
    unsigned long long graph_signature() const;
    et_status load(const int32_t *xyz, const int64_t *offsets, int nv, bool on_device, cudaStream_t st);
    Batch dev_batch() const;
    Work dev_work() const;
    Out dev_out() const;
    et_status enqueue(cudaStream_t st, bool record);
    et_status find(cudaStream_t st, bool use_graph);
    et_status read_ctl(Ctl &h);
    et_status settle(bool record);
    et_status fetch(int64_t *view_off, et_track *out, int64_t cap, int64_t *n_tracks, int32_t *mem,
                    int64_t mcap, int64_t *n_members);
    et_status seed_counts(int32_t *si, int32_t *sj, int32_t *cnt, int64_t cap, int64_t *n_seeds);
    void stats(et_stats *o);
    void mark(int stage, cudaStream_t st);
    int count_kernels();
};

}  // namespace et

// Opaque handles of the C ABI.
struct et_ctx : public et::Ctx {};
struct et_batch : public et::BatchRT {
    using et::BatchRT::BatchRT;
};

#define GUARD_BEGIN try {
#define GUARD_END                                                        \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        return et::fail(ET_ERR_OOM, "host allocation failed");           \
    }                                                                    \
    catch (...) {                                                        \
        return et::fail(ET_ERR_CUDA, "unexpected exception in the runtime"); \
    }

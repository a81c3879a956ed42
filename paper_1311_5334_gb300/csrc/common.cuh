// common.cuh -- device-side structures shared by the kernel translation units
// of libet (grain-pair seeded straight-line track finding, Section 2 of the
// paper).  Host code sees these through the launcher declarations at the end.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "et.h"   // ET_FLAG_* variant bits

namespace et {

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------- error bits
enum : u32 {
    ERRB_OUT_OF_RANGE = 1u << 0,
    ERRB_DUPLICATE = 1u << 1,
    ERRB_OVF_CAND = 1u << 3,
    ERRB_OVF_MEMBERS = 1u << 4,
    ERRB_TIMEOUT = 1u << 5,
    ERRB_OVF_RECORD = 1u << 6,
    ERRB_INPUT_MASK = ERRB_OUT_OF_RANGE | ERRB_DUPLICATE,
    ERRB_OVF_MASK = ERRB_OVF_CAND | ERRB_OVF_MEMBERS | ERRB_OVF_RECORD,
};

// Candidate states during the merge.
enum : unsigned char { CS_UNDECIDED = 0, CS_ACCEPTED = 1, CS_REJECTED = 2 };

// Device control block: counters written by the kernels, read back by the host.
struct Ctl {
    u64 n_seeds;        // seeds generated (inside the tube-count kernel)
    u64 n_tests;        // tube tests performed
    u64 n_hits;         // sum of counts over seeds
    u64 n_cand;         // candidates appended (may exceed capacity -> overflow bit)
    u64 n_members;      // sum of candidate counts (scan result)
    u64 n_acc;          // accepted tracks
    u64 n_out_members;  // members of accepted tracks
    u64 n_record;       // per-seed records written (diagnostic path)
    u32 error;          // ERRB_* bits
    u32 rounds;         // merge rounds run
    u32 bar[2];         // grid barrier of the cooperative kernels: arrivals, generation
    u32 active[2];      // merge: participants per round (ping-pong)
    u32 pad[2];
    u64 ncl[2];         // merge: lengths of the undecided-candidate lists (ping-pong)
    u32 round_active[64];   // merge: participants of the first 64 rounds (diagnostics)
    u64 ticket[2];          // work tickets of the tube-count and member-list kernels
    u64 n_pair_tests;       // seed-window tests of the seed generator
};

// Everything a kernel needs to know about the batch.  Passed by value.
struct Batch {
    int V;               // views
    int N;               // grains in all views
    const long long *goff;   // V + 1 grain offsets (device)
    // parameters
    int ext[3];
    int smin, smax, r, H;
    long long smin2, smax2, r2;
    unsigned flags;          // ET_FLAG_* variants
    long long spin_limit;    // polls before a bounded device wait gives up (0: defaults)
    int gen_origins;         // origins per work ticket of the seed generator (1, 2 or 4)
    int cut_base, cut_slope, cut_tmax;   // angle cut (ET_FLAG_ANGLE_CUT)
    // cell grid (identical for all views)
    int cs[3];           // cell edge per axis
    int nc[3];           // cells per axis
    float ics[3];        // 1 / cs
    int ncell;           // cells per view
    int cbits[3];        // bit widths of x, y, z in the canonical key
    int vshift;          // bit position of the view index in the canonical key
    int rbits;           // bit width of a per-view rank or count (largest view's grain count)
    // arrays
    const int *xyz_in;   // N x 3 input, caller order
    int4 *gr;            // canonical order: x, y, z, caller index within the view
    int4 *gc;            // cell order: x, y, z, canonical (global) index; the y-row
                         // list's order follows at gc + N (gcy)
    u64 *gp;             // cell order: x | y << 21 | z << 42 (the tube counts' 8-byte grain loads)
    u32 *cell_start;     // V * ncell + 1
    // second cell list with rows along y: cell edges (cs[1], cs[0], cs[2]),
    // index cy + ncy[1] * (cx + ncy[0] * cz); lines whose |w_y| > |w_x| walk it
    int dual;            // 1 if the second list is built and used
    int csy[3], ncy[3];
    float icsy[3];
    int ncelly;
    int4 *gcy;
    u64 *gpy;
    u32 *cell_start_y;   // V * ncelly + 1
    Ctl *ctl;
};

// Candidates (seeds are generated and walked inside the tube-count kernel).
struct Work {
    // candidates
    int *c_lo, *c_hi;    // canonical global indices
    u32 *c_cnt;          // tube count
    u64 *c_key;          // (2^21-1-count) << 42 | rank_lo << 21 | rank_hi
    u64 *c_moff;         // member offsets, cap + 1
    unsigned char *c_state;
    u32 *c_nfree;        // unused grains when accepted
    u64 cand_cap;
    int *members;        // canonical global indices
    u64 member_cap;
    // merge
    u64 *best[2];        // per grain
    int *owner;          // per grain: accepting candidate or -1
    int *clist[2];       // undecided candidates carried to the next round (cand_cap each)
    const u32 *corder;   // candidates in key order (the association's windows)
    u64 window;          // candidates per window (0: automatic)
    // diagnostic per-seed record (optional)
    int *rec_lo, *rec_hi, *rec_cnt;
    u64 rec_cap;
};

// Output stage.
struct Out {
    int *acc;            // accepted candidate ids, later sorted by (view, key)
    u64 acc_cap;
    u64 *sort_k[2];      // scratch keys for sorting the accepted list / members
    u32 *sort_v[2];
    int *trk_view;       // view of each accepted track (sorted order)
    u64 *trk_moff;       // member offsets of accepted tracks (sorted order), cap + 1
    long long *view_trk; // V + 1 track offsets
    void *tracks;        // et_track[acc_cap]
    int *out_members;    // caller indices, sorted within each track
    u64 out_member_cap;
};

__device__ __forceinline__ int view_of(const long long *goff, int V, long long g) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (goff[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Coordinates (each below 2^21) packed into 8 bytes and back.
__device__ __forceinline__ u64 pack_xyz(int x, int y, int z) {
    return (u64)(unsigned)x | ((u64)(unsigned)y << 21) | ((u64)(unsigned)z << 42);
}
__device__ __forceinline__ int4 unpack_xyz(u64 p) {
    return make_int4((int)(p & 0x1fffffu), (int)((p >> 21) & 0x1fffffu), (int)(p >> 42), 0);
}

// Sort key of a candidate key (2^21 - 1 - count) << 42 | rank_lo << 21 |
// rank_hi, in the same order but on 3 * rbits bits: fewer radix passes.
__device__ __forceinline__ u64 cand_sort_key(const Batch &b, u64 key) {
    const u64 m21 = (1ull << 21) - 1ull, mr = (1ull << b.rbits) - 1ull;
    const u64 cnt = m21 - (key >> 42), rlo = (key >> 21) & m21, rhi = key & m21;
    return ((mr - cnt) << (2 * b.rbits)) | (rlo << b.rbits) | rhi;
}

__device__ __forceinline__ bool input_failed(const Ctl *ctl) {
    return (*(volatile const u32 *)&ctl->error & (ERRB_INPUT_MASK | ERRB_OVF_MASK | ERRB_TIMEOUT)) != 0;
}

// Bounded grid barrier over the first nblocks blocks of a cooperative launch.
// bar[0] counts arrivals and is 0 between barriers (it must be 0 before a
// launch's first barrier); bar[1] is a generation that only grows.  A block
// that polls more than lim times, or sees err_bit set by another block, sets
// err_bit and returns false: the caller must then return.  With one block the
// barrier is a block barrier.
__device__ __forceinline__ bool coop_barrier(u32 *bar, unsigned nblocks, u32 *err, u32 err_bit,
                                             unsigned long long lim) {
    __syncthreads();
    if (nblocks > 1 && threadIdx.x == 0) {
        volatile u32 *gen = &bar[1];
        const u32 g = *gen;
        __threadfence();
        const u32 arrived = atomicAdd(&bar[0], 1u);
        if (arrived == nblocks - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            unsigned long long spins = 0;
            while (*gen == g) {
                if (++spins > lim || (*(volatile u32 *)err & err_bit)) {
                    atomicOr(err, err_bit);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return (*(volatile u32 *)err & err_bit) == 0;
}

// Programmatic dependent launch.  A kernel launched by launch_dep may be
// scheduled while the kernel before it on the stream is still running (that
// one lets it by griddep_launch at its start); griddep_wait, the first
// statement of every such kernel, then holds it until the kernel before has
// completed and its memory writes are visible.  The overlap hides the
// launch and block start-up of short kernels.  Cooperative launches keep a
// plain stream dependency, so their blocks never compete with waiting ones.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_dep(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

// Blocks of a cooperative launch of kernel fn with the given block size that
// fit on the device at once (0 if the query fails).
template <class F>
inline unsigned coop_grid_limit(F fn, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    return sms > 0 && per_sm > 0 ? (unsigned)(sms * per_sm) : 0u;
}

// ---------------------------------------------------------------- launchers
// scan_sort.cu
// Queries the cooperative launch limits of the scan and the sort (call once
// per process before any capture).
void init_scan_sort();
size_t radix_temp_bytes(long long n);
// Stable LSD radix sort of (key, value) pairs on bits [0, bits) of the key,
// over [0, min(*n_dev, n_cap)) (all n_cap when n_dev is null), in one
// cooperative launch.  Ping-pongs between (k0, v0) and (k1, v1); returns 0 if
// the result is in (k0, v0), 1 if in (k1, v1).  bar: two words of zero (a
// completed sort leaves them zero).  A wait (grid barrier, or a tile's wait
// on a predecessor) that polls more than spin_limit times (0: the default
// limit, about half a second) sets err_bit in *err and the sort stops; if
// err_bit is already set the sort does nothing.  Every write stays inside
// [0, n).
int radix_sort_pairs_dev(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap, const u64 *n_dev, int bits,
                         void *temp, cudaStream_t st, u32 *err, u32 err_bit, u32 *bar, long long spin_limit = 0);
inline int radix_sort_pairs(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n, int bits, void *temp,
                            cudaStream_t st, u32 *err, u32 err_bit, u32 *bar, long long spin_limit = 0) {
    return radix_sort_pairs_dev(k0, v0, k1, v1, n, nullptr, bits, temp, st, err, err_bit, bar, spin_limit);
}
// Kernel launches of one radix sort on bits bits.
inline int radix_sort_launches(int bits) { return bits > 0 ? 1 : 0; }
size_t scan_temp_bytes(long long n);
// Exclusive prefix sum of the first min(*n_dev, n_cap) values (n_cap when
// n_dev is null) in one cooperative launch; writes n + 1 outputs (the last =
// total), and the total to *total_out when total_out is not null.  In place
// allowed.  bar, err, err_bit and spin_limit as for the sort.
void exclusive_scan_u32(const u32 *in, u32 *out, long long n, void *temp, cudaStream_t st, u32 *err,
                        u32 err_bit, u32 *bar, long long spin_limit = 0);
void exclusive_scan_u64_dev(const u64 *in, u64 *out, long long n_cap, const u64 *n_dev, void *temp,
                            u64 *total_out, cudaStream_t st, u32 *err, u32 err_bit, u32 *bar,
                            long long spin_limit = 0);

// grid.cu
void launch_canonical_keys(const Batch &b, u64 *keys, u32 *vals, cudaStream_t st);
void launch_canonical_order(const Batch &b, const u64 *keys, const u32 *vals, u32 *cell_of, u32 *cell_count,
                            cudaStream_t st);
// cell_start: exclusive scan of the counts; cursor: zeroed per-cell counters
void launch_cell_scatter(const Batch &b, const u32 *cell_of, const u32 *cell_start, u32 *cursor, int ylist,
                         cudaStream_t st);
void launch_y_cells(const Batch &b, u32 *cell_of, u32 *cell_count, cudaStream_t st);

// count.cu
void launch_tube_count(const Batch &b, const Work &w, int record, cudaStream_t st);
// sort_k / sort_v: input of the candidate-order sort (null: not written)
void launch_cand_keys(const Batch &b, const Work &w, u64 *sort_k, u32 *sort_v, cudaStream_t st);
void launch_member_fill(const Batch &b, const Work &w, cudaStream_t st);
void launch_single_pass(const Batch &b, const Work &w, cudaStream_t st);
// candidates in key order, from the sort input written by launch_cand_keys
const u32 *launch_cand_order(const Batch &b, const Work &w, Out &o, void *temp, cudaStream_t st);

// merge.cu
int merge_grid_blocks(int device);

}  // namespace et

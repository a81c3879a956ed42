// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort, one
// cooperative launch each.
//
// Both run over a capacity-sized index range with an optional device-resident
// element count, so that a fixed launch sequence (capturable in a CUDA graph)
// can process data-dependent sizes.  The grid is sized for the capacity; its
// blocks first read the count and keep only as many blocks as the count has
// tiles (the others return at once), so a short sort or scan is done by one
// block with block barriers however large its capacity, and costs one launch.
// Longer ones separate their phases by bounded grid barriers.  The radix sort
// makes one histogram of all digits up front and then one pass per 8-bit
// digit, whose tiles find their output offsets by a decoupled look-back
// (details at the kernel).
#include <algorithm>

#include "common.cuh"

namespace et {

namespace {

constexpr int SC_T = 512;
constexpr int SC_I = 8;
constexpr int SC_TILE = SC_T * SC_I;
constexpr long long WAIT_LIMIT = 1ll << 22;   // polls of one wait (~0.5 s with the back-off)

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Lanes of the warp holding the same value d < 512 as this lane, from one
// ballot per bit of d (cheaper than a hardware match).
__device__ __forceinline__ unsigned warp_peers9(u32 d) {
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and the block total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T &total) {
    __shared__ T warp_sum[33];   // 32 warp prefixes + the block total
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? warp_sum[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < nw) warp_sum[lane] = si - s;
        if (lane == nw - 1) warp_sum[32] = si;
    }
    __syncthreads();
    T res = warp_sum[wid] + inc - v;
    total = warp_sum[32];
    __syncthreads();
    return res;
}

__device__ __forceinline__ long long eff_n(long long n_cap, const u64 *n_dev) {
    if (!n_dev) return n_cap;
    u64 n = *n_dev;
    return n < (u64)n_cap ? (long long)n : n_cap;
}

// Scan of [0, n) in tiles of SC_TILE.  The blocks in use (at most one per
// tile) take equal runs of consecutive tiles.  With more than one block: each
// sums its run, a grid barrier, each adds the sums of the runs before its
// own.  Then every block scans its run tile by tile with a running carry; the
// last block writes the total.
template <class T>
__global__ void __launch_bounds__(SC_T) k_scan(const T *in, T *out, long long n_cap, const u64 *n_dev, T *partial,
                                               u64 *total_out, u32 *bar, u32 *err, u32 err_bit,
                                               unsigned long long lim) {
    griddep_launch();
    griddep_wait();
    if (*(volatile u32 *)err & err_bit) return;
    const long long n = eff_n(n_cap, n_dev);
    const long long nt = n > 0 ? (n + SC_TILE - 1) / SC_TILE : 1;
    const unsigned nb = (unsigned)min((long long)gridDim.x, nt);
    if (blockIdx.x >= nb) return;   // uniform: every block read the same count
    const long long per = (nt + nb - 1) / nb;
    const long long t0 = (long long)blockIdx.x * per, t1 = min(nt, t0 + per);
    T carry = 0;
    if (nb > 1) {
        T s = 0;
        for (long long tl = t0; tl < t1; ++tl) {
            const long long base = tl * SC_TILE + (long long)threadIdx.x * SC_I;
#pragma unroll
            for (int i = 0; i < SC_I; ++i)
                if (base + i < n) s += in[base + i];
        }
        T tot;
        block_excl_scan(s, tot);
        if (threadIdx.x == 0) partial[blockIdx.x] = tot;
        if (!coop_barrier(bar, nb, err, err_bit, lim)) return;
        T pre = 0;   // runs before this block's (written by other SMs: read through L2)
        for (unsigned j = threadIdx.x; j < blockIdx.x; j += SC_T) pre += __ldcg(&partial[j]);
        block_excl_scan(pre, carry);
    }
    for (long long tl = t0; tl < t1; ++tl) {
        const long long base = tl * SC_TILE + (long long)threadIdx.x * SC_I;
        T v[SC_I];
        T s = 0;
#pragma unroll
        for (int i = 0; i < SC_I; ++i) {
            v[i] = (base + i < n) ? in[base + i] : T(0);
            s += v[i];
        }
        T tot;
        T ex = block_excl_scan(s, tot) + carry;
#pragma unroll
        for (int i = 0; i < SC_I; ++i) {
            if (base + i < n) out[base + i] = ex;
            ex += v[i];
        }
        carry += tot;
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) {
        out[n] = carry;
        if (total_out) *total_out = (u64)carry;
    }
}

template <class T>
unsigned scan_grid_limit() {
    static const unsigned limit = coop_grid_limit(k_scan<T>, SC_T);
    return limit;
}

template <class T>
void scan_impl(const T *in, T *out, long long n_cap, const u64 *n_dev, void *temp, u64 *total_out,
               cudaStream_t st, u32 *err, u32 err_bit, u32 *bar, long long spin_limit) {
    const unsigned limit = scan_grid_limit<T>();
    long long nt = (n_cap + SC_TILE - 1) / SC_TILE;
    if (nt == 0) nt = 1;
    unsigned grid = (unsigned)std::min<long long>(nt, limit ? (long long)limit : 1ll);
    T *partial = (T *)temp;
    unsigned long long lim = spin_limit > 0 ? (unsigned long long)spin_limit : (unsigned long long)WAIT_LIMIT;
    void *args[] = {(void *)&in, (void *)&out, (void *)&n_cap, (void *)&n_dev, (void *)&partial,
                    (void *)&total_out, (void *)&bar, (void *)&err, (void *)&err_bit, (void *)&lim};
    cudaLaunchCooperativeKernel((const void *)k_scan<T>, dim3(grid), dim3(SC_T), args, 0, st);
}

// ---------------------------------------------------------------- radix sort
//
// One cooperative launch.  The blocks in use (at most one per tile of the
// count) clear the histogram and the tile status; after a grid barrier they
// make a histogram of every digit of every key (one read), and after another
// each block turns it into per-pass digit offsets.  Then one pass per 8-bit
// digit, separated by grid barriers: block b takes tiles b, b + nb, ... in
// order, counts a tile's digits, and finds the offset of the tile inside each
// digit's output range by a decoupled look-back over the tiles before it:
// every tile publishes its count per digit, then (once its own prefix is
// known) the inclusive prefix, so a tile sums the counts of its predecessors
// back to the first inclusive prefix it meets.  All blocks run at once and
// take their tiles in increasing order, so a tile only waits for tiles being
// processed.  Every wait is bounded: past
// the limit the kernel sets the caller's timeout bit and stops at the next
// barrier (the result is then invalid and reported as such).  Inside a tile
// each warp owns 256 consecutive elements: the warps count their digits, one
// thread per digit adds up the warps before each warp, and each warp places
// its elements round by round (peer lanes from ballots + popcount), so equal
// digits keep their index order and the sort is stable.  A list of at most one
// tile is sorted by one block with every pass on chip (block_sort_small), as
// is a list whose capacity is at most RSS_MAX (k_rs_small, a plain launch).
// Keys and values written in one pass are read by other SMs in the next:
// those reads go through L2.

constexpr int RS_T = 256;
constexpr int RS_I = 8;
constexpr int RS_TILE = RS_T * RS_I;
constexpr int RS_W = RS_T / 32;
constexpr int RS_MAXP = 8;                    // passes of a 64-bit key
constexpr int RS_LB = 8;                      // predecessors read per look-back round trip
constexpr unsigned long long RS_VAL = (1ull << 54) - 1ull;
constexpr unsigned long long RS_AGG = 1ull << 54, RS_INC = 2ull << 54;

// temp: gbase[RS_MAXP][256] u32 | 256 B unused | status[ntiles][256] u64
struct RsTemp {
    u32 *gbase;
    unsigned long long *status;
};

__host__ __device__ inline size_t rs_status_offset() { return (size_t)RS_MAXP * 256 * sizeof(u32) + 256; }

// Sort of n <= NT * 8 pairs by one block of NT threads with every pass on
// chip: warp w owns elements [256 w, 256 w + 256), lane l holds 256 w + 32 r
// + l for r < 8 in registers.  Per pass the warps count their digits, one
// block scan over the (digit, warp) counts in digit-major order (8 per
// thread) gives every warp's first output position per digit, and each warp
// places its elements round by round (peer lanes from ballots + popcount), so
// equal digits keep their index order; the pairs are exchanged
// through shared memory (xk, xv) and read back in index order.  A pass whose
// digit is the same for every key is skipped (a stable pass over it is the
// identity).  The last pass writes (kout, vout), which may be (kin, vin): the
// input is read first.
template <int NT>
__device__ __forceinline__ void block_sort_small(const u64 *kin, const u32 *vin, u64 *kout, u32 *vout, int n,
                                                 int npass, u32 *wc, u64 *xk, u32 *xv) {
    constexpr int NW = NT / 32, IT = 8;
    static_assert(NT >= 256 && NT <= 1024 && (NT & (NT - 1)) == 0, "8 (digit, warp) entries per thread");
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    u64 key[IT];
    u32 val[IT];
    __shared__ unsigned long long s_or, s_and;
    if (n <= 0) return;
    u64 kor = 0ull, kand = ~0ull;
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        const int i = w * 256 + r * 32 + lane;
        key[r] = i < n ? __ldcg(&kin[i]) : 0ull;
        val[r] = i < n ? __ldcg(&vin[i]) : 0u;
        if (i < n) {
            kor |= key[r];
            kand &= key[r];
        }
    }
    // key bits that differ between keys: a pass whose digit is the same for
    // every key leaves the order as it is and is skipped
    if (t == 0) {
        s_or = 0ull;
        s_and = ~0ull;
    }
    __syncthreads();
    {
        const u64 wor = ((u64)__reduce_or_sync(0xffffffffu, (u32)(kor >> 32)) << 32) |
                        __reduce_or_sync(0xffffffffu, (u32)kor);
        const u64 wand = ((u64)__reduce_and_sync(0xffffffffu, (u32)(kand >> 32)) << 32) |
                         __reduce_and_sync(0xffffffffu, (u32)kand);
        if (lane == 0) {
            atomicOr(&s_or, wor);
            atomicAnd(&s_and, wand);
        }
    }
    __syncthreads();
    const u64 vary = s_or ^ s_and;
    int last_p = -1;
    for (int p = 0; p < npass; ++p)
        if ((vary >> (8 * p)) & 255u) last_p = p;
    if (last_p < 0) {   // already in order on the sorted bits
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int i = w * 256 + r * 32 + lane;
            if (i < n) {
                kout[i] = key[r];
                vout[i] = val[r];
            }
        }
        return;
    }
    for (int p = 0; p <= last_p; ++p) {
        const int shift = 8 * p;
        if (!((vary >> shift) & 255u)) continue;   // uniform
        for (int j = t; j < NW * 256; j += NT) wc[j] = 0;
        __syncthreads();
        u32 dig[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int i = w * 256 + r * 32 + lane;
            dig[r] = i < n ? (u32)(key[r] >> shift) & 255u : 256u + (u32)lane;   // invalid lanes never match
            if (i < n) atomicAdd(&wc[w * 256 + dig[r]], 1u);
        }
        __syncthreads();
        {   // (digit, warp) counts in digit-major order, 8 consecutive entries per thread
            u32 c8[8], s8 = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = t * 8 + j;
                c8[j] = wc[(e % NW) * 256 + e / NW];
                s8 += c8[j];
            }
            u32 all;
            u32 x = block_excl_scan(s8, all);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = t * 8 + j;
                wc[(e % NW) * 256 + e / NW] = x;
                x += c8[j];
            }
        }
        __syncthreads();
        const bool last = p == last_p;
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            if (w * 256 + r * 32 >= n) break;   // warp-uniform: no element in this round or later
            const u32 d = dig[r];
            const unsigned peers = warp_peers9(d);
            const bool valid = d < 256u;
            const u32 b = valid ? wc[w * 256 + d] : 0u;
            __syncwarp();
            if (valid) {
                const u32 rank = __popc(peers & lt), m = __popc(peers);
                const u32 pos = b + rank;
                if (last) {
                    kout[pos] = key[r];
                    vout[pos] = val[r];
                } else {
                    xk[pos] = key[r];
                    xv[pos] = val[r];
                }
                if (rank == m - 1) wc[w * 256 + d] = b + m;
            }
            __syncwarp();
        }
        if (!last) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < IT; ++r) {
                const int i = w * 256 + r * 32 + lane;
                if (i < n) {
                    key[r] = xk[i];
                    val[r] = xv[i];
                }
            }
        }
    }
}

constexpr int RSS_MAX = 1024 * 8;   // pairs the one-block sort takes (with 1024 threads)

template <int NT>
constexpr size_t rss_smem() {
    return (size_t)(NT / 32) * 256 * sizeof(u32) + (size_t)NT * 8 * (sizeof(u64) + sizeof(u32));
}

// One block of NT threads sorts a list whose capacity is at most NT * 8 pairs.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_rs_small(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap,
                                                    const u64 *n_dev, int npass, u32 *err, u32 err_bit) {
    griddep_launch();
    griddep_wait();
    extern __shared__ __align__(16) unsigned char rss_smem_buf[];
    if (*(volatile u32 *)err & err_bit) return;
    const int n = (int)eff_n(n_cap, n_dev);
    u32 *wc = (u32 *)rss_smem_buf;
    u64 *xk = (u64 *)(rss_smem_buf + (size_t)(NT / 32) * 256 * sizeof(u32));
    u32 *xv = (u32 *)(xk + NT * 8);
    block_sort_small<NT>(k0, v0, (npass & 1) ? k1 : k0, (npass & 1) ? v1 : v0, n, npass, wc, xk, xv);
}

__global__ void __launch_bounds__(RS_T, 4) k_rs_sort(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap,
                                                  const u64 *n_dev, int npass, RsTemp tp, u32 *bar, u32 *err,
                                                  u32 err_bit, unsigned long long lim) {
    griddep_launch();
    griddep_wait();
    struct Tiles {   // the tiled passes
        u32 base[RS_MAXP][256];   // the block's histogram, then per-pass digit offsets
        u32 wcnt[RS_W][256];      // per warp and digit: count, then output position
    };
    struct Small {   // one tile sorted on chip
        u32 wc[RS_W][256];
        u64 xk[RS_TILE];
        u32 xv[RS_TILE];
    };
    __shared__ union {
        Tiles l;
        Small s;
    } sm;
    u32 (*s_base)[256] = sm.l.base;
    u32 (*wcnt)[256] = sm.l.wcnt;
    if (*(volatile u32 *)err & err_bit) return;
    const long long n = eff_n(n_cap, n_dev);
    if (n <= RS_TILE) {   // one tile: block 0 alone, no waits (uniform: every block read the same count)
        if (blockIdx.x == 0 && n > 0)
            block_sort_small<RS_T>(k0, v0, (npass & 1) ? k1 : k0, (npass & 1) ? v1 : v0, (int)n, npass,
                                   &sm.s.wc[0][0], sm.s.xk, sm.s.xv);
        return;
    }
    const long long nt = (n + RS_TILE - 1) / RS_TILE;
    const unsigned nb = (unsigned)min((long long)gridDim.x, nt);
    if (blockIdx.x >= nb) return;   // uniform: every block read the same count
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    {   // clear the global histogram and the status of the tiles in use
        const long long gt = (long long)blockIdx.x * RS_T + t, nth = (long long)nb * RS_T;
        for (long long i = gt; i < (long long)npass * 256; i += nth) tp.gbase[i] = 0;
        for (long long i = gt; i < nt * 256; i += nth) tp.status[i] = 0;
    }
    for (int i = t; i < RS_MAXP * 256; i += RS_T) (&s_base[0][0])[i] = 0;
    if (!coop_barrier(bar, nb, err, err_bit, lim)) return;
    for (long long i = (long long)blockIdx.x * RS_T + t; i < n; i += (long long)nb * RS_T) {
        const u64 k = __ldcg(&k0[i]);
        for (int p = 0; p < npass; ++p) atomicAdd(&s_base[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = t; i < npass * 256; i += RS_T) {
        const u32 c = (&s_base[0][0])[i];
        if (c) atomicAdd(&tp.gbase[i], c);
    }
    if (!coop_barrier(bar, nb, err, err_bit, lim)) return;
    for (int p = 0; p < npass; ++p) {   // digit counts -> exclusive digit offsets
        const u32 c = __ldcg(&tp.gbase[p * 256 + t]);
        u32 tot;
        s_base[p][t] = block_excl_scan(c, tot);
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int p = 0; p < npass; ++p) {
        const u64 *kin = (p & 1) ? k1 : k0;
        const u32 *vin = (p & 1) ? v1 : v0;
        u64 *kout = (p & 1) ? k0 : k1;
        u32 *vout = (p & 1) ? v0 : v1;
        const int shift = 8 * p;
        const unsigned long long tag = (unsigned long long)(p + 1) << 56;
        // block b takes tiles b, b + nb, ... in order: every block runs at once,
        // so the tiles a tile waits for are always being processed
        for (long long tile = blockIdx.x; tile < nt; tile += nb) {
#pragma unroll
            for (int j = 0; j < RS_W; ++j) wcnt[j][t] = 0;
            __syncthreads();
            // warp w holds the tile's elements 256 w + 32 r + lane, r < RS_I
            const long long wbase = tile * RS_TILE + w * 256 + lane;
            u64 key[RS_I];
            u32 val[RS_I];
#pragma unroll
            for (int r = 0; r < RS_I; ++r) {
                const long long i = wbase + r * 32;
                const bool valid = i < n;
                key[r] = valid ? __ldcg(&kin[i]) : 0ull;
                val[r] = valid ? __ldcg(&vin[i]) : 0u;
                if (valid) atomicAdd(&wcnt[w][(u32)(key[r] >> shift) & 255u], 1u);
            }
            __syncthreads();
            {   // digit t: prefix over the warps, tile total, look-back over the tiles before
                u32 c = 0;
#pragma unroll
                for (int j = 0; j < RS_W; ++j) {
                    const u32 x = wcnt[j][t];
                    wcnt[j][t] = c;
                    c += x;
                }
                volatile unsigned long long *st = tp.status + (size_t)tile * 256 + t;
                unsigned long long excl = 0;
                if (tile > 0) {
                    *st = tag | RS_AGG | c;
                    // predecessors u, u - 1, ... are read RS_LB at a time (independent
                    // loads, one round trip); the window is summed nearest first up
                    // to the first inclusive prefix, and polled again from the first
                    // predecessor that has published nothing yet
                    long long u = tile - 1;
                    unsigned long long spins = 0;
                    while (u >= 0) {
                        unsigned long long sv[RS_LB];
#pragma unroll
                        for (int j = 0; j < RS_LB; ++j)
                            sv[j] = u - j >= 0 ? *((volatile unsigned long long *)(tp.status + (size_t)(u - j) * 256 + t))
                                               : 0ull;
                        int used = 0;
                        bool inc = false;
#pragma unroll
                        for (int j = 0; j < RS_LB; ++j) {
                            if (used < j || u - j < 0) break;   // stopped earlier, or before tile 0
                            const unsigned long long v = sv[j];
                            if ((v >> 56) != (unsigned long long)(p + 1) || (v & (RS_AGG | RS_INC)) == 0) break;
                            excl += v & RS_VAL;
                            used = j + 1;
                            if (v & RS_INC) {
                                inc = true;
                                break;
                            }
                        }
                        if (inc) break;
                        u -= used;
                        if (used < RS_LB && u >= 0) {   // predecessor u has not published yet
                            if (++spins > lim) {
                                atomicOr(err, err_bit);
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                }
                *st = tag | RS_INC | (excl + c);
                const u32 base = s_base[p][t] + (u32)excl;
#pragma unroll
                for (int j = 0; j < RS_W; ++j) wcnt[j][t] += base;
            }
            __syncthreads();
            // each warp places its elements round by round: equal digits keep index order
#pragma unroll
            for (int r = 0; r < RS_I; ++r) {
                const long long i = wbase + r * 32;
                if (wbase - lane + r * 32 >= n) break;   // warp-uniform: no element in this round or later
                const bool valid = i < n;
                const u32 d = valid ? (u32)(key[r] >> shift) & 255u : 256u + (u32)lane;   // invalid lanes never match
                const unsigned peers = warp_peers9(d);
                const u32 b = valid ? wcnt[w][d] : 0u;
                __syncwarp();
                if (valid) {
                    const u32 rank = __popc(peers & lt_mask), m = __popc(peers);
                    const u32 pos = b + rank;
                    if ((long long)pos < n) {   // always, unless a timed-out look-back left the offset invalid
                        kout[pos] = key[r];
                        vout[pos] = val[r];
                    }
                    if (rank == m - 1) wcnt[w][d] = b + m;
                }
                __syncwarp();
            }
            __syncthreads();   // the counters are reset for the next tile
        }
        if (p + 1 < npass && !coop_barrier(bar, nb, err, err_bit, lim)) return;
    }
}

unsigned sort_grid_limit() {
    static const unsigned limit = coop_grid_limit(k_rs_sort, RS_T);
    return limit;
}

}  // namespace

void init_scan_sort() {
    // the launch limits are queried once, outside any stream capture
    (void)scan_grid_limit<u32>();
    (void)scan_grid_limit<u64>();
    (void)sort_grid_limit();
    cudaFuncSetAttribute(k_rs_small<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rss_smem<512>());
    cudaFuncSetAttribute(k_rs_small<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rss_smem<1024>());
}

size_t scan_temp_bytes(long long n) {
    long long nb = (n + SC_TILE - 1) / SC_TILE + 2;
    return (size_t)nb * sizeof(u64);
}

void exclusive_scan_u32(const u32 *in, u32 *out, long long n, void *temp, cudaStream_t st, u32 *err, u32 err_bit,
                        u32 *bar, long long spin_limit) {
    scan_impl<u32>(in, out, n, nullptr, temp, nullptr, st, err, err_bit, bar, spin_limit);
}

void exclusive_scan_u64_dev(const u64 *in, u64 *out, long long n_cap, const u64 *n_dev, void *temp,
                            u64 *total_out, cudaStream_t st, u32 *err, u32 err_bit, u32 *bar, long long spin_limit) {
    scan_impl<u64>(in, out, n_cap, n_dev, temp, total_out, st, err, err_bit, bar, spin_limit);
}

size_t radix_temp_bytes(long long n) {
    long long ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles == 0) ntiles = 1;
    return rs_status_offset() + (size_t)ntiles * 256 * sizeof(unsigned long long);
}

int radix_sort_pairs_dev(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap, const u64 *n_dev, int bits,
                         void *temp, cudaStream_t st, u32 *err, u32 err_bit, u32 *bar, long long spin_limit) {
    const unsigned limit = sort_grid_limit();
    const long long ntiles = (n_cap + RS_TILE - 1) / RS_TILE;
    int npass = (bits + 7) / 8;
    if (ntiles == 0 || npass == 0) return 0;
    if (n_cap <= RSS_MAX) {   // a short list by capacity: one block, every pass on chip
        if (n_cap <= 256 * 8)
            launch_dep(k_rs_small<256>, dim3(1), dim3(256), rss_smem<256>(), st, k0, v0, k1, v1, n_cap, n_dev, npass, err, err_bit);
        else if (n_cap <= 512 * 8)
            launch_dep(k_rs_small<512>, dim3(1), dim3(512), rss_smem<512>(), st, k0, v0, k1, v1, n_cap, n_dev, npass, err, err_bit);
        else
            launch_dep(k_rs_small<1024>, dim3(1), dim3(1024), rss_smem<1024>(), st, k0, v0, k1, v1, n_cap, n_dev, npass, err, err_bit);
        return npass & 1;
    }
    RsTemp tp;
    tp.gbase = (u32 *)temp;
    tp.status = (unsigned long long *)((char *)temp + rs_status_offset());
    const unsigned grid = (unsigned)std::min<long long>(ntiles, limit ? (long long)limit : 1ll);
    unsigned long long lim = spin_limit > 0 ? (unsigned long long)spin_limit : (unsigned long long)WAIT_LIMIT;
    void *args[] = {(void *)&k0, (void *)&v0,  (void *)&k1,  (void *)&v1,      (void *)&n_cap, (void *)&n_dev,
                    (void *)&npass, (void *)&tp, (void *)&bar, (void *)&err, (void *)&err_bit, (void *)&lim};
    cudaLaunchCooperativeKernel((const void *)k_rs_sort, dim3(grid), dim3(RS_T), args, 0, st);
    return npass & 1;
}

}  // namespace et

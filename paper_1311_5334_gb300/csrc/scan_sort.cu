// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both run over a capacity-sized index range with an optional device-resident
// element count, so that a fixed launch sequence (capturable in a CUDA graph)
// can process data-dependent sizes.  The radix sort makes one histogram of all
// digits up front and then one kernel per 8-bit digit, whose tiles find their
// output offsets by a decoupled look-back (details at the kernels).
#include <algorithm>

#include "common.cuh"

namespace et {

namespace {

constexpr int SC_T = 512;
constexpr int SC_I = 8;
constexpr int SC_TILE = SC_T * SC_I;

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

template <class T>
__global__ void k_scan_reduce(const T *in, long long n_cap, const u64 *n_dev, T *partial) {
    const long long n = eff_n(n_cap, n_dev);
    const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_I;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SC_I; ++i)
        if (base + i < n) s += in[base + i];
    T tot;
    block_excl_scan(s, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_top(T *partial, long long nb) {
    T carry = 0;
    for (long long off = 0; off < nb; off += blockDim.x) {
        long long i = off + threadIdx.x;
        T v = i < nb ? partial[i] : T(0);
        T tot;
        T ex = block_excl_scan(v, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) partial[nb] = carry;
}

template <class T>
__global__ void k_scan_down(const T *in, T *out, long long n_cap, const u64 *n_dev, const T *partial,
                            long long nb, u64 *total_out) {
    const long long n = eff_n(n_cap, n_dev);
    const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_I;
    T v[SC_I];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SC_I; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T tot;
    T ex = block_excl_scan(s, tot) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SC_I; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[n] = partial[nb];
        if (total_out) *total_out = (u64)partial[nb];
    }
}

template <class T>
void scan_impl(const T *in, T *out, long long n_cap, const u64 *n_dev, void *temp, u64 *total_out,
               cudaStream_t st) {
    long long nb = (n_cap + SC_TILE - 1) / SC_TILE;
    if (nb == 0) nb = 1;
    T *partial = (T *)temp;
    k_scan_reduce<T><<<(unsigned)nb, SC_T, 0, st>>>(in, n_cap, n_dev, partial);
    k_scan_top<T><<<1, 1024, 0, st>>>(partial, nb);
    k_scan_down<T><<<(unsigned)nb, SC_T, 0, st>>>(in, out, n_cap, n_dev, partial, nb, total_out);
}

// ---------------------------------------------------------------- radix sort
//
// One pass per 8-bit digit, one kernel per pass.  A histogram of every digit
// of every key (one read) and its per-digit exclusive scans are made first.
// In a pass each block takes the next tile from a ticket counter, counts the
// tile's digits, and finds the offset of its tile inside each digit's output
// range by a decoupled look-back over the tiles before it: every tile
// publishes its count per digit, then (once its own prefix is known) the
// inclusive prefix, so a tile sums the counts of its predecessors back to the
// first inclusive prefix it meets.  Tickets are taken in start order, so a
// tile only waits for tiles whose blocks are already running.  The wait is
// bounded: past the limit the kernel sets the caller's timeout bit and
// carries on (the result is then invalid and reported as such).  Inside a
// tile, equal digits are ranked by warp match + popcount in index order, so
// the sort is stable.

constexpr int RS_T = 256;
constexpr int RS_I = 8;
constexpr int RS_TILE = RS_T * RS_I;
constexpr int RS_W = RS_T / 32;
constexpr int RS_MAXP = 8;                    // passes of a 64-bit key
constexpr unsigned long long RS_VAL = (1ull << 54) - 1ull;
constexpr unsigned long long RS_AGG = 1ull << 54, RS_INC = 2ull << 54;
constexpr long long RS_SPIN_LIMIT = 1ll << 22;   // polls of one predecessor (~0.5 s with the back-off)

// temp: gbase[RS_MAXP][256] u32 | tickets[RS_MAXP] u32 (256 B) | status[ntiles][256] u64
struct RsTemp {
    u32 *gbase;
    u32 *tickets;
    unsigned long long *status;
};

__host__ __device__ inline size_t rs_status_offset() { return (size_t)RS_MAXP * 256 * sizeof(u32) + 256; }

__global__ void k_rs_hist(const u64 *keys, long long n_cap, const u64 *n_dev, int npass, u32 *gbase) {
    __shared__ u32 cnt[RS_MAXP][256];
    for (int i = threadIdx.x; i < RS_MAXP * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const long long n = eff_n(n_cap, n_dev);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const u64 k = keys[i];
        for (int p = 0; p < npass; ++p) atomicAdd(&cnt[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += blockDim.x) {
        const u32 c = (&cnt[0][0])[i];
        if (c) atomicAdd(&gbase[i], c);
    }
}

// Per pass, digit counts -> exclusive digit offsets (in place).
__global__ void k_rs_bases(u32 *gbase, int npass) {
    for (int p = 0; p < npass; ++p) {
        const u32 c = gbase[p * 256 + threadIdx.x];
        u32 tot;
        const u32 ex = block_excl_scan(c, tot);
        gbase[p * 256 + threadIdx.x] = ex;
    }
}

__global__ void __launch_bounds__(RS_T) k_rs_pass(const u64 *kin, const u32 *vin, u64 *kout, u32 *vout,
                                                  long long n_cap, const u64 *n_dev, int pass, RsTemp tp,
                                                  u32 *err, u32 err_bit, long long spin_limit) {
    __shared__ u32 s_tile;
    __shared__ u32 cnt[256];
    __shared__ u32 base_off[256];
    __shared__ u32 running[256];
    __shared__ u32 wcnt[RS_W][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_tile = atomicAdd(&tp.tickets[pass], 1u);
    cnt[t] = 0;
    running[t] = 0;
#pragma unroll
    for (int j = 0; j < RS_W; ++j) wcnt[j][t] = 0;
    __syncthreads();
    const long long tile = s_tile;
    const long long n = eff_n(n_cap, n_dev);
    const long long tbase = tile * RS_TILE;
    if (tbase >= n) return;
    const int shift = 8 * pass;
    u64 key[RS_I];
    u32 val[RS_I], dig[RS_I];
#pragma unroll
    for (int k = 0; k < RS_I; ++k) {
        const long long i = tbase + k * RS_T + t;
        const bool valid = i < n;
        key[k] = valid ? kin[i] : 0ull;
        val[k] = valid ? vin[i] : 0u;
        dig[k] = valid ? (u32)(key[k] >> shift) & 255u : 256u + (u32)lane;   // invalid lanes never match
        if (valid) atomicAdd(&cnt[dig[k]], 1u);
    }
    __syncthreads();
    {   // look-back for digit t
        const u32 c = cnt[t];
        volatile unsigned long long *st = tp.status + (size_t)tile * 256 + t;
        const unsigned long long tag = (unsigned long long)(pass + 1) << 56;
        unsigned long long excl = 0;
        if (tile > 0) {
            *st = tag | RS_AGG | c;
            long long u = tile - 1;
            long long spins = 0;
            while (u >= 0) {
                const unsigned long long sv = *((volatile unsigned long long *)(tp.status + (size_t)u * 256 + t));
                if ((sv >> 56) != (unsigned long long)(pass + 1) || (sv & (RS_AGG | RS_INC)) == 0) {
                    if (++spins > spin_limit) {
                        if (err) atomicOr(err, err_bit);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                excl += sv & RS_VAL;
                if (sv & RS_INC) break;
                --u;
            }
        }
        __threadfence();
        *st = tag | RS_INC | (excl + c);
        base_off[t] = tp.gbase[pass * 256 + t] + (u32)excl;
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int k = 0; k < RS_I; ++k) {
        const bool valid = dig[k] < 256u;
        const u32 d = dig[k];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const u32 rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {   // per digit: prefix over warps, carry across sub-passes
            u32 s = running[t];
#pragma unroll
            for (int j = 0; j < RS_W; ++j) {
                const u32 c = wcnt[j][t];
                wcnt[j][t] = s;
                s += c;
            }
            running[t] = s;
        }
        __syncthreads();
        if (valid) {
            const u32 pos = base_off[d] + wcnt[w][d] + rank;
            if ((long long)pos < n) {   // always, unless a timed-out look-back left the offset invalid
                kout[pos] = key[k];
                vout[pos] = val[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RS_W; ++j) wcnt[j][t] = 0;
        __syncthreads();
    }
}

unsigned rs_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return (unsigned)sms;
}

}  // namespace

size_t scan_temp_bytes(long long n) {
    long long nb = (n + SC_TILE - 1) / SC_TILE + 2;
    return (size_t)nb * sizeof(u64);
}

void exclusive_scan_u32(const u32 *in, u32 *out, long long n, void *temp, cudaStream_t st) {
    scan_impl<u32>(in, out, n, nullptr, temp, nullptr, st);
}

void exclusive_scan_u64_dev(const u64 *in, u64 *out, long long n_cap, const u64 *n_dev, void *temp,
                            u64 *total_out, cudaStream_t st) {
    scan_impl<u64>(in, out, n_cap, n_dev, temp, total_out, st);
}

size_t radix_temp_bytes(long long n) {
    long long ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles == 0) ntiles = 1;
    return rs_status_offset() + (size_t)ntiles * 256 * sizeof(unsigned long long);
}

int radix_sort_pairs_dev(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap, const u64 *n_dev, int bits,
                         void *temp, cudaStream_t st, u32 *err, u32 err_bit, long long spin_limit) {
    if (spin_limit <= 0) spin_limit = RS_SPIN_LIMIT;
    const long long ntiles = (n_cap + RS_TILE - 1) / RS_TILE;
    const int npass = (bits + 7) / 8;
    if (ntiles == 0 || npass == 0) return 0;
    RsTemp tp;
    tp.gbase = (u32 *)temp;
    tp.tickets = tp.gbase + RS_MAXP * 256;
    tp.status = (unsigned long long *)((char *)temp + rs_status_offset());
    cudaMemsetAsync(temp, 0, radix_temp_bytes(n_cap), st);
    const unsigned hg = (unsigned)std::min<long long>(ntiles, (long long)rs_sm_count() * 4);
    k_rs_hist<<<hg, 256, 0, st>>>(k0, n_cap, n_dev, npass, tp.gbase);
    k_rs_bases<<<1, 256, 0, st>>>(tp.gbase, npass);
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        u64 *ki = cur ? k1 : k0, *ko = cur ? k0 : k1;
        u32 *vi = cur ? v1 : v0, *vo = cur ? v0 : v1;
        k_rs_pass<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, vi, ko, vo, n_cap, n_dev, p, tp, err, err_bit, spin_limit);
        cur ^= 1;
    }
    return cur;
}

int radix_sort_pairs(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n, int bits, void *temp, cudaStream_t st,
                     u32 *err, u32 err_bit, long long spin_limit) {
    return radix_sort_pairs_dev(k0, v0, k1, v1, n, nullptr, bits, temp, st, err, err_bit, spin_limit);
}

}  // namespace et

// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both run over a capacity-sized index range with an optional device-resident
// element count, so that a fixed launch sequence (capturable in a CUDA graph)
// can process data-dependent sizes.  The radix sort is the classic three-step
// pass per 8-bit digit: per-tile digit histograms, one exclusive scan over
// (digit, tile), and a stable scatter that ranks equal digits inside a tile by
// warp match + popcount in index order.
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

constexpr int RS_T = 256;
constexpr int RS_I = 8;
constexpr int RS_TILE = RS_T * RS_I;
constexpr int RS_W = RS_T / 32;

__global__ void k_rs_hist(const u64 *keys, long long n_cap, const u64 *n_dev, int shift, u32 *hist,
                          long long ntiles) {
    __shared__ u32 cnt[256];
    const long long n = eff_n(n_cap, n_dev);
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_I; ++k) {
        long long i = base + k * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const u64 *kin, const u32 *vin, u64 *kout, u32 *vout, long long n_cap,
                             const u64 *n_dev, int shift, const u32 *offs, long long ntiles) {
    __shared__ u32 base_off[256];
    __shared__ u32 running[256];
    __shared__ u32 wcnt[RS_W][256];
    const long long n = eff_n(n_cap, n_dev);
    const long long tbase = (long long)blockIdx.x * RS_TILE;
    if (tbase >= n) return;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    base_off[t] = offs[(long long)t * ntiles + blockIdx.x];
    running[t] = 0;
#pragma unroll
    for (int j = 0; j < RS_W; ++j) wcnt[j][t] = 0;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int k = 0; k < RS_I; ++k) {
        long long i = tbase + k * RS_T + t;
        bool valid = i < n;
        u64 key = valid ? kin[i] : 0ull;
        u32 val = valid ? vin[i] : 0u;
        u32 d = valid ? (u32)(key >> shift) & 255u : 256u + (u32)lane;   // invalid lanes never match
        unsigned peers = __match_any_sync(0xffffffffu, d);
        u32 rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {   // per digit: prefix over warps, carry across sub-passes
            u32 s = running[t];
#pragma unroll
            for (int j = 0; j < RS_W; ++j) {
                u32 c = wcnt[j][t];
                wcnt[j][t] = s;
                s += c;
            }
            running[t] = s;
        }
        __syncthreads();
        if (valid) {
            u32 pos = base_off[d] + wcnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        // wcnt now holds prefixes; zero it for the next sub-pass
#pragma unroll
        for (int j = 0; j < RS_W; ++j) wcnt[j][t] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t scan_temp_bytes(long long n) {
    long long nb = (n + SC_TILE - 1) / SC_TILE + 2;
    return (size_t)nb * sizeof(u64);
}

void exclusive_scan_u64(const u64 *in, u64 *out, long long n, void *temp, u64 *total_out,
                        cudaStream_t st) {
    scan_impl<u64>(in, out, n, nullptr, temp, total_out, st);
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
    size_t hist = (size_t)256 * ntiles + 1;
    size_t bytes = (hist * sizeof(u32) + 255) / 256 * 256;
    return bytes + scan_temp_bytes((long long)hist);
}

int radix_sort_pairs_dev(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n_cap, const u64 *n_dev,
                         int bits, void *temp, cudaStream_t st) {
    long long ntiles = (n_cap + RS_TILE - 1) / RS_TILE;
    if (ntiles == 0) return 0;
    size_t hist_n = (size_t)256 * ntiles;
    u32 *hist = (u32 *)temp;
    size_t hist_bytes = ((hist_n + 1) * sizeof(u32) + 255) / 256 * 256;
    void *stemp = (char *)temp + hist_bytes;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        u64 *ki = cur ? k1 : k0, *ko = cur ? k0 : k1;
        u32 *vi = cur ? v1 : v0, *vo = cur ? v0 : v1;
        k_rs_hist<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, n_cap, n_dev, shift, hist, ntiles);
        scan_impl<u32>(hist, hist, (long long)hist_n, nullptr, stemp, nullptr, st);
        k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, vi, ko, vo, n_cap, n_dev, shift, hist, ntiles);
        cur ^= 1;
    }
    return cur;
}

int radix_sort_pairs(u64 *k0, u32 *v0, u64 *k1, u32 *v1, long long n, int bits, void *temp,
                     cudaStream_t st) {
    return radix_sort_pairs_dev(k0, v0, k1, v1, n, nullptr, bits, temp, st);
}

}  // namespace et

// count.cu -- seeds, tube counts, candidates and their member lists.
//
// Seeds (Section 2, Fig. 4a): for each grain a, every grain b of higher
// canonical rank with seed_min^2 <= |g_b - g_a|^2 < seed_max^2.  Higher rank
// means lexicographically larger (x, y, z), so only cells with cx >= cx(a)
// can hold partners.
//
// Tube count (Section 2, Fig. 4b): for each seed, the grains of the whole
// view within tube_r of the infinite line, by the exact test of tube.cuh over
// the cell cover.  Seeds whose count reaches min_hits become candidates.
#include "common.cuh"
#include "tube.cuh"

namespace et {

namespace {

constexpr int CT = 256;

__device__ __forceinline__ u64 warp_sum_u64(u64 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Visits the partners of the grain at cell-order position q.
template <class F>
__device__ __forceinline__ void seed_partners(const Batch &b, long long q, F &&f) {
    const int4 g = b.gc[q];
    const int v = view_of(b.goff, b.V, g.w);
    const u32 *cs = b.cell_start + (size_t)v * b.ncell;
    const int reach = b.smax - 1;
    if (reach < 0) return;
    const int cx0 = g.x / b.cs[0];
    const int cx1 = min(b.nc[0] - 1, (g.x + reach) / b.cs[0]);
    const int cy0 = max(0, g.y - reach) / b.cs[1];
    const int cy1 = min(b.nc[1] - 1, (g.y + reach) / b.cs[1]);
    const int cz0 = max(0, g.z - reach) / b.cs[2];
    const int cz1 = min(b.nc[2] - 1, (g.z + reach) / b.cs[2]);
    for (int cz = cz0; cz <= cz1; ++cz)
        for (int cy = cy0; cy <= cy1; ++cy) {
            const int row = (cz * b.nc[1] + cy) * b.nc[0];
            const u32 e = cs[row + cx1 + 1];
            for (u32 k = cs[row + cx0]; k < e; ++k) {
                const int4 h = b.gc[k];
                if (h.w <= g.w) continue;
                const long long dx = h.x - g.x, dy = h.y - g.y, dz = h.z - g.z;
                const long long d2 = dx * dx + dy * dy + dz * dz;
                if (d2 >= b.smin2 && d2 < b.smax2) f(g.w, h.w);
            }
        }
}

__global__ void __launch_bounds__(CT) k_seed_count(Batch b, Work w) {
    if (input_failed(b.ctl)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < b.N; q += stride) {
        u64 n = 0;
        seed_partners(b, q, [&](int, int) { ++n; });
        w.seed_off[q] = n;
    }
}

__global__ void __launch_bounds__(CT) k_seed_fill(Batch b, Work w) {
    if (input_failed(b.ctl)) return;
    if (b.ctl->n_seeds > w.seed_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&b.ctl->error, ERRB_OVF_SEEDS);
        return;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < b.N; q += stride) {
        u64 o = w.seed_off[q];
        seed_partners(b, q, [&](int lo, int hi) { w.seeds[o++] = make_int2(lo, hi); });
    }
}

__global__ void __launch_bounds__(CT) k_tube_count(Batch b, Work w, int record) {
    if (input_failed(b.ctl)) return;
    const u64 ns = b.ctl->n_seeds;
    if (record && ns > w.rec_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&b.ctl->error, ERRB_OVF_RECORD);
        return;
    }
    const u64 stride = (u64)gridDim.x * blockDim.x;
    u64 tests = 0, hits = 0;
    // every lane of a warp runs the same number of iterations (warp-uniform bound)
    const u64 first = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (u64 base = first; base < ns; base += stride) {
        const u64 s = base + (threadIdx.x & 31u);
        const bool valid = s < ns;
        u32 count = 0;
        int lo = 0, hi = 0;
        if (valid) {
            const int2 sd = w.seeds[s];
            lo = sd.x;
            hi = sd.y;
            const int4 ga = b.gr[lo], gb = b.gr[hi];
            const int3 a = make_int3(ga.x, ga.y, ga.z);
            const int3 d = make_int3(gb.x - ga.x, gb.y - ga.y, gb.z - ga.z);
            const long long R = b.r2 * ((long long)d.x * d.x + (long long)d.y * d.y + (long long)d.z * d.z);
            const int v = view_of(b.goff, b.V, lo);
            const u32 *cs = b.cell_start + (size_t)v * b.ncell;
            const int4 *__restrict__ gc = b.gc;
            tube_cover(b, cs, a, d, [&](u32 beg, u32 end) {
                tests += end - beg;
                for (u32 k = beg; k < end; ++k) count += in_tube(gc[k], a, d, R);
            });
            hits += count;
            if (record) {
                w.rec_lo[s] = ga.w;
                w.rec_hi[s] = gb.w;
                w.rec_cnt[s] = (int)count;
            }
        }
        const bool is_cand = valid && count >= (u32)b.H;
        const unsigned m = __ballot_sync(0xffffffffu, is_cand);
        if (m) {
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(m) - 1;
            u64 base_idx = 0;
            if (lane == leader) base_idx = atomicAdd(&b.ctl->n_cand, (u64)__popc(m));
            base_idx = __shfl_sync(0xffffffffu, base_idx, leader);
            if (is_cand) {
                const u64 idx = base_idx + __popc(m & ((1u << lane) - 1u));
                if (idx < w.cand_cap) {
                    w.c_lo[idx] = lo;
                    w.c_hi[idx] = hi;
                    w.c_cnt[idx] = count;
                } else {
                    atomicOr(&b.ctl->error, ERRB_OVF_CAND);
                }
            }
        }
    }
    tests = warp_sum_u64(tests);
    hits = warp_sum_u64(hits);
    if ((threadIdx.x & 31) == 0) {
        if (tests) atomicAdd(&b.ctl->n_tests, tests);
        if (hits) atomicAdd(&b.ctl->n_hits, hits);
    }
}

// Candidate keys: (2^21 - 1 - count) << 42 | rank_lo << 21 | rank_hi, so that
// ascending keys visit candidates by count descending, then ranks ascending.
__global__ void k_cand_keys(Batch b, Work w) {
    if (input_failed(b.ctl)) return;
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
        const int lo = w.c_lo[c], hi = w.c_hi[c];
        const int v = view_of(b.goff, b.V, lo);
        const u64 rlo = (u64)(lo - b.goff[v]), rhi = (u64)(hi - b.goff[v]);
        const u64 cnt = w.c_cnt[c];
        w.c_key[c] = ((((1ull << 21) - 1ull) - cnt) << 42) | (rlo << 21) | rhi;
        w.c_moff[c] = cnt;
        w.c_state[c] = CS_UNDECIDED;
    }
}

__global__ void __launch_bounds__(CT) k_member_fill(Batch b, Work w) {
    if (input_failed(b.ctl)) return;
    if (b.ctl->n_members > w.member_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&b.ctl->error, ERRB_OVF_MEMBERS);
        return;
    }
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
        const int lo = w.c_lo[c], hi = w.c_hi[c];
        const int4 ga = b.gr[lo], gb = b.gr[hi];
        const int3 a = make_int3(ga.x, ga.y, ga.z);
        const int3 d = make_int3(gb.x - ga.x, gb.y - ga.y, gb.z - ga.z);
        const long long R = b.r2 * ((long long)d.x * d.x + (long long)d.y * d.y + (long long)d.z * d.z);
        const int v = view_of(b.goff, b.V, lo);
        const u32 *cs = b.cell_start + (size_t)v * b.ncell;
        u64 o = w.c_moff[c];
        const u64 oend = w.c_moff[c + 1];
        tube_cover(b, cs, a, d, [&](u32 beg, u32 end) {
            for (u32 k = beg; k < end; ++k) {
                const int4 g = b.gc[k];
                if (in_tube(g, a, d, R) && o < oend) w.members[o++] = g.w;
            }
        });
    }
}

unsigned persistent_grid(int blocks_per_sm) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return (unsigned)(sms * blocks_per_sm);
}

}  // namespace

void launch_seed_count(const Batch &b, const Work &w, cudaStream_t st) {
    k_seed_count<<<persistent_grid(8), CT, 0, st>>>(b, w);
}

void launch_seed_fill(const Batch &b, const Work &w, cudaStream_t st) {
    k_seed_fill<<<persistent_grid(8), CT, 0, st>>>(b, w);
}

void launch_tube_count(const Batch &b, const Work &w, int record, cudaStream_t st) {
    k_tube_count<<<persistent_grid(8), CT, 0, st>>>(b, w, record);
}

void launch_cand_keys(const Batch &b, const Work &w, cudaStream_t st) {
    k_cand_keys<<<persistent_grid(4), 256, 0, st>>>(b, w);
}

void launch_member_fill(const Batch &b, const Work &w, cudaStream_t st) {
    k_member_fill<<<persistent_grid(8), CT, 0, st>>>(b, w);
}

}  // namespace et

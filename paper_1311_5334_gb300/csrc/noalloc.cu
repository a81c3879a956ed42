// noalloc.cu -- tube counts for caller-chosen grain pairs of one small view,
// with every intermediate buffer in one fixed, file-scope device array.
//
// Who needs this: callers that cannot call cudaMalloc.  Examples are a
// scanning microscope's acquisition loop that may not block (cudaMalloc can
// synchronise the whole device), code running inside a host function enqueued
// on a stream (CUDA API calls are not allowed there), and applications whose
// framework has reserved the free device memory for its own pool.  They pass
// device pointers to their grains, their pairs and an output array, and this
// entry point uses only the scratch array below.
//
// The scratch array lives on every GPU that loads the library until the
// process exits.  In host code its name is only a stand-in: the device
// address is obtained once per device with cudaGetSymbolAddress (on the first
// call on that device, which should therefore happen before any stream
// capture) and passed to the kernels.  The address is cached together with
// the device's current CUDA context; after a device reset the context
// differs, and the next call looks the address up again.  Every call shares
// the array and leaves its contents behind; calls whose work overlaps on the
// GPU race with each other, so callers must order them (one stream, or
// events).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "runtime.h"
#include "tube.cuh"

namespace et {

namespace {

constexpr long long NA_MAX_GRAINS = ET_NOALLOC_MAX_GRAINS;
constexpr long long NA_MAX_CELLS = ET_NOALLOC_MAX_CELLS;

// Layout of the scratch array (byte offsets, 256-aligned).
constexpr size_t NA_OFF_GRAINS = 0;                                              // int4[MAX_GRAINS]
constexpr size_t NA_OFF_START = NA_OFF_GRAINS + sizeof(int4) * NA_MAX_GRAINS;    // u32[MAX_CELLS + 1]
constexpr size_t NA_OFF_CURSOR = NA_OFF_START + ((sizeof(u32) * (NA_MAX_CELLS + 1) + 255) / 256) * 256;
constexpr size_t NA_OFF_FLAG = NA_OFF_CURSOR + sizeof(u32) * NA_MAX_CELLS;       // u32 error word
constexpr size_t NA_BYTES = NA_OFF_FLAG + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaScratch {
    int4 *grains;
    u32 *start;
    u32 *cursor;
    u32 *flag;
};

NaScratch carve(unsigned char *base) {
    NaScratch s;
    s.grains = (int4 *)(base + NA_OFF_GRAINS);
    s.start = (u32 *)(base + NA_OFF_START);
    s.cursor = (u32 *)(base + NA_OFF_CURSOR);
    s.flag = (u32 *)(base + NA_OFF_FLAG);
    return s;
}

__global__ void k_na_clear(NaScratch s, int ncell) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncell; c += gridDim.x * blockDim.x) {
        s.start[c] = 0;
        if (c < ncell) s.cursor[c] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.flag = 0;
}

__device__ __forceinline__ int na_cell(const Batch &b, int x, int y, int z) {
    const int cx = min(x / b.cs[0], b.nc[0] - 1), cy = min(y / b.cs[1], b.nc[1] - 1);
    const int cz = min(z / b.cs[2], b.nc[2] - 1);
    return cx + b.nc[0] * (cy + b.nc[1] * cz);
}

__global__ void k_na_count(Batch b, const int *xyz, NaScratch s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.N; i += gridDim.x * blockDim.x) {
        const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (x < 0 || x >= b.ext[0] || y < 0 || y >= b.ext[1] || z < 0 || z >= b.ext[2]) {
            atomicOr(s.flag, 1u);
            continue;
        }
        atomicAdd(&s.cursor[na_cell(b, x, y, z)], 1u);
    }
}

// One block: exclusive scan of the per-cell counts into cell starts; the
// counts are turned into fill cursors at the same time.
__global__ void k_na_scan(NaScratch s, int ncell) {
    __shared__ u32 part[1024];
    __shared__ u32 carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += 1024) {
        const int c = base + threadIdx.x;
        const u32 v = c < ncell ? s.cursor[c] : 0u;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
            const u32 add = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        const u32 ex = carry + part[threadIdx.x] - v;
        if (c < ncell) {
            s.start[c] = ex;
            s.cursor[c] = ex;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) s.start[ncell] = carry;
}

__global__ void k_na_scatter(Batch b, const int *xyz, NaScratch s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.N; i += gridDim.x * blockDim.x) {
        const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (x < 0 || x >= b.ext[0] || y < 0 || y >= b.ext[1] || z < 0 || z >= b.ext[2]) continue;
        const u32 pos = atomicAdd(&s.cursor[na_cell(b, x, y, z)], 1u);
        s.grains[pos] = make_int4(x, y, z, i);
    }
}

// One thread per pair: the exact tube test over the conservative cell cover.
// A pair with an index outside [0, n) or equal indices, a pair whose two
// grains coincide or lie seed_max or more apart on some axis, and every pair
// when a coordinate was out of range, gets -1.  The separation bound keeps
// every cross-product component an exact int32 (|d_e w_f| + |d_f w_e| <
// (extent_e + extent_f) seed_max < 2^31, the parameter precondition) and the
// squared norms within 64 bits, as for the seeds of the regular path.
__global__ void k_na_tube(Batch b, const int *xyz, const int *pairs, long long n_pairs, int *counts,
                          NaScratch s) {
    const bool bad_view = *(volatile u32 *)s.flag != 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        if (bad_view || i < 0 || i >= b.N || j < 0 || j >= b.N || i == j) {
            counts[k] = -1;
            continue;
        }
        const int3 a = make_int3(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
        const int3 d = make_int3(xyz[3 * j] - a.x, xyz[3 * j + 1] - a.y, xyz[3 * j + 2] - a.z);
        if ((d.x == 0 && d.y == 0 && d.z == 0) || abs(d.x) >= b.smax || abs(d.y) >= b.smax ||
            abs(d.z) >= b.smax) {
            counts[k] = -1;
            continue;
        }
        const long long R = b.r2 * ((long long)d.x * d.x + (long long)d.y * d.y + (long long)d.z * d.z);
        int c = 0;
        const int4 *__restrict__ g = s.grains;
        tube_cover(b, s.start, a, d, [&](u32 beg, u32 end) {
            for (u32 q = beg; q < end; ++q) c += in_tube(g[q], a, d, R);
        });
        counts[k] = c;
    }
}

std::mutex g_na_mu;
unsigned char *g_na_base[64] = {};
void *g_na_ctx[64] = {};   // the CUDA context the cached address belongs to

// The calling thread's current CUDA context (a driver handle), through the
// runtime's driver entry point so that the library needs no -lcuda.
void *current_context() {
    typedef int (*GetCurrent)(void **);
    static GetCurrent fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (GetCurrent)f;
        cudaGetLastError();
        looked = true;
    }
    void *c = nullptr;
    if (fn && fn(&c) != 0) c = nullptr;
    return c;
}

}  // namespace

}  // namespace et

using namespace et;

extern "C" et_status et_tube_count_noalloc(const int32_t *d_xyz, int64_t n, const et_params *params,
                                           const int32_t *d_pairs, int64_t n_pairs, int32_t *d_counts,
                                           void *stream) {
    et_status st = check_params(params);
    if (st != ET_OK) return st;
    if (n < 0 || n_pairs < 0) return fail(ET_ERR_INVALID_ARG, "negative size");
    if (n > NA_MAX_GRAINS)
        return fail(ET_ERR_INVALID_ARG, "view of %lld grains exceeds the fixed scratch limit of %lld grains",
                    (long long)n, NA_MAX_GRAINS);
    if (n_pairs == 0) return ET_OK;
    if (!d_xyz || !d_pairs || !d_counts) return fail(ET_ERR_INVALID_ARG, "null device pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(ET_ERR_INVALID_ARG, "device %d beyond the supported 64", dev);
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mu);
        void *cur = current_context();
        if (!g_na_base[dev] || cur != g_na_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
            g_na_base[dev] = (unsigned char *)p;
            g_na_ctx[dev] = current_context();
        }
        base = g_na_base[dev];
    }
    // cell grid: about one grain per cell, coarsened until it fits the scratch limit
    Batch b;
    memset(&b, 0, sizeof b);
    b.V = 1;
    b.N = (int)n;
    for (int k = 0; k < 3; ++k) b.ext[k] = params->extent[k];
    b.r = params->tube_r;
    b.r2 = (long long)params->tube_r * params->tube_r;
    b.smax = params->seed_max;
    const double vol = (double)b.ext[0] * b.ext[1] * b.ext[2];
    double sz = std::cbrt(vol / (double)std::max<int64_t>(n, 1));
    long long ncell = 0;
    for (int tries = 0; tries < 64; ++tries) {
        ncell = 1;
        for (int k = 0; k < 3; ++k) {
            b.cs[k] = std::max(1, std::min((int)std::ceil(sz), b.ext[k]));
            b.nc[k] = (b.ext[k] + b.cs[k] - 1) / b.cs[k];
            b.ics[k] = 1.0f / (float)b.cs[k];
            ncell *= b.nc[k];
        }
        if (ncell <= NA_MAX_CELLS) break;
        sz *= 1.26;
    }
    if (ncell > NA_MAX_CELLS) return fail(ET_ERR_INVALID_ARG, "no cell grid fits the fixed scratch limit");
    b.ncell = (int)ncell;
    const NaScratch s = carve(base);
    cudaStream_t cst = (cudaStream_t)stream;
    k_na_clear<<<64, 256, 0, cst>>>(s, (int)ncell);
    if (n > 0) {
        const unsigned gn = (unsigned)std::min<long long>((n + 255) / 256, 1024);
        k_na_count<<<gn, 256, 0, cst>>>(b, d_xyz, s);
        k_na_scan<<<1, 1024, 0, cst>>>(s, (int)ncell);
        k_na_scatter<<<gn, 256, 0, cst>>>(b, d_xyz, s);
    }
    const unsigned gp = (unsigned)std::min<long long>((n_pairs + 255) / 256, 152 * 16);
    k_na_tube<<<gp, 256, 0, cst>>>(b, d_xyz, d_pairs, n_pairs, d_counts, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc tube count launch");
    return ET_OK;
}

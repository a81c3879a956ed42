// grid.cu -- canonical order and cell list of every view in a batch.
//
// Canonical rank: the position of a grain in lexicographic (x, y, z) order of
// its view.  It orders seeds (lo = lower rank) and breaks ties between
// candidates, so every result is independent of the caller's grain order and
// of the cell size.  The cell list bins the grains of each view in a uniform
// 3D grid (the paper's 3D hash tables, Section 3 footnote), x fastest, so that
// a run of cells along x is one contiguous range of grains.  The list is a
// counting sort: per-cell counts, their exclusive scan (cell starts), and a
// scatter that takes slots with an atomic cursor per cell.  The order of the
// grains inside one cell is therefore arbitrary; no result depends on it
// (counts, keys and fits are order-independent, member lists are sorted on
// output).
#include "common.cuh"

namespace et {

namespace {

__global__ void k_canonical_keys(Batch b, u64 *keys, u32 *vals) {
    griddep_launch();
    griddep_wait();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int sy = b.cbits[2], sx = b.cbits[1] + b.cbits[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < b.N; i += stride) {
        int v = view_of(b.goff, b.V, i);
        int x = b.xyz_in[3 * i + 0], y = b.xyz_in[3 * i + 1], z = b.xyz_in[3 * i + 2];
        bool ok = (x >= 0) & (x < b.ext[0]) & (y >= 0) & (y < b.ext[1]) & (z >= 0) & (z < b.ext[2]);
        if (!ok) {
            atomicOr(&b.ctl->error, ERRB_OUT_OF_RANGE);
            x = min(max(x, 0), b.ext[0] - 1);
            y = min(max(y, 0), b.ext[1] - 1);
            z = min(max(z, 0), b.ext[2] - 1);
        }
        keys[i] = ((u64)v << b.vshift) | ((u64)x << sx) | ((u64)y << sy) | (u64)z;
        vals[i] = (u32)i;
    }
}

__global__ void k_canonical_order(Batch b, const u64 *keys, const u32 *vals, u32 *cell_of,
                                  u32 *cell_count) {
    griddep_launch();
    griddep_wait();
    // a coordinate out of range is reported as such; a timed-out sort leaves
    // invalid indices: either way nothing after this point may run
    if (input_failed(b.ctl)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < b.N; p += stride) {
        const int v = view_of(b.goff, b.V, p);
        const long long i = vals[p];
        int x = b.xyz_in[3 * i + 0], y = b.xyz_in[3 * i + 1], z = b.xyz_in[3 * i + 2];
        x = min(max(x, 0), b.ext[0] - 1);
        y = min(max(y, 0), b.ext[1] - 1);
        z = min(max(z, 0), b.ext[2] - 1);
        b.gr[p] = make_int4(x, y, z, (int)(i - b.goff[v]));
        if (p > b.goff[v] && keys[p] == keys[p - 1]) atomicOr(&b.ctl->error, ERRB_DUPLICATE);
        int cx = min(x / b.cs[0], b.nc[0] - 1);
        int cy = min(y / b.cs[1], b.nc[1] - 1);
        int cz = min(z / b.cs[2], b.nc[2] - 1);
        u32 cell = (u32)v * (u32)b.ncell + (u32)(cx + b.nc[0] * (cy + b.nc[1] * cz));
        cell_of[p] = cell;
        atomicAdd(&cell_count[cell], 1u);
    }
}

// Scatter of the canonical order into a cell list: grain p takes the next
// slot of its cell (cursor zeroed before the launch).
__global__ void k_cell_scatter(Batch b, const u32 *cell_of, const u32 *cell_start, u32 *cursor, int4 *gc,
                               u64 *gp) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < b.N; p += stride) {
        const u32 c = cell_of[p];
        const u32 q = cell_start[c] + atomicAdd(&cursor[c], 1u);
        const int4 g = b.gr[p];
        gc[q] = make_int4(g.x, g.y, g.z, (int)p);
        gp[q] = pack_xyz(g.x, g.y, g.z);
    }
}

// Cells of the second cell list (rows along y) for the canonical order.
__global__ void k_y_cells(Batch b, u32 *cell_of, u32 *cell_count) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < b.N; p += stride) {
        const int v = view_of(b.goff, b.V, p);
        const int4 g = b.gr[p];
        const int cx = min(g.x / b.csy[0], b.ncy[0] - 1);
        const int cy = min(g.y / b.csy[1], b.ncy[1] - 1);
        const int cz = min(g.z / b.csy[2], b.ncy[2] - 1);
        const u32 cell = (u32)v * (u32)b.ncelly + (u32)(cy + b.ncy[1] * (cx + b.ncy[0] * cz));
        cell_of[p] = cell;
        atomicAdd(&cell_count[cell], 1u);
    }
}

unsigned grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)g;
}

}  // namespace

void launch_canonical_keys(const Batch &b, u64 *keys, u32 *vals, cudaStream_t st) {
    launch_dep(k_canonical_keys, dim3(grid_for(b.N, 256)), dim3(256), 0, st, b, keys, vals);
}

void launch_canonical_order(const Batch &b, const u64 *keys, const u32 *vals, u32 *cell_of, u32 *cell_count,
                            cudaStream_t st) {
    launch_dep(k_canonical_order, dim3(grid_for(b.N, 256)), dim3(256), 0, st, b, keys, vals, cell_of, cell_count);
}

void launch_cell_scatter(const Batch &b, const u32 *cell_of, const u32 *cell_start, u32 *cursor, int ylist,
                         cudaStream_t st) {
    launch_dep(k_cell_scatter, dim3(grid_for(b.N, 256)), dim3(256), 0, st, b, cell_of, cell_start, cursor, ylist ? b.gcy : b.gc,
                                                       ylist ? b.gpy : b.gp);
}

void launch_y_cells(const Batch &b, u32 *cell_of, u32 *cell_count, cudaStream_t st) {
    launch_dep(k_y_cells, dim3(grid_for(b.N, 256)), dim3(256), 0, st, b, cell_of, cell_count);
}

}  // namespace et

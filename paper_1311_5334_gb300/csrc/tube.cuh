// tube.cuh -- the cell cover of a seed's tube and the exact membership test.
//
// Membership (Section 2, Fig. 4b; exact): grain k lies on the seed line
// through g_a with direction w = g_b - g_a iff
//     |(g_k - g_a) x w|^2 <= r^2 |w|^2 .
// Cross-product components are exact int32 under the parameter precondition
// (|d_e w_f| + |d_f w_e| < 2^31); each square is below 2^62, so their sum is
// below 3 * 2^62 and exact in unsigned 64 bits, and so is r^2 |w|^2 (the
// parameters keep 3 r^2 seed_max^2 below 2^63).
//
// Cover.  The tube is an infinite cylinder across the view.  A grain p in the
// tube has a foot point q(t) = g_a + t w with |p - q| <= r, so on every axis
// |p_e - q_e(t)| <= r.  Grains are grouped in rows (cy, cz) of cells along x,
// each row a contiguous range of the cell-ordered grain array.  For each row
// the parameter interval where q_y and q_z can serve a grain of that row is
// intersected with the interval where q stays near the view; over it q_x
// spans an interval, widened by r, that gives the row's run of x cells.  All
// bounds are computed in FP32 and widened by r + COVER_PAD: with coordinates
// below 2^22 every rounding error is under one unit while the extra pad is
// COVER_PAD units, so the cover is a superset of the tube and the exact test
// decides.  The cover depends on the cell size; the count does not.
#pragma once
#include "common.cuh"

namespace et {

constexpr float COVER_PAD = 4.0f;

__device__ __forceinline__ bool in_tube(int4 g, int3 a, int3 w, long long R) {
    const int dx = g.x - a.x, dy = g.y - a.y, dz = g.z - a.z;
    const int cx = dy * w.z - dz * w.y;
    const int cy = dz * w.x - dx * w.z;
    const int cz = dx * w.y - dy * w.x;
    const unsigned long long s = (unsigned long long)((long long)cx * cx) +
                                 (unsigned long long)((long long)cy * cy) +
                                 (unsigned long long)((long long)cz * cz);
    return s <= (unsigned long long)R;
}

__device__ __forceinline__ int floor_i(float x) { return __float2int_rd(x); }

// Calls f(begin, end) for every row run of cells that may hold tube grains.
// cs: the view's cell_start (ncell + 1 entries).
template <class F>
__device__ __forceinline__ void tube_cover(const Batch &b, const u32 *__restrict__ cs, int3 a, int3 w,
                                           F &&f) {
    const float pad = (float)b.r + COVER_PAD;
    const float ax = (float)a.x, ay = (float)a.y, az = (float)a.z;
    const float wx = (float)w.x, wy = (float)w.y, wz = (float)w.z;
    float t0 = -3.0e38f, t1 = 3.0e38f;
    const float iwx = w.x ? 1.0f / wx : 0.0f;
    const float iwy = w.y ? 1.0f / wy : 0.0f;
    const float iwz = w.z ? 1.0f / wz : 0.0f;
    if (w.x) {
        float ta = (-pad - ax) * iwx, tb = ((float)(b.ext[0] - 1) + pad - ax) * iwx;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (w.y) {
        float ta = (-pad - ay) * iwy, tb = ((float)(b.ext[1] - 1) + pad - ay) * iwy;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (w.z) {
        float ta = (-pad - az) * iwz, tb = ((float)(b.ext[2] - 1) + pad - az) * iwz;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    const int nx = b.nc[0], ny = b.nc[1], nz = b.nc[2];
    const float csy = (float)b.cs[1], csz = (float)b.cs[2];
    const float yl = ay + fminf(t0 * wy, t1 * wy) - pad, yh = ay + fmaxf(t0 * wy, t1 * wy) + pad;
    const int cy0 = max(0, floor_i(yl * b.ics[1])), cy1 = min(ny - 1, floor_i(yh * b.ics[1]));
    for (int cy = cy0; cy <= cy1; ++cy) {
        float ya = t0, yb = t1;
        if (w.y) {
            float ua = ((float)cy * csy - pad - ay) * iwy;
            float ub = ((float)cy * csy + csy - 1.0f + pad - ay) * iwy;
            ya = fmaxf(t0, fminf(ua, ub));
            yb = fminf(t1, fmaxf(ua, ub));
            if (ya > yb) continue;
        }
        const float zl = az + fminf(ya * wz, yb * wz) - pad, zh = az + fmaxf(ya * wz, yb * wz) + pad;
        const int cz0 = max(0, floor_i(zl * b.ics[2])), cz1 = min(nz - 1, floor_i(zh * b.ics[2]));
        for (int cz = cz0; cz <= cz1; ++cz) {
            float za = ya, zb = yb;
            if (w.z) {
                float va = ((float)cz * csz - pad - az) * iwz;
                float vb = ((float)cz * csz + csz - 1.0f + pad - az) * iwz;
                za = fmaxf(ya, fminf(va, vb));
                zb = fminf(yb, fmaxf(va, vb));
                if (za > zb) continue;
            }
            const float xl = ax + fminf(za * wx, zb * wx) - pad, xh = ax + fmaxf(za * wx, zb * wx) + pad;
            const int cx0 = max(0, floor_i(xl * b.ics[0])), cx1 = min(nx - 1, floor_i(xh * b.ics[0]));
            if (cx0 > cx1) continue;
            const int row = (cz * ny + cy) * nx;
            f(cs[row + cx0], cs[row + cx1 + 1]);
        }
    }
}

}  // namespace et

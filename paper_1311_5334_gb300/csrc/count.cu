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

__device__ __forceinline__ u64 warp_sum_u64(u64 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Work tickets of the warp-balanced walks below.
constexpr int TW = 8;   // warps per block
constexpr int SEED_CHUNK = 32 * 8;   // largest work ticket of a warp (lines)

// Ticket size: SEED_CHUNK lines, smaller when there are too few lines to give
// every warp of the grid a few tickets.
__device__ __forceinline__ u64 ticket_size(u64 n) {
    const u64 unit = 32;
    u64 c = (n / ((u64)gridDim.x * TW * 4) + unit - 1) / unit * unit;
    return c < unit ? unit : (c > (u64)SEED_CHUNK ? (u64)SEED_CHUNK : c);
}

// floor(sqrt(v)) for 0 <= v < 2^62: the float estimate, corrected exactly.
__device__ __forceinline__ int isqrt_ll(long long v) {
    int r = (int)sqrtf((float)v);
    while ((long long)r * r > v) --r;
    while ((long long)(r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Tube walks with warp-level load balancing (tube counts and member lists).
//
// A warp takes 32 lines (one per lane).  Each line's cover is split into work
// items: the slabs of cells along whichever of y or z the line crosses more
// cells of ("outer" axis).  Within one slab the tube meets only 1-3 rows of
// the other ("inner") axis, each row a run of x cells that is one contiguous
// range of the cell-ordered grains, so items cost about the same.  The items
// of the 32 lines are dealt to the lanes in rounds of 32: a lane finds the
// line owning its item from the start positions of the lines that begin in
// the round (an OR-reduction of one-hot masks and a popcount).  Line geometry
// is resolved once into shared memory; per-line results are merged with
// shared-memory atomics.  The geometry is the conservative cover of
// tube_cover() (tube.cuh), with the per-slab terms hoisted.
// Cover geometry of one line, resolved once per line into eight 16-byte
// vectors (an item loads the six it needs, a grain test the first two).  Slab t-intervals
// are kept as (lower end at cell 0, step per cell, width) with the direction's
// sign already folded in, so the walk needs no min/max to order their ends.
struct __align__(16) SeedSm {
    int4 e0;      // ax, ay, az, wx
    int4 e1;      // wy, wz, R low, R high           (R = r^2 |w|^2)
    float4 e2;    // t0, t1 (span of the line near the view), o0, excl (int bits)
    float4 e3;    // outer slab: lower base, step, width; inner cell count (int bits)
    float4 e4;    // inner slab: lower base, step, width, 1 / inner cell edge
    float4 e5;    // inner axis: a - pad, a + pad, w, flags (int bits: 1 second list, 2 w_inner < 0, 4 w_run < 0)
    float4 e6;    // run axis: a - pad, a + pad, w, 1 / run cell edge
    int4 e7;      // run cell count, row stride of outer cell, of inner cell, view offset in the start table
};

// The records of a warp's 32 lines, vector k of line i at v[k][i]: a lane
// storing its own record writes consecutive 16-byte slots (no bank
// conflicts), and lanes reading different lines' vector k mostly hit
// different banks.
struct SeedTab {
    int4 v[8][32];
    __device__ __forceinline__ void put(int i, const SeedSm &q) {
        v[0][i] = q.e0;
        v[1][i] = q.e1;
        v[2][i] = f4i(q.e2);
        v[3][i] = f4i(q.e3);
        v[4][i] = f4i(q.e4);
        v[5][i] = f4i(q.e5);
        v[6][i] = f4i(q.e6);
        v[7][i] = q.e7;
    }
    __device__ __forceinline__ int4 i4(int k, int i) const { return v[k][i]; }
    __device__ __forceinline__ float4 f4(int k, int i) const {
        const int4 t = v[k][i];
        return make_float4(__int_as_float(t.x), __int_as_float(t.y), __int_as_float(t.z), __int_as_float(t.w));
    }
    static __device__ __forceinline__ int4 f4i(float4 f) {
        return make_int4(__float_as_int(f.x), __float_as_int(f.y), __float_as_int(f.z), __float_as_int(f.w));
    }
};

// Slab k of a cell grid with edge cs spans coordinates [k cs, (k+1) cs - 1];
// padded by pad, the line a + t w meets it for t in
//   [base + k step, base + k step + width]
// (w != 0).  w = 0: every t (the caller restricts k to the cells the line's
// constant coordinate can reach).
__device__ __forceinline__ float3 slab_coeffs(float a, float w, float iw, float cs, float pad) {
    if (w == 0.0f) return make_float3(-3.0e38f, 0.0f, 6.0e38f);
    const float step = cs * iw;
    if (w > 0.0f) return make_float3((-pad - a) * iw, step, (cs - 1.0f + 2.0f * pad) * iw);
    return make_float3((cs - 1.0f + pad - a) * iw, step, -(cs - 1.0f + 2.0f * pad) * iw);
}

// Resolves the cover geometry of the line through ga and gb into q and
// returns its number of items (outer slabs).
__device__ __forceinline__ int seed_setup(const Batch &b, int4 ga, int4 gb, int view, SeedSm &q) {
    const float pad = (float)b.r + COVER_PAD;
    const int wxi = gb.x - ga.x, wyi = gb.y - ga.y, wzi = gb.z - ga.z;
    const long long R = b.r2 * ((long long)wxi * wxi + (long long)wyi * wyi + (long long)wzi * wzi);
    q.e0 = make_int4(ga.x, ga.y, ga.z, wxi);
    q.e1 = make_int4(wyi, wzi, (int)(unsigned)(R & 0xffffffffll), (int)(R >> 32));
    const float ax = (float)ga.x, ay = (float)ga.y, az = (float)ga.z;
    const float wx = (float)wxi, wy = (float)wyi, wz = (float)wzi;
    const float iwx = wxi ? 1.0f / wx : 0.0f;
    const float iwy = wyi ? 1.0f / wy : 0.0f;
    const float iwz = wzi ? 1.0f / wz : 0.0f;
    float t0 = -3.0e38f, t1 = 3.0e38f;
    if (wxi) {
        float ta = (-pad - ax) * iwx, tb = ((float)(b.ext[0] - 1) + pad - ax) * iwx;
        t0 = fmaxf(t0, fminf(ta, tb)); t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (wyi) {
        float ta = (-pad - ay) * iwy, tb = ((float)(b.ext[1] - 1) + pad - ay) * iwy;
        t0 = fmaxf(t0, fminf(ta, tb)); t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (wzi) {
        float ta = (-pad - az) * iwz, tb = ((float)(b.ext[2] - 1) + pad - az) * iwz;
        t0 = fmaxf(t0, fminf(ta, tb)); t1 = fminf(t1, fmaxf(ta, tb));
    }
    const float xl = ax + fminf(t0 * wx, t1 * wx) - pad, xh = ax + fmaxf(t0 * wx, t1 * wx) + pad;
    const float yl = ay + fminf(t0 * wy, t1 * wy) - pad, yh = ay + fmaxf(t0 * wy, t1 * wy) + pad;
    const float zl = az + fminf(t0 * wz, t1 * wz) - pad, zh = az + fmaxf(t0 * wz, t1 * wz) + pad;
    // rows follow the line's dominant horizontal axis: x rows (first list) or y rows (second)
    const bool ylist = b.dual && abs(wyi) > abs(wxi);
    // per axis: a, w, 1/w, cell edge, 1/cell edge, cells
    float ra, rw, oa, ow, oiw, ocs, ia, iw, iiw, ics_, iinv, rinv;
    int nr, o0, nitems, nci, mo, mi;
    u32 cs_off;
    if (!ylist) {
        const int nx = b.nc[0], ny = b.nc[1], nz = b.nc[2];
        cs_off = (u32)view * (u32)b.ncell;
        ra = ax; rw = wx; rinv = b.ics[0]; nr = nx;
        const int cy0 = max(0, floor_i(yl * b.ics[1])), cy1 = min(ny - 1, floor_i(yh * b.ics[1]));
        const int cz0 = max(0, floor_i(zl * b.ics[2])), cz1 = min(nz - 1, floor_i(zh * b.ics[2]));
        const int nyc = max(0, cy1 - cy0 + 1), nzc = max(0, cz1 - cz0 + 1);
        if (nyc >= nzc) {   // outer y, inner z; row = (cz * ny + cy) * nx
            oa = ay; ow = wy; oiw = iwy; ocs = (float)b.cs[1];
            ia = az; iw = wz; iiw = iwz; ics_ = (float)b.cs[2]; iinv = b.ics[2]; nci = nz;
            mo = nx; mi = ny * nx; o0 = cy0; nitems = nyc;
        } else {            // outer z, inner y
            oa = az; ow = wz; oiw = iwz; ocs = (float)b.cs[2];
            ia = ay; iw = wy; iiw = iwy; ics_ = (float)b.cs[1]; iinv = b.ics[1]; nci = ny;
            mo = ny * nx; mi = nx; o0 = cz0; nitems = nzc;
        }
    } else {                // second list: rows along y, index cy + ny * (cx + nx * cz)
        const int nx = b.ncy[0], ny = b.ncy[1], nz = b.ncy[2];
        cs_off = (u32)view * (u32)b.ncelly;
        ra = ay; rw = wy; rinv = b.icsy[1]; nr = ny;
        const int cx0 = max(0, floor_i(xl * b.icsy[0])), cx1 = min(nx - 1, floor_i(xh * b.icsy[0]));
        const int cz0 = max(0, floor_i(zl * b.icsy[2])), cz1 = min(nz - 1, floor_i(zh * b.icsy[2]));
        const int nxc = max(0, cx1 - cx0 + 1), nzc = max(0, cz1 - cz0 + 1);
        if (nxc >= nzc) {   // outer x, inner z; row = (cz * nx + cx) * ny
            oa = ax; ow = wx; oiw = iwx; ocs = (float)b.csy[0];
            ia = az; iw = wz; iiw = iwz; ics_ = (float)b.csy[2]; iinv = b.icsy[2]; nci = nz;
            mo = ny; mi = nx * ny; o0 = cx0; nitems = nxc;
        } else {            // outer z, inner x
            oa = az; ow = wz; oiw = iwz; ocs = (float)b.csy[2];
            ia = ax; iw = wx; iiw = iwx; ics_ = (float)b.csy[0]; iinv = b.icsy[0]; nci = nx;
            mo = nx * ny; mi = ny; o0 = cz0; nitems = nzc;
        }
    }
    const float3 os = slab_coeffs(oa, ow, oiw, ocs, pad);
    const float3 is = slab_coeffs(ia, iw, iiw, ics_, pad);
    const int flags = (ylist ? 1 : 0) | (iw < 0.0f ? 2 : 0) | (rw < 0.0f ? 4 : 0);
    q.e2 = make_float4(t0, t1, __int_as_float(o0), __int_as_float(0));
    q.e3 = make_float4(os.x, os.y, os.z, __int_as_float(nci));
    q.e4 = make_float4(is.x, is.y, is.z, iinv);
    q.e5 = make_float4(ia - pad, ia + pad, iw, __int_as_float(flags));
    q.e6 = make_float4(ra - pad, ra + pad, rw, rinv);
    q.e7 = make_int4(nr, mo, mi, (int)cs_off);
    return nitems;
}

// Deals the items of the 32 lines in sp to the lanes of the warp and tests
// the grains of their cell runs; hit(owner_line, g) is called for every grain
// g inside the owner line's tube.  n_items is this lane's own line's item
// count (0 for an idle lane); tests counts the membership tests this lane
// performs.
//
// A round gives one item to each lane.  The lane resolves the item's non-empty
// row ranges (usually one or two; a rare third or later row is tested by the
// lane itself).  The warp then deals all grains of the round's first two row
// ranges to its lanes, 32 at a time: lane j takes grain base + j of the
// concatenated ranges, finds the range owning it from the ranges that start
// in this pass (an OR-reduction of one-hot start bits and a popcount) and reads
// the range from a per-warp table (tbl) indexed by that rank.  So every pass
// tests 32 grains, however unevenly the rows of the round hold them.
// Grain k of the two cell orders back to back (k < N: x-row list, k >= N:
// y-row list): 8-byte packed coordinates (PACKED, w = 0) or the 16-byte
// record with the canonical index.
template <bool PACKED>
__device__ __forceinline__ int4 grain_at(const Batch &b, u32 k) {
    if (PACKED) return unpack_xyz(b.gp[k]);
    return b.gc[k];
}

// Grains of its own rows a lane tests itself before the rest is dealt (1 was
// the fastest of 0, 1, 2, 3, 4 and 6 on the batched, dense, PR1 and stress
// workloads: the lane's own loads touch up to 32 lines per warp load, so more
// than one costs more than dealing them).
constexpr int WALK_SERIAL = 1;

// Adds 1 to a shared-memory counter when p holds, without a branch.
__device__ __forceinline__ void red_add_if(bool p, u32 *addr) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared.add.u32 [%1], 1;\n\t}" ::"r"((unsigned)p),
                 "r"(a)
                 : "memory");
}

// COUNT: in the dealt passes every grain inside the tube of line s adds 1 to
// cnt[s] by a predicated reduction; otherwise hit(s, g) is called for it.
template <bool PACKED, bool COUNT, int SERIAL, class Hit>
__device__ __forceinline__ void warp_items(const Batch &b, SeedTab &sp, int4 *tbl, int n_items, u32 &tests,
                                           u32 *cnt, Hit &&hit) {
    const int lane = threadIdx.x & 31;
    const unsigned lane_le = 0xffffffffu >> (31 - lane);
    const unsigned lane_lt = lane_le >> 1;
    int incl = n_items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - n_items;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (n_items > 0) sp.v[2][lane].w = excl;
    __syncwarp();
    for (int ibase = 0; ibase < total; ibase += 32) {
        // lines whose first item falls in this round mark its position;
        // a lane's owner is the last line started at or before it
        const bool starts = n_items > 0 && excl >= ibase && excl < ibase + 32;
        const unsigned smask = __reduce_or_sync(0xffffffffu, starts ? (1u << (excl - ibase)) : 0u);
        const int before = __popc(__ballot_sync(0xffffffffu, n_items > 0 && excl < ibase));
        const int own = before + __popc(smask & lane_le) - 1;
        const int item = ibase + lane;
        u32 b0 = 0, n0 = 0, b1 = 0, n1 = 0;
        u32 loff = 0;   // N for the y-row list (its cell order follows the x-row one)
        if (item < total) {
            const float4 e2 = sp.f4(2, own), e3 = sp.f4(3, own);
            const int co = __float_as_int(e2.z) + (item - __float_as_int(e2.w));
            const float olo = fmaf((float)co, e3.y, e3.x);
            const float ta = fmaxf(e2.x, olo), tb = fminf(e2.y, olo + e3.z);
            if (ta <= tb) {
                const float4 e4 = sp.f4(4, own), e5 = sp.f4(5, own), e6 = sp.f4(6, own);
                const int4 e7 = sp.i4(7, own);
                const int flags = __float_as_int(e5.w);
                const int list = flags & 1;
                loff = list ? (u32)b.N : 0u;
                const bool ineg = (flags & 2) != 0, rneg = (flags & 4) != 0;
                // inner cells reached over [ta, tb]
                const float il = fmaf(ineg ? tb : ta, e5.z, e5.x), ih = fmaf(ineg ? ta : tb, e5.z, e5.y);
                const int nci = __float_as_int(e3.w);
                const int ci0 = max(0, floor_i(il * e4.w)), ci1 = min(nci - 1, floor_i(ih * e4.w));
                const u32 *__restrict__ cs = (list ? b.cell_start_y : b.cell_start) + (u32)e7.w;
                const int rowo = co * e7.y;
                // cell run of inner cell ci: [s0, s1) into cs, or s0 = s1 = 0
                auto run = [&](int ci, int &s0, int &s1) {
                    s0 = s1 = 0;
                    const float vlo = fmaf((float)ci, e4.y, e4.x);
                    const float za = fmaxf(ta, vlo), zb = fminf(tb, vlo + e4.z);
                    const float r0 = fmaf(rneg ? zb : za, e6.z, e6.x), r1 = fmaf(rneg ? za : zb, e6.z, e6.y);
                    const int cr0 = max(0, floor_i(r0 * e6.w)), cr1 = min(e7.x - 1, floor_i(r1 * e6.w));
                    if (za <= zb && cr0 <= cr1 && ci <= ci1) {
                        const int row = rowo + ci * e7.z;
                        s0 = row + cr0;
                        s1 = row + cr1 + 1;
                    }
                };
                // the first two inner cells (almost every item has at most two):
                // their four start-table loads are issued together
                int sa0, sa1, sb0, sb1;
                run(ci0, sa0, sa1);
                run(ci0 + 1, sb0, sb1);
                const u32 ba = cs[sa0], ea = cs[sa1], bb = cs[sb0], eb = cs[sb1];
                if (ea != ba) {
                    b0 = ba;
                    n0 = ea - ba;
                }
                if (eb != bb) {
                    if (n0 == 0) {
                        b0 = bb;
                        n0 = eb - bb;
                    } else {
                        b1 = bb;
                        n1 = eb - bb;
                    }
                }
                for (int ci = ci0 + 2; ci <= ci1; ++ci) {
                    int s0, s1;
                    run(ci, s0, s1);
                    const u32 beg = cs[s0], end = cs[s1];
                    if (end == beg) continue;
                    if (n0 == 0) {
                        b0 = beg;
                        n0 = end - beg;
                    } else if (n1 == 0) {
                        b1 = beg;
                        n1 = end - beg;
                    } else {   // rare: a third row, tested by this lane alone
                        const int4 e0 = sp.i4(0, own), e1 = sp.i4(1, own);
                        const int3 a = make_int3(e0.x, e0.y, e0.z), d = make_int3(e0.w, e1.x, e1.y);
                        const long long R =
                            (long long)(((unsigned long long)(unsigned)e1.w << 32) | (unsigned)e1.z);
                        tests += end - beg;
                        for (u32 k = beg; k < end; ++k) {
                            const int4 g = grain_at<PACKED>(b, loff + k);
                            if (in_tube(g, a, d, R)) hit(own, g);
                        }
                    }
                }
            }
        }
        tests += n0 + n1;
        if (SERIAL > 0 && __any_sync(0xffffffffu, n0 + n1 > 0)) {
            // the first SERIAL grains of its rows each lane tests itself, with its
            // line's parameters in registers (cheaper per test than dealing);
            // only the grains beyond them are dealt over the warp
            const u32 s0 = min(n0, (u32)SERIAL), s1 = min(n1, (u32)SERIAL - s0);
            if (s0 + s1 > 0) {
                const int4 e0 = sp.i4(0, own), e1 = sp.i4(1, own);
                const long long R = (long long)(((unsigned long long)(unsigned)e1.w << 32) | (unsigned)e1.z);
                const int3 a = make_int3(e0.x, e0.y, e0.z), d = make_int3(e0.w, e1.x, e1.y);
#pragma unroll
                for (int j = 0; j < SERIAL; ++j) {
                    if ((u32)j < s0 + s1) {
                        const u32 k = loff + ((u32)j < s0 ? b0 + (u32)j : b1 + ((u32)j - s0));
                        const int4 g = grain_at<PACKED>(b, k);
                        const bool h = in_tube(g, a, d, R);
                        if (COUNT) red_add_if(h, &cnt[own]);
                        else if (h) hit(own, g);
                    }
                }
            }
            b0 += s0;
            n0 -= s0;
            b1 += s1;
            n1 -= s1;
        }
        // deal the remaining grains of all lanes' first two rows over the warp
        const u32 n = n0 + n1;
        u32 rin = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(0xffffffffu, rin, o);
            if (lane >= o) rin += v;
        }
        const u32 rtotal = __shfl_sync(0xffffffffu, rin, 31);
        const u32 rex = rin - n;
        const unsigned nonempty = __ballot_sync(0xffffffffu, n > 0);
        if (n > 0)   // offsets into the two lists back to back
            tbl[__popc(nonempty & lane_lt)] =
                make_int4((int)(b0 + loff - rex), (int)(rex + n0), (int)(b1 + loff - rex - n0), own);
        __syncwarp();
        // two passes per iteration, so that their table, geometry and grain
        // loads overlap; a last part of at most 32 grains takes one pass
        u32 base = 0;
        for (; base + 32 < rtotal; base += 64) {
            const bool st0 = n > 0 && rex >= base && rex < base + 32;
            const bool st1 = n > 0 && rex >= base + 32 && rex < base + 64;
            const unsigned sm0 = __reduce_or_sync(0xffffffffu, st0 ? (1u << (rex - base)) : 0u);
            const unsigned sm1 = __reduce_or_sync(0xffffffffu, st1 ? (1u << (rex - base - 32)) : 0u);
            const unsigned bm = __ballot_sync(0xffffffffu, n > 0 && rex < base);
            const int bef0 = __popc(bm), bef1 = bef0 + __popc(sm0);
            const u32 i0 = base + lane, i1 = i0 + 32;
            const bool v1 = i1 < rtotal;
            const int4 t0 = tbl[bef0 + __popc(sm0 & lane_le) - 1];
            const int4 t1 = tbl[v1 ? bef1 + __popc(sm1 & lane_le) - 1 : 0];
            const u32 k0 = i0 + (u32)(i0 < (u32)t0.y ? t0.x : t0.z);
            const u32 k1 = i1 + (u32)(i1 < (u32)t1.y ? t1.x : t1.z);
            const int ow0 = t0.w, ow1 = t1.w;
            const int4 p0 = sp.i4(0, ow0), q0 = sp.i4(1, ow0), p1 = sp.i4(0, ow1), q1 = sp.i4(1, ow1);
            const int4 g0 = grain_at<PACKED>(b, k0);
            int4 g1 = make_int4(0, 0, 0, 0);
            if (v1) g1 = grain_at<PACKED>(b, k1);
            const long long R0 = (long long)(((unsigned long long)(unsigned)q0.w << 32) | (unsigned)q0.z);
            const long long R1 = (long long)(((unsigned long long)(unsigned)q1.w << 32) | (unsigned)q1.z);
            const bool h0 = in_tube(g0, make_int3(p0.x, p0.y, p0.z), make_int3(p0.w, q0.x, q0.y), R0);
            const bool h1 = v1 && in_tube(g1, make_int3(p1.x, p1.y, p1.z), make_int3(p1.w, q1.x, q1.y), R1);
            if (COUNT) {
                red_add_if(h0, &cnt[ow0]);
                red_add_if(h1, &cnt[ow1]);
            } else {
                if (h0) hit(ow0, g0);
                if (h1) hit(ow1, g1);
            }
        }
        if (base < rtotal) {
            const bool st = n > 0 && rex >= base && rex < base + 32;
            const unsigned sm = __reduce_or_sync(0xffffffffu, st ? (1u << (rex - base)) : 0u);
            const int bef = __popc(__ballot_sync(0xffffffffu, n > 0 && rex < base));
            const u32 i = base + lane;
            if (i < rtotal) {
                const int4 t = tbl[bef + __popc(sm & lane_le) - 1];
                const u32 k = i + (u32)(i < (u32)t.y ? t.x : t.z);
                const int ow = t.w;
                const int4 e0 = sp.i4(0, ow), e1 = sp.i4(1, ow);
                const int4 g = grain_at<PACKED>(b, k);
                const long long R = (long long)(((unsigned long long)(unsigned)e1.w << 32) | (unsigned)e1.z);
                const bool h = in_tube(g, make_int3(e0.x, e0.y, e0.z), make_int3(e0.w, e1.x, e1.y), R);
                if (COUNT) red_add_if(h, &cnt[ow]);
                else if (h) hit(ow, g);
            }
        }
        __syncwarp();   // the table is rewritten by the next round
    }
}

// Seed generation inside the tube-count kernel.
//
// Seeds (Section 2) are the pairs of grains of one view with
// seed_min^2 <= |g_b - g_a|^2 < seed_max^2, each pair once (a of lower
// canonical rank).  A warp takes SG origins a at a time (1, 2 or 4, a tuning
// choice compiled into one kernel each; consecutive in the
// x-row cell order, one work ticket).  The cell rows that can hold their
// partners -- the (y, z) cells within seed_max - 1 of a, each an x run from
// a's cell to the largest admissible dx -- are dealt to the lanes in rounds
// of 32, and the grains of a round's rows are tested 32 per pass (owner row
// found from one-hot start bits, as in the tube walk).  Accepted pairs queue
// in shared memory; the tube walk takes them 32 at a time.  So seeds are
// walked in the order origin, row, x, and concurrently running warps work on
// nearby origins: no seed list is written to memory.
constexpr int SQ = 64;         // seed queue: < 32 waiting + one pass

template <int SG>
struct GenSm {
    int4 og[SG];      // origin: x, y, z, canonical index
    int4 oc[SG];      // cx0, cx1, cy0, cz0
    int2 on[SG];      // y cells per z slab, cell-table offset of the view
    int ofirst[SG];   // first row item of each origin (the group's total if none)
    int2 tbl[32];     // round's non-empty rows: first position minus pass position, owner origin
    uint2 rr[32];     // per lane: pass position and length of the lane's row in the round
    int ov[SG];       // view of each origin
    int2 q[SQ];       // seeds waiting for the tube walk (lo, hi)
    int qv[SQ];       // their views
};

struct GenState {
    int gtotal = 0;   // row items of the current origin group
    int ibase = 0;    // first row item of the current round
    u32 rtotal = 0;   // grains of the current round
    u32 pbase = 0;    // next pass position in the round
    u32 cnt = 0;      // queued seeds
    u32 pair_tests = 0;   // seed-window tests made by this lane (far below 2^32 in one launch)
};

// Takes the next SG origins; false when none is left.
template <int SG>
__device__ __forceinline__ bool gen_group(const Batch &b, GenSm<SG> &sm, GenState &gs) {
    const int lane = threadIdx.x & 31;
    u64 g0 = 0;
    if (lane == 0) g0 = atomicAdd(&b.ctl->ticket[0], (u64)SG);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    const u64 N = (u64)b.N;
    if (g0 >= N) return false;
    const int reach = b.smax - 1;   // >= 0: seed_max >= 1
    int nrows = 0;
    if (lane < SG && g0 + lane < N) {
        const int4 g = b.gc[g0 + lane];
        const int v = view_of(b.goff, b.V, g.w);
        const int cx0 = g.x / b.cs[0];
        const int cx1 = min(b.nc[0] - 1, (g.x + reach) / b.cs[0]);
        const int cy0 = max(0, g.y - reach) / b.cs[1];
        const int cy1 = min(b.nc[1] - 1, (g.y + reach) / b.cs[1]);
        const int cz0 = max(0, g.z - reach) / b.cs[2];
        const int cz1 = min(b.nc[2] - 1, (g.z + reach) / b.cs[2]);
        const int ny = cy1 - cy0 + 1;
        nrows = ny * (cz1 - cz0 + 1);
        sm.og[lane] = g;
        sm.oc[lane] = make_int4(cx0, cx1, cy0, cz0);
        sm.on[lane] = make_int2(ny, (int)((u32)v * (u32)b.ncell));
        sm.ov[lane] = v;
    }
    int incl = nrows;
#pragma unroll
    for (int o = 1; o < SG; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane < SG) sm.ofirst[lane] = incl - nrows;
    gs.gtotal = __shfl_sync(0xffffffffu, incl, SG - 1);
    gs.ibase = 0;
    __syncwarp();
    return true;
}

// Resolves the rows of the round at gs.ibase into the pass table.
template <int SG>
__device__ __forceinline__ void gen_round(const Batch &b, GenSm<SG> &sm, GenState &gs) {
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const int item = gs.ibase + lane;
    u32 beg = 0, n = 0;
    int own = 0;
    if (item < gs.gtotal) {
        // owner: the last origin whose first item is at or before this one
        // (an origin without rows has ofirst = gtotal and is never chosen)
#pragma unroll
        for (int o = 1; o < SG; ++o) own += sm.ofirst[o] <= item ? 1 : 0;
        const int4 g = sm.og[own], oc = sm.oc[own];
        const int2 on = sm.on[own];
        const int j = item - sm.ofirst[own];
        const int jz = j / on.x;
        const int cy = oc.z + (j - jz * on.x), cz = oc.w + jz;
        const long long rz = max(0, max(cz * b.cs[2] - g.z, g.z - (cz * b.cs[2] + b.cs[2] - 1)));
        const long long ry = max(0, max(cy * b.cs[1] - g.y, g.y - (cy * b.cs[1] + b.cs[1] - 1)));
        // the row's nearest point is at least (ry, rz) away in (y, z): it holds
        // partners only up to dx^2 <= seed_max^2 - 1 - ry^2 - rz^2
        const long long left = b.smax2 - 1 - ry * ry - rz * rz;
        if (left >= 0) {
            const int cxr = min(oc.y, (g.x + isqrt_ll(left)) / b.cs[0]);
            const u32 *cs = b.cell_start + (u32)on.y + (size_t)(cz * b.nc[1] + cy) * b.nc[0];
            beg = cs[oc.x];
            n = cs[cxr + 1] - beg;
        }
    }
    u32 rin = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, rin, o);
        if (lane >= o) rin += t;
    }
    const u32 rex = rin - n;
    const unsigned nonempty = __ballot_sync(0xffffffffu, n > 0);
    if (n > 0) sm.tbl[__popc(nonempty & lane_lt)] = make_int2((int)(beg - rex), own);
    sm.rr[lane] = make_uint2(rex, n);
    gs.rtotal = __shfl_sync(0xffffffffu, rin, 31);
    gs.pbase = 0;
    __syncwarp();
}

// One pass of 32 grain tests, appending the accepted pairs to the queue;
// false when every origin is done.
template <int SG>
__device__ __forceinline__ bool gen_pass(const Batch &b, GenSm<SG> &sm, GenState &gs) {
    while (gs.pbase >= gs.rtotal) {
        gs.ibase += 32;
        if (gs.ibase >= gs.gtotal && !gen_group(b, sm, gs)) return false;
        gen_round(b, sm, gs);
    }
    const int lane = threadIdx.x & 31;
    const unsigned lane_le = 0xffffffffu >> (31 - lane), lane_lt = lane_le >> 1;
    const uint2 r = sm.rr[lane];
    const u32 base = gs.pbase;
    const bool st = r.y > 0 && r.x >= base && r.x < base + 32;
    const unsigned pm = __reduce_or_sync(0xffffffffu, st ? (1u << (r.x - base)) : 0u);
    const int bef = __popc(__ballot_sync(0xffffffffu, r.y > 0 && r.x < base));
    const u32 i = base + lane;
    bool hit = false;
    int lo = 0, hi = 0, view = 0;
    if (i < gs.rtotal) {
        const int2 t = sm.tbl[bef + __popc(pm & lane_le) - 1];
        const int4 h = b.gc[i + (u32)t.x];
        const int4 g = sm.og[t.y];
        const long long dx = h.x - g.x, dy = h.y - g.y, dz = h.z - g.z;
        const long long d2 = dx * dx + dy * dy + dz * dz;
        hit = h.w > g.w && d2 >= b.smin2 && d2 < b.smax2;
        lo = g.w;
        hi = h.w;
        view = sm.ov[t.y];
        ++gs.pair_tests;
    }
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (hit) {
        const int slot = gs.cnt + __popc(hm & lane_lt);
        sm.q[slot] = make_int2(lo, hi);
        sm.qv[slot] = view;
    }
    gs.cnt += __popc(hm);
    gs.pbase = base + 32;
    __syncwarp();
    return true;
}

template <int SG>
__global__ void __launch_bounds__(TW * 32, 4) k_tube_count(Batch b, Work w, int record) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    __shared__ SeedTab sp[TW];
    __shared__ int4 tbl[TW][32];
    __shared__ u32 scount[TW][32];
    __shared__ GenSm<SG> gsm[TW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    u32 tests = 0, hits = 0;   // per thread: far below 2^32 in one launch
    u64 nseeds = 0;            // per warp (lane 0)
    GenState gs;               // empty: the first pass takes a work ticket
    bool more = true;
    for (;;) {
        while (gs.cnt < 32 && more) more = gen_pass(b, gsm[wib], gs);
        if (gs.cnt == 0) break;
        const u32 m = min(gs.cnt, 32u);
        const bool valid = lane < (int)m;
        int lo = 0, hi = 0, view = 0, n_items = 0;
        if (valid) {
            const int2 sd = gsm[wib].q[lane];
            lo = sd.x;
            hi = sd.y;
            view = gsm[wib].qv[lane];
        }
        __syncwarp();
        if (lane + 32 < (int)gs.cnt) {
            gsm[wib].q[lane] = gsm[wib].q[lane + 32];
            gsm[wib].qv[lane] = gsm[wib].qv[lane + 32];
        }
        gs.cnt -= m;
        nseeds += m;
        if (valid) {
            SeedSm q;
            n_items = seed_setup(b, b.gr[lo], b.gr[hi], view, q);
            sp[wib].put(lane, q);
        }
        scount[wib][lane] = 0;
        __syncwarp();
        warp_items<true, true, WALK_SERIAL>(b, sp[wib], tbl[wib], n_items, tests, scount[wib],
                               [&](int own, int4) { atomicAdd(&scount[wib][own], 1u); });
        __syncwarp();
        const u32 count = valid ? scount[wib][lane] : 0u;
        hits += count;
        if (record) {   // diagnostic per-seed records, appended in blocks of 32
            u64 r0 = 0;
            if (lane == 0) r0 = atomicAdd(&b.ctl->n_record, (u64)m);
            r0 = __shfl_sync(0xffffffffu, r0, 0);
            if (valid) {
                const u64 s = r0 + lane;
                if (s < w.rec_cap) {   // indices into the batch's grains back to back
                    const int vbase = (int)b.goff[view];
                    w.rec_lo[s] = vbase + b.gr[lo].w;
                    w.rec_hi[s] = vbase + b.gr[hi].w;
                    w.rec_cnt[s] = (int)count;
                } else {
                    atomicOr(&b.ctl->error, ERRB_OVF_RECORD);
                }
            }
        }
        const bool is_cand = valid && count >= (u32)b.H;
        const unsigned cm = __ballot_sync(0xffffffffu, is_cand);
        if (cm) {
            const int leader = __ffs(cm) - 1;
            u64 base_idx = 0;
            if (lane == leader) base_idx = atomicAdd(&b.ctl->n_cand, (u64)__popc(cm));
            base_idx = __shfl_sync(0xffffffffu, base_idx, leader);
            if (is_cand) {
                const u64 idx = base_idx + __popc(cm & ((1u << lane) - 1u));
                if (idx < w.cand_cap) {
                    w.c_lo[idx] = lo;
                    w.c_hi[idx] = hi;
                    w.c_cnt[idx] = count;
                } else {
                    atomicOr(&b.ctl->error, ERRB_OVF_CAND);
                }
            }
        }
        __syncwarp();
    }
    const u64 wtests = warp_sum_u64(tests), whits = warp_sum_u64(hits);
    const u64 wpairs = warp_sum_u64(gs.pair_tests);
    if (lane == 0) {
        if (wtests) atomicAdd(&b.ctl->n_tests, wtests);
        if (wpairs) atomicAdd(&b.ctl->n_pair_tests, wpairs);
        if (whits) atomicAdd(&b.ctl->n_hits, whits);
        if (nseeds) atomicAdd(&b.ctl->n_seeds, nseeds);
    }
}

// Candidate keys: (2^21 - 1 - count) << 42 | rank_lo << 21 | rank_hi, so that
// ascending keys visit candidates by count descending, then ranks ascending.
// With sk not null, also the input of the candidate-order sort: the key on
// 3 * rbits bits and the candidate index.
__global__ void k_cand_keys(Batch b, Work w, u64 *sk, u32 *sv) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
        const int lo = w.c_lo[c], hi = w.c_hi[c];
        const int v = view_of(b.goff, b.V, lo);
        const u64 rlo = (u64)(lo - b.goff[v]), rhi = (u64)(hi - b.goff[v]);
        const u64 cnt = w.c_cnt[c];
        const u64 key = ((((1ull << 21) - 1ull) - cnt) << 42) | (rlo << 21) | rhi;
        w.c_key[c] = key;
        w.c_moff[c] = cnt;
        w.c_state[c] = CS_UNDECIDED;
        if (sk) {
            sk[c] = cand_sort_key(b, key);
            sv[c] = (u32)c;
        }
    }
}

// Member lists of the candidates: the same warp-balanced walk as the counts;
// each in-tube grain takes the next slot of its candidate's member range
// (a shared-memory cursor), so the order inside a list is arbitrary.
__global__ void __launch_bounds__(TW * 32, 4) k_member_fill(Batch b, Work w) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    if (b.ctl->n_members > w.member_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&b.ctl->error, ERRB_OVF_MEMBERS);
        return;
    }
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    __shared__ SeedTab sp[TW];
    __shared__ int4 tbl[TW][32];
    __shared__ u32 cursor[TW][32];            // next slot, relative to the candidate's first
    __shared__ unsigned long long mbase[TW][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *__restrict__ members = w.members;
    // lines walked together by a warp: 32, or fewer (at least 4) when the
    // candidates cannot give every warp of the grid 32; the rounds a warp
    // walks in sequence, not the work, then set the kernel's duration
    const u64 nwarps = (u64)gridDim.x * TW;
    const u64 per_warp = (nc + nwarps - 1) / nwarps;
    const int lines = per_warp >= 32 ? 32 : (per_warp < 4 ? 4 : (int)per_warp);
    const u64 tsize = lines == 32 ? ticket_size(nc) : (u64)lines;
    for (;;) {
    u64 c0 = 0;
    if (lane == 0) c0 = atomicAdd(&b.ctl->ticket[1], tsize);
    c0 = __shfl_sync(0xffffffffu, c0, 0);
    if (c0 >= nc) break;
    const u64 c1 = min(c0 + tsize, nc);
    for (u64 base = c0; base < c1; base += (u64)lines) {
        const u64 c = base + lane;
        int n_items = 0;
        if (lane < lines && c < c1) {
            const int lo = __ldcs(&w.c_lo[c]), hi = __ldcs(&w.c_hi[c]);
            SeedSm q;
            n_items = seed_setup(b, b.gr[lo], b.gr[hi], view_of(b.goff, b.V, lo), q);
            sp[wib].put(lane, q);
            cursor[wib][lane] = 0;
            mbase[wib][lane] = w.c_moff[c];
        }
        __syncwarp();
        u32 tests = 0;
        warp_items<false, false, WALK_SERIAL>(b, sp[wib], tbl[wib], n_items, tests, cursor[wib], [&](int own, int4 g) {
            members[mbase[wib][own] + atomicAdd(&cursor[wib][own], 1u)] = g.w;
        });
        __syncwarp();
    }
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

void launch_tube_count(const Batch &b, const Work &w, int record, cudaStream_t st) {
    if (b.gen_origins == 1) launch_dep(k_tube_count<1>, dim3(persistent_grid(8)), dim3(TW * 32), 0, st, b, w, record);
    else if (b.gen_origins == 4) launch_dep(k_tube_count<4>, dim3(persistent_grid(8)), dim3(TW * 32), 0, st, b, w, record);
    else launch_dep(k_tube_count<2>, dim3(persistent_grid(8)), dim3(TW * 32), 0, st, b, w, record);
}

void launch_cand_keys(const Batch &b, const Work &w, u64 *sort_k, u32 *sort_v, cudaStream_t st) {
    launch_dep(k_cand_keys, dim3(persistent_grid(4)), dim3(256), 0, st, b, w, sort_k, sort_v);
}

void launch_member_fill(const Batch &b, const Work &w, cudaStream_t st) {
    launch_dep(k_member_fill, dim3(persistent_grid(8)), dim3(TW * 32), 0, st, b, w);
}

}  // namespace et

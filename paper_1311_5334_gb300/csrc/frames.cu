// frames.cu -- the image front end: filtering and 3D grain recognition of raw
// camera frames (Section 2 of the paper, Fig. 2), from a batch of views to
// their grains, and the C ABI of include/et_frames.h.
//
// One kernel does both steps.  A block owns a tile of TX x TY pixels of one
// view and walks its frames front to back.  The frames reach shared memory
// by TMA (a 3D tensor map over the raw bytes, one box of TX x (TY + 2)
// pixels per frame: the tile plus one halo row above and below), through a
// ring of NSTAGE buffers with one mbarrier each.  The block's warps then run
// independently: each scans its four rows of the tile and, once done with
// a frame, counts itself out of that frame's stage; the last warp to let go
// of a stage loads the frame NSTAGE further on into it.  No block-wide
// barrier is taken inside the frame loop.
//
// Filtering is monotone in the raw value (non-increasing), so f > T holds
// exactly for raw values below a per-pixel cutoff: the count of raw values
// whose filtered value exceeds T, computed once per calibration by
// k_cutoff from the same formula.  The scan of a frame therefore compares 16
// raw bytes per lane against 16 cutoffs held in registers (four byte-wise
// SIMD compares).  The warp then evaluates its rare candidates one at a time
// with one neighbour of the 3 x 3 x 3 box per lane (halo columns outside the
// tile come from global memory): one ballot decides the maximum test with the
// raster-order tie rule (lanes are in raster order, the candidate is lane 13),
// warp reductions give the exact centre-of-mass sums.  A grain is appended
// with its key (view, frame, row, column); a radix sort by key then gives
// every view's grains in raster order, independent of the order blocks ran in.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "et_frames.h"
#include "runtime.h"

namespace et {

namespace {

constexpr int TX = 256, TY = 16, FT = 256;
constexpr int LPR = TX / 16;              // lanes per tile row (16 pixels each)
constexpr int RPW = 32 / LPR;             // tile rows per warp
constexpr int NSTAGE = 6;
constexpr int STAGE_BYTES = TX * (TY + 2);
// calibration tile: the pixel tile with one halo row above and below and 16
// columns on either side (so that it loads as aligned 16-byte vectors); pixel
// column lx of the tile is calibration column lx + 16
constexpr int HX = TX + 32, HY = TY + 2;
static_assert(FT == LPR * TY, "one thread per 16 pixels of the tile");
static_assert(STAGE_BYTES % 128 == 0, "stage buffers stay 128-byte aligned");
static_assert(TX <= 256 && TY + 2 <= 256, "TMA box edges are at most 256 elements");

enum : u32 { FRB_OVF = 1u << 0, FRB_TIMEOUT = 1u << 1 };

struct FrCtl {
    u64 n_grains;   // grains appended (may exceed the capacity)
    u64 n_cand;     // voxels with f > T
    u32 error;      // FRB_* bits
    u32 bar[2];     // grid barrier of the sort and the scan
    u32 pad;
};

struct FrArgs {
    int W, H, D, P, V;
    int T;
    int num[3], den[3];
    int tiles_x;
    const unsigned char *raw;   // device copy of the views (halo columns of candidates)
    const unsigned char *gain, *thr, *cut;   // padded tables: pixel (x, y) at (y + 1) * TP + x + 16
    int TP;
    FrCtl *ctl;
    u64 *keys;
    u32 *vals;
    int4 *rec;
    u64 cap;
    u32 *view_count;
};

__device__ __forceinline__ int filt(int raw, int g, int t) {
    const int v = min(255, ((255 - raw) * g + 64) >> 7);
    return max(0, v - t);
}

// Per pixel: the number of raw values r in [0, 255] with filt(r) > T; by
// monotonicity exactly the r below it.  filt(255) = 0, so it is at most 255.
__global__ void k_cutoff(const unsigned char *gain, const unsigned char *thr, unsigned char *cut, int n, int T) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = gain[i], t = thr[i];
        int c = 0;
        for (int r = 0; r < 256; ++r) c += filt(r, g, t) > T;
        cut[i] = (unsigned char)c;
    }
}

__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 global_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase `parity` of the mbarrier at bar; false after about a
// second without completion (the caller records a timeout and leaves).
__device__ __forceinline__ bool mbar_try(u32 bar, u32 parity) {
    u32 done;
    // suspends for up to 2 us while the phase is pending instead of spinning
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(2000)
        : "memory");
    return done != 0;
}

__device__ __noinline__ bool mbar_wait_slow(u32 bar, u32 parity) {
    const u64 t0 = global_ns();
    for (u32 it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 7) == 7 && global_ns() - t0 > 1000000000ull) return false;
        if (it > (1u << 26)) return false;
    }
}

// Waits for the phase `parity` of the mbarrier at bar; false after about a
// second without completion (the caller records a timeout and leaves).
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity) {
    return mbar_try(bar, parity) || mbar_wait_slow(bar, parity);
}

__global__ void __launch_bounds__(FT, 5) k_recognize(const __grid_constant__ CUtensorMap tmap, FrArgs a) {
    __shared__ __align__(128) unsigned char stage[NSTAGE][STAGE_BYTES];
    __shared__ __align__(16) unsigned char gsm[HY][HX];
    __shared__ __align__(16) unsigned char tsm[HY][HX];
    __shared__ __align__(8) u64 mbar[NSTAGE];
    __shared__ int released[NSTAGE];   // warps done with the frame a stage holds
    __shared__ int issued;             // frames whose load has been issued

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int v = blockIdx.y;
    const int x0 = (blockIdx.x % a.tiles_x) * TX, y0 = (blockIdx.x / a.tiles_x) * TY;
    const int D = a.D;

    auto issue = [&](int j, int s) {   // TMA of frame j of this view into stage s = j % NSTAGE
        const u32 bar = smem_addr(&mbar[s]);
        // the stage was last read by ordinary loads of every warp (released below)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_addr(stage[s])),
            "l"(&tmap), "r"(x0), "r"(y0 - 1), "r"(v * D + j), "r"(bar)
            : "memory");
    };

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[s])) : "memory");
            released[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issued = min(D, NSTAGE);
    }
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < min(D, NSTAGE); ++j) issue(j, j);

    // calibration of the tile with its halo and margins (zero outside the frame)
    for (int i = tid; i < HY * (HX / 16); i += FT) {
        const int row = i / (HX / 16), c16 = (i % (HX / 16)) * 16;
        const size_t off = (size_t)(y0 + row) * a.TP + x0 + c16;
        *(uint4 *)&gsm[row][c16] = __ldg((const uint4 *)(a.gain + off));
        *(uint4 *)&tsm[row][c16] = __ldg((const uint4 *)(a.thr + off));
    }
    // this lane's 16 pixels: row ry of the tile (warp w scans rows RPW w ..
    // RPW w + RPW - 1), columns cx .. cx + 15, and their cutoffs
    const int ry = tid / LPR, cx = (tid % LPR) * 16;
    u32 cw[4];   // cutoffs of the 16 pixels, 4 per word, low 7 bits of each byte
    u32 ch[4];   // and their high bits
    {
        const uint4 c = __ldg((const uint4 *)(a.cut + (size_t)(y0 + ry + 1) * a.TP + x0 + cx + 16));
        const u32 cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cw[k] = cv[k] & 0x7f7f7f7fu;
            ch[k] = cv[k] & 0x80808080u;
        }
    }
    __syncthreads();   // calibration tiles complete; from here on the warps run independently

    // this lane's neighbour in a candidate's 3 x 3 x 3 box (lanes 0..26, raster
    // order, so lane 13 is the candidate and lanes below it come before it)
    const int ndz = lane / 9 - 1, ndy = (lane / 3) % 3 - 1, ndx = lane % 3 - 1;
    // the centroid coordinate this lane computes for a grain (lanes 0, 1, 2)
    const int cnum = lane == 0 ? a.num[0] : (lane == 1 ? a.num[1] : a.num[2]);
    const int cden = lane == 0 ? a.den[0] : (lane == 1 ? a.den[1] : a.den[2]);
    u32 ncand = 0;
    u32 fprev[4] = {0u, 0u, 0u, 0u};
    bool timed_out = false;
    // stages of frames z - 1, z, z + 1 and the phase parity of frame z + 1
    int sm1 = NSTAGE - 1, s0 = 0, sp1 = 1;
    u32 par1 = 0;
    if (!mbar_wait(smem_addr(&mbar[0]), 0)) timed_out = true;
    for (int z = 0; z < D && !timed_out; ++z) {
        if (z + 1 < D && !mbar_wait(smem_addr(&mbar[sp1]), par1)) {
            timed_out = true;
            break;
        }
        // scan: this lane's pixels of frame z whose raw value is below the cutoff
        const unsigned char *f0 = stage[s0];
        const uint4 rw = *(const uint4 *)&f0[(ry + 1) * TX + cx];
        // per byte raw < cutoff, four bytes a word (SWAR): with the byte's high
        // bits ra, ca and d = (raw | 0x80) - (cutoff & 0x7f) (no borrow between
        // bytes), raw < cutoff iff (!ra & ca) | (ra == ca & !d7)
        const u32 rwv[4] = {rw.x, rw.y, rw.z, rw.w};
        u32 lt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const u32 d = (rwv[k] | 0x80808080u) - cw[k];
            lt[k] = ((~rwv[k] & ch[k]) | (~(rwv[k] ^ ch[k]) & ~d)) & 0x80808080u;
        }
        u32 bits = 0;   // bit k: pixel cx + k
        if (lt[0] | lt[1] | lt[2] | lt[3]) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const u32 m = lt[k] >> 7;   // bits 0, 8, 16, 24
                bits |= ((m & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u)) << (4 * k);
            }
        }
        // exact pruning inside the lane, before the warp-wide test: filtered
        // values of the lane's candidates (only candidates can beat a
        // candidate: every other voxel has f <= T).  Of two candidates next to
        // each other in x, the earlier loses iff the later is brighter, else
        // the later loses; a candidate loses to the same pixel one frame back
        // if that was at least as bright.  fprev: this lane's filtered values
        // of frame z - 1 (candidates only, else 0), a byte per pixel.
        u32 fnow[4] = {0u, 0u, 0u, 0u};
        if (bits) {
            ncand += __popc(bits);
            u32 keep = bits, b = bits;
            int pk = -2, pf = 0;
            while (b) {
                const int k = __ffs(b) - 1;
                b &= b - 1;
                const int wsel = k >> 2, sh = 8 * (k & 3);
                const u32 word = wsel == 0 ? rwv[0] : (wsel == 1 ? rwv[1] : (wsel == 2 ? rwv[2] : rwv[3]));
                const u32 prev = wsel == 0 ? fprev[0] : (wsel == 1 ? fprev[1] : (wsel == 2 ? fprev[2] : fprev[3]));
                const int f = filt((word >> sh) & 0xffu, gsm[ry + 1][cx + k + 16], tsm[ry + 1][cx + k + 16]);
                if ((int)((prev >> sh) & 0xffu) >= f) keep &= ~(1u << k);
                if (pk == k - 1) {
                    if (pf >= f) keep &= ~(1u << k);
                    else keep &= ~(1u << pk);
                }
                pk = k;
                pf = f;
                const u32 ins = (u32)f << sh;
                fnow[0] |= wsel == 0 ? ins : 0u;
                fnow[1] |= wsel == 1 ? ins : 0u;
                fnow[2] |= wsel == 2 ? ins : 0u;
                fnow[3] |= wsel == 3 ? ins : 0u;
            }
            bits = keep;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) fprev[k] = fnow[k];
        unsigned pend = __ballot_sync(0xffffffffu, bits != 0);
        if (pend) {
            // per frame: this lane's neighbour (frame, and offsets in the stage and
            // calibration tiles) and whether its frame exists
            const int zz = z + ndz;
            const bool zin = lane < 27 && zz >= 0 && zz < D;
            const unsigned char *fr = stage[ndz < 0 ? sm1 : (ndz == 0 ? s0 : sp1)] + ndy * TX + ndx;
            // the warp evaluates its candidates one at a time, a neighbour per lane
            for (; pend; pend = __ballot_sync(0xffffffffu, bits != 0)) {
                const int src = __ffs(pend) - 1;
                const int k = __ffs(__shfl_sync(0xffffffffu, bits, src)) - 1;
                if (lane == src) bits &= bits - 1;
                const int lx = (src % LPR) * 16 + k, ly = warp * RPW + src / LPR;   // uniform
                const int gx = x0 + lx, gy = y0 + ly;
                const bool in = zin && (unsigned)(gy + ndy) < (unsigned)a.H && (unsigned)(gx + ndx) < (unsigned)a.W;
                const int sb = (ly + 1) * TX + lx;
                int r = 0;
                if (lx > 0 && lx < TX - 1) {   // uniform: the whole box is in the stage
                    if (in) r = fr[sb];
                } else if (in) {               // tile edge: halo columns from global memory
                    r = ((unsigned)(lx + ndx) < (unsigned)TX)
                            ? fr[sb]
                            : __ldg(&a.raw[(((size_t)v * D + zz) * a.H + gy + ndy) * (size_t)a.P + gx + ndx]);
                }
                const int cb = (ly + 1 + ndy) * HX + lx + ndx + 16;
                const int fq = in ? filt(r, (&gsm[0][0])[cb], (&tsm[0][0])[cb]) : -1;
                const int fpv = __shfl_sync(0xffffffffu, fq, 13);
                const bool beats = lane < 13 ? fq >= fpv : fq > fpv;
                if (__ballot_sync(0xffffffffu, beats)) continue;   // not a local maximum
                // centre-of-mass sums, two per reduction: S (< 2^13) below
                // Sx = sum w dx above; Sy + 4096 (sum of w dy + 128 over 32 lanes, in
                // [1801, 6391]) below Sz = sum w dz above
                const int w = max(fq, 0);
                const int p1 = __reduce_add_sync(0xffffffffu, (u32)(w + ndx * w * 65536));
                const int p2 = __reduce_add_sync(0xffffffffu, (u32)(ndy * w + 128 + ndz * w * 65536));
                const int S = p1 & 0xffff, SXo = (p1 - S) >> 16;
                const int SYo = (p2 & 0xffff) - 4096, SZo = (p2 - (p2 & 0xffff)) >> 16;
                // coordinate of axis `lane` (lanes 0..2), rounded half up:
                // floor((2 S g num + 2 So num + S den) / (2 S den)) with the voxel
                // index g and So the offset sum.  With A = 2 g num = a1 (2 den) + a0
                // it is a1 + floor((S a0 + 2 So num + S den) / (2 S den)), all in
                // int32: A < 2^30, S a0 < 9.1e8, |2 So num| < 3.1e8, S den < 4.6e8
                int c = 0;
                if (lane < 3) {
                    const int g = lane == 0 ? gx : (lane == 1 ? gy : z);
                    const int So = lane == 0 ? SXo : (lane == 1 ? SYo : SZo);
                    const int A = 2 * g * cnum, twoden = 2 * cden;
                    const int a1 = A / twoden, a0 = A - a1 * twoden;
                    const int n = S * a0 + 2 * So * cnum + S * cden, Q = S * twoden;
                    int q = n / Q;
                    if (n < 0 && q * Q != n) --q;
                    c = a1 + q;
                }
                const int Y = __shfl_sync(0xffffffffu, c, 1), Z = __shfl_sync(0xffffffffu, c, 2);
                if (lane == 0) {
                    const u64 slot = atomicAdd(&a.ctl->n_grains, 1ull);
                    if (slot < a.cap) {
                        a.keys[slot] = (u64)v * ((u64)D * a.H * a.W) + ((u64)z * a.H + gy) * a.W + gx;
                        a.vals[slot] = (u32)slot;
                        a.rec[slot] = make_int4(c, Y, Z, S);
                    } else {
                        atomicOr(&a.ctl->error, FRB_OVF);
                    }
                    atomicAdd(&a.view_count[v], 1u);
                }
            }
        }
        // frame z - 1 is no longer needed by this warp; the last warp to let go
        // of it reloads its stage with frame z + NSTAGE - 1
        __syncwarp();
        if (lane == 0 && z >= 1) {
            __threadfence_block();
            if (atomicAdd(&released[sm1], 1) == FT / 32 - 1) {
                released[sm1] = 0;
                __threadfence_block();
                const int j = z - 1 + NSTAGE;
                if (j < D) {
                    issue(j, sm1);
                    atomicAdd(&issued, 1);
                }
            }
        }
        sm1 = s0;
        s0 = sp1;
        if (++sp1 == NSTAGE) {
            sp1 = 0;
            par1 ^= 1u;
        }
    }
    ncand = __reduce_add_sync(0xffffffffu, ncand);
    if (lane == 0 && ncand) atomicAdd(&a.ctl->n_cand, (u64)ncand);
    if (timed_out && lane == 0) {
        // record the failure; the block's first warp then gives the copies still
        // in flight into its buffers a bounded chance to land before it exits
        atomicOr(&a.ctl->error, FRB_TIMEOUT);
    }
    __syncthreads();
    if (tid == 0 && (*(volatile u32 *)&a.ctl->error & FRB_TIMEOUT)) {
        const int n = *(volatile int *)&issued;
        for (int j = max(0, n - NSTAGE); j < n; ++j)
            if (!mbar_wait(smem_addr(&mbar[j % NSTAGE]), (j / NSTAGE) & 1)) break;
    }
}

// Grains in key order: xyz (int32 [n][3]) and pulse (int32 [n]).
__global__ void k_fr_gather(const FrCtl *ctl, u64 cap, const u32 *sorted_vals, const int4 *rec, int *xyz,
                            int *pulse) {
    const u64 n = min(ctl->n_grains, cap);
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const int4 r = rec[sorted_vals[i]];
        xyz[3 * i + 0] = r.x;
        xyz[3 * i + 1] = r.y;
        xyz[3 * i + 2] = r.z;
        pulse[i] = r.w;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

}  // namespace

// The front end of one camera (geometry and calibration) with its device buffers.
struct FramesRT {
    Ctx *ctx;
    et_frame_params p;
    Group g_tab, g_raw, g_out, g_ctl;
    unsigned char *gain = nullptr, *thr = nullptr, *cut = nullptr;
    FrCtl *ctl = nullptr;
    // run state
    int V = 0;
    const unsigned char *d_raw = nullptr;
    u64 cap = 0, want = 0;
    u64 *keys[2] = {nullptr, nullptr};
    u32 *vals[2] = {nullptr, nullptr};
    int4 *rec = nullptr;
    int *xyz = nullptr, *pulse = nullptr;
    u32 *view_count = nullptr, *view_off = nullptr;
    void *temp = nullptr;
    int sorted = 0, launches = 0;
    cudaStream_t run_stream = nullptr;
    cudaEvent_t ev[4] = {};   // run start, kernel start, kernel end, done
    cudaEvent_t handoff = nullptr;   // a batch's copy of the grains (et_frames_to_batch)
    bool handoff_pending = false;
    bool ran = false, settled = false;
    FrCtl hctl{};
    et_status run_status = ET_OK;
    float kernel_ms = 0.0f, run_ms = 0.0f;

    FramesRT(Ctx *c, const et_frame_params &pp) : ctx(c), p(pp) {}
    ~FramesRT() {
        if (ran) cudaEventSynchronize(ev[3]);
        if (handoff_pending) cudaEventSynchronize(handoff);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (handoff) cudaEventDestroy(handoff);
        g_tab.release(ctx);
        g_raw.release(ctx);
        g_out.release(ctx);
        g_ctl.release(ctx);
    }

    size_t pixels() const { return (size_t)p.width * p.height; }
    // padded calibration tables: pitch covering every tile plus 16-byte margins,
    // one row above and enough below for the last tile's halo
    int tiles_x() const { return (p.width + TX - 1) / TX; }
    int tiles_y() const { return (p.height + TY - 1) / TY; }
    int table_pitch() const { return tiles_x() * TX + 32; }
    size_t table_bytes() const { return (size_t)table_pitch() * ((size_t)tiles_y() * TY + 2); }
    size_t view_bytes() const { return (size_t)p.depth * p.height * p.row_pitch; }

    et_status init() {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(ET_ERR_CUDA, "event creation failed");
        if (cudaEventCreateWithFlags(&handoff, cudaEventDisableTiming) != cudaSuccess)
            return fail(ET_ERR_CUDA, "event creation failed");
        const size_t tb = align_up(table_bytes(), 256);
        if (!g_tab.reserve(ctx, 3 * tb)) return fail(ET_ERR_OOM, "calibration tables");
        gain = (unsigned char *)g_tab.base;
        thr = gain + tb;
        cut = thr + tb;
        if (!g_ctl.reserve(ctx, sizeof(FrCtl))) return fail(ET_ERR_OOM, "control block");
        ctl = (FrCtl *)g_ctl.base;
        return ET_OK;
    }

    et_status calibrate(const unsigned char *hg, const unsigned char *ht) {
        if (ran) cudaEventSynchronize(ev[3]);
        cudaStream_t st = ctx->stream;
        const size_t tp = (size_t)table_pitch();
        cudaError_t e = cudaMemsetAsync(gain, 0, 2 * align_up(table_bytes(), 256), st);   // gain and thr
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(gain + tp + 16, tp, hg, p.width, p.width, p.height, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(thr + tp + 16, tp, ht, p.width, p.width, p.height, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "calibration upload");
        // zero gain outside the frame gives a zero cutoff there
        const int n = (int)table_bytes();
        k_cutoff<<<std::min((n + 255) / 256, 152 * 8), 256, 0, st>>>(gain, thr, cut, n, p.grain_threshold);
        e = cudaStreamSynchronize(st);   // the caller may free its tables on return
        return e == cudaSuccess ? ET_OK : cuda_fail(e, "cutoff table");
    }

    et_status reserve_out(u64 need) {
        Carver c;
        auto carve = [&](Carver &cv) {
            keys[0] = cv.take<u64>(need);
            keys[1] = cv.take<u64>(need);
            vals[0] = cv.take<u32>(need);
            vals[1] = cv.take<u32>(need);
            rec = cv.take<int4>(need);
            xyz = cv.take<int>(3 * need);
            pulse = cv.take<int>(need);
            view_count = cv.take<u32>((size_t)V + 1);
            view_off = cv.take<u32>((size_t)V + 1);
            temp = cv.take<char>(std::max(radix_temp_bytes((long long)need), scan_temp_bytes((long long)V)));
        };
        carve(c);
        if (!g_out.reserve(ctx, c.off)) return fail(ET_ERR_OOM, "grain buffers (%llu grains)", (unsigned long long)need);
        Carver d;
        d.base = g_out.base;
        carve(d);
        cap = need;
        return ET_OK;
    }

    et_status enqueue(cudaStream_t st) {
        const int tiles_x = (p.width + TX - 1) / TX, tiles_y = (p.height + TY - 1) / TY;
        EncodeTiledFn enc = encode_fn();
        if (!enc) return fail(ET_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        CUtensorMap tmap;
        const cuuint64_t dims[3] = {(cuuint64_t)p.width, (cuuint64_t)p.height, (cuuint64_t)V * p.depth};
        const cuuint64_t strides[2] = {(cuuint64_t)p.row_pitch, (cuuint64_t)p.row_pitch * p.height};
        const cuuint32_t box[3] = {TX, TY + 2, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)d_raw, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(ET_ERR_CUDA, "tensor map encoding failed (%d)", (int)r);
        cudaMemsetAsync(ctl, 0, sizeof(FrCtl), st);
        cudaMemsetAsync(view_count, 0, sizeof(u32) * ((size_t)V + 1), st);
        FrArgs a;
        a.W = p.width;
        a.H = p.height;
        a.D = p.depth;
        a.P = p.row_pitch;
        a.V = V;
        a.T = p.grain_threshold;
        for (int k = 0; k < 3; ++k) {
            a.num[k] = p.pitch_num[k];
            a.den[k] = p.pitch_den[k];
        }
        a.tiles_x = tiles_x;
        a.raw = d_raw;
        a.gain = gain;
        a.thr = thr;
        a.cut = cut;
        a.TP = table_pitch();
        a.ctl = ctl;
        a.keys = keys[0];
        a.vals = vals[0];
        a.rec = rec;
        a.cap = cap;
        a.view_count = view_count;
        cudaEventRecord(ev[1], st);
        k_recognize<<<dim3(tiles_x * tiles_y, V), FT, 0, st>>>(tmap, a);
        cudaEventRecord(ev[2], st);
        const int bits = bits_for((u64)V * p.depth * p.height * p.width - 1);
        sorted = radix_sort_pairs_dev(keys[0], vals[0], keys[1], vals[1], (long long)cap, &ctl->n_grains, bits,
                                      temp, st, &ctl->error, FRB_TIMEOUT, ctl->bar);
        // recognition, the sort, the gather and the scan of the view counts
        launches = 1 + radix_sort_launches(bits) + 1 + 1;
        k_fr_gather<<<152 * 4, 256, 0, st>>>(ctl, cap, vals[sorted], rec, xyz, pulse);
        exclusive_scan_u32(view_count, view_off, (long long)V, temp, st, &ctl->error, FRB_TIMEOUT,
                           ctl->bar);   // view_off[V] = total
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? ET_OK : cuda_fail(e, "front-end launch");
    }

    et_status run(const unsigned char *raw, int nv, bool on_device, cudaStream_t st) {
        if (ran) cudaEventSynchronize(ev[3]);
        if (handoff_pending) cudaEventSynchronize(handoff);   // buffers may be regrown below
        handoff_pending = false;
        V = nv;
        const size_t bytes = (size_t)nv * view_bytes();
        cudaEventRecord(ev[0], st);
        if (on_device) {
            d_raw = raw;
        } else {
            if (!g_raw.reserve(ctx, bytes)) return fail(ET_ERR_OOM, "raw frame buffer (%zu bytes)", bytes);
            cudaError_t e = cudaMemcpyAsync(g_raw.base, raw, bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "raw frame upload");
            d_raw = (const unsigned char *)g_raw.base;
        }
        if (want == 0) want = 65536;
        const u64 guess = std::max<u64>(65536, (u64)nv * p.depth * p.height * p.width / 2000);
        want = std::max(want, guess);
        if (cap < want || view_count == nullptr || (size_t)V + 1 > last_views) {
            et_status s = reserve_out(std::max(want, cap));
            if (s != ET_OK) return s;
            last_views = (size_t)V + 1;
        }
        et_status s = enqueue(st);
        if (s != ET_OK) return s;
        cudaEventRecord(ev[3], st);
        run_stream = st;
        ran = true;
        settled = false;
        return ET_OK;
    }
    size_t last_views = 0;

    // Waits for the run; regrows and reruns after an output overflow.
    et_status settle() {
        if (!ran) return fail(ET_ERR_NOT_READY, "nothing has been run");
        if (settled) return run_status;
        for (int attempt = 0; attempt < 4; ++attempt) {
            cudaError_t e = cudaEventSynchronize(ev[3]);
            if (e != cudaSuccess) return run_status = cuda_fail(e, "front-end run");
            e = cudaMemcpy(&hctl, ctl, sizeof(FrCtl), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return run_status = cuda_fail(e, "control block read");
            if (hctl.error & FRB_TIMEOUT) {
                settled = true;
                return run_status = fail(ET_ERR_TIMEOUT, "a frame load did not complete in time");
            }
            if (!(hctl.error & FRB_OVF)) {
                cudaEventElapsedTime(&kernel_ms, ev[1], ev[2]);
                cudaEventElapsedTime(&run_ms, ev[0], ev[3]);
                settled = true;
                return run_status = ET_OK;
            }
            want = hctl.n_grains + hctl.n_grains / 8 + 1024;
            et_status s = reserve_out(want);
            if (s != ET_OK) return run_status = s;
            cudaStream_t st = ctx->stream;
            cudaEventRecord(ev[0], st);
            s = enqueue(st);
            if (s != ET_OK) return run_status = s;
            cudaEventRecord(ev[3], st);
        }
        settled = true;
        return run_status = fail(ET_ERR_CAPACITY, "grain buffer kept overflowing");
    }

    u64 n_grains() const { return std::min(hctl.n_grains, cap); }
};

}  // namespace et

using namespace et;

struct et_frames : public FramesRT {
    using FramesRT::FramesRT;
};

static et_status check_frame_params(const et_frame_params *p) {
    if (!p) return fail(ET_ERR_INVALID_ARG, "params is NULL");
    if (p->width < 1 || p->width > 4096 || p->height < 1 || p->height > 4096 || p->depth < 1 || p->depth > 1024)
        return fail(ET_ERR_INVALID_ARG, "frame size %d x %d x %d outside the limits", p->width, p->height, p->depth);
    if (p->row_pitch < p->width || p->row_pitch % 16 != 0)
        return fail(ET_ERR_INVALID_ARG, "row_pitch %d must be >= width and a multiple of 16", p->row_pitch);
    for (int k = 0; k < 3; ++k)
        if (p->pitch_num[k] < 1 || p->pitch_num[k] > 65535 || p->pitch_den[k] < 1 || p->pitch_den[k] > 65535)
            return fail(ET_ERR_INVALID_ARG, "voxel pitch of axis %d outside [1, 65535]", k);
    if (p->grain_threshold < 0 || p->grain_threshold > 254)
        return fail(ET_ERR_INVALID_ARG, "grain_threshold %d outside [0, 254]", p->grain_threshold);
    if (p->flags != 0) return fail(ET_ERR_INVALID_ARG, "flags must be 0");
    return ET_OK;
}

extern "C" {

et_status et_frames_create(et_ctx *ctx, const et_frame_params *params, const uint8_t *gain, const uint8_t *thr,
                           et_frames **out) {
    GUARD_BEGIN
    if (!ctx || !out || !gain || !thr) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    et_status s = check_frame_params(params);
    if (s != ET_OK) return s;
    cudaSetDevice(ctx->device);
    et_frames *fr = new et_frames(ctx, *params);
    s = fr->init();
    if (s == ET_OK) s = fr->calibrate(gain, thr);
    if (s != ET_OK) {
        delete fr;
        return s;
    }
    *out = fr;
    return ET_OK;
    GUARD_END
}

et_status et_frames_set_calibration(et_frames *fr, const uint8_t *gain, const uint8_t *thr) {
    GUARD_BEGIN
    if (!fr || !gain || !thr) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(fr->ctx->device);
    return fr->calibrate(gain, thr);
    GUARD_END
}

et_status et_frames_run(et_frames *fr, const uint8_t *raw, int32_t n_views, int32_t on_device, void *stream) {
    GUARD_BEGIN
    if (!fr || !raw) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    if (n_views < 1 || n_views > 65535)
        return fail(ET_ERR_INVALID_ARG, "n_views %d outside the limits", n_views);
    if (on_device && ((uintptr_t)raw & 15u)) return fail(ET_ERR_INVALID_ARG, "device frames must be 16-byte aligned");
    cudaSetDevice(fr->ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : fr->ctx->stream;
    return fr->run(raw, n_views, on_device != 0, st);
    GUARD_END
}

et_status et_frames_sync(et_frames *fr) {
    GUARD_BEGIN
    if (!fr) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(fr->ctx->device);
    return fr->settle();
    GUARD_END
}

et_status et_frames_fetch(et_frames *fr, int64_t *view_offsets, int32_t *xyz, int32_t *pulse, int64_t cap,
                          int64_t *n_grains) {
    GUARD_BEGIN
    if (!fr || !n_grains) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(fr->ctx->device);
    et_status s = fr->settle();
    if (s != ET_OK) return s;
    const int64_t n = (int64_t)fr->n_grains();
    *n_grains = n;
    if (n > 0 && (!xyz || cap < n)) return fail(ET_ERR_CAPACITY, "need room for %lld grains", (long long)n);
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpy(xyz, fr->xyz, sizeof(int32_t) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n > 0 && pulse) e = cudaMemcpy(pulse, fr->pulse, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && view_offsets) {
        std::vector<u32> off((size_t)fr->V + 1);
        e = cudaMemcpy(off.data(), fr->view_off, sizeof(u32) * off.size(), cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < off.size(); ++i) view_offsets[i] = off[i];
    }
    return e == cudaSuccess ? ET_OK : cuda_fail(e, "grain download");
    GUARD_END
}

et_status et_frames_to_batch(et_frames *fr, et_batch *batch, void *stream) {
    GUARD_BEGIN
    if (!fr || !batch) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    if (batch->ctx != fr->ctx) return fail(ET_ERR_INVALID_ARG, "batch and front end belong to different contexts");
    cudaSetDevice(fr->ctx->device);
    et_status s = fr->settle();
    if (s != ET_OK) return s;
    std::vector<u32> off((size_t)fr->V + 1);
    cudaError_t e = cudaMemcpy(off.data(), fr->view_off, sizeof(u32) * off.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "view offsets");
    std::vector<int64_t> off64(off.begin(), off.end());
    cudaStream_t st = stream ? (cudaStream_t)stream : fr->ctx->stream;
    if (batch->ran) cudaEventSynchronize(batch->done);
    s = batch->load(fr->xyz, off64.data(), fr->V, true, st);
    if (s == ET_OK) {
        cudaEventRecord(fr->handoff, st);   // the next run waits for this copy
        fr->handoff_pending = true;
    }
    return s;
    GUARD_END
}

et_status et_frames_stats_get(et_frames *fr, et_frames_stats *out) {
    if (!fr || !out) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    if (!fr->ran || !fr->settled || fr->run_status != ET_OK) return ET_OK;
    out->n_views = fr->V;
    out->n_voxels = (int64_t)fr->V * fr->p.depth * fr->p.height * fr->p.width;
    out->n_candidates = (int64_t)fr->hctl.n_cand;
    out->n_grains = (int64_t)fr->n_grains();
    out->kernel_ms = fr->kernel_ms;
    out->run_ms = fr->run_ms;
    out->kernel_launches = fr->launches;
    return ET_OK;
}

et_status et_frames_destroy(et_frames *fr) {
    if (!fr) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(fr->ctx->device);
    delete fr;
    return ET_OK;
}

}  // extern "C"

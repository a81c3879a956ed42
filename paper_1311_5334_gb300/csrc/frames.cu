// frames.cu -- the image front end: filtering and 3D grain recognition of raw
// camera frames (Section 2 of the paper, Fig. 2), from a batch of views to
// their grains, and the C ABI of include/et_frames.h.
//
// One kernel does both steps.  A block owns a tile of TX x TY pixels of one
// view and walks its frames front to back.  The frames reach shared memory
// by TMA (a 3D tensor map over the raw bytes, one box of TX x (TY + 2)
// pixels per frame: the tile plus one halo row above and below), through a
// ring of NSTAGE buffers with one mbarrier each, LOOKAHEAD frames ahead.
//
// Filtering is monotone in the raw value (non-increasing), so f > T holds
// exactly for raw values below a per-pixel cutoff: the count of raw values
// whose filtered value exceeds T, computed once per calibration by
// k_cutoff from the same formula.  The scan of a frame therefore compares 16
// raw bytes per thread against 16 cutoffs held in registers (four byte-wise
// SIMD compares) and queues the rare candidates in shared memory.  The block
// then evaluates the queued candidates one per thread: the filtered values
// of the 3 x 3 x 3 neighbourhood (halo columns outside the tile come from
// global memory), the maximum test with the raster-order tie rule, and the
// exact centre of mass in 64-bit integers.  A grain is appended with its key
// (view, frame, row, column); a radix sort by key then gives every view's
// grains in raster order, independent of the order blocks ran in.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "et_frames.h"
#include "runtime.h"

namespace et {

namespace {

constexpr int TX = 128, TY = 32, FT = 256;
constexpr int NSTAGE = 6, LOOKAHEAD = NSTAGE - 2;
constexpr int STAGE_BYTES = TX * (TY + 2);
constexpr int HX = TX + 2, HY = TY + 2;   // calibration tile with a one-pixel halo
static_assert(FT == (TX / 16) * TY, "one thread per 16 pixels of the tile");
static_assert(STAGE_BYTES % 128 == 0, "stage buffers stay 128-byte aligned");

enum : u32 { FRB_OVF = 1u << 0, FRB_TIMEOUT = 1u << 1 };

struct FrCtl {
    u64 n_grains;   // grains appended (may exceed the capacity)
    u64 n_cand;     // voxels with f > T
    u32 error;      // FRB_* bits
    u32 pad;
};

struct FrArgs {
    int W, H, D, P, V;
    int T;
    int num[3], den[3];
    int tiles_x;
    const unsigned char *raw;   // device copy of the views (halo columns of candidates)
    const unsigned char *gain, *thr, *cut;
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
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity) {
    const u64 t0 = global_ns();
    for (u32 it = 0;; ++it) {
        u32 done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
        if (it > (1u << 26)) return false;
    }
}

__global__ void __launch_bounds__(FT) k_recognize(const __grid_constant__ CUtensorMap tmap, FrArgs a) {
    __shared__ __align__(128) unsigned char stage[NSTAGE][STAGE_BYTES];
    __shared__ unsigned char gsm[HY][HX], tsm[HY][HX];
    __shared__ unsigned short queue[TX * TY];
    __shared__ __align__(8) u64 mbar[NSTAGE];
    __shared__ int qn[2];

    const int tid = threadIdx.x;
    const int v = blockIdx.y;
    const int x0 = (blockIdx.x % a.tiles_x) * TX, y0 = (blockIdx.x / a.tiles_x) * TY;
    const int D = a.D;

    auto issue = [&](int j) {   // TMA of frame j of this view into its stage
        const int s = j % NSTAGE;
        const u32 bar = smem_addr(&mbar[s]);
        // the stage was last read by ordinary loads (before a block barrier)
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
        for (int s = 0; s < NSTAGE; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        qn[0] = qn[1] = 0;
    }
    __syncthreads();
    int issued = 0, last_z = 0;   // frames issued (thread 0), step reached
    if (tid == 0)
        for (; issued < min(D, LOOKAHEAD); ++issued) issue(issued);

    // calibration of the tile and its halo (pixels outside the frame: 0)
    for (int i = tid; i < HY * HX; i += FT) {
        const int ly = i / HX, lx = i % HX;
        const int gy = y0 + ly - 1, gx = x0 + lx - 1;
        const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
        gsm[ly][lx] = in ? a.gain[(size_t)gy * a.W + gx] : 0;
        tsm[ly][lx] = in ? a.thr[(size_t)gy * a.W + gx] : 0;
    }
    // this thread's 16 pixels: row ry of the tile, columns cx .. cx + 15
    const int ry = tid / (TX / 16), cx = (tid % (TX / 16)) * 16;
    u32 cw[4];
    {
        const int gy = y0 + ry;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            u32 wv = 0;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const int gx = x0 + cx + 4 * k + bb;
                const u32 c = (gy < a.H && gx < a.W) ? a.cut[(size_t)gy * a.W + gx] : 0u;
                wv |= c << (8 * bb);
            }
            cw[k] = wv;
        }
    }
    __syncthreads();

    u32 ncand = 0;
    bool timed_out = false;
    for (int z = 0; z < D; ++z) {
        last_z = z;
        if (tid == 0 && z + LOOKAHEAD < D) issue(issued++);   // frame z + LOOKAHEAD; its stage held frame z - 2
        bool ok = true;
        if (z == 0) ok = mbar_wait(smem_addr(&mbar[0]), 0);
        if (ok && z + 1 < D) ok = mbar_wait(smem_addr(&mbar[(z + 1) % NSTAGE]), ((z + 1) / NSTAGE) & 1);
        if (tid == 0) qn[(z + 1) & 1] = 0;
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        // scan: queue the pixels of frame z whose raw value is below the cutoff
        const unsigned char *f0 = stage[z % NSTAGE];
        const uint4 rw = *(const uint4 *)&f0[(ry + 1) * TX + cx];
        const u32 m[4] = {__vcmpltu4(rw.x, cw[0]), __vcmpltu4(rw.y, cw[1]), __vcmpltu4(rw.z, cw[2]),
                          __vcmpltu4(rw.w, cw[3])};
        if (m[0] | m[1] | m[2] | m[3]) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                u32 mk = m[k] & 0x01010101u;
                while (mk) {
                    const int bb = (__ffs(mk) - 1) >> 3;
                    mk &= mk - 1;
                    const int slot = atomicAdd(&qn[z & 1], 1);
                    queue[slot] = (unsigned short)(((cx + 4 * k + bb) << 5) | ry);
                }
            }
        }
        __syncthreads();
        const int nq = qn[z & 1];
        ncand += tid == 0 ? (u32)nq : 0u;
        const unsigned char *fm = stage[(z + NSTAGE - 1) % NSTAGE], *fp1 = stage[(z + 1) % NSTAGE];
        for (int i = tid; i < nq; i += FT) {
            const int lx = queue[i] >> 5, ly = queue[i] & 31;
            const int gx = x0 + lx, gy = y0 + ly;
            const int fpv = filt(f0[(ly + 1) * TX + lx], gsm[ly + 1][lx + 1], tsm[ly + 1][lx + 1]);
            long long S = 0, SX = 0, SY = 0, SZ = 0;
            bool is_max = true;
            for (int dz = -1; dz <= 1 && is_max; ++dz) {
                const int zz = z + dz;
                if (zz < 0 || zz >= D) continue;
                const unsigned char *fr = dz < 0 ? fm : (dz == 0 ? f0 : fp1);
                for (int dy = -1; dy <= 1 && is_max; ++dy) {
                    const int yy = gy + dy;
                    if (yy < 0 || yy >= a.H) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int xx = gx + dx;
                        if (xx < 0 || xx >= a.W) continue;
                        const int lxx = lx + dx;
                        const int r = (lxx >= 0 && lxx < TX)
                                          ? fr[(ly + dy + 1) * TX + lxx]
                                          : __ldg(&a.raw[(((size_t)v * D + zz) * a.H + yy) * (size_t)a.P + xx]);
                        const int fq = filt(r, gsm[ly + dy + 1][lxx + 1], tsm[ly + dy + 1][lxx + 1]);
                        const bool before = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                        if (before ? fq >= fpv : fq > fpv) {
                            is_max = false;
                            break;
                        }
                        S += fq;
                        SX += (long long)fq * xx;
                        SY += (long long)fq * yy;
                        SZ += (long long)fq * zz;
                    }
                }
            }
            if (!is_max) continue;
            // centre of mass in coordinate units, rounded half up (all terms positive)
            const int X = (int)((2 * SX * a.num[0] + S * a.den[0]) / (2 * S * a.den[0]));
            const int Y = (int)((2 * SY * a.num[1] + S * a.den[1]) / (2 * S * a.den[1]));
            const int Z = (int)((2 * SZ * a.num[2] + S * a.den[2]) / (2 * S * a.den[2]));
            const u64 slot = atomicAdd(&a.ctl->n_grains, 1ull);
            if (slot < a.cap) {
                a.keys[slot] = (u64)v * ((u64)D * a.H * a.W) + ((u64)z * a.H + gy) * a.W + gx;
                a.vals[slot] = (u32)slot;
                a.rec[slot] = make_int4(X, Y, Z, (int)S);
            } else {
                atomicOr(&a.ctl->error, FRB_OVF);
            }
            atomicAdd(&a.view_count[v], 1u);
        }
        __syncthreads();   // stage z - 1 and the queue are reused from here on
    }
    if (timed_out) {
        // record the failure, then give the copies still in flight into this
        // block's buffers a bounded chance to land before the block exits
        if (tid == 0) {
            atomicOr(&a.ctl->error, FRB_TIMEOUT);
            for (int j = max(0, last_z); j < issued; ++j)
                if (!mbar_wait(smem_addr(&mbar[j % NSTAGE]), (j / NSTAGE) & 1)) break;
        }
        return;
    }
    if (tid == 0 && ncand) atomicAdd(&a.ctl->n_cand, (u64)ncand);
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
    int sorted = 0;
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
    size_t view_bytes() const { return (size_t)p.depth * p.height * p.row_pitch; }

    et_status init() {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(ET_ERR_CUDA, "event creation failed");
        if (cudaEventCreateWithFlags(&handoff, cudaEventDisableTiming) != cudaSuccess)
            return fail(ET_ERR_CUDA, "event creation failed");
        if (!g_tab.reserve(ctx, 3 * align_up(pixels(), 256))) return fail(ET_ERR_OOM, "calibration tables");
        gain = (unsigned char *)g_tab.base;
        thr = gain + align_up(pixels(), 256);
        cut = thr + align_up(pixels(), 256);
        if (!g_ctl.reserve(ctx, sizeof(FrCtl))) return fail(ET_ERR_OOM, "control block");
        ctl = (FrCtl *)g_ctl.base;
        return ET_OK;
    }

    et_status calibrate(const unsigned char *hg, const unsigned char *ht) {
        if (ran) cudaEventSynchronize(ev[3]);
        cudaStream_t st = ctx->stream;
        cudaError_t e = cudaMemcpyAsync(gain, hg, pixels(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(thr, ht, pixels(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "calibration upload");
        const int n = (int)pixels();
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
                                      temp, st);
        k_fr_gather<<<152 * 4, 256, 0, st>>>(ctl, cap, vals[sorted], rec, xyz, pulse);
        exclusive_scan_u32(view_count, view_off, (long long)V, temp, st);   // view_off[V] = total
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
    return ET_OK;
}

et_status et_frames_destroy(et_frames *fr) {
    if (!fr) return fail(ET_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(fr->ctx->device);
    delete fr;
    return ET_OK;
}

}  // extern "C"

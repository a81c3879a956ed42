// probe.cu -- integer issue throughput of the device (et_probe.h): the
// measured denominator for the roofline of the integer-bound tube counts.
#include "et_probe.h"
#include "runtime.h"

namespace et {

namespace {

constexpr int PB_T = 256;        // threads per block
constexpr int PB_CHAINS = 8;     // independent chains per thread
constexpr int PB_STEPS = 16;     // unrolled steps per iteration
constexpr int PB_ITERS = 2048;

// MODE 0: a = (a ^ y) + z; MODE 1: a = a * a + z; MODE 2: both in turn.
// The chains depend on themselves non-linearly, so no step can be folded
// into another; the result is kept alive by a store that never happens.
template <int MODE>
__global__ void __launch_bounds__(PB_T) k_int_probe(unsigned *sink, unsigned y, unsigned z, int iters) {
    unsigned a[PB_CHAINS];
#pragma unroll
    for (int k = 0; k < PB_CHAINS; ++k) a[k] = (threadIdx.x + 1u) * (2u * k + 1u) ^ blockIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < PB_STEPS; ++s) {
#pragma unroll
            for (int k = 0; k < PB_CHAINS; ++k) {
                if (MODE != 1) a[k] = (a[k] ^ y) + z;
                if (MODE != 0) a[k] = a[k] * a[k] + z;
            }
        }
    }
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < PB_CHAINS; ++k) r ^= a[k];
    if (r == y + z + 0x9e3779b9u) sink[0] = r;
}

template <int MODE>
cudaError_t time_probe(unsigned *sink, unsigned grid, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                       float &ms) {
    k_int_probe<MODE><<<grid, PB_T, 0, st>>>(sink, 0x2545f491u, 0x61c88647u, PB_ITERS / 8);   // warm-up
    cudaEventRecord(e0, st);
    k_int_probe<MODE><<<grid, PB_T, 0, st>>>(sink, 0x2545f491u, 0x61c88647u, PB_ITERS);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    return e;
}

}  // namespace

}  // namespace et

using namespace et;

extern "C" et_status et_probe_int_throughput(et_ctx *ctx, double out[3]) {
    GUARD_BEGIN
    if (!ctx || !out) return fail(ET_ERR_INVALID_ARG, "ctx or out is NULL");
    cudaSetDevice(ctx->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sms <= 0) return fail(ET_ERR_CUDA, "no multiprocessors reported");
    const unsigned grid = (unsigned)sms * 8u;
    unsigned *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms[3] = {0, 0, 0};
    if (e == cudaSuccess) e = time_probe<0>(sink, grid, ctx->stream, e0, e1, ms[0]);
    if (e == cudaSuccess) e = time_probe<1>(sink, grid, ctx->stream, e0, e1, ms[1]);
    if (e == cudaSuccess) e = time_probe<2>(sink, grid, ctx->stream, e0, e1, ms[2]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "integer throughput probe");
    const double steps = (double)grid * PB_T * PB_CHAINS * PB_STEPS * PB_ITERS;
    const double ops[3] = {2.0, 1.0, 3.0};
    for (int k = 0; k < 3; ++k) out[k] = ms[k] > 0 ? steps * ops[k] / (ms[k] * 1e-3) : 0.0;
    return ET_OK;
    GUARD_END
}

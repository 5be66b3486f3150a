// lbm_static.cu -- lbm_saturation_static: the FP64 saturation / mass
// reduction for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: their device memory is owned by
// another allocator that has reserved it all (a framework's caching pool, a
// fixed arena on an embedded or shared GPU), or they run in a loop that must
// not pay for an allocation or for the device-wide synchronisation that
// cudaMalloc / cudaFree can cause.  This entry point takes caller-owned
// inputs and outputs only; its scratch space (one FP64 partial sum per block)
// lives in a file-scope __device__ array that every GPU loading the library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                                 // densities per thread
constexpr int kChunk = kThreads * kItems;                  // 4096 nodes per block
constexpr int kMaxBlocks = 4096;                           // scratch capacity in blocks
constexpr int kSmoothSlot = 4;                             // sum of rho1 / (rho1 + rho2)
constexpr int kStride = 8;                                 // doubles per block partial

// Scratch: kMaxBlocks * kStride doubles = 256 KB per device.
static __device__ __align__(256) double g_partials[kMaxBlocks * kStride];

// Device address of g_partials, looked up once per device and context (host
// code may not use the symbol itself: on the host it names a stand-in, not
// device memory).  The context is part of the key: after cudaDeviceReset the
// next call runs in a new primary context, where the module and its array are
// loaded again at another address.
constexpr int kMaxDevices = 64;
struct Scratch {
    void *ctx;
    double *ptr;
};
Scratch g_scratch[kMaxDevices] = {};
std::mutex g_mutex;

// The driver's current context (cuCtxGetCurrent, reached through the runtime
// so that the library needs no link against the driver library); nullptr when
// the entry point is unavailable.
using CtxGetCurrent = int (*)(void **);
CtxGetCurrent ctx_get_current()
{
    static CtxGetCurrent fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrent)p;
    }
    return fn;
}

void *current_context()
{
    void *ctx = nullptr;
    CtxGetCurrent fn = ctx_get_current();
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

__global__ void __launch_bounds__(kThreads) k_partials(const float *rho1, const float *rho2,
                                                       const uint8_t *sample, int64_t n, double *partials)
{
    double acc[5] = {0, 0, 0, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kChunk;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i >= n) break;
        const float a = rho1[i], b = rho2[i];
        acc[0] += (double)a;
        acc[1] += (double)b;
        if (sample == nullptr || sample[i]) {
            acc[2] += 1.0;
            acc[3] += (b > a) ? 1.0 : 0.0;
            acc[4] += (double)a / ((double)a + (double)b);
        }
    }
    __shared__ double sm[kThreads / 32][5];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[wid][q] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double v = lane < kThreads / 32 ? sm[lane][q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) partials[(int64_t)blockIdx.x * kStride + q] = v;
        }
    }
}

// One block sums the partials of every block in a fixed order and writes
// out[0..3] = S_w, smooth S_nw, mass1, mass2.
__global__ void __launch_bounds__(kThreads) k_finish(const double *partials, int nblocks, double *out)
{
    __shared__ double sm[kThreads / 32][5];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < 5; ++q) acc[q] += partials[(int64_t)b * kStride + q];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 5; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < kThreads / 32; ++w)
            for (int q = 0; q < 5; ++q) t[q] += sm[w][q];
        out[0] = t[2] > 0 ? t[3] / t[2] : 0.0;
        out[1] = t[2] > 0 ? t[kSmoothSlot] / t[2] : 0.0;
        out[2] = t[0];
        out[3] = t[1];
    }
}

// Device address of the scratch array on the current device (set-up on the
// first call per device, and again on the first call in a new context of
// that device).
lbm_status scratch_for_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    Scratch &sc = g_scratch[dev];
    void *ctx = current_context();
    if (!sc.ptr || !ctx || ctx != sc.ctx) {
        double *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_partials);
        if (e != cudaSuccess || ptr == nullptr) return LBM_ERR_CUDA;
        sc.ptr = ptr;
        sc.ctx = current_context();  // the lookup made the device's context current if none was
    }
    *out = sc.ptr;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_saturation_static(const float *rho1, const float *rho2, const uint8_t *sample, int64_t n,
                                            double *out, void *stream)
{
    if (n < 0 || !out || (n > 0 && (!rho1 || !rho2))) return LBM_ERR_ARG;
    if (n > (int64_t)kMaxBlocks * kChunk) return LBM_ERR_ARG;  // beyond LBM_SATURATION_STATIC_MAX_N
    double *scratch = nullptr;
    lbm_status st = scratch_for_current_device(&scratch);
    if (st != LBM_OK) return st;
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t s = (cudaStream_t)stream;
    if (nblocks > 0) k_partials<<<nblocks, kThreads, 0, s>>>(rho1, rho2, sample, n, scratch);
    k_finish<<<1, kThreads, 0, s>>>(scratch, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

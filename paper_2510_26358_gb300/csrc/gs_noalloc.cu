// gs_image_l1_noalloc: the L1 photometric loss for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: a hard real-time mapping loop
// whose memory is fixed at start-up (cudaMalloc can block and synchronise the
// device), or code embedded in a host program that only hands over its input
// and output buffers.  This variant of gs_image_l1 needs no workspace: its
// only scratch, one double per block of CHUNK values, is the file-scope
// device array below, which every GPU that loads the library holds until the
// process exits.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.  Later calls reuse the address and
// call nothing that allocates.  The cached address is checked on every call
// (cudaPointerGetAttributes: still device memory of this device): after a
// device reset has unloaded the library's module, the check fails and the
// call resolves the address again, so the first call after a reset is a
// set-up call too and also belongs outside any stream capture.  All calls
// share the array, so calls whose kernels overlap on the GPU race on it;
// every partial a call reads is first written by that same call, so nothing
// needs clearing between calls.
#include <mutex>
#include <string>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kStaticBlocks = GS_IMAGE_L1_NOALLOC_BLOCKS;  // partials held by the array
constexpr int64_t kChunk = GS_IMAGE_L1_NOALLOC_CHUNK;      // values summed per block
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_l1_partials[kStaticBlocks];

std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double block_sum(double v, double *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) t += sm[i];
    return t;
}

// block b sums |rgb - target| over [b*kChunk, (b+1)*kChunk) and adds the
// gradient sign(rgb - target)/n there
__global__ void __launch_bounds__(kThreads) k_l1_static_partial(const float *rgb, const float *target, int64_t n,
                                                               float *grad, double *partials) {
    __shared__ double sm[32];
    const int64_t lo = (int64_t)blockIdx.x * kChunk;
    const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
    const float inv = (float)(1.0 / (double)n);
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        float d = rgb[i] - target[i];
        s += fabs((double)d);
        if (grad) grad[i] += d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    double t = block_sum(s, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) k_l1_static_final(const double *partials, int nb, int64_t n,
                                                             float *loss) {
    __shared__ double sm[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) s += partials[i];
    double t = block_sum(s, sm);
    if (threadIdx.x == 0) *loss = n > 0 ? (float)(t / (double)n) : 0.f;
}

// device address of g_l1_partials on the current device (resolved once)
gs_status partials_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_image_l1_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("gs_image_l1_noalloc: device index beyond the supported 64");
        return GS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_partials_addr[dev]) {
        // still this device's memory?  (a device reset unloads the module)
        cudaPointerAttributes a{};
        e = cudaPointerGetAttributes(&a, g_partials_addr[dev]);
        if (e != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
            (void)cudaGetLastError();  // the failed query is not an error of this call
            g_partials_addr[dev] = nullptr;
        }
    }
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_l1_partials);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("gs_image_l1_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return GS_ERR_CUDA;
        }
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partials_addr[dev];
    return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_image_l1_noalloc(const float *rgb, const float *target, int64_t n, float *loss,
                                         float *dL_drgb, void *stream) {
    using namespace gs;
    if (!rgb || !target || !loss) {
        set_last_error("gs_image_l1_noalloc: rgb, target and loss must not be NULL");
        return GS_ERR_INVALID_ARG;
    }
    if (n < 0 || n > (int64_t)kStaticBlocks * kChunk) {
        set_last_error("gs_image_l1_noalloc: n = " + std::to_string(n) + " is outside [0, " +
                       std::to_string((int64_t)kStaticBlocks * kChunk) +
                       "], the most values its static scratch can reduce");
        return GS_ERR_INVALID_ARG;
    }
    double *partials = nullptr;
    gs_status st = partials_address(&partials);
    if (st != GS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int nb = (int)((n + kChunk - 1) / kChunk);
    if (nb > 0) k_l1_static_partial<<<nb, kThreads, 0, s>>>(rgb, target, n, dL_drgb, partials);
    k_l1_static_final<<<1, kThreads, 0, s>>>(partials, nb, n, loss);
    return check_launch("gs_image_l1_noalloc");
}

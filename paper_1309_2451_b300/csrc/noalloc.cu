// noalloc.cu -- ctap_norm_noalloc: the FP64 norm reduction of a state,
// sum |psi|^2 dV (the value ctap_observables returns in out[0]), for callers
// that must not allocate device memory.
//
// Why it exists: ctap_observables keeps its per-CTA partial sums in scratch
// that the plan allocates with cudaMalloc.  Some callers cannot allow that:
// a process whose device memory is already held by another framework's
// caching allocator (a raw cudaMalloc may then fail or fragment it), or a
// latency-critical loop that cannot accept cudaMalloc's implicit device
// synchronisation.  This entry point needs no plan and allocates nothing:
// its partial sums go to a fixed file-scope device array.
//
// The array (kMaxBlocks doubles, 64 KiB) lives on every GPU that loads the
// library, until the process exits.  Every call shares it, so two calls
// that overlap on the GPU (different streams, or different host threads)
// race on it; calls issued to one stream are ordered and safe.  Each call
// writes every slot it later reads, so nothing needs clearing between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/ctap.h"

namespace {

constexpr long long kChunk = 16384;      // elements reduced by one block
constexpr int kMaxBlocks = 8192;         // => at most 2^27 elements per call
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks];

// Host-side device address of g_noalloc_partials, one per device.  In host
// code the symbol itself is only a stand-in and must never reach a kernel.
double *g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ double block_sum(double v)
{
    __shared__ double warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kThreads / 32 ? warp_sums[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// partials[b] = sum over block b's chunk of |psi|^2 (FP64 accumulation)
template <class V>
__global__ void __launch_bounds__(kThreads) norm_partials_kernel(const V *psi, long long n,
                                                                 double *partials)
{
    const long long i0 = (long long)blockIdx.x * kChunk;
    const long long i1 = i0 + kChunk < n ? i0 + kChunk : n;
    double acc = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += kThreads) {
        const V v = psi[i];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// *out = dV * sum of the first nblk partials, in a fixed order
__global__ void __launch_bounds__(kThreads) norm_finish_kernel(const double *partials, int nblk,
                                                               double dV, double *out)
{
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kThreads) acc += partials[b];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) *out = t * dV;
}

// Device address of the array on the current device.  Outside stream
// capture it is looked up again on every call (the query is cheap and
// allocates nothing), so a context that was torn down and recreated -- a
// cudaDeviceReset, say -- never leaves a stale address behind.  During
// capture the address found by the last call outside capture on this
// device is used; with none yet the call fails.
ctap_status partials_address(cudaStream_t st, double **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CTAP_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return CTAP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return CTAP_ERR_CUDA;
        }
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    if (!g_partials_addr[dev]) return CTAP_ERR_CUDA;
    *addr = g_partials_addr[dev];
    return CTAP_OK;
}

}  // namespace

extern "C" ctap_status ctap_norm_noalloc(const void *psi, long long n, ctap_dtype dtype,
                                         double dV, void *cuda_stream, double *out)
{
    if (!psi || !out || n < 1 || !std::isfinite(dV)) return CTAP_ERR_INVALID_ARG;
    if (dtype != CTAP_C64 && dtype != CTAP_C128) return CTAP_ERR_DTYPE;
    const long long nblk = (n + kChunk - 1) / kChunk;
    if (nblk > kMaxBlocks) return CTAP_ERR_UNSUPPORTED_SIZE;   // n > CTAP_NOALLOC_MAX_ELEMENTS
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *partials = nullptr;
    ctap_status s = partials_address(st, &partials);
    if (s != CTAP_OK) return s;
    if (dtype == CTAP_C64)
        norm_partials_kernel<float2><<<(int)nblk, kThreads, 0, st>>>(
            static_cast<const float2 *>(psi), n, partials);
    else
        norm_partials_kernel<double2><<<(int)nblk, kThreads, 0, st>>>(
            static_cast<const double2 *>(psi), n, partials);
    norm_finish_kernel<<<1, kThreads, 0, st>>>(partials, (int)nblk, dV, out);
    if (cudaGetLastError() != cudaSuccess) return CTAP_ERR_CUDA;
    return CTAP_OK;
}

// peaks.cu -- ctap_measure_fma_peaks: the arithmetic peaks the roofline of
// the passes is quoted against, measured on the device in use.
//
// Each probe kernel runs eight independent chains of fused multiply-adds per
// thread (enough independent work to keep every pipe busy) over a grid of
// eight CTAs of 256 threads per SM, timed with CUDA events on the caller's
// stream after a warm-up launch.  FP32 is measured twice: as scalar FFMA and
// as the packed FP32-pair form (fma.rn.f32x2) the packed passes use; FP64 as
// DFMA.  A fused multiply-add counts as two floating-point operations.
#include <cuda_runtime.h>

#include "../../include/ctap.h"

namespace {

constexpr int kIters = 8192;
constexpr int kThreads = 256;

// Never written (the guarded stores cannot fire); a real device address
// keeps the probes well defined.
__device__ double sink_dev[kThreads];

__global__ void __launch_bounds__(kThreads) fma32_kernel(float *sink, float a, float b)
{
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __fmaf_rn(x[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5f) sink[threadIdx.x] = s;     // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) fma32x2_kernel(float *sink, float a, float b)
{
    float2 x[8];
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = make_float2(threadIdx.x * 1e-3f + j, 0.5f * j);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], A, B);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma64_kernel(double *sink, double a, double b)
{
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < kIters / 8; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __fma_rn(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" ctap_status ctap_measure_fma_peaks(void *cuda_stream, double *out)
{
    if (!out) return CTAP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CTAP_ERR_CUDA;
    }
    const int blocks = 8 * nsm;
    const double threads = (double)blocks * kThreads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return CTAP_ERR_CUDA;
    }
    ctap_status s = CTAP_OK;
    void *sink = nullptr;
    if (cudaGetSymbolAddress(&sink, sink_dev) != cudaSuccess) s = CTAP_ERR_CUDA;
    for (int k = 0; k < 3 && s == CTAP_OK; ++k) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {          // warm-up, then the timed launch
            if (rep == 1) cudaEventRecord(e0, st);
            if (k == 0) fma32_kernel<<<blocks, kThreads, 0, st>>>(static_cast<float *>(sink), 0.999f, 1e-3f);
            if (k == 1) fma32x2_kernel<<<blocks, kThreads, 0, st>>>(static_cast<float *>(sink), 0.999f, 1e-3f);
            if (k == 2) fma64_kernel<<<blocks, kThreads, 0, st>>>(static_cast<double *>(sink), 0.999, 1e-3);
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.0f) {
            s = CTAP_ERR_CUDA;
            break;
        }
        const double fmas = threads * 8.0 * (k == 2 ? kIters / 8 : kIters) * (k == 1 ? 2.0 : 1.0);
        out[k] = 2.0 * fmas / (ms * 1e-3) / 1e12;    // TFLOP/s
    }
    if (cudaGetLastError() != cudaSuccess && s == CTAP_OK) s = CTAP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

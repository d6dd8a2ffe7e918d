// peak.cu -- issue-rate probes of the arithmetic pipes the particle pass uses, for
// the FP64-pipe roofline of the passes: dependent chains of FP64 fused
// multiply-adds (the DFMA rate), of FP32 fused multiply-adds, and of FP64 <-> FP32
// conversion pairs, each timed with CUDA events on the caller's stream.  The paper
// has no counterpart; these are measurements of the machine, not of the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "fdf_internal.cuh"

namespace fdf {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;      // independent chains per thread (hides the pipe latency)
constexpr int kIters = 4096;    // loop trips per launch

// written only if a chain's sum is exactly 12345, which never happens (the chains
// converge to 1): a store the compiler cannot remove, so the chains stay live
__device__ double g_peak_sink;

// x <- x a + b converges to b / (1 - a) = 1 with no denormals.
__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 0.01 * c + 1e-6 * threadIdx.x;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.0) g_peak_sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 0.01f * c + 1e-6f * threadIdx.x;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) g_peak_sink = s;
}

// One trip of a chain: FP64 -> FP32, one FP32 FMA, FP32 -> FP64 (two conversions).
__global__ void __launch_bounds__(kPeakThreads) k_peak_cvt(float a, float b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 0.01 * c + 1e-6 * threadIdx.x;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = (double)fmaf(__double2float_rn(x[c]), a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.0) g_peak_sink = s;
}

}  // namespace
}  // namespace fdf

using namespace fdf;

extern "C" int fdf_pipe_rates(void* stream, double* dfma_per_s, double* ffma_per_s, double* cvt_per_s)
{
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, (std::string("fdf_pipe_rates: ") + cudaGetErrorString(e)).c_str());
    // eight resident blocks of 256 threads per SM: 64 warps, the SM's limit
    const unsigned blocks = (unsigned)sms * 8;
    const double per_launch = (double)blocks * kPeakThreads * kChains * kIters;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best[3] = {0.0, 0.0, 0.0};
    for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (kind == 0) k_peak_dfma<<<blocks, kPeakThreads, 0, s>>>(0.9999999, 1e-7);
            else if (kind == 1) k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(0.999f, 1e-3f);
            else k_peak_cvt<<<blocks, kPeakThreads, 0, s>>>(0.999f, 1e-3f);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            // the first launch of each kind is a warm-up
            if (e == cudaSuccess && rep > 0 && ms > 0.f) best[kind] = std::max(best[kind], per_launch / (ms * 1e-3));
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, (std::string("fdf_pipe_rates: ") + cudaGetErrorString(e)).c_str());
    if (dfma_per_s) *dfma_per_s = best[0];
    if (ffma_per_s) *ffma_per_s = best[1];
    if (cvt_per_s) *cvt_per_s = best[2];
    return FDF_OK;
}

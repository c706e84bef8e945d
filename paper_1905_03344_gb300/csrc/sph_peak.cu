// sph_peak.cu -- sph_fma_peak: the FP32 or FP64 fused multiply-add rate this
// GPU sustains, measured by a kernel of independent FMA chains.  It is the
// denominator of the pair kernels' roofline fractions (they are bound by the
// FP32 pipe on the mixed path and the FP64 pipe on the FP64 path; neither
// peak is a copy or a GEMM rate).  The paper has no counterpart.
#include <string>

#include "sph_internal.cuh"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kUnroll = 16;       // chain steps per loop iteration
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ float g_sink_f;
__device__ double g_sink_d;

// each chain: a <- a * b + c, b and c unknown at compile time
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int64_t iters, T b, T c, T* sink)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (T)(threadIdx.x + k);
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == (T)-1.25e-30) *sink = s;  // keeps the chains live; never true for these b, c
}

thread_local std::string g_peak_error;

sph_status peak_fail(sph_status s, const std::string& msg)
{
    g_peak_error = msg;
    return s;
}

template <typename T>
sph_status time_once(int blocks, int64_t iters, T b, T c, T* sink, cudaStream_t st, cudaEvent_t e0,
                     cudaEvent_t e1, float* ms)
{
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, b, c, sink);
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return peak_fail(SPH_ECUDA, std::string("sph_fma_peak: ") + cudaGetErrorString(e));
    cudaEventElapsedTime(ms, e0, e1);
    return SPH_OK;
}

template <typename T>
sph_status run_peak(int sms, cudaStream_t st, double* out, T* sink)
{
    const int blocks = sms * kBlocksPerSm;
    const double flops_per_iter = 2.0 * kChains * kUnroll * (double)kThreads * blocks;
    const T b = (T)0.999999, c = (T)1e-6;  // b slightly below 1: the chains stay finite
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return peak_fail(SPH_ECUDA, "sph_fma_peak: event creation failed");
    }
    // grow the run to at least 50 ms, then keep the best of three runs
    int64_t iters = 64;
    float ms = 0.f;
    sph_status s = SPH_OK;
    for (int k = 0; k < 24; k++) {
        s = time_once<T>(blocks, iters, b, c, sink, st, e0, e1, &ms);
        if (s != SPH_OK || ms >= 50.f) break;
        iters *= 2;
    }
    double best = 0.0;
    for (int k = 0; k < 3 && s == SPH_OK; k++) {
        s = time_once<T>(blocks, iters, b, c, sink, st, e0, e1, &ms);
        if (s == SPH_OK && ms > 0.f) {
            const double rate = flops_per_iter * (double)iters / (ms * 1e-3);
            if (rate > best) best = rate;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SPH_OK) return s;
    if (best <= 0.0) return peak_fail(SPH_ECUDA, "sph_fma_peak: no timing");
    *out = best;
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_fma_peak(int32_t precision, double* flop_per_s, void* cuda_stream)
{
    if (!flop_per_s || (precision != SPH_MIXED && precision != SPH_FP64))
        return peak_fail(SPH_EINVAL, "sph_fma_peak: precision must be SPH_MIXED or SPH_FP64, out non-NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1)
        return peak_fail(SPH_ECUDA, std::string("sph_fma_peak: no usable device: ") + cudaGetErrorString(e));
    void* sink = nullptr;
    e = precision == SPH_FP64 ? cudaGetSymbolAddress(&sink, g_sink_d) : cudaGetSymbolAddress(&sink, g_sink_f);
    if (e != cudaSuccess) return peak_fail(SPH_ECUDA, std::string("sph_fma_peak: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (precision == SPH_FP64) return run_peak<double>(sms, st, flop_per_s, (double*)sink);
    return run_peak<float>(sms, st, flop_per_s, (float*)sink);
}

extern "C" const char* sph_fma_peak_last_error(void) { return g_peak_error.c_str(); }

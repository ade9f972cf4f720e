// sfhk_peak.cu -- throughput probes of the FP32 and FP64 FMA pipes: the
// measured denominators of the integrators' rooflines (sfhk_fma_peak in
// include/sfhk.h).  Not a step of the method.
//
// Every thread runs kChains independent FMA recurrences x <- x a + b for
// `iters` rounds, so that the pipe never waits on a dependency: with 32
// resident warps per SM (8 per scheduler) and 8 chains per thread there are
// 64 independent FMAs in flight per scheduler, well above the pipe latency.
// The chains converge to the fixed point b / (1 - a) without overflow or
// denormals; their sum is written out so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include "sfhk_internal.h"

namespace sfhk {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float* out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0f + 0.125f * k + 1e-3f * threadIdx.x;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the packed form: one f32x2 instruction = two FP32 FMAs
__global__ void __launch_bounds__(kThreads) k_peak_ffma2(float* out, int iters, float a, float b)
{
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = make_float2(1.0f + 0.125f * k, 2.0f - 1e-3f * threadIdx.x);
    const float2 va = make_float2(a, a), vb = make_float2(b, b);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], va, vb);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(double* out, int iters, double a,
                                                          double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 0.125 * k + 1e-3 * threadIdx.x;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sfhk

extern "C" int sfhk_fma_peak(int device, int kind, int iters, double* tflops, float* ms)
{
    using namespace sfhk;
    if (!tflops || kind < 0 || kind > 2 || iters < 1) return SFHK_E_INVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
        cudaGetLastError();
        return SFHK_E_CUDA;
    }
    SFHK_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    SFHK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * kBlocksPerSM;
    const size_t n_out = (size_t)blocks * kThreads;
    void* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SFHK_OK;
    if (cudaMalloc(&out, n_out * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = SFHK_E_CUDA;
    float t = 0.0f;
    // a warm-up launch, then the timed one
    for (int rep = 0; rep < 2 && rc == SFHK_OK; ++rep) {
        if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = SFHK_E_CUDA;
        if (kind == 0)
            k_peak_ffma<<<blocks, kThreads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        else if (kind == 1)
            k_peak_ffma2<<<blocks, kThreads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        else
            k_peak_dfma<<<blocks, kThreads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = SFHK_E_CUDA;
        if (rep == 1 && rc == SFHK_OK &&
            (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
             cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            rc = SFHK_E_CUDA;
    }
    if (rc == SFHK_OK) {
        // FMAs per thread per round: kChains (x2 for the packed form); 2 flops each
        const double fma = (double)n_out * iters * kChains * (kind == 1 ? 2.0 : 1.0);
        *tflops = 2.0 * fma / (t * 1e-3) / 1e12;
        if (ms) *ms = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    cudaGetLastError();
    return rc;
}

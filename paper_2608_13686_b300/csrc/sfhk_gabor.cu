// sfhk_gabor.cu -- Gabor time-frequency map of the dipole velocity, the
// analysis of Sec. III.D:
//   G(t_m, w_k) = | sum_n v_z(t_n) exp(-(t_n - t_m)^2 / (2 sigma^2)) e^{i w_k t_n} dt |^2
// on the grids t_m = t_first + m t_step, w_k = w_first + k w_step.
//
// One block per window centre t_m.  The block stages the windowed samples
// u_n = v_z(t_n) exp(-(t_n - t_m)^2 / (2 sigma^2)) dt of its window in shared
// memory, a chunk at a time, and every thread accumulates sum_n u_n e^{i w_k t_n}
// for its frequencies, advancing the phase factor by e^{i w_k dt} per sample
// and re-anchoring it with sincos at the start of every chunk (the recurrence
// drifts by ~1e-16 per sample).  Samples farther than kHalfWidth sigma from
// t_m carry a window factor below 1e-16 and are skipped.  FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>

#include "sfhk_internal.h"

namespace sfhk {

namespace {

constexpr int kChunk = 1024;           // samples staged per pass
constexpr double kHalfWidth = 8.6;     // exp(-8.6^2 / 2) = 8.6e-17

__global__ void __launch_bounds__(256) k_gabor(const double* __restrict__ vz, int nt, double dt,
                                               double t_origin, double sigma, double t_first,
                                               double t_step, double w_first, double w_step,
                                               int n_w, double* __restrict__ out)
{
    __shared__ double u[kChunk];
    const int m = blockIdx.x;
    const double tm = t_first + m * t_step;
    const double reach = kHalfWidth * sigma;
    // window [lo, hi] on the sample grid, clipped to the signal
    const double flo = ceil((tm - reach - t_origin) / dt);
    const double fhi = floor((tm + reach - t_origin) / dt);
    const long long lo = (long long)fmin(fmax(flo, 0.0), (double)nt);
    const long long hi = (long long)fmax(fmin(fhi, (double)(nt - 1)), -1.0);
    const double inv2s2 = 0.5 / (sigma * sigma);
    for (int k0 = 0; k0 < n_w; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const double w = w_first + k * w_step;
        double zr = 1.0, zi = 0.0;           // e^{i w dt}
        if (k < n_w) sincos(w * dt, &zi, &zr);
        double ar = 0.0, ai = 0.0;
        for (long long c0 = lo; c0 <= hi; c0 += kChunk) {
            const int len = (int)min((long long)kChunk, hi - c0 + 1);
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const double t = t_origin + (double)(c0 + i) * dt;
                const double d = t - tm;
                u[i] = vz[c0 + i] * exp(-d * d * inv2s2) * dt;
            }
            __syncthreads();
            if (k < n_w) {
                double pr, pi;               // e^{i w t_{c0}}
                sincos(w * (t_origin + (double)c0 * dt), &pi, &pr);
                for (int i = 0; i < len; ++i) {
                    const double x = u[i];
                    ar = fma(x, pr, ar);
                    ai = fma(x, pi, ai);
                    const double nr = pr * zr - pi * zi;
                    pi = fma(pr, zi, pi * zr);
                    pr = nr;
                }
            }
        }
        if (k < n_w) out[(size_t)m * n_w + k] = ar * ar + ai * ai;
    }
}

}  // namespace

int launch_gabor(const double* vz, int nt, double dt, double t_origin, double sigma,
                 double t_first, double t_step, int n_t, double w_first, double w_step, int n_w,
                 double* out, cudaStream_t s)
{
    const int threads = n_w >= 256 ? 256 : ((n_w + 31) / 32) * 32;
    count_launch();
    k_gabor<<<n_t, threads, 0, s>>>(vz, nt, dt, t_origin, sigma, t_first, t_step, w_first,
                                    w_step, n_w, out);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

}  // namespace sfhk

using namespace sfhk;

extern "C" {

int sfhk_gabor(const double* vz, size_t nt, double dt, double t_origin, double sigma,
               double t_first, double t_step, size_t n_t, double omega_first,
               double omega_step, size_t n_w, double* out, int device_ptrs, void* stream)
{
    if (!vz || !out || nt < 1 || nt > (size_t)(1 << 27) || n_t < 1 || n_t > (size_t)(1 << 20) ||
        n_w < 1 || n_w > (size_t)(1 << 20) || n_t * n_w > ((size_t)1 << 31))
        return SFHK_E_INVAL;
    if (!(dt > 0.0) || !(sigma > 0.0) || !std::isfinite(dt) || !std::isfinite(sigma) ||
        !std::isfinite(t_origin) || !std::isfinite(t_first) || !std::isfinite(t_step) ||
        !std::isfinite(omega_first) || !std::isfinite(omega_step))
        return SFHK_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)nt, T = (int)n_t, K = (int)n_w;
    if (device_ptrs)
        return launch_gabor(vz, N, dt, t_origin, sigma, t_first, t_step, T, omega_first,
                            omega_step, K, out, s);
    // host buffers: dipole | map, one allocation, synchronous
    void* buf = nullptr;
    const size_t bytes = sizeof(double) * ((size_t)N + (size_t)T * K);
    SFHK_CUDA_TRY(cudaMallocAsync(&buf, bytes, s));
    double* dvz = (double*)buf;
    double* dG = dvz + N;
    int rc = SFHK_OK;
    if (cudaMemcpyAsync(dvz, vz, sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc)
        rc = launch_gabor(dvz, N, dt, t_origin, sigma, t_first, t_step, T, omega_first,
                          omega_step, K, dG, s);
    if (!rc && cudaMemcpyAsync(out, dG, sizeof(double) * T * K, cudaMemcpyDeviceToHost, s) !=
                   cudaSuccess)
        rc = SFHK_E_CUDA;
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SFHK_E_CUDA;
    return rc;
}

}  // extern "C"

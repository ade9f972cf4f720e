// sfhk_spectrum.cu -- Hann-windowed Fourier transform of the dipole velocity
// and the harmonic yield (Eq. 3):
//   v(omega_k) = sum_n v_z(t_n) W_H(t_n) e^{i omega_k t_n} dt,
//   W_H(t) = [1 + cos(pi t / tau_H)]/2 (|t| <= tau_H), omega_k = 2 pi k/(Nt dt),
//   yield = omega^2 |v|^2, phase = arg v.
// With omega_k t_n = omega_k t_0 + 2 pi k n / Nt, the phase factor is looked
// up in a table of e^{2 pi i m / Nt} at m = (k n) mod Nt (exact integer
// reduction), so the sum is a plain DFT on the time grid; one warp per
// frequency, FP64 throughout.
#include <cuda_runtime.h>

#include "sfhk_internal.h"

namespace sfhk {

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void k_twiddle_window(const double* vz, int nt, double dt, double t_origin,
                                 double tau_H, double2* tw, double* u)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nt) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)nt, &s, &c);
    tw[m] = make_double2(c, s);
    const double t = t_origin + m * dt;
    const double w = fabs(t) <= tau_H ? 0.5 * (1.0 + cos(kPi * t / tau_H)) : 0.0;
    u[m] = vz[m] * w * dt;
}

__global__ void k_dft(const double* __restrict__ u, const double2* __restrict__ tw, int nt,
                      double dt, double t_origin, int n_out, double* omega, double* yield,
                      double* phase)
{
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n_out) return;
    const long long K = k;
    long long idx = (K * lane) % nt;
    const long long step = (K * 32) % nt;
    double re = 0.0, im = 0.0;
    for (int m = lane; m < nt; m += 32) {
        const double2 t = tw[idx];
        re += u[m] * t.x;
        im += u[m] * t.y;
        idx += step;
        if (idx >= nt) idx -= nt;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) {
        const double w = 2.0 * kPi * (double)k / ((double)nt * dt);
        double s, c;
        sincos(w * t_origin, &s, &c);
        const double vr = re * c - im * s, vi = re * s + im * c;
        if (omega) omega[k] = w;
        if (yield) yield[k] = w * w * (vr * vr + vi * vi);
        if (phase) phase[k] = atan2(vi, vr);
    }
}

}  // namespace

int launch_spectrum(const double* vz, int nt, double dt, double t_origin, double tau_H,
                    double* omega, double* yield, double* phase, int n_out, double2* twiddle,
                    cudaStream_t s)
{
    // twiddle holds nt double2 followed by nt doubles of windowed samples
    double* u = reinterpret_cast<double*>(twiddle + nt);
    count_launch(2);
    k_twiddle_window<<<(nt + 255) / 256, 256, 0, s>>>(vz, nt, dt, t_origin, tau_H, twiddle, u);
    const long long threads = (long long)n_out * 32;
    k_dft<<<(int)((threads + 255) / 256), 256, 0, s>>>(u, twiddle, nt, dt, t_origin, n_out, omega,
                                                       yield, phase);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

}  // namespace sfhk

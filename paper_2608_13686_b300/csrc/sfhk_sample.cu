// sfhk_sample.cu -- pulse tables, the ionization step (initial ensemble) and
// the counting sorts that order trajectories by birth time.
//
// Ionization step (Sec. II.A, Eqs. 1-2, 6), one thread per trajectory, FP64:
//   t0 on the time grid by inverse CDF of p_n ~ exp(-2 (2Ip)^{3/2}/(3|E(t_n)|)),
//   k_perp ~ N(0, |E(t0)| / (2 sqrt(2 Ip))) per component (Box-Muller),
//   molecular axis per trajectory (Eq. 6) from the alignment distribution,
//   saddle t_s = t0 + i tt of Eq. 2 by safeguarded Newton on
//     Y(tt) = Im A(t0 + i tt) = -sgn(E(t0)) sqrt(2 Ip + k_perp^2),
//   k_z = -Re[A(t_s) - A(t0)], exit q0 = Re int_{t_s}^{t0} A, tunnelling action
//   S_down = Ip t_s - int_{t_s}^{t0} [k + A - A(t0)]^2/2, all in closed form
//   from the three-sinusoid form of the sin^2 pulse, and the amplitude
//   a = <kappa| z E(t_s) |psi0> / sqrt(E(t_s) kappa_z) e^{i(S_down + k.q0)}
//   with the analytic Fourier transform of the Gaussian orbital; w = a / pdf.
#include <cuda_runtime.h>

#include <cmath>

#include "sfhk_device.cuh"
#include "sfhk_internal.h"

namespace sfhk {

namespace {

constexpr double kPi = 3.14159265358979323846;

// E(t) from its definition E = -dA/dt of A = -(E0/w) cos^2(pi t/Tp) sin(w t + cep).
__device__ double field_direct(double omega, double E0, double Tp, double cep, double t)
{
    if (fabs(t) > 0.5 * Tp) return 0.0;
    const double c = cos(kPi * t / Tp);
    const double ph = omega * t + cep;
    return E0 * c * c * cos(ph) - (E0 * kPi / (omega * Tp)) * sin(2.0 * kPi * t / Tp) * sin(ph);
}

__global__ void k_field_table(double omega, double E0, double Tp, double cep, double t_origin,
                              double dt, int nt, double* Eh, float* Ehf)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= 2 * nt - 1) return;
    const int n = m >> 1;
    double t = t_origin + n * dt;
    if (m & 1) t += 0.5 * dt;
    const double e = field_direct(omega, E0, Tp, cep, t);
    Eh[m] = e;
    Ehf[m] = (float)e;
}

__global__ void k_phase_table(double Ip, double t_origin, double dt, int nt, double2* ph,
                              float2* phf)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nt) return;
    double s, c;
    sincos(Ip * (t_origin + n * dt), &s, &c);
    ph[n] = make_double2(c, -s);
    phf[n] = make_float2((float)c, (float)-s);
}

// ADK weights and their inclusive prefix sum, one block of 1024 threads:
// contiguous chunks, chunk totals scanned in shared memory.  The same pass
// fills the per-birth-step table after the CDF (row layout at kBirthTab):
// the field, the transverse width, the pulse terms' phases, and W_m, scaled
// by 1 / (pi dt total) once the total is known.
__global__ void __launch_bounds__(1024) k_adk_cdf(double omega, double E0, double Tp, double cep,
                                                  double t_origin, double dt, int nt, double Ip,
                                                  double* cdf)
{
    __shared__ double part[1024];
    __shared__ double s_total;
    const int tid = threadIdx.x;
    const int chunk = (nt + 1023) / 1024;
    const int b = tid * chunk, e = min(nt, b + chunk);
    const double cst = 2.0 * pow(2.0 * Ip, 1.5) / 3.0;
    const double sqrt2Ip = sqrt(2.0 * Ip);
    const PulseTerms PT = pulse_terms(omega, E0, Tp, cep);
    double* tab = cdf + birth_tab_offset(nt);
    double acc = 0.0;
    for (int n = b; n < e; ++n) {
        const double t = t_origin + n * dt;
        const double E = field_direct(omega, E0, Tp, cep, t);
        const double f = fabs(E);
        const double w = f > 0.0 ? exp(-cst / f) : 0.0;
        acc += w;
        cdf[n] = acc;
        double* row = tab + (size_t)kBirthTab * n;
        row[0] = E;
        row[1] = sqrt(f / (2.0 * sqrt2Ip));
        row[2] = f > 0.0 ? sqrt2Ip / f : 0.0;
        row[3] = w;
#pragma unroll
        for (int q = 0; q < 3; ++q) sincos(PT.k[q] * t + PT.cep, &row[4 + 2 * q], &row[5 + 2 * q]);
    }
    part[tid] = acc;
    __syncthreads();
    if (tid == 0) {
        double run = 0.0;
        for (int i = 0; i < 1024; ++i) {
            const double v = part[i];
            part[i] = run;
            run += v;
        }
        s_total = run;
    }
    __syncthreads();
    const double off = part[tid];
    const double sc = s_total > 0.0 ? 1.0 / (kPi * dt * s_total) : 0.0;
    for (int n = b; n < e; ++n) {
        cdf[n] += off;
        tab[(size_t)kBirthTab * n + 3] *= sc;
    }
}

struct SampleParams {
    PulseTerms P;
    double omega, E0, Tp, t_origin, dt;
    int nt;
    double Ip;
    int align_kind;
    double theta, phi;
    int n_nodes;                              // quadrature: K, nodes x_k and weights K W_k
    double qx[SFHK_MAX_QUAD_NODES], qkw[SFHK_MAX_QUAD_NODES];
    uint64_t seed;
    uint32_t instance;
    long long n;
    double R;
    int n_prim;
    int ionization;                           // SFHK_IONIZE_SFA / SFHK_IONIZE_MODIFIED
    int sampling;                             // SFHK_SAMPLE_PROPOSAL / SFHK_SAMPLE_ABS_AMPLITUDE
    double norm;
    double pexp[SFHK_MAX_PRIM], pcoef[SFHK_MAX_PRIM];
    // per-draw constants formed once on the host: coef_p (pi/a_p)^{3/2} and
    // N (2 pi)^{-3/2}
    double pfac[SFHK_MAX_PRIM];
    double mz_scale;
    // 1/(2 a_p) and 1/(4 a_p) of the primitives' exponents (0 for an unused slot)
    double i2a[SFHK_MAX_PRIM], i4a[SFHK_MAX_PRIM];
    // a fixed axis (SFHK_ALIGN_FIXED): sin, cos of theta and phi
    double fsth, fcth, fsph, fcph;
    // reciprocals of the pulse's frequencies k_q and of k_q -+ k_r (0 where
    // the frequency is 0)
    double ik[3], ikd[3][3], iks[3][3];
    int pkind[SFHK_MAX_PRIM];
    double cchi, schi;                        // pi lobe azimuth (cos, sin)
    // polyatomic targets: Euler-angle orientation, primitives on their own centres
    int poly;
    double psi;                               // third Euler angle (FIXED)
    int n_centres;
    double cpos[SFHK_MAX_CENTRES][3];         // molecular frame
    int pcentre[SFHK_MAX_PRIM];
    double pdir[SFHK_MAX_PRIM][3];            // unit, molecular frame (p-type)
};

// sinh x and cosh x - 1 from em = e^x - 1 and r = 1 / e^x (formed once by
// the caller), without cancellation
__device__ __forceinline__ void sh_cm1(double em, double r, double& sh, double& cm1)
{
    const double d = 0.5 * r;
    sh = em * (em + 2.0) * d;
    cm1 = em * em * d;
}

// int_0^T cos(al + i be s) ds = (cos(al) sinh(x) - i sin(al) (cosh x - 1)) / be,
// x = be T, given cos(al), sin(al), ibe = 1/be (0 for be = 0), em = e^x - 1
// and r = 1 / e^x
__device__ __forceinline__ double2 int_cos(double ca, double sa, double ibe, double em, double r,
                                           double T)
{
    if (ibe == 0.0) return make_double2(T * ca, 0.0);
    double sh, cm1;
    sh_cm1(em, r, sh, cm1);
    return make_double2(ca * sh * ibe, -sa * cm1 * ibe);
}

// One draw of the proposal from the six uniforms u (trajectory index j for
// the quadrature node) and its amplitude: f receives the 12 SoA fields
// (n0 | q0[3] | p0[3] | axis[3] | w_re w_im, w = a / pdf, zero without a
// saddle root); returns whether the saddle has a root.
__device__ __forceinline__ bool propose(const SampleParams& S, long long j, const double u[6],
                                        const double* __restrict__ cdf, double f[12])
{
    // ---- birth time: smallest m with cdf[m] > u0 * total
    const double total = cdf[S.nt - 1];
    const double thr = u[0] * total;
    int lo = 0, hi = S.nt - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > thr) hi = mid; else lo = mid + 1;
    }
    const int m = lo;
    const double t0 = S.t_origin + m * S.dt;
    // what depends on the birth step alone, from the table after the CDF
    const double* brow = cdf + birth_tab_offset(S.nt) + (size_t)kBirthTab * m;
    const double Et0 = brow[0];
    const double sigma = brow[1];
    const double rr = sqrt(-2.0 * log(u[1]));
    double sb, cb;
    sincos(2.0 * kPi * u[2], &sb, &cb);
    const double kx = sigma * rr * cb, ky = sigma * rr * sb;
    // ---- molecular axis (Eq. 6)
    double th = S.theta, phv = S.phi;
    if (S.align_kind == SFHK_ALIGN_ISOTROPIC) {
        th = acos(2.0 * u[3] - 1.0);
        phv = 2.0 * kPi * u[4];
    } else if (S.align_kind == SFHK_ALIGN_COS2) {
        th = acos(cbrt(2.0 * u[3] - 1.0));
        phv = 2.0 * kPi * u[4];
    } else if (S.align_kind == SFHK_ALIGN_QUADRATURE) {
        th = acos(S.qx[j % S.n_nodes]);
        phv = 2.0 * kPi * u[4];
    }
    double sth = S.fsth, cth = S.fcth, sph = S.fsph, cph = S.fcph;
    if (S.align_kind != SFHK_ALIGN_FIXED) {
        sincos(th, &sth, &cth);
        sincos(phv, &sph, &cph);
    }
    const double nx = sth * cph, ny = sth * sph, nz = cth;
    // polyatomic: the third Euler angle, uniform for the isotropic and cos^2
    // distributions (the Haar measure over all three angles for isotropic)
    double psi = S.psi;
    if (S.poly && (S.align_kind == SFHK_ALIGN_ISOTROPIC || S.align_kind == SFHK_ALIGN_COS2))
        psi = 2.0 * kPi * u[5];
    // SFHK2: the emitting centre (eta = +1: the one at -(R/2) n, drawn with
    // probability 1/2, weight x 2) and the saddle's offset c = eta (R/2) n_z
    int only = -1;
    double cmod = 0.0, side_w = 1.0;
    if (S.ionization == SFHK_IONIZE_MODIFIED) {
        const double eta = u[5] < 0.5 ? 1.0 : -1.0;
        only = eta > 0.0 ? 1 : 0;
        cmod = eta * 0.5 * S.R * nz;
        side_w = 2.0;
    }

    double qz = 0.0, kz = 0.0;
    double2 w = make_double2(0.0, 0.0);
    bool ok = fabs(Et0) > 0.0;
    double tt = 0.0;
    double cthm[3], sthm[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        sthm[q] = brow[4 + 2 * q];
        cthm[q] = brow[5 + 2 * q];
    }
    const double kp2 = kx * kx + ky * ky;
    const double target = 2.0 * S.Ip + kp2;
    if (ok) {
        // ---- saddle point: g(s) = Y(s) - Y*, Y(s) = sum a cos(th) sinh(k s)
        const double Ystar = (Et0 > 0.0 ? -1.0 : 1.0) * sqrt(target);
        double ac[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) ac[q] = S.P.a[q] * cthm[q];
        // Y(s) - Y* and Y'(s); the terms' exponentials e^{k_q s} for k = w,
        // w + W, w - W as products of e^{w s} and e^{W s} (two exponentials
        // and two reciprocals per evaluation)
        const double kW = S.P.k[1] - S.P.k[0];
        auto g = [&](double s, double* dg) {
            const double e0 = exp(S.P.k[0] * s), eW = exp(kW * s);
            const double ie0 = 1.0 / e0, ieW = 1.0 / eW;
            const double e[3] = {e0, e0 * eW, e0 * ieW}, ie[3] = {ie0, ie0 * ieW, ie0 * eW};
            double y = 0.0, yp = 0.0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                y += ac[q] * (e[q] - ie[q]);
                yp += ac[q] * S.P.k[q] * (e[q] + ie[q]);
            }
            *dg = 0.5 * yp;
            return 0.5 * y - Ystar;
        };
        // SFHK2 (Sec. III.D): with E(t_s) = E_r + i E_i the imaginary part of
        // the modified saddle gives X = k_z + Re A(t_s) - A(t0) = c E_i / Y and
        // the real part F(s) = Y^2 - X^2 - target + 2 c E_r = 0, F(0+) < 0;
        // Y' = -E_r, E_r' = -Im dE/dt, E_i' = Re dE/dt along t0 + i s
        double Xlast = 0.0;
        auto gmod = [&](double s, double* dF) {
            double Y = 0.0, dY = 0.0, Ei = 0.0, dEr = 0.0, dEi = 0.0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double k = S.P.k[q], a = S.P.a[q];
                const double e = exp(k * s), ie = 1.0 / e;
                const double sh = 0.5 * (e - ie), ch = 0.5 * (e + ie);
                Y += a * cthm[q] * sh;
                dY += a * k * cthm[q] * ch;
                Ei += a * k * sthm[q] * sh;
                dEr -= a * k * k * cthm[q] * sh;
                dEi += a * k * k * sthm[q] * ch;
            }
            const double Er = -dY;
            const double X = cmod * Ei / Y;
            const double dX = cmod * (dEi * Y - Ei * dY) / (Y * Y);
            Xlast = X;
            *dF = 2.0 * Y * dY - 2.0 * X * dX + 2.0 * cmod * dEr;
            return Y * Y - X * X - target + 2.0 * cmod * Er;
        };
        // first sign change by marching up from the quasi-static estimate,
        // then safeguarded Newton from the bracket's upper end
        auto solve = [&](auto&& fn, double sg0, double* s_out) -> bool {
            const double s0 = sqrt(target) / fabs(Et0);
            double slo = 0.0, shi = s0, dg;
            double ghi = fn(shi, &dg);
            bool found = false;
            for (int it = 0; it < 64; ++it) {
                if ((ghi > 0.0) != (sg0 > 0.0) || ghi == 0.0) { found = true; break; }
                slo = shi;
                shi *= 1.25;
                if (shi > 64.0 * s0) break;
                ghi = fn(shi, &dg);
            }
            if (!found) return false;
            double s = shi, gs = ghi;
            for (int it = 0; it < 200; ++it) {
                if (gs == 0.0) break;
                if ((gs > 0.0) == (sg0 > 0.0)) slo = s; else shi = s;
                double sn = s - gs / dg;
                if (!(sn > slo && sn < shi)) sn = 0.5 * (slo + shi);
                const bool done = fabs(sn - s) <= 4e-16 * s || shi - slo <= 4e-16 * shi;
                s = sn;
                if (done) break;
                gs = fn(s, &dg);
            }
            *s_out = s;
            return true;
        };
        double Xs = 0.0;
        if (S.ionization == SFHK_IONIZE_MODIFIED) {
            ok = solve(gmod, -1.0, &tt);
            if (ok) {
                double d;
                gmod(tt, &d);
                Xs = Xlast;
            }
        } else {
            ok = solve(g, -Ystar, &tt);     // g(0) = -Y*
        }
        if (ok) {
            // ---- k_z, exit and action in closed form; em[q] = e^{k_q tt} - 1,
            // ir[q] = e^{-k_q tt}: the one division per term, every other
            // quotient a product with it or with the pulse's 1/k (host)
            double em[3], ep[3], ir[3], shq[3], cmq[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                em[q] = expm1(S.P.k[q] * tt);
                ep[q] = 1.0 + em[q];
                ir[q] = 1.0 / ep[q];
                sh_cm1(em[q], ir[q], shq[q], cmq[q]);
            }
            double At0 = 0.0, dRe = 0.0, q0 = 0.0, Yt = 0.0;
            double2 Es = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double a = S.P.a[q], k = S.P.k[q];
                const double sh = shq[q], cm1 = cmq[q];
                At0 += a * sthm[q];
                dRe += a * sthm[q] * cm1;                  // Re A(t_s) - A(t0)
                Yt += a * cthm[q] * sh;                    // Im A(t_s)
                if (k != 0.0) q0 += a * cthm[q] * cm1 * S.ik[q];   // int_0^tt Im A(t0+is) ds
                // E(t_s) = -sum a k cos(th + i k tt)
                Es.x -= a * k * cthm[q] * (cm1 + 1.0);
                Es.y += a * k * sthm[q] * sh;
            }
            kz = Xs - dRe;
            qz = q0;
            const double2 kapz = make_double2(kz + dRe, Yt);
            // int_0^tt B(s)^2 ds, B = c' + sum a sin(th + i k s), c' = kz - A(t0)
            const double cp = kz - At0;
            // int_0^tt sin(th + i k s) ds = (sin th sinh x + i cos th (cosh x - 1)) / k
            // with x = k tt; the products sin(th_q + i k_q s) sin(th_r + i k_r s)
            // = [cos(difference) - cos(sum)] / 2, the (q, r) and (r, q) terms
            // equal, e^{(k_q -+ k_r) tt} - 1 formed from em[q] and em[r].
            double2 IB = make_double2(cp * cp * tt, 0.0);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double k = S.P.k[q];
                double2 is;
                if (k == 0.0) {
                    is = make_double2(tt * sthm[q], 0.0);
                } else {
                    is = make_double2(sthm[q] * shq[q] * S.ik[q], cthm[q] * cmq[q] * S.ik[q]);
                }
                IB = cadd(IB, cscale(is, 2.0 * cp * S.P.a[q]));
#pragma unroll
                for (int r = q; r < 3; ++r) {
                    const double cc = cthm[q] * cthm[r], ss = sthm[q] * sthm[r];
                    const double sc = sthm[q] * cthm[r], cs = cthm[q] * sthm[r];
                    // e^{(k_q - k_r) tt} - 1 and e^{(k_q + k_r) tt} - 1, with their
                    // reciprocal exponentials e^{-(k_q -+ k_r) tt}
                    const double emd = (em[q] - em[r]) * ir[r];
                    const double ems = em[q] + em[r] + em[q] * em[r];
                    const double2 d1 =
                        q == r ? make_double2(tt, 0.0)
                               : int_cos(cc + ss, sc - cs, S.ikd[q][r], emd, ep[r] * ir[q], tt);
                    const double2 d2 =
                        int_cos(cc - ss, sc + cs, S.iks[q][r], ems, ir[q] * ir[r], tt);
                    const double f = (q == r ? 0.5 : 1.0) * S.P.a[q] * S.P.a[r];
                    IB = cadd(IB, cscale(csub(d1, d2), f));
                }
            }
            // S_down = Ip (t0 + i tt) + (i/2)(kp2 tt + IB)
            const double2 Sd = make_double2(S.Ip * t0 - 0.5 * IB.y, S.Ip * tt + 0.5 * (kp2 * tt + IB.x));
            // <kappa| z |psi0>, kappa = (kx, ky, kapz)
            const double2 kk = make_double2(kp2 + kapz.x * kapz.x - kapz.y * kapz.y,
                                            2.0 * kapz.x * kapz.y);
            double2 mz = make_double2(0.0, 0.0);
            if (S.poly) {
                // each primitive on its own centre A = Rot x_c (lab), s-type
                // (A_z - i kappa_z/(2a)) F or p-type along u = Rot d:
                // [u_z/(2a) - kappa_z (u.kappa)/(4a^2) - i A_z (u.kappa)/(2a)] F
                double sps, cps, Rot[9];
                sincos(psi, &sps, &cps);
                euler_rotation<double>(cph, sph, cth, sth, cps, sps, Rot);
                for (int p = 0; p < S.n_prim; ++p) {
                    const double* x = S.cpos[S.pcentre[p]];
                    const double A[3] = {Rot[0] * x[0] + Rot[1] * x[1] + Rot[2] * x[2],
                                         Rot[3] * x[0] + Rot[4] * x[1] + Rot[5] * x[2],
                                         Rot[6] * x[0] + Rot[7] * x[1] + Rot[8] * x[2]};
                    const double2 kA = make_double2(kx * A[0] + ky * A[1] + kapz.x * A[2],
                                                    kapz.y * A[2]);
                    const double i4a = S.i4a[p];
                    const double2 ex = make_double2(kA.y - kk.x * i4a, -kA.x - kk.y * i4a);
                    const double2 F = cscale(cexp_(ex), S.pfac[p]);
                    double2 f;
                    if (S.pkind[p]) {
                        const double* d = S.pdir[p];
                        const double uu[3] = {Rot[0] * d[0] + Rot[1] * d[1] + Rot[2] * d[2],
                                              Rot[3] * d[0] + Rot[4] * d[1] + Rot[5] * d[2],
                                              Rot[6] * d[0] + Rot[7] * d[1] + Rot[8] * d[2]};
                        const double2 uk = make_double2(uu[0] * kx + uu[1] * ky + uu[2] * kapz.x,
                                                        uu[2] * kapz.y);
                        const double2 ku = cmul(kapz, uk);
                        const double i2a = S.i2a[p], i4a2 = i2a * i2a;
                        f = make_double2(uu[2] * i2a - ku.x * i4a2 + A[2] * uk.y * i2a,
                                         -ku.y * i4a2 - A[2] * uk.x * i2a);
                    } else {
                        f = make_double2(A[2] + kapz.y * S.i2a[p], -kapz.x * S.i2a[p]);
                    }
                    mz = cadd(mz, cmul(F, f));
                }
            }
            for (int c = 0; c < (S.poly ? 0 : 2); ++c) {
                if (only >= 0 && c != only) continue;
                const double sgn = c == 0 ? 1.0 : -1.0;
                const double Ax = sgn * 0.5 * S.R * nx, Ay = sgn * 0.5 * S.R * ny,
                             Az = sgn * 0.5 * S.R * nz;
                // kappa.A (complex)
                const double2 kA = make_double2(kx * Ax + ky * Ay + kapz.x * Az, kapz.y * Az);
                for (int p = 0; p < S.n_prim; ++p) {
                    const double i4a = S.i4a[p];
                    // -i kappa.A - kappa.kappa / (4a)
                    const double2 ex = make_double2(kA.y - kk.x * i4a, -kA.x - kk.y * i4a);
                    const double2 F = cscale(cexp_(ex), S.pfac[p]);
                    double2 f;
                    if (S.pkind[p]) {
                        // p-type, x' = r - A, factor s u.x' (sigma: u = n, s = s_c;
                        // pi: u = m, s = 1): int e^{-i kappa.r} (A_z + x'_z) s u.x'
                        // e^{-a x'^2} = s [u_z/(2a) - kappa_z (u.kappa)/(4a^2)
                        // - i A_z (u.kappa)/(2a)] F (the derivatives of F in kappa)
                        double u[3] = {nx, ny, nz}, s = sgn;
                        if (S.pkind[p] == 2) {
                            pi_direction<double>(nx, ny, nz, S.cchi, S.schi, u);
                            s = 1.0;
                        }
                        const double2 uk = make_double2(u[0] * kx + u[1] * ky + u[2] * kapz.x,
                                                        u[2] * kapz.y);
                        const double2 ku = cmul(kapz, uk);
                        const double i2a = S.i2a[p], i4a2 = i2a * i2a;
                        f = make_double2(s * (u[2] * i2a - ku.x * i4a2 + Az * uk.y * i2a),
                                         s * (-ku.y * i4a2 - Az * uk.x * i2a));
                    } else {
                        // (A_z - i kappa_z / (2a))
                        f = make_double2(Az + kapz.y * S.i2a[p], -kapz.x * S.i2a[p]);
                    }
                    mz = cadd(mz, cmul(F, f));
                }
            }
            mz = cscale(mz, S.mz_scale);
            // amplitude and weight
            const double2 num = cmul(Es, mz);
            double2 curv = cmul(Es, kapz);
            if (S.ionization == SFHK_IONIZE_MODIFIED) {
                // + c dE/dt(t_s), dE/dt = sum a k^2 sin(th + i k tt)
                double2 Ed = make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double ak2 = S.P.a[q] * S.P.k[q] * S.P.k[q];
                    Ed.x += ak2 * sthm[q] * (cmq[q] + 1.0);
                    Ed.y += ak2 * cthm[q] * shq[q];
                }
                curv = cadd(curv, cscale(Ed, cmod));
            }
            const double2 den = csqrt_(curv);
            const double2 Z = make_double2(Sd.x + kz * qz, Sd.y);     // S_down + k.q0
            const double2 eiz = cexp_(make_double2(-Z.y, Z.x));        // e^{iZ}
            const double2 amp = cmul(cdiv(num, den), eiz);
            // proposal density: W_m / (total dt) for the birth step times the
            // Gaussian of k_perp, e^{-kp2/(2 sigma^2)} / (2 pi sigma^2)
            const double i2s2 = brow[2];
            const double pdf = brow[3] * i2s2 * exp(-kp2 * i2s2);
            // the quadrature node's weight K W_k (1 otherwise)
            const double f = side_w *
                             (S.align_kind == SFHK_ALIGN_QUADRATURE ? S.qkw[j % S.n_nodes] : 1.0);
            const double fp = f / pdf;
            w = make_double2(fp * amp.x, fp * amp.y);
        }
    }
    f[0] = (double)m;
    f[1] = 0.0;
    f[2] = 0.0;
    f[3] = qz;
    f[4] = kx;
    f[5] = ky;
    f[6] = kz;
    // orientation: the axis, or the Euler angles of a polyatomic molecule
    f[7] = S.poly ? phv : nx;
    f[8] = S.poly ? th : ny;
    f[9] = S.poly ? psi : nz;
    f[10] = w.x;
    f[11] = w.y;
    return ok;
}

__device__ __forceinline__ void uniforms_at(const SampleParams& S, long long j, uint32_t d0,
                                            double u[6])
{
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
#pragma unroll
    for (uint32_t d = 0; d < 3; ++d) {
        const uint4 r =
            philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), S.instance, d0 + d), key);
        u[2 * d] = u01(r.x, r.y);
        u[2 * d + 1] = u01(r.z, r.w);
    }
}

// Initial points distributed ~ |a| (sampling 1): exact rejection with weight
// correction on the proposal.  A draw of weight w is accepted with
// alpha = min(1, |w|/M) and carries P w / alpha (= P M w/|w| when |w| <= M),
// which keeps every weighted mean unbiased for any M.  M = kappa x mean |w|
// over the first half of a pilot of proposal draws, P = mean alpha over the
// second half (k_pilot, k_pilot_constants), then k_sample_abs.  Attempt k of trajectory j uses
// draws 3k..3k+2 (attempt 0 = the plain sampler's draws) and acceptance
// uniform draw kAccBase + k; pilot draw i uses draws kPilotBase.. of index i.
// A trajectory still unaccepted after kAttempts = K attempts gets weight 0;
// every attempt succeeds with the same probability P, so that happens with
// probability (1 - P)^K and the kept weights carry the extra factor
// 1 / (1 - (1 - P)^K), which keeps the mean over all N trajectories (the
// dipole's 1/N counts the unaccepted ones) unbiased for any kappa.
constexpr int kPilot = 16384;
constexpr int kAttempts = 256;
constexpr uint32_t kAccBase = 1u << 20;
constexpr uint32_t kPilotBase = 1u << 24;

__global__ void k_sample(SampleParams S, const double* __restrict__ cdf, double* __restrict__ soa,
                         int* __restrict__ n0_out, unsigned long long* n_invalid)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= S.n) return;
    const long long n = S.n;
    // ---- random numbers: Philox4x32-10, key = seed, counter = (j, instance, draw)
    double u[6], f[12];
    uniforms_at(S, j, 0u, u);
    const bool ok = propose(S, j, u, cdf, f);
    if (!ok) atomicAdd(n_invalid, 1ull);
#pragma unroll
    for (int q = 0; q < 12; ++q) soa[q * n + j] = f[q];
    n0_out[j] = (int)f[0];
}

// Sampling 1 without lanes idling: a persistent kernel in which every lane
// makes one proposal draw per iteration for its current trajectory, and a
// lane whose draw is accepted writes that trajectory and takes the next one
// from a global counter.  A trajectory's draws depend only on (j, attempt),
// so the result is the same as attempting each trajectory in turn; what
// changes is that a warp no longer waits for its slowest lane.
__global__ void k_sample_abs(SampleParams S, const double* __restrict__ cdf,
                             double* __restrict__ soa, int* __restrict__ n0_out,
                             unsigned long long* n_invalid, const double* __restrict__ mp,
                             unsigned long long* __restrict__ next)
{
    const long long n = S.n;
    const double M = mp[0], keep = mp[1];
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    long long j = (long long)atomicAdd(next, 1ull);
    int k = 0;
    while (j < n) {
        double u[6], f[12];
        uniforms_at(S, j, 3u * (uint32_t)k, u);
        bool done = false, ok = false;
        if (propose(S, j, u, cdf, f)) {
            const double aw = hypot(f[10], f[11]);
            const double alpha = M > 0.0 ? fmin(1.0, aw / M) : 0.0;
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)j, (uint32_t)(j >> 32), S.instance, kAccBase + (uint32_t)k),
                key);
            if (alpha > 0.0 && u01(r.x, r.y) < alpha) {
                f[10] *= keep / alpha;
                f[11] *= keep / alpha;
                done = ok = true;
            }
        }
        if (!done && k + 1 >= kAttempts) {
            done = true;               // no acceptance: invalid, weight 0
            f[10] = f[11] = 0.0;
        }
        if (done) {
            if (!ok) atomicAdd(n_invalid, 1ull);
#pragma unroll
            for (int q = 0; q < 12; ++q) soa[q * n + j] = f[q];
            n0_out[j] = (int)f[0];
            j = (long long)atomicAdd(next, 1ull);
            k = 0;
        } else {
            ++k;
        }
    }
}

// |w| of the pilot draws (sampling 1)
__global__ void k_pilot(SampleParams S, const double* __restrict__ cdf, double* __restrict__ aw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPilot) return;
    double u[6], f[12];
    uniforms_at(S, i, kPilotBase, u);
    propose(S, i, u, cdf, f);
    aw[i] = hypot(f[10], f[11]);
}

// M and P from the pilot |w| (one block of 1024 threads): mp[0] = M,
// mp[1] = P / (1 - (1 - P)^kAttempts), the factor of an accepted draw's weight
__global__ void __launch_bounds__(1024) k_pilot_constants(const double* __restrict__ aw,
                                                          double kappa, double* __restrict__ mp)
{
    __shared__ double part[1024];
    const int t = threadIdx.x;
    constexpr int half = kPilot / 2;
    double acc = 0.0;
    for (int i = t; i < half; i += 1024) acc += aw[i];
    part[t] = acc;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if (t < off) part[t] += part[t + off];
        __syncthreads();
    }
    const double M = kappa * part[0] / half;
    __syncthreads();
    acc = 0.0;
    for (int i = half + t; i < kPilot; i += 1024) acc += M > 0.0 ? fmin(1.0, aw[i] / M) : 0.0;
    part[t] = acc;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if (t < off) part[t] += part[t + off];
        __syncthreads();
    }
    if (t == 0) {
        const double P = part[0] / half;
        mp[0] = M;
        mp[1] = P > 0.0 ? P / -expm1((double)kAttempts * log1p(-P)) : 0.0;
    }
}

__global__ void k_n0_from_soa(const double* soa, long long n, int* n0)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j < n) n0[j] = (int)soa[j];
}

// ------------------------------------------------------------------ counting sort
__global__ void k_hist(const int* keys, long long n, int* hist)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        atomicAdd(&hist[keys[j]], 1);
}

// exclusive scan of K ints in one block (chunked)
__global__ void __launch_bounds__(1024) k_exscan(int* a, int K)
{
    __shared__ long long part[1024];
    const int tid = threadIdx.x;
    const int chunk = (K + 1023) / 1024;
    const int b = tid * chunk, e = min(K, b + chunk);
    long long acc = 0;
    for (int i = b; i < e; ++i) acc += a[i];
    part[tid] = acc;
    __syncthreads();
    if (tid == 0) {
        long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const long long v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = part[tid];
    for (int i = b; i < e; ++i) {
        const int v = a[i];
        a[i] = (int)run;
        run += v;
    }
}

__global__ void k_scatter(const int* keys, long long n, int* cursor, int* perm)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        perm[atomicAdd(&cursor[keys[j]], 1)] = (int)j;
}

__global__ void k_build_items(const int* perm, const int* n0, long long n, int inst,
                              WorkItem* items)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long first = i * kWarp;
    if (first >= n) return;
    WorkItem it;
    it.inst = inst;
    it.first = (int)first;
    it.count = (int)min((long long)kWarp, n - first);
    // the smallest n0 of the item (counting sort orders by n0)
    int m = n0[perm[first]];
    for (int k = 1; k < it.count; ++k) m = min(m, n0[perm[first + k]]);
    it.n_start = m;
    items[i] = it;
}

__global__ void k_item_keys(const WorkItem* items, int n_items, const int* inst_nt, int K,
                            int* keys)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const WorkItem it = items[i];
    const int len = inst_nt[it.inst] - it.n_start;      // 1..K
    keys[i] = K - len;                                   // longest first
}

__global__ void k_gather_items(const WorkItem* in, const int* perm, int n_items, WorkItem* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_items) out[i] = in[perm[i]];
}

int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }

}  // namespace

int launch_field_table(const Pulse& P, double* Eh, float* Ehf, cudaStream_t s)
{
    const int m = 2 * P.nt - 1;
    count_launch();
    k_field_table<<<grid_for(m, 256), 256, 0, s>>>(P.omega, P.E0, P.Tp, P.desc.cep, P.t_origin,
                                                    P.dt, P.nt, Eh, Ehf);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int launch_phase_table(const Pulse& P, double Ip, double2* ph, float2* phf, cudaStream_t s)
{
    count_launch();
    k_phase_table<<<grid_for(P.nt, 256), 256, 0, s>>>(Ip, P.t_origin, P.dt, P.nt, ph, phf);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int launch_adk_cdf(const Pulse& P, double Ip, double* cdf, cudaStream_t s)
{
    count_launch();
    k_adk_cdf<<<1, 1024, 0, s>>>(P.omega, P.E0, P.Tp, P.desc.cep, P.t_origin, P.dt, P.nt, Ip, cdf);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

bool align_valid(const sfhk_align_desc& al)
{
    if (al.kind == SFHK_ALIGN_QUADRATURE)
        return al.n_nodes >= 1 && al.n_nodes <= SFHK_MAX_QUAD_NODES;
    return al.kind == SFHK_ALIGN_FIXED || al.kind == SFHK_ALIGN_ISOTROPIC ||
           al.kind == SFHK_ALIGN_COS2;
}

// K-point Gauss-Legendre rule on [0, 1]: the roots of P_K by Newton's method
// from the estimate cos(pi (i + 3/4) / (K + 1/2)), P_K and P_K' by the
// three-term recurrence, weights 2 / ((1 - x^2) P_K'(x)^2) on [-1, 1], then
// mapped to [0, 1] (x -> (1 + x)/2, w -> w/2); nodes in descending order.
void quadrature_nodes(int K, double* x01, double* w01)
{
    for (int i = 0; i < K; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (K + 0.5));
        double pk = 0.0, dpk = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm = 1.0;
            pk = x;
            for (int m = 2; m <= K; ++m) {
                const double pn = ((2 * m - 1) * x * pk - (m - 1) * pm) / m;
                pm = pk;
                pk = pn;
            }
            dpk = K * (pm - x * pk) / (1.0 - x * x);
            const double step = pk / dpk;
            x -= step;
            if (std::fabs(step) <= 1e-16) break;
        }
        double pm = 1.0;
        pk = x;
        for (int m = 2; m <= K; ++m) {
            const double pn = ((2 * m - 1) * x * pk - (m - 1) * pm) / m;
            pm = pk;
            pk = pn;
        }
        dpk = K * (pm - x * pk) / (1.0 - x * x);
        x01[i] = 0.5 * (1.0 + x);
        w01[i] = 1.0 / ((1.0 - x * x) * dpk * dpk);
    }
}

int launch_sample(const Target& T, const Pulse& P, const sfhk_align_desc& al, long long n,
                  uint64_t seed, uint32_t instance, const double* cdf, double* soa, int* n0,
                  unsigned long long* n_invalid, double* pilot, cudaStream_t s)
{
    if (!align_valid(al)) return SFHK_E_INVAL;
    if (T.desc.sampling == SFHK_SAMPLE_ABS_AMPLITUDE && pilot == nullptr) return SFHK_E_INVAL;
    const bool poly = T.desc.kind == SFHK_POT_POLYATOMIC;
    if (poly && (al.kind == SFHK_ALIGN_QUADRATURE || !std::isfinite(al.psi))) return SFHK_E_INVAL;
    SampleParams S;
    S.n_nodes = al.kind == SFHK_ALIGN_QUADRATURE ? al.n_nodes : 1;
    for (int k = 0; k < SFHK_MAX_QUAD_NODES; ++k) S.qx[k] = S.qkw[k] = 0.0;
    if (al.kind == SFHK_ALIGN_QUADRATURE) {
        quadrature_nodes(al.n_nodes, S.qx, S.qkw);
        for (int k = 0; k < al.n_nodes; ++k) S.qkw[k] *= al.n_nodes;
    }
    S.P = pulse_terms(P.omega, P.E0, P.Tp, P.desc.cep);
    for (int q = 0; q < 3; ++q) {
        S.ik[q] = S.P.k[q] != 0.0 ? 1.0 / S.P.k[q] : 0.0;
        for (int r = 0; r < 3; ++r) {
            const double d = S.P.k[q] - S.P.k[r], m = S.P.k[q] + S.P.k[r];
            S.ikd[q][r] = d != 0.0 ? 1.0 / d : 0.0;
            S.iks[q][r] = m != 0.0 ? 1.0 / m : 0.0;
        }
    }
    S.omega = P.omega;
    S.E0 = P.E0;
    S.Tp = P.Tp;
    S.t_origin = P.t_origin;
    S.dt = P.dt;
    S.nt = P.nt;
    S.Ip = T.desc.Ip;
    S.align_kind = al.kind;
    S.theta = al.theta;
    S.phi = al.phi;
    S.seed = seed;
    S.instance = instance;
    S.n = n;
    S.R = T.desc.R;
    S.n_prim = T.desc.n_prim;
    S.ionization = T.desc.ionization;
    S.sampling = T.desc.sampling;
    S.norm = T.dev.norm;
    for (int k = 0; k < SFHK_MAX_PRIM; ++k) {
        S.pexp[k] = T.desc.prim_exp[k];
        S.pcoef[k] = T.desc.prim_coef[k];
        S.pkind[k] = T.desc.prim_kind[k];
        S.pfac[k] = S.pexp[k] > 0.0 ? S.pcoef[k] * std::pow(kPi / S.pexp[k], 1.5) : 0.0;
        S.i2a[k] = S.pexp[k] > 0.0 ? 0.5 / S.pexp[k] : 0.0;
        S.i4a[k] = S.pexp[k] > 0.0 ? 0.25 / S.pexp[k] : 0.0;
    }
    S.fsth = std::sin(al.theta);
    S.fcth = std::cos(al.theta);
    S.fsph = std::sin(al.phi);
    S.fcph = std::cos(al.phi);
    S.mz_scale = S.norm * std::pow(2.0 * kPi, -1.5);
    S.cchi = std::cos(T.desc.pi_azimuth);
    S.schi = std::sin(T.desc.pi_azimuth);
    S.poly = poly ? 1 : 0;
    S.psi = al.psi;
    S.n_centres = poly ? T.desc.n_centres : 0;
    for (int c = 0; c < SFHK_MAX_CENTRES; ++c)
        for (int a = 0; a < 3; ++a) S.cpos[c][a] = poly ? T.desc.centre_pos[c][a] : 0.0;
    for (int k = 0; k < SFHK_MAX_PRIM; ++k) {
        S.pcentre[k] = poly ? T.desc.prim_centre[k] : 0;
        for (int a = 0; a < 3; ++a) S.pdir[k][a] = T.dev.pdir[k][a];
    }
    if (S.sampling == SFHK_SAMPLE_ABS_AMPLITUDE) {
        // pilot: |w| of kPilot proposal draws, then M and P; then the
        // persistent rejection sampler over a trajectory counter
        double* mp = pilot + kPilot;
        unsigned long long* next = reinterpret_cast<unsigned long long*>(pilot + kPilot + 2);
        const double kappa = T.desc.sampling_factor > 0.0 ? T.desc.sampling_factor : 5.0;
        int dev = 0, sms = 0, occ = 0;
        SFHK_CUDA_TRY(cudaGetDevice(&dev));
        SFHK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SFHK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_abs, 128, 0));
        long long grid = (long long)sms * (occ > 0 ? occ : 1);
        const long long need = (n + 127) / 128;
        if (grid > need) grid = need;
        SFHK_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
        count_launch(3);
        k_pilot<<<kPilot / 128, 128, 0, s>>>(S, cdf, pilot);
        k_pilot_constants<<<1, 1024, 0, s>>>(pilot, kappa, mp);
        k_sample_abs<<<(int)grid, 128, 0, s>>>(S, cdf, soa, n0, n_invalid, mp, next);
    } else {
        count_launch();
        k_sample<<<grid_for(n, 128), 128, 0, s>>>(S, cdf, soa, n0, n_invalid);
    }
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

// pilot |w| | M, P | trajectory counter
size_t sample_pilot_doubles() { return (size_t)kPilot + 3; }

int launch_n0_from_soa(const double* soa, long long n, int* n0, cudaStream_t s)
{
    count_launch();
    k_n0_from_soa<<<grid_for(n, 256), 256, 0, s>>>(soa, n, n0);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int launch_counting_sort(const int* keys, long long n, int K, int* perm, int* hist, cudaStream_t s)
{
    SFHK_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * K, s));
    const int g = (int)std::min<long long>(grid_for(n, 256), 148 * 16);
    count_launch(3);
    k_hist<<<g, 256, 0, s>>>(keys, n, hist);
    k_exscan<<<1, 1024, 0, s>>>(hist, K);
    k_scatter<<<g, 256, 0, s>>>(keys, n, hist, perm);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int launch_build_items(const int* perm, const int* n0, long long n, int inst, WorkItem* items,
                       cudaStream_t s)
{
    const long long n_items = (n + kWarp - 1) / kWarp;
    count_launch();
    k_build_items<<<grid_for(n_items, 128), 128, 0, s>>>(perm, n0, n, inst, items);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int launch_sort_items(const WorkItem* in, int n_items, const int* inst_nt, WorkItem* out,
                      int* keys, int* perm, int* hist, int K, cudaStream_t s)
{
    count_launch(2);
    k_item_keys<<<grid_for(n_items, 256), 256, 0, s>>>(in, n_items, inst_nt, K, keys);
    int rc = launch_counting_sort(keys, n_items, K, perm, hist, s);
    if (rc) return rc;
    k_gather_items<<<grid_for(n_items, 256), 256, 0, s>>>(in, perm, n_items, out);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

}  // namespace sfhk

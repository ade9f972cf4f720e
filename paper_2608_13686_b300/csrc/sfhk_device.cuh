// sfhk_device.cuh -- device-side building blocks of libsfhk: counter-based
// random numbers, complex and two-float arithmetic, the sin^2 pulse in closed
// form (real and complex time), and the potential of Eq. 7 with its gradient
// and Hessian.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <math_constants.h>

#include <cstdint>

#include "sfhk_internal.h"

namespace sfhk {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64-bit
// multiplies (0xD2511F53, 0xCD9E8D57) with the Weyl key schedule
// (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// 53-bit uniform in (0,1): ((a >> 5) 2^26 + (b >> 6) + 1/2) 2^-53.
__device__ __forceinline__ double u01(uint32_t a, uint32_t b)
{
    return (__uint2double_rn(a >> 5) * 67108864.0 + __uint2double_rn(b >> 6) + 0.5) *
           (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------------------ complex (double2)
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    const double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
// e^{z}
__device__ __forceinline__ double2 cexp_(double2 z)
{
    double s, c;
    sincos(z.y, &s, &c);
    const double m = exp(z.x);
    return make_double2(m * c, m * s);
}
// principal square root
__device__ __forceinline__ double2 csqrt_(double2 z)
{
    const double r = hypot(z.x, z.y);
    if (r == 0.0) return make_double2(0.0, 0.0);
    if (z.x >= 0.0) {
        const double t = sqrt(0.5 * (r + z.x));
        return make_double2(t, 0.5 * z.y / t);
    }
    const double t = sqrt(0.5 * (r - z.x));
    return make_double2(0.5 * fabs(z.y) / t, copysign(t, z.y));
}
// sin and cos of a + i b
__device__ __forceinline__ void csincos(double a, double b, double2* s, double2* c)
{
    double sa, ca;
    sincos(a, &sa, &ca);
    const double sh = sinh(b), ch = cosh(b);
    *s = make_double2(sa * ch, ca * sh);
    *c = make_double2(ca * ch, -sa * sh);
}

// ------------------------------------------------------------------ two-float
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x, renormalised (Dekker's FastTwoSum at the end).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// ------------------------------------------------------------------ pulse
// A(t) = -(E0/w) cos^2(pi t/Tp) sin(w t + cep)
//      = sum_m a_m sin(k_m t + cep),  (a, k) = (-E0/(2w), w), (-E0/(4w), w+W),
//        (-E0/(4w), w-W), W = 2 pi / Tp  (cos^2 x = (1 + cos 2x)/2, product to sum).
struct PulseTerms {
    double a[3], k[3], cep;
};

__host__ __device__ inline PulseTerms pulse_terms(double omega, double E0, double Tp, double cep)
{
    const double W = 2.0 * 3.14159265358979323846 / Tp;
    PulseTerms P;
    P.a[0] = -E0 / (2.0 * omega);
    P.a[1] = -E0 / (4.0 * omega);
    P.a[2] = -E0 / (4.0 * omega);
    P.k[0] = omega;
    P.k[1] = omega + W;
    P.k[2] = omega - W;
    P.cep = cep;
    return P;
}

// E(t) = -dA/dt for real t inside the pulse.
__device__ __forceinline__ double pulse_E(const PulseTerms& P, double t)
{
    double e = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) e -= P.a[m] * P.k[m] * cos(P.k[m] * t + P.cep);
    return e;
}
__device__ __forceinline__ double pulse_A(const PulseTerms& P, double t)
{
    double a = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) a += P.a[m] * sin(P.k[m] * t + P.cep);
    return a;
}

// ------------------------------------------------------------------ potential
// Eq. 7 per centre with the softened distance s = sqrt(|d|^2 + a^2), u = 1/s:
//   V    = -(Zinf + dZ e) u,                     e = exp(-alpha s)
//   grad = g1 d,     g1 = Zinf u^3 + dZ e (alpha u^2 + u^3)
//   Hess = g1 I + g2 d d^T,
//          g2 = -u^2 (3 Zinf u^3 + dZ e u (alpha^2 + 3 alpha u + 3 u^2))
// (from f(s) = -(Zinf + dZ e^{-alpha s})/s: g1 = f'/s, g2 = (f'' - f'/s)/s^2).
template <typename R>
struct Sym3 {
    R xx, yy, zz, xy, xz, yz;
};

template <typename R>
__device__ __forceinline__ R rsqrt_t(R x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ R exp_t(R x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return __expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

template <typename R>
struct PotConst {
    R cx, cy, cz;          // centre offset (R/2) n
    R Zinf, dZ, alpha, a2, w2;
    int kind, screened;
};

// Rotation of a polyatomic molecule, molecular frame -> lab, from the ZYZ
// Euler angles (phi, theta, psi): Rot = Rz(phi) Ry(theta) Rz(psi) multiplied
// out, row-major, given the angles' cosines and sines.  Rot z = n(theta, phi).
template <typename R>
__device__ __forceinline__ void euler_rotation(R cph, R sph, R cth, R sth, R cps, R sps, R Rot[9])
{
    Rot[0] = cph * cth * cps - sph * sps;
    Rot[1] = -cph * cth * sps - sph * cps;
    Rot[2] = cph * sth;
    Rot[3] = sph * cth * cps + cph * sps;
    Rot[4] = -sph * cth * sps + cph * cps;
    Rot[5] = sph * sth;
    Rot[6] = -sth * cps;
    Rot[7] = sth * sps;
    Rot[8] = cth;
}

// Lobe direction of a pi p-type primitive: the unit vector perpendicular to
// the axis n = (sin th cos ph, sin th sin ph, cos th) at azimuth chi about n,
// m = cos(chi) theta_hat + sin(chi) phi_hat with theta_hat =
// (cos th cos ph, cos th sin ph, -sin th) and phi_hat = (-sin ph, cos ph, 0);
// ph = 0 on the z axis.
template <typename R>
__device__ __forceinline__ void pi_direction(R nx, R ny, R nz, R cchi, R schi, R m[3])
{
    const R rho = sqrt(nx * nx + ny * ny);
    R cp = R(1), sp = R(0);
    if (rho > R(0)) {
        cp = nx / rho;
        sp = ny / rho;
    }
    m[0] = cchi * nz * cp - schi * sp;
    m[1] = cchi * nz * sp + schi * cp;
    m[2] = -cchi * rho;
}

// Differences of a step's base point from the two centres +-(R/2)n,
// e_c = (q - c_c) + l, with l the low part of a two-float position (LO; zero
// in FP64).  The centre is subtracted from the high part first (exact near a
// nucleus) and the low part added to that small difference, so the distance
// to a nearby nucleus keeps the two-float precision of the position.  They
// are formed once per RK4 step and shared by its four stages.
template <typename R, bool LO>
__device__ __forceinline__ void centre_diffs(const PotConst<R>& K, const R q[3], const R l[3],
                                             R e[2][3])
{
    const R c[3] = {K.cx, K.cy, K.cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e[0][a] = LO ? (q[a] - c[a]) + l[a] : q[a] - c[a];
        e[1][a] = LO ? (q[a] + c[a]) + l[a] : q[a] + c[a];
    }
}

// V, force F = -grad V and Hessian at the stage point base + o, given the
// base point's centre differences e (centre_diffs) and the RK4 stage offset
// o; OFS = false: the stage point is the base point itself (o ignored).  The
// harmonic test potential (R = 0) reads the position from e[0].
// PK, the form of the potential when it is known at compile time (kPot*,
// sfhk_internal.h); each form runs the same arithmetic as the run-time
// branches it replaces.

template <typename R, bool OFS = true, int PK = kPotAny>
__device__ __forceinline__ void potential(const PotConst<R>& K, const R e[2][3], R ox, R oy,
                                          R oz, R& V, R& Fx, R& Fy, R& Fz, Sym3<R>& H)
{
    // the screening of a molecular target (K.screened when decided at run time)
    const bool screened = PK == kPotBare ? false : PK == kPotScreened ? true : K.screened != 0;
    if (PK == kPotAny && K.kind != 0) {            // harmonic test potential
        const R x = OFS ? e[0][0] + ox : e[0][0];
        const R y = OFS ? e[0][1] + oy : e[0][1];
        const R z = OFS ? e[0][2] + oz : e[0][2];
        V = R(0.5) * K.w2 * (x * x + y * y + z * z);
        Fx = -K.w2 * x;
        Fy = -K.w2 * y;
        Fz = -K.w2 * z;
        H.xx = H.yy = H.zz = K.w2;
        H.xy = H.xz = H.yz = R(0);
        return;
    }
    if constexpr (std::is_same<R, float>::value) {
        // FP32: the two centres side by side in the lanes of float2 values,
        // so that each per-centre operation is one f32x2 instruction
        float2 dx = make_float2(e[0][0], e[1][0]), dy = make_float2(e[0][1], e[1][1]),
               dz = make_float2(e[0][2], e[1][2]);
        if (OFS) {
            dx = __fadd2_rn(dx, make_float2(ox, ox));
            dy = __fadd2_rn(dy, make_float2(oy, oy));
            dz = __fadd2_rn(dz, make_float2(oz, oz));
        }
        const float2 s2 = __ffma2_rn(
            dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(K.a2, K.a2))));
        const float2 u = make_float2(rsqrtf(s2.x), rsqrtf(s2.y));
        const float2 u2 = __fmul2_rn(u, u), u3 = __fmul2_rn(u2, u);
        const float2 zi = make_float2(K.Zinf, K.Zinf);
        float2 vc, g1, g2n;        // g2n = -g2
        if (screened) {
            const float2 sr = __fmul2_rn(s2, u);
            const float2 e = make_float2(__expf(-K.alpha * sr.x), __expf(-K.alpha * sr.y));
            const float2 de = __fmul2_rn(make_float2(K.dZ, K.dZ), e);
            const float2 al = make_float2(K.alpha, K.alpha);
            vc = __fmul2_rn(__fadd2_rn(zi, de), u);
            g1 = __ffma2_rn(de, __ffma2_rn(al, u2, u3), __fmul2_rn(zi, u3));
            const float2 poly = __ffma2_rn(make_float2(3.0f, 3.0f), u2,
                                           __ffma2_rn(make_float2(3.0f * K.alpha, 3.0f * K.alpha),
                                                      u, __fmul2_rn(al, al)));
            g2n = __fmul2_rn(u2, __ffma2_rn(__fmul2_rn(de, u), poly,
                                            __fmul2_rn(make_float2(3.0f * K.Zinf, 3.0f * K.Zinf),
                                                       u3)));
        } else {
            vc = __fmul2_rn(zi, u);
            g1 = __fmul2_rn(zi, u3);
            g2n = __fmul2_rn(make_float2(3.0f * K.Zinf, 3.0f * K.Zinf), __fmul2_rn(u3, u2));
        }
        V = -(vc.x + vc.y);
        Fx = -(g1.x * dx.x + g1.y * dx.y);
        Fy = -(g1.x * dy.x + g1.y * dy.y);
        Fz = -(g1.x * dz.x + g1.y * dz.y);
        const float gs = g1.x + g1.y;
        const float2 gx = __fmul2_rn(g2n, dx), gy = __fmul2_rn(g2n, dy), gz = __fmul2_rn(g2n, dz);
        H.xx = gs - (gx.x * dx.x + gx.y * dx.y);
        H.yy = gs - (gy.x * dy.x + gy.y * dy.y);
        H.zz = gs - (gz.x * dz.x + gz.y * dz.y);
        H.xy = -(gx.x * dy.x + gx.y * dy.y);
        H.xz = -(gx.x * dz.x + gx.y * dz.y);
        H.yz = -(gy.x * dz.x + gy.y * dz.y);
    } else {
        const R o[3] = {ox, oy, oz};
        R d[2][3];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a) d[c][a] = OFS ? e[c][a] + o[a] : e[c][a];
        R g1[2], g2[2], vc[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const R dx = d[c][0], dy = d[c][1], dz = d[c][2];
            const R s2 = dx * dx + dy * dy + dz * dz + K.a2;
            R u = rsqrt_t<R>(s2);
            const R u2 = u * u, u3 = u2 * u;
            if (screened) {
                const R e = exp_t<R>(-K.alpha * (s2 * u));
                const R de = K.dZ * e;
                vc[c] = (K.Zinf + de) * u;
                g1[c] = K.Zinf * u3 + de * (K.alpha * u2 + u3);
                g2[c] = -u2 * (R(3) * K.Zinf * u3 +
                               de * u * (K.alpha * K.alpha + R(3) * K.alpha * u + R(3) * u2));
            } else {
                vc[c] = K.Zinf * u;
                g1[c] = K.Zinf * u3;
                g2[c] = R(-3) * K.Zinf * u3 * u2;
            }
        }
        // sum over the two centres: V = -sum vc, F = -sum g1 d,
        // H = (sum g1) I + sum g2 d d^T
        V = -(vc[0] + vc[1]);
        Fx = -(g1[0] * d[0][0] + g1[1] * d[1][0]);
        Fy = -(g1[0] * d[0][1] + g1[1] * d[1][1]);
        Fz = -(g1[0] * d[0][2] + g1[1] * d[1][2]);
        const R gs = g1[0] + g1[1];
        R gd[2][3];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a) gd[c][a] = g2[c] * d[c][a];
        H.xx = gd[0][0] * d[0][0] + (gd[1][0] * d[1][0] + gs);
        H.yy = gd[0][1] * d[0][1] + (gd[1][1] * d[1][1] + gs);
        H.zz = gd[0][2] * d[0][2] + (gd[1][2] * d[1][2] + gs);
        H.xy = gd[0][0] * d[0][1] + gd[1][0] * d[1][1];
        H.xz = gd[0][0] * d[0][2] + gd[1][0] * d[1][2];
        H.yz = gd[0][1] * d[0][2] + gd[1][1] * d[1][2];
    }
}

// Row r of this lane's column of the per-warp centre table: FP32 rows are
// float4 (x, y, z, 0), one 16-byte shared load, 32 rows of lanes apart; FP64
// rows are three doubles, 32 apart.  kTabWords: words per row and lane.
template <typename R>
constexpr int kTabWords = std::is_same<R, float>::value ? 4 : 3;

template <typename R>
__device__ __forceinline__ void tab_row(const R* tab, int r, R& x, R& y, R& z)
{
    if constexpr (std::is_same<R, float>::value) {
        const float4 v = reinterpret_cast<const float4*>(tab)[r * 32];
        x = v.x;
        y = v.y;
        z = v.z;
    } else {
        x = tab[(3 * r) * 32];
        y = tab[(3 * r + 1) * 32];
        z = tab[(3 * r + 2) * 32];
    }
}

template <typename R>
__device__ __forceinline__ void tab_store(R* tab, int r, R x, R y, R z)
{
    if constexpr (std::is_same<R, float>::value) {
        reinterpret_cast<float4*>(tab)[r * 32] = make_float4(x, y, z, 0.0f);
    } else {
        tab[(3 * r) * 32] = x;
        tab[(3 * r + 1) * 32] = y;
        tab[(3 * r + 2) * 32] = z;
    }
}

// Polyatomic potential (Eq. 7 summed over the N centres of the target, each
// with its own Z_inf, Z0 - Z_inf and alpha): V, F = -grad V and the Hessian
// at the stage point ((q - c) + l) + o for every centre c.  The centres' lab
// positions are this lane's rows of a per-warp shared-memory table (tab_row;
// the lanes of a warp read consecutive words).  Per centre, with u = 1/s,
// s^2 = |d|^2 + a^2:
//   vc = (Zinf + dZ e^{-alpha s}) u,  g1 = Zinf u^3 + dZ e^{-alpha s}(alpha u^2 + u^3),
//   g2 = -u^2 [3 Zinf u^3 + dZ e^{-alpha s} u (alpha^2 + 3 alpha u + 3 u^2)],
//   V = -sum vc,  F = -sum g1 d,  H = (sum g1) I + sum g2 d d^T.
template <typename R>
struct PolyAcc {
    R V, Fx, Fy, Fz, gs, hxx, hyy, hzz, hxy, hxz, hyz;
};

// one centre's terms added to the sums.  BRANCH: skip the screening terms
// of a centre whose dZ is 0 (the generic loop); without it they are
// computed and vanish through dZ = 0 exactly (the unrolled loops, where a
// branch per centre costs more than the arithmetic it saves)
template <typename R, bool LO, bool OFS, bool BRANCH, typename Target>
__device__ __forceinline__ void poly_centre(const Target& T, const R* tab, int c, R a2,
                                            const R q[3], const R l[3], const R o[3],
                                            PolyAcc<R>& A)
{
    constexpr bool F32 = std::is_same<R, float>::value;
    R cc[3], d[3];
    tab_row(tab, c, cc[0], cc[1], cc[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = LO ? (q[a] - cc[a]) + l[a] : q[a] - cc[a];
        if (OFS) d[a] += o[a];
    }
    R Zinf, dZ, al;
    if constexpr (F32) {
        const float4 k = T.cq_f[c];           // one 16-byte load
        Zinf = k.x;
        dZ = k.y;
        al = k.z;
    } else {
        Zinf = T.cZinf[c];
        dZ = T.cdZ[c];
        al = T.calpha[c];
    }
    const R s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + a2;
    const R u = rsqrt_t<R>(s2);
    const R u2 = u * u, u3 = u2 * u;
    R vc, g1, g2;
    if (!BRANCH || dZ != R(0)) {
        const R de = dZ * exp_t<R>(-al * (s2 * u));
        vc = (Zinf + de) * u;
        g1 = Zinf * u3 + de * (al * u2 + u3);
        g2 = -u2 * (R(3) * Zinf * u3 + de * u * (al * al + R(3) * al * u + R(3) * u2));
    } else {
        vc = Zinf * u;
        g1 = Zinf * u3;
        g2 = R(-3) * Zinf * u3 * u2;
    }
    A.V -= vc;
    A.Fx -= g1 * d[0];
    A.Fy -= g1 * d[1];
    A.Fz -= g1 * d[2];
    A.gs += g1;
    const R gx = g2 * d[0], gy = g2 * d[1], gz = g2 * d[2];
    A.hxx += gx * d[0];
    A.hyy += gy * d[1];
    A.hzz += gz * d[2];
    A.hxy += gx * d[1];
    A.hxz += gx * d[2];
    A.hyz += gy * d[2];
}

// NC > 0: the target has exactly NC centres (the loop unrolled); 0: any
// number (a loop over T.n_centres)
template <typename R, bool LO, bool OFS, int NC, typename Target>
__device__ __forceinline__ void potential_poly(const Target& T, const R* tab, R a2,
                                               const R q[3], const R l[3], R ox, R oy, R oz,
                                               R& V, R& Fx, R& Fy, R& Fz, Sym3<R>& H)
{
    PolyAcc<R> A = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    const R o[3] = {ox, oy, oz};
    if constexpr (NC > 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) poly_centre<R, LO, OFS, false>(T, tab, c, a2, q, l, o, A);
    } else {
#pragma unroll 1
        for (int c = 0; c < T.n_centres; ++c)
            poly_centre<R, LO, OFS, true>(T, tab, c, a2, q, l, o, A);
    }
    V = A.V;
    Fx = A.Fx;
    Fy = A.Fy;
    Fz = A.Fz;
    H.xx = A.hxx + A.gs;
    H.yy = A.hyy + A.gs;
    H.zz = A.hzz + A.gs;
    H.xy = A.hxy;
    H.xz = A.hxz;
    H.yz = A.hyz;
}

// Three centres in FP32 (the unrolled three-centre kernel): centres 0 and 1
// side by side in the lanes of float2 values, so that each of their
// per-centre operations is one f32x2 instruction, and centre 2 alone.  The
// base differences e_c = (q - c) + l are formed once per RK4 step from the
// lane's table rows (centre subtracted from the high part first, as in
// centre_diffs) and shared by the step's four stages.
struct Poly3Base {
    float2 x, y, z;        // centres 0 and 1
    float x2, y2, z2;      // centre 2
};

__device__ __forceinline__ void poly3_base(const float* tab, const float q[3], const float l[3],
                                           Poly3Base& B)
{
    float c0[3], c1[3], c2[3];
    tab_row(tab, 0, c0[0], c0[1], c0[2]);
    tab_row(tab, 1, c1[0], c1[1], c1[2]);
    tab_row(tab, 2, c2[0], c2[1], c2[2]);
    B.x = make_float2((q[0] - c0[0]) + l[0], (q[0] - c1[0]) + l[0]);
    B.y = make_float2((q[1] - c0[1]) + l[1], (q[1] - c1[1]) + l[1]);
    B.z = make_float2((q[2] - c0[2]) + l[2], (q[2] - c1[2]) + l[2]);
    B.x2 = (q[0] - c2[0]) + l[0];
    B.y2 = (q[1] - c2[1]) + l[1];
    B.z2 = (q[2] - c2[2]) + l[2];
}

// V, F and the Hessian at the stage point base + o (OFS; else the base
// point), the same terms as poly_centre summed over the three centres
template <bool OFS, typename Target>
__device__ __forceinline__ void potential_poly3(const Target& T, const Poly3Base& B, float a2,
                                                float ox, float oy, float oz, float& V,
                                                float& Fx, float& Fy, float& Fz, Sym3<float>& H)
{
    float2 dx = B.x, dy = B.y, dz = B.z;
    float d2x = B.x2, d2y = B.y2, d2z = B.z2;
    if (OFS) {
        dx = __fadd2_rn(dx, make_float2(ox, ox));
        dy = __fadd2_rn(dy, make_float2(oy, oy));
        dz = __fadd2_rn(dz, make_float2(oz, oz));
        d2x += ox;
        d2y += oy;
        d2z += oz;
    }
    // centres 0 and 1
    const float4 k0 = T.cq2_f[0][0], k1 = T.cq2_f[0][1];
    const float2 zi = make_float2(k0.x, k0.y), dZ = make_float2(k0.z, k0.w),
                 al = make_float2(k1.x, k1.y);
    const float2 s2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(a2, a2))));
    const float2 u = make_float2(rsqrtf(s2.x), rsqrtf(s2.y));
    const float2 u2 = __fmul2_rn(u, u), u3 = __fmul2_rn(u2, u);
    const float2 sr = __fmul2_rn(s2, u);
    const float2 de = __fmul2_rn(dZ, make_float2(__expf(-al.x * sr.x), __expf(-al.y * sr.y)));
    const float2 vc = __fmul2_rn(__fadd2_rn(zi, de), u);
    const float2 g1 = __ffma2_rn(de, __ffma2_rn(al, u2, u3), __fmul2_rn(zi, u3));
    const float2 three = make_float2(3.0f, 3.0f);
    const float2 poly = __ffma2_rn(three, u2, __ffma2_rn(__fmul2_rn(three, al), u, __fmul2_rn(al, al)));
    const float2 g2n =          // -g2
        __fmul2_rn(u2, __ffma2_rn(__fmul2_rn(de, u), poly, __fmul2_rn(__fmul2_rn(three, zi), u3)));
    // centre 2
    const float4 k2 = T.cq_f[2];
    const float zi2 = k2.x, dZ2 = k2.y, al2 = k2.z;
    const float s22 = d2z * d2z + (d2y * d2y + (d2x * d2x + a2));
    const float v = rsqrtf(s22);
    const float v2 = v * v, v3 = v2 * v;
    const float de2 = dZ2 * __expf(-al2 * (s22 * v));
    const float vc2 = (zi2 + de2) * v;
    const float g12 = de2 * (al2 * v2 + v3) + zi2 * v3;
    const float g2n2 =
        v2 * ((de2 * v) * (3.0f * v2 + (3.0f * al2 * v + al2 * al2)) + 3.0f * zi2 * v3);
    // sums over the centres: V = -sum vc, F = -sum g1 d, H = (sum g1) I - sum g2n d d^T
    V = -(vc.x + vc.y + vc2);
    Fx = -(g1.x * dx.x + g1.y * dx.y + g12 * d2x);
    Fy = -(g1.x * dy.x + g1.y * dy.y + g12 * d2y);
    Fz = -(g1.x * dz.x + g1.y * dz.y + g12 * d2z);
    const float gs = g1.x + g1.y + g12;
    const float2 gx = __fmul2_rn(g2n, dx), gy = __fmul2_rn(g2n, dy), gz = __fmul2_rn(g2n, dz);
    const float gx2 = g2n2 * d2x, gy2 = g2n2 * d2y, gz2 = g2n2 * d2z;
    H.xx = gs - (gx.x * dx.x + gx.y * dx.y + gx2 * d2x);
    H.yy = gs - (gy.x * dy.x + gy.y * dy.y + gy2 * d2y);
    H.zz = gs - (gz.x * dz.x + gz.y * dz.y + gz2 * d2z);
    H.xy = -(gx.x * dy.x + gx.y * dy.y + gx2 * d2y);
    H.xz = -(gx.x * dz.x + gx.y * dz.y + gx2 * d2z);
    H.yz = -(gy.x * dz.x + gy.y * dz.y + gy2 * d2z);
}

}  // namespace sfhk

// sfhk_propagate.cu -- the persistent trajectory integrator with the fused
// Herman-Kluk prefactor, recombination element and dipole reduction
// (Sec. II.A and Eq. 4).
//
// One lane = one trajectory; a warp takes a work item of 32 trajectories
// sorted by birth time from a global queue (atomic counter), longest first,
// and walks the time grid from the item's earliest birth in chunks of 32
// steps.  Per step and lane:
//   1. prefactor C = sqrt(det[(M_qq + M_pp - i g M_qp + (i/g) M_pq)/2]) on a
//      continuous branch (sign chosen so that C moves by less than a right
//      angle from the previous step), the finiteness check, the prefactor
//      filter and the stability filter (hard, or tapered in the running
//      maximum of |M|);
//   2. contribution x = Re[w C e^{iS} e^{-i Ip t_n} <psi0|k_z|p,q>] (times the
//      taper weight), stored in the warp's shared-memory tile at (step, lane);
//   3. one RK4 step of (q, p, S) collecting the four stage Hessians, then the
//      six stability-matrix columns advanced by the same RK4 with those
//      Hessians (identical to RK4 on the full 43-component system because the
//      columns obey the linear system dMq/dt = Mp, dMp/dt = -Hess V(q(t)) Mq).
// After each chunk lane l sums row l of the tile (step nb + l over the 32
// trajectories) and adds it, scaled by -2/N, into the FP64 dipole with one
// atomic: no per-trajectory time series reaches HBM.  The field E at the
// chunk's half steps and e^{-i Ip t_n} are loaded once per chunk (one element
// per lane) and broadcast by shuffles.
//
// Diatomic targets run k_propagate (two centres at +-(R/2) n, in the lanes of
// float2 values in FP32); polyatomic targets run k_propagate_poly, the same
// integrator with the N-centre potential over a per-warp table of the
// molecule's lab-frame centres.
//
// Precision policies
//   FP64:  everything in double.
//   MIXED: q, p, M, the stage arithmetic, the determinant and the
//          recombination element in float; q and p accumulated as two-float
//          pairs kept normalised at every step (compensated RK4 update), the
//          action S as a two-float pair, its phase reduced modulo 2 pi in
//          two-float before sincos, the warp sum as two-float, the
//          cross-warp reduction in FP64 atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "sfhk_device.cuh"
#include "sfhk_internal.h"

namespace sfhk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct C2 {
    R x, y;
};

template <typename R>
__device__ __forceinline__ C2<R> cm(C2<R> a, C2<R> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Stability matrix storage.  Column c of M (c < 3: d/dq0_c, c >= 3:
// d/dp0_{c-3}) has the q rows Q(c, r) and the p rows P(c, r), r = 0..2.
template <typename R>
struct Mono {
    R q[6][3], p[6][3];
    __device__ __forceinline__ R Q(int c, int r) const { return q[c][r]; }
    __device__ __forceinline__ R P(int c, int r) const { return p[c][r]; }
    __device__ __forceinline__ void identity(R)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                q[c][r] = (c == r) ? R(1) : R(0);
                p[c][r] = (c == r + 3) ? R(1) : R(0);
            }
    }
};
// FP32: columns k and k + 3 share one float2, so that the RK4 update runs on
// packed pairs (two FP32 operations per f32x2 instruction), and column k + 3
// is stored times -gamma: a float2 is then (Re, Im) of a column of
// Y = M [I; -i gamma I], from which the prefactor matrix
// B = Y_q + (i/gamma) Y_p takes two FMAs per element.  The update is linear
// and column by column, so the scaling does not change it.
template <>
struct Mono<float> {
    float2 q[3][3], p[3][3];
    float nig;                      // -1/gamma
    __device__ __forceinline__ float Q(int c, int r) const
    {
        return c < 3 ? q[c][r].x : q[c - 3][r].y * nig;
    }
    __device__ __forceinline__ float P(int c, int r) const
    {
        return c < 3 ? p[c][r].x : p[c - 3][r].y * nig;
    }
    __device__ __forceinline__ void identity(float gam)
    {
        nig = -1.0f / gam;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                q[k][r] = make_float2(k == r ? 1.0f : 0.0f, 0.0f);
                p[k][r] = make_float2(0.0f, k == r ? -gam : 0.0f);
            }
    }
};

template <typename R>
__device__ __forceinline__ R hypot_t(R a, R b);
template <>
__device__ __forceinline__ float hypot_t<float>(float a, float b) { return hypotf(a, b); }
template <>
__device__ __forceinline__ double hypot_t<double>(double a, double b) { return hypot(a, b); }

// principal square root of z, given r = |z|:  sqrt(z) = (t, y/(2t)) with
// t = sqrt((r + x)/2) for x >= 0, and the mirrored form for x < 0.
template <typename R>
__device__ __forceinline__ C2<R> csqrt_p(C2<R> z, R r)
{
    if (r == R(0)) return {R(0), R(0)};
    const R a = R(0.5) * (r + fabs(z.x));
    const R ra = rsqrt_t<R>(a);
    const R t = a * ra;                      // sqrt(a)
    const R u = R(0.5) * fabs(z.y) * ra;     // |y| / (2 sqrt(a))
    if (z.x >= R(0)) return {t, copysign(u, z.y)};
    return {u, copysign(t, z.y)};
}

// max(a, b, c) in one instruction on sm_100+
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double fmax3(double a, double b, double c) { return fmax(fmax(a, b), c); }

// largest |element| of the stability matrix
__device__ __forceinline__ float max_abs_M(const Mono<float>& M)
{
    // unscaled columns from .x, the -gamma-scaled ones from .y
    float mx[6], my[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mx[2 * k] = fmax3(fabsf(M.q[k][0].x), fabsf(M.q[k][1].x), fabsf(M.q[k][2].x));
        mx[2 * k + 1] = fmax3(fabsf(M.p[k][0].x), fabsf(M.p[k][1].x), fabsf(M.p[k][2].x));
        my[2 * k] = fmax3(fabsf(M.q[k][0].y), fabsf(M.q[k][1].y), fabsf(M.q[k][2].y));
        my[2 * k + 1] = fmax3(fabsf(M.p[k][0].y), fabsf(M.p[k][1].y), fabsf(M.p[k][2].y));
    }
    const float ax = fmax3(fmax3(mx[0], mx[1], mx[2]), mx[3], fmax(mx[4], mx[5]));
    const float ay = fmax3(fmax3(my[0], my[1], my[2]), my[3], fmax(my[4], my[5]));
    return fmax(ax, ay * fabsf(M.nig));
}

template <typename R>
__device__ __forceinline__ R max_abs_M(const Mono<R>& M)
{
    R m[12];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        m[2 * c] = fmax3(fabs(M.Q(c, 0)), fabs(M.Q(c, 1)), fabs(M.Q(c, 2)));
        m[2 * c + 1] = fmax3(fabs(M.P(c, 0)), fabs(M.P(c, 1)), fabs(M.P(c, 2)));
    }
    const R a = fmax3(m[0], m[1], m[2]), b = fmax3(m[3], m[4], m[5]);
    const R c = fmax3(m[6], m[7], m[8]), d = fmax3(m[9], m[10], m[11]);
    return fmax3(a, b, fmax(c, d));
}

// (hi, lo) += x, keeping the pair normalised (|lo| <= ulp(hi)/2, hi the
// correctly rounded value of hi + lo): the increment first takes up the low
// part, t = x + lo, and Dekker's FastTwoSum then splits hi + t into the new
// pair.  The stage arithmetic reads only hi, so hi must carry the pair's
// value at every step: with the low part left to collect rounding errors
// over many steps, hi lags the true state by several ulp, and a chaotic
// trajectory amplifies that lag (measured on an H2 trajectory that ends with
// max |M| = 2e3: 5e-4 relative error of its prefactor against 3e-5 with
// the pair kept normalised, the floor set by the FP32 force evaluation).
// Same four operations as the unnormalised update; the rounding of t loses
// about an ulp of the increment, as its FP32 evaluation already does.
__device__ __forceinline__ void acc2(float& hi, float& lo, float x)
{
    const float t = __fadd_rn(x, lo);
    const float s = __fadd_rn(hi, t);
    lo = __fsub_rn(t, __fsub_rn(s, hi));
    hi = s;
}
// the same for two pairs at once (f32x2); s - hi and t - (s - hi) as FMAs
// with -1, which round exactly like the subtractions
__device__ __forceinline__ void acc2x2(float& h0, float& h1, float& l0, float& l1, float x0,
                                       float x1)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 hi = make_float2(h0, h1);
    const float2 t = __fadd2_rn(make_float2(x0, x1), make_float2(l0, l1));
    const float2 s = __fadd2_rn(hi, t);
    const float2 lo = __ffma2_rn(__ffma2_rn(hi, m1, s), m1, t);
    h0 = s.x;
    h1 = s.y;
    l0 = lo.x;
    l1 = lo.y;
}

template <typename R>
__device__ __forceinline__ R shfl(R v, int src)
{
    return __shfl_sync(kFull, v, src);
}


// 3-vector helpers of the stage arithmetic; in FP32 the (x, y) components go
// through one f32x2 instruction and z through a scalar one.
template <typename R>
__device__ __forceinline__ void scale3(R a, const R x[3], R y[3])      // y = a x
{
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = a * x[i];
}
template <typename R>
__device__ __forceinline__ void axpy3(R a, const R x[3], const R y[3], R z[3])   // z = y + a x
{
#pragma unroll
    for (int i = 0; i < 3; ++i) z[i] = y[i] + a * x[i];
}
// z = a ((u + 2 (v + w)) + x)
template <typename R>
__device__ __forceinline__ void rk4sum3(R a, const R u[3], const R v[3], const R w[3],
                                        const R x[3], R z[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) z[i] = a * (u[i] + R(2) * (v[i] + w[i]) + x[i]);
}
template <>
__device__ __forceinline__ void scale3<float>(float a, const float x[3], float y[3])
{
    const float2 r = __fmul2_rn(make_float2(a, a), make_float2(x[0], x[1]));
    y[0] = r.x;
    y[1] = r.y;
    y[2] = a * x[2];
}
template <>
__device__ __forceinline__ void axpy3<float>(float a, const float x[3], const float y[3],
                                             float z[3])
{
    const float2 r =
        __ffma2_rn(make_float2(a, a), make_float2(x[0], x[1]), make_float2(y[0], y[1]));
    z[0] = r.x;
    z[1] = r.y;
    z[2] = y[2] + a * x[2];
}
template <>
__device__ __forceinline__ void rk4sum3<float>(float a, const float u[3], const float v[3],
                                               const float w[3], const float x[3], float z[3])
{
    const float2 t = __fadd2_rn(
        __ffma2_rn(make_float2(2.0f, 2.0f),
                   __fadd2_rn(make_float2(v[0], v[1]), make_float2(w[0], w[1])),
                   make_float2(u[0], u[1])),
        make_float2(x[0], x[1]));
    const float2 r = __fmul2_rn(make_float2(a, a), t);
    z[0] = r.x;
    z[1] = r.y;
    z[2] = a * (u[2] + 2.0f * (v[2] + w[2]) + x[2]);
}

// The field at a stage point base + o: the two-centre potential from the
// step's centre differences e, or (POLY) the N-centre potential from this
// lane's column of the centre table.
// the packed three-centre form serves mixed-precision three-centre targets
template <typename R, bool MIXED, bool POLY, int NC>
constexpr bool kPoly3 = POLY && MIXED && NC == 3 && std::is_same<R, float>::value;

template <typename R, bool MIXED, bool POLY, bool OFS, int NC = 0, int PK = kPotAny>
__device__ __forceinline__ void field_at(const PotConst<R>& K, const R e[2][3], const DevTarget* T,
                                         const R* tab, const Poly3Base& B3, const R q[3],
                                         const R ql[3], R ox, R oy, R oz, R& V, R F[3],
                                         Sym3<R>& H)
{
    if constexpr (kPoly3<R, MIXED, POLY, NC>)
        potential_poly3<OFS>(*T, B3, K.a2, ox, oy, oz, V, F[0], F[1], F[2], H);
    else if constexpr (POLY)
        potential_poly<R, MIXED, OFS, NC>(*T, tab, K.a2, q, ql, ox, oy, oz, V, F[0], F[1], F[2],
                                          H);
    else
        potential<R, OFS, PK>(K, e, ox, oy, oz, V, F[0], F[1], F[2], H);
}

// One RK4 step's stage evaluations from (q, p) (high part q, low part ql):
// the four stage Hessians and the increments dq, dp, dS of the step.  Stage
// points are formed as base + offset (see potential()).
template <typename R, bool MIXED, bool POLY = false, int NC = 0, int PK = kPotAny>
__device__ __forceinline__ void stage_eval(const PotConst<R>& K, const R q[3], const R ql[3],
                                           const R p[3], R E1, R E2, R E4, R h, R h2, R h6,
                                           Sym3<R> H[4], R dq[3], R dp[3], R& dS,
                                           const DevTarget* T = nullptr, const R* tab = nullptr)
{
    R V, F[3], e[2][3];
    Poly3Base B3;
    if constexpr (!POLY) centre_diffs<R, MIXED>(K, q, ql, e);
    if constexpr (kPoly3<R, MIXED, POLY, NC>) poly3_base(tab, q, ql, B3);
    const R z0 = R(0);
    field_at<R, MIXED, POLY, false, NC, PK>(K, e, T, tab, B3, q, ql, z0, z0, z0, V, F, H[0]);
    const R k1p[3] = {F[0], F[1], F[2] - E1};
    const R k1s = R(0.5) * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) - V - q[2] * E1;
    R o[3], p2[3];
    scale3(h2, p, o);
    axpy3(h2, k1p, p, p2);
    field_at<R, MIXED, POLY, true, NC, PK>(K, e, T, tab, B3, q, ql, o[0], o[1], o[2], V, F, H[1]);
    const R k2p[3] = {F[0], F[1], F[2] - E2};
    const R k2s =
        R(0.5) * (p2[0] * p2[0] + p2[1] * p2[1] + p2[2] * p2[2]) - V - (q[2] + o[2]) * E2;
    R p3[3];
    scale3(h2, p2, o);
    axpy3(h2, k2p, p, p3);
    field_at<R, MIXED, POLY, true, NC, PK>(K, e, T, tab, B3, q, ql, o[0], o[1], o[2], V, F, H[2]);
    const R k3p[3] = {F[0], F[1], F[2] - E2};
    const R k3s =
        R(0.5) * (p3[0] * p3[0] + p3[1] * p3[1] + p3[2] * p3[2]) - V - (q[2] + o[2]) * E2;
    R p4[3];
    scale3(h, p3, o);
    axpy3(h, k3p, p, p4);
    field_at<R, MIXED, POLY, true, NC, PK>(K, e, T, tab, B3, q, ql, o[0], o[1], o[2], V, F, H[3]);
    const R k4s =
        R(0.5) * (p4[0] * p4[0] + p4[1] * p4[1] + p4[2] * p4[2]) - V - (q[2] + o[2]) * E4;
    dS = h6 * (k1s + R(2) * (k2s + k3s) + k4s);
    const R k4p[3] = {F[0], F[1], F[2] - E4};
    rk4sum3(h6, p, p2, p3, p4, dq);
    rk4sum3(h6, k1p, k2p, k3p, k4p, dp);
}

// The six stability-matrix columns advanced by the same RK4 step with the
// four stage Hessians H1..H4 (dMq/dt = Mp, dMp/dt = -Hess V Mq).  With
// a_i = H_i x_i the stage accelerations (x_1 = Mq, x_2 = Mq + h/2 Mp,
// x_3 = x_2 - h^2/4 a_1, x_4 = Mq + h Mp - h^2/2 a_2), the RK4 sums collapse to
//   Mq' = Mq + h Mp - h^2/6 (a_1 + a_2 + a_3)
//   Mp' = Mp - h/6 (a_1 + 2 a_2 + 2 a_3 + a_4),
// the same step up to rounding order; every Hessian term enters as a small
// correction added to the larger part last, so it keeps its own precision.
template <typename R>
__device__ __forceinline__ void hx(const Sym3<R>& H, const R x[3], R y[3])
{
    y[0] = H.xx * x[0] + H.xy * x[1] + H.xz * x[2];
    y[1] = H.xy * x[0] + H.yy * x[1] + H.yz * x[2];
    y[2] = H.xz * x[0] + H.yz * x[1] + H.zz * x[2];
}

template <typename R>
__device__ __forceinline__ void m_update(Mono<R>& M, const Sym3<R> H[4], R h, R h2, R h6, R hh4,
                                         R hh2, R hh6)
{
    // hh4 = h^2/4, hh2 = h^2/2, hh6 = h^2/6
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        R x0[3], v0[3], xs[3], xb[3], a1[3], a2[3], a3[3], a4[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            x0[r] = M.q[c][r];
            v0[r] = M.p[c][r];
            xs[r] = x0[r] + h2 * v0[r];
            xb[r] = x0[r] + h * v0[r];
        }
        hx(H[0], x0, a1);
        hx(H[1], xs, a2);
#pragma unroll
        for (int r = 0; r < 3; ++r) xs[r] = xs[r] - hh4 * a1[r];
        hx(H[2], xs, a3);
#pragma unroll
        for (int r = 0; r < 3; ++r) xs[r] = xb[r] - hh2 * a2[r];
        hx(H[3], xs, a4);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            M.q[c][r] = xb[r] - hh6 * ((a1[r] + a2[r]) + a3[r]);
            M.p[c][r] = v0[r] - h6 * ((a1[r] + a4[r]) + R(2) * (a2[r] + a3[r]));
        }
    }
}

// The same update on packed column pairs, every operation one f32x2
// instruction for two columns.  The stage sums are accumulated inside the
// Hessian products instead of after them (hxa: y = H x + acc), which saves
// the separate adds:
//   s12 = a1 + a2,  sA = H3 x3 + s12 = a1 + a2 + a3,
//   Mq' = xb - h^2/6 sA,
//   Mp' = v0 - h/6 (H4 x4 + (2 sA - a1)) = v0 - h/6 (a1 + 2 a2 + 2 a3 + a4).
// a1 is formed negated (from -H1), so that all three of its uses are FMAs.
__device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }

__device__ __forceinline__ void hx2(const Sym3<float>& H, const float2 x[3], float2 y[3])
{
    y[0] = __ffma2_rn(bc(H.xz), x[2], __ffma2_rn(bc(H.xy), x[1], __fmul2_rn(bc(H.xx), x[0])));
    y[1] = __ffma2_rn(bc(H.yz), x[2], __ffma2_rn(bc(H.yy), x[1], __fmul2_rn(bc(H.xy), x[0])));
    y[2] = __ffma2_rn(bc(H.zz), x[2], __ffma2_rn(bc(H.yz), x[1], __fmul2_rn(bc(H.xz), x[0])));
}

__device__ __forceinline__ void hxa2(const Sym3<float>& H, const float2 x[3], const float2 acc[3],
                                     float2 y[3])
{
    y[0] = __ffma2_rn(bc(H.xz), x[2], __ffma2_rn(bc(H.xy), x[1], __ffma2_rn(bc(H.xx), x[0], acc[0])));
    y[1] = __ffma2_rn(bc(H.yz), x[2], __ffma2_rn(bc(H.yy), x[1], __ffma2_rn(bc(H.xy), x[0], acc[1])));
    y[2] = __ffma2_rn(bc(H.zz), x[2], __ffma2_rn(bc(H.yz), x[1], __ffma2_rn(bc(H.xz), x[0], acc[2])));
}

__device__ __forceinline__ void m_update(Mono<float>& M, const Sym3<float> H[4], float h,
                                         float h2, float h6, float hh4, float hh2, float hh6)
{
    const float2 vh = bc(h), vh2 = bc(h2), mh6 = bc(-h6), phh4 = bc(hh4), mhh2 = bc(-hh2),
                 mhh6 = bc(-hh6), two = bc(2.0f), m1 = bc(-1.0f);
    const Sym3<float> nH1 = {-H[0].xx, -H[0].yy, -H[0].zz, -H[0].xy, -H[0].xz, -H[0].yz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float2 x0[3], v0[3], xs[3], xb[3], a1[3], a2[3], t[3];   // a1 holds -a1
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            x0[r] = M.q[k][r];
            v0[r] = M.p[k][r];
            xs[r] = __ffma2_rn(vh2, v0[r], x0[r]);
            xb[r] = __ffma2_rn(vh, v0[r], x0[r]);
        }
        hx2(nH1, x0, a1);                               // -a1
        hx2(H[1], xs, a2);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            xs[r] = __ffma2_rn(phh4, a1[r], xs[r]);     // x3 = x2 - h^2/4 a1
            t[r] = __ffma2_rn(m1, a1[r], a2[r]);        // s12 = a1 + a2
        }
        hxa2(H[2], xs, t, t);                           // sA
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            xs[r] = __ffma2_rn(mhh2, a2[r], xb[r]);     // x4
            M.q[k][r] = __ffma2_rn(mhh6, t[r], xb[r]);
            t[r] = __ffma2_rn(two, t[r], a1[r]);        // 2 sA - a1
        }
        hxa2(H[3], xs, t, t);
#pragma unroll
        for (int r = 0; r < 3; ++r) M.p[k][r] = __ffma2_rn(mh6, t[r], v0[r]);
    }
}

// Element (r, c) of 2 x the prefactor matrix, M_qq + M_pp + i (M_pq / g - g M_qp).
template <typename R>
__device__ __forceinline__ C2<R> b_elem(const Mono<R>& M, int r, int c, R gam, R igam)
{
    return {M.Q(c, r) + M.P(3 + c, r), igam * M.P(c, r) - gam * M.Q(3 + c, r)};
}
// FP32 (column c + 3 stored times -g): Re = Q_c + P_{c+3} = q.x - p.y / g,
// Im = P_c / g - g Q_{c+3} = p.x / g + q.y
__device__ __forceinline__ C2<float> b_elem(const Mono<float>& M, int r, int c, float,
                                            float igam)
{
    const float2 q = M.q[c][r], p = M.p[c][r];
    return {fmaf(-igam, p.y, q.x), fmaf(igam, p.x, q.y)};
}

// Prefactor of the current M on the continuous branch (sign kept within a
// right angle of the previous C), then the per-step checks in the order:
// finiteness, prefactor filter, stability filter.
template <typename R>
__device__ __forceinline__ void prefactor_and_checks(const Mono<R>& M, R gam,
                                                     R igam, C2<R>& Cp, const R q[3],
                                                     const R p[3], R S, R cut2, R stab,
                                                     R stab_hi, R& Mhat, int& status)
{
    C2<R> B[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            B[3 * r + c] = b_elem(M, r, c, gam, igam);
    const C2<R> m0 = cm(B[4], B[8]), m1 = cm(B[5], B[7]);
    const C2<R> m2 = cm(B[3], B[8]), m3 = cm(B[5], B[6]);
    const C2<R> m4 = cm(B[3], B[7]), m5 = cm(B[4], B[6]);
    const C2<R> c0 = cm(B[0], {m0.x - m1.x, m0.y - m1.y});
    const C2<R> c1 = cm(B[1], {m2.x - m3.x, m2.y - m3.y});
    const C2<R> c2 = cm(B[2], {m4.x - m5.x, m4.y - m5.y});
    // det of the half-sum matrix = det(B) / 8
    const C2<R> det = {R(0.125) * (c0.x - c1.x + c2.x), R(0.125) * (c0.y - c1.y + c2.y)};
    // |det| from its square where that neither overflows nor underflows
    R rdet;
    const R r2 = det.x * det.x + det.y * det.y;
    if (r2 > R(1e-30) && r2 < R(1e30)) rdet = r2 * rsqrt_t<R>(r2);
    else rdet = hypot_t<R>(det.x, det.y);
    C2<R> C = csqrt_p(det, rdet);
    if (C.x * Cp.x + C.y * Cp.y < R(0)) {
        C.x = -C.x;
        C.y = -C.y;
    }
    Cp = C;
    const bool fin = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(p[0]) &&
                     isfinite(p[1]) && isfinite(p[2]) && isfinite(S) && isfinite(rdet);
    if (!fin) status = 2;
    else if (cut2 > R(0) && rdet > cut2) status = 1;
    else if (stab > R(0)) {
        const R mm = max_abs_M(M);
        if (stab_hi > R(0)) {
            // tapered filter: running maximum, stop at the taper's end
            Mhat = fmax(Mhat, mm);
            if (Mhat >= stab_hi) status = 3;
        } else if (mm > stab) {
            status = 3;
        }
    }
}

// Weight of the tapered stability filter for a running maximum Mhat above
// the cutoff m0: (1 + cos(pi ln(Mhat/m0) / ln r)) / 2.
template <typename R>
__device__ __forceinline__ R taper_weight(R Mhat, R m0, R inv_log_r)
{
    if constexpr (std::is_same<R, float>::value)
        return 0.5f * (1.0f + __cosf(3.14159265f * __logf(Mhat / m0) * inv_log_r));
    else
        return 0.5 * (1.0 + cos(3.141592653589793 * log(Mhat / m0) * inv_log_r));
}

// <psi0|k_z|p,q> summed over both centres and the primitives, FP32, with the
// two centres in the lanes of float2 values (one f32x2 instruction per
// per-centre operation).  Both centres are evaluated unless both are beyond
// the far-field bound; a primitive whose exponent is below kSkipMixed is
// dropped in its lane.  Per centre and primitive the term is
//   K4 e^{K1 |d|^2 + K2 |p|^2} (p_z - i g d_z) e^{i K3 p.d}
// for an s-type primitive and
//   s_c K4 e^{K1 |d|^2 + K2 |p|^2} [(P1 n.d + i P2 n.p)(p_z - i g d_z) + i P3 n_z] e^{i K3 p.d}
// for a sigma p-type one (s_c = +-1 the centre's sign; n the axis, read
// only when the target has p-type primitives), and the same with s_c n
// replaced by the lobe direction m for a pi p-type one.
constexpr float kSkipMixed = -30.0f;

// recomb_pair's loop for a target with sigma p-type primitives
__device__ __forceinline__ C2<float> recomb_pair_sp(const DevInstance& I, const float q[3],
                                                    const float p[3], float pp, int n_prim, int j,
                                                    float2 dz, float2 dd, float2 pdd, float2 gdz)
{
    C2<float> Rk;
    float2 P = make_float2(0.0f, 0.0f), Q = P, U = P, Wv = P;
    const long long n = I.n;
    const double* nhat = I.soa + 7 * n + j;
    const float nx = (float)nhat[0], ny = (float)nhat[n], nz = (float)nhat[2 * n];
    const float hR = (float)I.tgt.half_R;
    const float nq = nx * q[0] + ny * q[1] + nz * q[2];
    const float np = nx * p[0] + ny * p[1] + nz * p[2];
    const float2 snd = make_float2(nq - hR, -nq - hR);          // s_c n.d
    const float2 snp = make_float2(np, -np);                    // s_c n.p
    const float2 snz = make_float2(nz, -nz);                    // s_c n_z
    const float2 pz2 = make_float2(p[2], p[2]);
    // pi lobe m (m.d = m.q, as m is perpendicular to the axis), both centres
    float2 md = make_float2(0.0f, 0.0f), mp = md, mz = md;
    if (I.rec.has_p & 2) {
        float m[3];
        pi_direction<float>(nx, ny, nz, (float)I.rec.cchi, (float)I.rec.schi, m);
        const float mq = m[0] * q[0] + m[1] * q[1] + m[2] * q[2];
        const float mpp = m[0] * p[0] + m[1] * p[1] + m[2] * p[2];
        md = make_float2(mq, mq);
        mp = make_float2(mpp, mpp);
        mz = make_float2(m[2], m[2]);
    }
#pragma unroll 1
    for (int k = 0; k < n_prim; ++k) {
        const float K1 = I.rec.K1f[k], K2 = I.rec.K2f[k], K3 = I.rec.K3f[k], K4 = I.rec.K4f[k];
        const float2 ex = __ffma2_rn(make_float2(K1, K1), dd, make_float2(K2 * pp, K2 * pp));
        const float2 arg = __fmul2_rn(make_float2(K3, K3), pdd);
        float2 mag, sn, cs;
        mag.x = ex.x > kSkipMixed ? K4 * __expf(ex.x) : 0.0f;
        mag.y = ex.y > kSkipMixed ? K4 * __expf(ex.y) : 0.0f;
        __sincosf(arg.x, &sn.x, &cs.x);
        __sincosf(arg.y, &sn.y, &cs.y);
        float2 br = pz2, bi = gdz;                              // s-type bracket
        const int kind = I.rec.kind[k];
        if (kind) {
            // sigma: s_c (n.d, n.p, n_z); pi: (m.d, m.p, m_z)
            const float2 ud = kind == 1 ? snd : md;
            const float2 up = kind == 1 ? snp : mp;
            const float2 uz = kind == 1 ? snz : mz;
            const float P1 = I.rec.P1f[k], P2 = I.rec.P2f[k], P3 = I.rec.P3f[k];
            const float2 u = __fmul2_rn(make_float2(P1, P1), ud);
            const float2 v = __fmul2_rn(make_float2(P2, P2), up);
            // (u + i v)(p_z + i gdz) + i P3 u_z
            const float2 vg = __fmul2_rn(v, gdz);
            br = __ffma2_rn(u, pz2, make_float2(-vg.x, -vg.y));
            bi = __ffma2_rn(u, gdz, __ffma2_rn(v, pz2, __fmul2_rn(make_float2(P3, P3), uz)));
        }
        const float2 A = __fmul2_rn(mag, br);
        const float2 B = __fmul2_rn(mag, bi);
        P = __ffma2_rn(A, cs, P);
        Q = __ffma2_rn(B, sn, Q);
        U = __ffma2_rn(A, sn, U);
        Wv = __ffma2_rn(B, cs, Wv);
    }
    Rk.x = (P.x + P.y) - (Q.x + Q.y);
    Rk.y = (U.x + U.y) + (Wv.x + Wv.y);
    return Rk;
}

__device__ __forceinline__ C2<float> recomb_pair(const DevInstance& I, const PotConst<float>& K,
                                                 const float q[3], const float p[3], float pp,
                                                 float gam, float K1max, float K2max, int n_prim,
                                                 int j)
{
    const float2 dx = make_float2(q[0] - K.cx, q[0] + K.cx);
    const float2 dy = make_float2(q[1] - K.cy, q[1] + K.cy);
    const float2 dz = make_float2(q[2] - K.cz, q[2] + K.cz);
    const float2 dd = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const float2 far = __ffma2_rn(make_float2(K1max, K1max), dd, make_float2(K2max * pp, K2max * pp));
    C2<float> Rk = {0.0f, 0.0f};
    if (far.x <= kSkipMixed && far.y <= kSkipMixed) return Rk;
    const float2 pdd = __ffma2_rn(make_float2(p[2], p[2]), dz,
                                  __ffma2_rn(make_float2(p[1], p[1]), dy,
                                             __fmul2_rn(make_float2(p[0], p[0]), dx)));
    const float2 gdz = __fmul2_rn(make_float2(-gam, -gam), dz);     // -g d_z
    float2 P = make_float2(0.0f, 0.0f), Q = P, U = P, Wv = P;
    if (I.rec.has_p) return recomb_pair_sp(I, q, p, pp, n_prim, j, dz, dd, pdd, gdz);
#pragma unroll 1
    for (int k = 0; k < n_prim; ++k) {
        const float K1 = I.rec.K1f[k], K2 = I.rec.K2f[k], K3 = I.rec.K3f[k], K4 = I.rec.K4f[k];
        const float2 ex = __ffma2_rn(make_float2(K1, K1), dd, make_float2(K2 * pp, K2 * pp));
        const float2 arg = __fmul2_rn(make_float2(K3, K3), pdd);
        float2 mag, sn, cs;
        mag.x = ex.x > kSkipMixed ? K4 * __expf(ex.x) : 0.0f;
        mag.y = ex.y > kSkipMixed ? K4 * __expf(ex.y) : 0.0f;
        __sincosf(arg.x, &sn.x, &cs.x);
        __sincosf(arg.y, &sn.y, &cs.y);
        const float2 A = __fmul2_rn(mag, make_float2(p[2], p[2]));   // mag p_z
        const float2 B = __fmul2_rn(mag, gdz);                       // -mag g d_z
        // (A + i B)(cs + i sn) = (A cs - B sn) + i (A sn + B cs)
        P = __ffma2_rn(A, cs, P);
        Q = __ffma2_rn(B, sn, Q);
        U = __ffma2_rn(A, sn, U);
        Wv = __ffma2_rn(B, cs, Wv);
    }
    Rk.x = (P.x + P.y) - (Q.x + Q.y);
    Rk.y = (U.x + U.y) + (Wv.x + Wv.y);
    return Rk;
}

// <psi0|k_z|p,q> of a polyatomic target: every primitive on its own centre
// (lab position from this lane's column of the table), term
//   K4 e^{K1 |d|^2 + K2 |p|^2 + i K3 p.d} (p_z - i g d_z)               (s-type)
//   K4 e^{...} [(P1 u.d + i P2 u.p)(p_z - i g d_z) + i P3 u_z]          (p-type, u)
// with d = q - A_c; terms below e^skip of their peak are not evaluated.
template <typename R>
__device__ __forceinline__ C2<R> recomb_poly(const DevInstance& I, const R* tab, const R q[3],
                                             const R p[3], R pp, R gam, int n_prim, R skip)
{
    constexpr bool F32 = std::is_same<R, float>::value;
    const int nc = I.tgt.n_centres;
    C2<R> Rk = {R(0), R(0)};
#pragma unroll 1
    for (int k = 0; k < n_prim; ++k) {
        const int c = I.tgt.pcentre[k];
        R cx, cy, cz;
        tab_row(tab, c, cx, cy, cz);
        const R dx = q[0] - cx, dy = q[1] - cy, dz = q[2] - cz;
        const R dd = dx * dx + dy * dy + dz * dz;
        const R K1 = F32 ? R(I.rec.K1f[k]) : R(I.rec.K1[k]);
        const R K2 = F32 ? R(I.rec.K2f[k]) : R(I.rec.K2[k]);
        const R ex = K1 * dd + K2 * pp;
        if (!(ex > skip)) continue;
        const R K3 = F32 ? R(I.rec.K3f[k]) : R(I.rec.K3[k]);
        const R K4 = F32 ? R(I.rec.K4f[k]) : R(I.rec.K4[k]);
        const R mag = K4 * exp_t<R>(ex);
        const R pdd = p[0] * dx + p[1] * dy + p[2] * dz;
        R sn, cs;
        if constexpr (F32) __sincosf(K3 * pdd, &sn, &cs);
        else sincos(K3 * pdd, &sn, &cs);
        R ar = mag * p[2], ai = -mag * gam * dz;
        if (I.rec.kind[k] == SFHK_PRIM_P_DIR) {
            R ux, uy, uz;
            tab_row(tab, nc + k, ux, uy, uz);
            const R P1 = F32 ? R(I.rec.P1f[k]) : R(I.rec.P1[k]);
            const R P2 = F32 ? R(I.rec.P2f[k]) : R(I.rec.P2[k]);
            const R P3 = F32 ? R(I.rec.P3f[k]) : R(I.rec.P3[k]);
            const R u = P1 * (ux * dx + uy * dy + uz * dz);
            const R v = P2 * (ux * p[0] + uy * p[1] + uz * p[2]);
            ar = mag * (u * p[2] + v * gam * dz);
            ai = mag * (-u * gam * dz + v * p[2] + P3 * uz);
        }
        Rk.x += ar * cs - ai * sn;
        Rk.y += ar * sn + ai * cs;
    }
    return Rk;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A lane's dynamic state in a park entry: column `lane` of kParkWords rows,
// 32 words apart (STORE: write it there; else read it back).  Integers are
// kept bit for bit in FP32 words and exactly in FP64 ones.
template <typename R>
__device__ __forceinline__ R park_from_int(int v)
{
    if constexpr (std::is_same<R, float>::value) return __int_as_float(v);
    else return R(v);
}
template <typename R>
__device__ __forceinline__ int park_to_int(R v)
{
    if constexpr (std::is_same<R, float>::value) return __float_as_int(v);
    else return int(v);
}

template <typename R, bool STORE>
__device__ __forceinline__ void park_io(R* col, R q[3], R ql[3], R p[3], R pl[3], Mono<R>& M,
                                        R& S, R& Sl, C2<R>& Cp, R& Mhat, int& status,
                                        int& n_ret, bool& left, R& e_ret, unsigned int& steps)
{
    int k = 0;
    auto io = [&](R& v) {
        if constexpr (STORE) col[k * kWarp] = v;
        else v = col[k * kWarp];
        ++k;
    };
    auto io_int = [&](int& v) {
        R w = park_from_int<R>(v);
        io(w);
        if constexpr (!STORE) v = park_to_int<R>(w);
    };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        io(q[a]);
        io(ql[a]);
        io(p[a]);
        io(pl[a]);
    }
    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                io(M.q[c][r].x);
                io(M.q[c][r].y);
                io(M.p[c][r].x);
                io(M.p[c][r].y);
            }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                io(M.q[c][r]);
                io(M.p[c][r]);
            }
    }
    io(S);
    io(Sl);
    io(Cp.x);
    io(Cp.y);
    io(Mhat);
    io(e_ret);
    int lf = left ? 1 : 0, st = (int)steps;
    io_int(status);
    io_int(n_ret);
    io_int(lf);
    io_int(st);
    if constexpr (!STORE) {
        left = lf != 0;
        steps = (unsigned int)st;
    }
}

// per-warp buffer of the chunk's contributions: 32 steps x 32 trajectories,
// row stride 33
constexpr int kRedStride = kWarp + 1;
constexpr int kRedElems = kWarp * kRedStride;

// POLY: a polyatomic target; tab is this lane's column of the warp's table
// of lab-frame centre positions and p directions (rows of 32 words); NC > 0:
// every such target of the launch has exactly NC centres.
// PARK (server slices): resume >= 0 restores the item's state from entry
// `resume` of pk->in_*; with a deadline, the item is parked at the first
// chunk boundary past it that has chunks left.  Returns whether the item
// ran to its end (false: parked).
template <bool MIXED, bool POLY = false, int NC = 0, bool FIXED = false, bool PARK = false,
          int PK = kPotAny>
__device__ __forceinline__ bool process_item(const DevInstance& I, const WorkItem& W, int lane,
                                             typename std::conditional<MIXED, float, double>::type* red,
                                             typename std::conditional<MIXED, float, double>::type* tab = nullptr,
                                             const ParkBufs* pk = nullptr, int resume = -1,
                                             unsigned long long deadline = 0)
{
    using R = typename std::conditional<MIXED, float, double>::type;

    const int nt = I.nt;
    const bool has = lane < W.count;
    const long long n = I.n;
    const int j = has ? I.perm[W.first + lane] : 0;
    const int n0 = has ? I.n0[j] : nt;

    // ---- per-trajectory inputs (FP64 in memory)
    const double* soa = I.soa;
    double qd[3], pd[3], nh[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        qd[a] = has ? soa[(1 + a) * n + j] : 0.0;
        pd[a] = has ? soa[(4 + a) * n + j] : 0.0;
        nh[a] = has ? soa[(7 + a) * n + j] : 0.0;
    }
    const double wr = has ? soa[10 * n + j] : 0.0, wi = has ? soa[11 * n + j] : 0.0;

    PotConst<R> K;
    K.cx = R(I.tgt.half_R * nh[0]);
    K.cy = R(I.tgt.half_R * nh[1]);
    K.cz = R(I.tgt.half_R * nh[2]);
    K.Zinf = R(I.tgt.Zinf);
    K.dZ = R(I.tgt.dZ);
    K.alpha = R(I.tgt.alpha);
    K.a2 = R(I.tgt.a2);
    K.w2 = R(I.tgt.w2);
    K.kind = I.tgt.kind;
    K.screened = I.tgt.screened;
    const int n_prim = I.tgt.n_prim;
    if constexpr (POLY) {
        // fields 7..9 are the Euler angles: the molecule's lab-frame centres
        // and p directions, Rot x, into this lane's column of the table
        K.cx = K.cy = K.cz = R(0);
        K.kind = 0;
        double sph, cph, sth, cth, sps, cps, Rot[9];
        sincos(nh[0], &sph, &cph);
        sincos(nh[1], &sth, &cth);
        sincos(nh[2], &sps, &cps);
        euler_rotation<double>(cph, sph, cth, sth, cps, sps, Rot);
        const int nc = I.tgt.n_centres;
        for (int r = 0; r < I.tgt.n_slots; ++r) {
            const double* x = r < nc ? I.tgt.cpos[r] : I.tgt.pdir[r - nc];
            R v[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                v[a] = R(Rot[3 * a] * x[0] + Rot[3 * a + 1] * x[1] + Rot[3 * a + 2] * x[2]);
            tab_store(tab, r, v[0], v[1], v[2]);
        }
    }
    // FIXED: the launch's instances all have FixedParams' values, which are
    // then compile-time constants (equal to the instance's, value for value)
    using F = FixedParams;
    const R gam = FIXED ? R(F::gamma) : R(I.gamma);
    const R igam = FIXED ? R(1.0 / F::gamma) : R(I.inv_gamma);
    const R wR = R(wr), wI = R(wi);
    const R cut2 = FIXED ? R(F::cutoff * F::cutoff) : R(I.cutoff2);   // |det| = |C|^2 threshold (0 = off)
    const R stab = FIXED ? R(F::stab) : R(I.stab_cut);
    const R stab_hi = FIXED ? R(F::taper * F::stab) : R(I.stab_hi);   // tapered filter (0 = hard cut)
    R Mhat = R(0);                            // running max of max |M_ij| (tapered filter)
    // far-field bound of the recombination exponent over the primitives:
    // K1 |d|^2 + K2 |p|^2 <= K1max |d|^2 + K2max |p|^2 (all K1, K2 < 0)
    R K1max = R(-1e30), K2max = R(-1e30);
    for (int k = 0; k < n_prim; ++k) {
        K1max = fmax(K1max, R(I.rec.K1[k]));
        K2max = fmax(K2max, R(I.rec.K2[k]));
    }
    // a Gaussian overlap below e^kSkip of its peak is not evaluated: in MIXED
    // such a term is below 1e-13 of the same trajectory's terms near the
    // nucleus, far under the FP32 resolution of the sum
    constexpr R kSkip = MIXED ? R(kSkipMixed) : R(-200);

    // ---- state
    R q[3], p[3], ql[3], pl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q[a] = R(qd[a]);
        p[a] = R(pd[a]);
        ql[a] = R(qd[a] - double(q[a]));
        pl[a] = R(pd[a] - double(p[a]));
    }
    Mono<R> M;
    M.identity(gam);
    // first returns (optional; the fixed-parameter integrators do not record
    // them, fixed_params sends such launches to the generic one)
    double* const ret = FIXED ? nullptr : I.returns;
    const R r_out = R(I.ret_out), r_in = R(I.ret_in);
    bool left = false;
    int n_ret = -1;
    R e_ret = R(0);
    R S = R(0), Sl = R(0);          // action (two-float in MIXED, Sl unused in FP64)
    C2<R> Cp = {R(1), R(0)};        // prefactor at the previous step
    int status = 0;                 // 0 alive, 1 prefactor filter, 2 non-finite, 3 stability filter
    unsigned int steps = 0;          // RK4 steps taken (< Nt)
    int nb_first = W.n_start;        // first step of the first chunk this call runs
    if constexpr (PARK) {
        if (resume >= 0) {
            R* col = (R*)pk->in_state + (size_t)resume * kParkWords * kWarp + lane;
            park_io<R, false>(col, q, ql, p, pl, M, S, Sl, Cp, Mhat, status, n_ret, left, e_ret,
                              steps);
            nb_first = pk->in_hdr[resume].nb;
        }
    }

    const double dt = FIXED ? F::dt : I.dt;
    const R h = R(dt), h2 = R(0.5 * dt), h6 = R(dt / 6.0);
    const R hh4 = R(dt * dt / 4.0), hh2 = R(dt * dt / 2.0), hh6 = R(dt * dt / 6.0);
    const int nE = 2 * nt - 1;

    // Carried only within a step: the stage Hessians and increments.
    Sym3<R> Hs[4];
    R dq[3], dp[3], dS;
    for (int nb = nb_first; nb < nt; nb += kWarp) {
        // chunk tables: E at the half steps of step nb+lane, e^{-i Ip t} at
        // nb+lane; broadcast by shuffles
        const int nl = nb + lane;
        R e0, e1, e2;
        C2<R> phl;
        if constexpr (MIXED) {
            e0 = I.Ehf[min(2 * nl, nE - 1)];
            e1 = I.Ehf[min(2 * nl + 1, nE - 1)];
            e2 = I.Ehf[min(2 * nl + 2, nE - 1)];
            const float2 t = I.phf[min(nl, nt - 1)];
            phl = {t.x, t.y};
        } else {
            e0 = I.Eh[min(2 * nl, nE - 1)];
            e1 = I.Eh[min(2 * nl + 1, nE - 1)];
            e2 = I.Eh[min(2 * nl + 2, nE - 1)];
            const double2 t = I.ph[min(nl, nt - 1)];
            phl = {t.x, t.y};
        }
        bool contributed = false;
        const int send = min(kWarp, nt - nb);
        for (int s = 0; s < send; ++s) {
            const int nn = nb + s;
            const R E1 = shfl(e0, s), E2 = shfl(e1, s), E4 = shfl(e2, s);
            const C2<R> ph = {shfl(phl.x, s), shfl(phl.y, s)};
            const bool live = (nn >= n0) && status == 0;
            // ---- prefactor at t_nn (C = 1 at birth) and the checks
            if (live)
                prefactor_and_checks(M, gam, igam, Cp, q, p, S, cut2, stab, stab_hi, Mhat, status);
            // ---- contribution at t_nn: Re[w C e^{iS} e^{-i Ip t} <psi0|k_z|p,q>]
            R x = R(0);
            if (live && status == 0) {
                const R pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
                // first return along the polarisation axis (optional)
                if (ret != nullptr && n_ret < 0) {
                    const R az = fabs(q[2]);
                    if (az > r_out) left = true;
                    else if (left && az < r_in) {
                        n_ret = nn;
                        e_ret = R(0.5) * pp;
                    }
                }
                C2<R> Rk = {R(0), R(0)};
                if constexpr (POLY) {
                    Rk = recomb_poly<R>(I, tab, q, p, pp, gam, n_prim, kSkip);
                } else if constexpr (MIXED) {
                    Rk = recomb_pair(I, K, q, p, pp, gam, K1max, K2max, n_prim, j);
                } else {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const R dx = c == 0 ? q[0] - K.cx : q[0] + K.cx;
                    const R dy = c == 0 ? q[1] - K.cy : q[1] + K.cy;
                    const R dz = c == 0 ? q[2] - K.cz : q[2] + K.cz;
                    const R dd = dx * dx + dy * dy + dz * dz;
                    if (K1max * dd + K2max * pp <= kSkip) continue;   // far from this centre
                    const R pdd = p[0] * dx + p[1] * dy + p[2] * dz;
#pragma unroll 1
                    for (int k = 0; k < n_prim; ++k) {
                        R K1, K2, K3, K4;
                        if constexpr (MIXED) {
                            K1 = I.rec.K1f[k]; K2 = I.rec.K2f[k];
                            K3 = I.rec.K3f[k]; K4 = I.rec.K4f[k];
                        } else {
                            K1 = I.rec.K1[k]; K2 = I.rec.K2[k];
                            K3 = I.rec.K3[k]; K4 = I.rec.K4[k];
                        }
                        const R ex = K1 * dd + K2 * pp;
                        if (ex > kSkip) {
                            const R mag = K4 * exp_t<R>(ex);
                            R sn, cs;
                            if constexpr (MIXED) __sincosf(K3 * pdd, &sn, &cs);
                            else sincos(K3 * pdd, &sn, &cs);
                            // mag (p_z - i g d_z)(cs + i sn), or for a p-type
                            // primitive mag s [(P1 u.d + i P2 u.p)(p_z - i g d_z)
                            // + i P3 u_z](cs + i sn) (sigma: u = n, s = s_c; pi:
                            // u = m, s = 1)
                            R ar = mag * p[2], ai = -mag * gam * dz;
                            if (I.rec.kind[k]) {
                                // sigma: u = n, sign s_c; pi: u = m, sign 1
                                const double* nv = soa + 7 * n + j;
                                R u3[3] = {R(nv[0]), R(nv[n]), R(nv[2 * n])};
                                R sc = c == 0 ? R(1) : R(-1);
                                if (I.rec.kind[k] == 2) {
                                    R m[3];
                                    pi_direction<R>(u3[0], u3[1], u3[2], R(I.rec.cchi),
                                                    R(I.rec.schi), m);
                                    u3[0] = m[0]; u3[1] = m[1]; u3[2] = m[2];
                                    sc = R(1);
                                }
                                const R u = R(I.rec.P1[k]) * (u3[0] * dx + u3[1] * dy + u3[2] * dz);
                                const R v = R(I.rec.P2[k]) * (u3[0] * p[0] + u3[1] * p[1] + u3[2] * p[2]);
                                const R br = u * p[2] + v * gam * dz;
                                const R bi = -u * gam * dz + v * p[2] + R(I.rec.P3[k]) * u3[2];
                                ar = sc * mag * br;
                                ai = sc * mag * bi;
                            }
                            Rk.x += ar * cs - ai * sn;
                            Rk.y += ar * sn + ai * cs;
                        }
                    }
                }
                }
                if (Rk.x != R(0) || Rk.y != R(0)) {
                    R sn, cs;
                    if constexpr (MIXED) {
                        // two-float reduction of S modulo 2 pi (Cody-Waite split)
                        const float k = rintf(S * 0.15915494309189535f);
                        float r = fmaf(-k, 6.28318548202514648f, S);
                        r = fmaf(-k, -1.7484555314695172e-07f, r);
                        r += Sl;
                        __sincosf(r, &sn, &cs);
                    } else {
                        sincos(S, &sn, &cs);
                    }
                    const C2<R> eS = {cs, sn};
                    const C2<R> a = cm(cm(C2<R>{wR, wI}, Cp), eS);
                    const C2<R> b = cm(a, ph);
                    x = b.x * Rk.x - b.y * Rk.y;
                    if (Mhat > stab) x *= taper_weight<R>(Mhat, stab, R(I.inv_log_taper));
                }
            }
            // ---- this step's contribution, summed over the warp after the chunk
            red[s * kRedStride + lane] = x;
            contributed |= (x != R(0));
            // ---- one RK4 step to t_{nn+1}
            if (live && status == 0 && nn < nt - 1) {
                ++steps;
                stage_eval<R, MIXED, POLY, NC, PK>(K, q, ql, p, E1, E2, E4, h, h2, h6, Hs, dq, dp, dS,
                                           &I.tgt, tab);
                if constexpr (MIXED) {
                    acc2x2(q[0], q[1], ql[0], ql[1], dq[0], dq[1]);
                    acc2x2(p[0], p[1], pl[0], pl[1], dp[0], dp[1]);
                    acc2x2(q[2], p[2], ql[2], pl[2], dq[2], dp[2]);
                } else {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        q[a] += dq[a];
                        p[a] += dp[a];
                    }
                }
                if constexpr (MIXED) {
                    acc2(S, Sl, dS);
                } else {
                    S += dS;
                }
                m_update(M, Hs, h, h2, h6, hh4, hh2, hh6);
            }
        }
        // lane l sums row l (step nb + l) over the 32 trajectories: two-float
        // in MIXED; rows are 33 apart so that both the writes above and these
        // reads hit 32 different banks
        __syncwarp();
        // the recombination evaluations of the chunk are its nonzero
        // contributions, counted here so that no counter stays live in the
        // step loop
        const bool any = __any_sync(kFull, contributed);
        unsigned int n_nz = 0;
        if (any && lane < send) {
            const R* row = red + lane * kRedStride;
            if constexpr (MIXED) {
                float sv = 0.0f, ev = 0.0f;
#pragma unroll 8
                for (int k = 0; k < kWarp; ++k) {
                    float t;
                    two_sum(sv, row[k], sv, t);
                    ev += t;
                    n_nz += row[k] != 0.0f;
                }
                if (sv != 0.0f || ev != 0.0f)
                    atomicAdd(&I.vz[nb + lane], I.scale * (double(sv) + double(ev)));
            } else {
                double sv = 0.0;
#pragma unroll 8
                for (int k = 0; k < kWarp; ++k) {
                    sv += row[k];
                    n_nz += row[k] != 0.0;
                }
                if (sv != 0.0) atomicAdd(&I.vz[nb + lane], I.scale * sv);
            }
        }
        if (any) {
            const unsigned int tot = __reduce_add_sync(kFull, n_nz);
            if (lane == 0 && tot) atomicAdd(&I.counters[5], (unsigned long long)tot);
        }
        __syncwarp();
        if (!__any_sync(kFull, has && status == 0)) break;
        if constexpr (PARK) {
            // time is up and chunks are left: park the item for the next slice
            if (deadline != 0 && nb + kWarp < nt) {
                unsigned long long now = 0;
                if (lane == 0) now = global_ns();
                now = __shfl_sync(kFull, now, 0);
                if (now >= deadline) {
                    unsigned int slot = 0;
                    if (lane == 0) slot = atomicAdd(pk->out_ctr, 1u);
                    slot = __shfl_sync(kFull, slot, 0);
                    if (slot < (unsigned int)pk->cap) {
                        R* col = (R*)pk->out_state + (size_t)slot * kParkWords * kWarp + lane;
                        park_io<R, true>(col, q, ql, p, pl, M, S, Sl, Cp, Mhat, status, n_ret,
                                         left, e_ret, steps);
                        if (lane == 0) {
                            ParkHdr hd;
                            hd.W = W;
                            hd.nb = nb + kWarp;
                            hd.pad[0] = hd.pad[1] = hd.pad[2] = 0;
                            pk->out_hdr[slot] = hd;
                            // remaining work in the host's units (Nt per item):
                            // the remaining fraction of the item's steps
                            const long long left_steps = nt - (nb + kWarp);
                            const long long all_steps = max(1, nt - W.n_start);
                            atomicAdd(pk->out_work,
                                      (unsigned long long)((long long)nt * left_steps / all_steps));
                        }
                        return false;
                    }
                }
            }
        }
    }

    // ---- counters and optional final state
    const unsigned filt = __ballot_sync(kFull, has && status == 1);
    const unsigned nonf = __ballot_sync(kFull, has && status == 2);
    const unsigned unst = __ballot_sync(kFull, has && status == 3);
    unsigned long long st = steps;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) st += __shfl_xor_sync(kFull, st, off);
    if (lane == 0) {
        if (filt) atomicAdd(&I.counters[0], (unsigned long long)__popc(filt));
        if (nonf) atomicAdd(&I.counters[1], (unsigned long long)__popc(nonf));
        if (unst) atomicAdd(&I.counters[4], (unsigned long long)__popc(unst));
        atomicAdd(&I.counters[2], st);
    }
    if (ret != nullptr && has) {
        ret[j] = double(n_ret);
        ret[n + j] = double(e_ret);
    }
    if (I.dump != nullptr && has) {
        double* d = I.dump;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[(size_t)a * n + j] = double(q[a]) + double(ql[a]) * (MIXED ? 1.0 : 0.0);
            d[(size_t)(3 + a) * n + j] = double(p[a]) + double(pl[a]) * (MIXED ? 1.0 : 0.0);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                d[(size_t)(6 + 6 * r + c) * n + j] = double(M.Q(c, r));
                d[(size_t)(6 + 6 * (r + 3) + c) * n + j] = double(M.P(c, r));
            }
        d[(size_t)42 * n + j] = double(S) + (MIXED ? double(Sl) : 0.0);
        d[(size_t)43 * n + j] = double(Cp.x);
        d[(size_t)44 * n + j] = double(Cp.y);
        d[(size_t)45 * n + j] = double(n0 + (long long)steps);   // time index of this state
        d[(size_t)46 * n + j] = double(status);
    }
    return true;
}

// The persistent loop over the work-item queue.  POLY: after the blocks'
// reduction buffers, every warp has a table of `slots` rows x kTabWords x 32
// words (this lane's column starts kTabWords words per lane in for FP32
// float4 rows, one word for the FP64 rows).
template <bool MIXED, bool POLY = false, int NC = 0, bool FIXED = false, int PK = kPotAny>
__device__ __forceinline__ void run_queue(const DevInstance* __restrict__ insts,
                                          const WorkItem* __restrict__ items, int n_items,
                                          unsigned int* __restrict__ counter, int slots = 0)
{
    using R = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* red = reinterpret_cast<R*>(smem_raw) + (threadIdx.x / kWarp) * kRedElems;
    const int lane = threadIdx.x & (kWarp - 1);
    R* tab = nullptr;
    if constexpr (POLY)
        tab = reinterpret_cast<R*>(smem_raw) + (blockDim.x / kWarp) * kRedElems +
              (threadIdx.x / kWarp) * (slots * kTabWords<R> * kWarp) +
              lane * (MIXED ? kTabWords<R> : 1);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const WorkItem W = items[it];
        process_item<MIXED, POLY, NC, FIXED, false, PK>(insts[W.inst], W, lane, red, tab);
    }
}


// Server slice of the same integrator: items come from a ring, warps stop
// taking new items once the slice's time is up, count finished items per
// instance, and skip the items of cancelled instances.  No thread waits on
// another: a warp only ever reads the clock and atomic counters.
// POLY: the ring holds polyatomic requests' items, and every warp has its
// centre table of `slots` rows after the reduction buffers (as run_queue).
// Parked items of the previous slice are resumed first, whatever the time
// (each then runs at least one chunk), then new items are taken until the
// deadline; an item is parked at the first chunk boundary past the deadline
// (process_item) and only an item that ran to its end counts as done.
template <bool MIXED, bool POLY = false, bool FIXED = false, int PK = kPotAny>
__device__ __forceinline__ void run_slice(const DevInstance* __restrict__ insts,
                                          const WorkItem* __restrict__ ring, unsigned int mask,
                                          unsigned int base, int n_items,
                                          unsigned int* __restrict__ counter,
                                          unsigned long long slice_ns,
                                          unsigned long long* __restrict__ t0,
                                          const ParkBufs* pk, int slots = 0)
{
    using R = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* red = reinterpret_cast<R*>(smem_raw) + (threadIdx.x / kWarp) * kRedElems;
    const int lane = threadIdx.x & (kWarp - 1);
    R* tab = nullptr;
    if constexpr (POLY)
        tab = reinterpret_cast<R*>(smem_raw) + (blockDim.x / kWarp) * kRedElems +
              (threadIdx.x / kWarp) * (slots * kTabWords<R> * kWarp) +
              lane * (MIXED ? kTabWords<R> : 1);
    unsigned long long deadline = 0;
    if (lane == 0 && slice_ns) {
        const unsigned long long now = global_ns();
        const unsigned long long prev = atomicCAS(t0, 0ull, now);
        deadline = (prev == 0ull ? now : prev) + slice_ns;
    }
    deadline = __shfl_sync(kFull, deadline, 0);
    for (;;) {
        int it = n_items, r = -1;
        if (lane == 0) {
            if (pk->n_in > 0) {
                const unsigned int k = atomicAdd(pk->in_ctr, 1u);
                if (k < (unsigned int)pk->n_in) r = (int)k;
            }
            if (r < 0 && (slice_ns == 0 || global_ns() < deadline))
                it = (int)atomicAdd(counter, 1u);
        }
        r = __shfl_sync(kFull, r, 0);
        it = __shfl_sync(kFull, it, 0);
        if (r < 0 && it >= n_items) break;
        const WorkItem W = r >= 0 ? pk->in_hdr[r].W : ring[(base + (unsigned int)it) & mask];
        const DevInstance& I = insts[W.inst];
        bool done = true;
        if (I.cancel == nullptr || *I.cancel == 0)
            done = process_item<MIXED, POLY, 0, FIXED, true, PK>(I, W, lane, red, tab, pk, r,
                                                             slice_ns ? deadline : 0ull);
        if (done && lane == 0 && I.done_items != nullptr) atomicAdd(I.done_items, 1u);
    }
}

// Register-cap variants of both kernels: no cap, or at most MAXREG registers
// per thread (more resident warps, possibly spills); the autotuner picks.
template <bool MIXED>
__global__ void __launch_bounds__(128)
    k_propagate_nocap(const DevInstance* __restrict__ insts, const WorkItem* __restrict__ items,
                      int n_items, unsigned int* __restrict__ counter)
{
    run_queue<MIXED>(insts, items, n_items, counter);
}
template <bool MIXED, int MAXREG>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate(const DevInstance* __restrict__ insts, const WorkItem* __restrict__ items,
                int n_items, unsigned int* __restrict__ counter)
{
    run_queue<MIXED>(insts, items, n_items, counter);
}
// The mixed-precision diatomic integrator with FixedParams' values compiled
// in, for the molecular two-centre potential (PK: the screening known for
// the whole launch, kPotBare or kPotScreened, or decided per instance,
// kPotMolecule), with the same register-cap variants
template <int PK>
__global__ void __launch_bounds__(128)
    k_propagate_fixed_nocap(const DevInstance* __restrict__ insts,
                            const WorkItem* __restrict__ items, int n_items,
                            unsigned int* __restrict__ counter)
{
    run_queue<true, false, 0, true, PK>(insts, items, n_items, counter);
}
template <int MAXREG, int PK>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_fixed(const DevInstance* __restrict__ insts, const WorkItem* __restrict__ items,
                      int n_items, unsigned int* __restrict__ counter)
{
    run_queue<true, false, 0, true, PK>(insts, items, n_items, counter);
}
// the three-centre polyatomic integrator with FixedParams' values compiled in
__global__ void __launch_bounds__(128)
    k_propagate_poly_fixed_nocap(const DevInstance* __restrict__ insts,
                                 const WorkItem* __restrict__ items, int n_items,
                                 unsigned int* __restrict__ counter, int slots)
{
    run_queue<true, true, 3, true>(insts, items, n_items, counter, slots);
}
template <int MAXREG>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_poly_fixed(const DevInstance* __restrict__ insts,
                           const WorkItem* __restrict__ items, int n_items,
                           unsigned int* __restrict__ counter, int slots)
{
    run_queue<true, true, 3, true>(insts, items, n_items, counter, slots);
}
// Polyatomic targets, with the same register-cap variants; NC = 3: every
// target of the launch has three centres (loop over the centres unrolled),
// 0: any number.
template <bool MIXED, int NC>
__global__ void __launch_bounds__(128)
    k_propagate_poly_nocap(const DevInstance* __restrict__ insts,
                           const WorkItem* __restrict__ items, int n_items,
                           unsigned int* __restrict__ counter, int slots)
{
    run_queue<MIXED, true, NC>(insts, items, n_items, counter, slots);
}
template <bool MIXED, int MAXREG, int NC>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_poly(const DevInstance* __restrict__ insts, const WorkItem* __restrict__ items,
                     int n_items, unsigned int* __restrict__ counter, int slots)
{
    run_queue<MIXED, true, NC>(insts, items, n_items, counter, slots);
}
template <bool MIXED>
__global__ void __launch_bounds__(128)
    k_propagate_slice_nocap(const DevInstance* __restrict__ insts,
                            const WorkItem* __restrict__ ring, unsigned int mask,
                            unsigned int base, int n_items, unsigned int* __restrict__ counter,
                            unsigned long long slice_ns, unsigned long long* __restrict__ t0,
                            __grid_constant__ const ParkBufs pk)
{
    run_slice<MIXED>(insts, ring, mask, base, n_items, counter, slice_ns, t0, &pk);
}
template <bool MIXED, int MAXREG>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_slice(const DevInstance* __restrict__ insts, const WorkItem* __restrict__ ring,
                      unsigned int mask, unsigned int base, int n_items,
                      unsigned int* __restrict__ counter, unsigned long long slice_ns,
                      unsigned long long* __restrict__ t0, __grid_constant__ const ParkBufs pk)
{
    run_slice<MIXED>(insts, ring, mask, base, n_items, counter, slice_ns, t0, &pk);
}

// the mixed diatomic slice with FixedParams' values compiled in
__global__ void __launch_bounds__(128)
    k_propagate_slice_fixed_nocap(const DevInstance* __restrict__ insts,
                                  const WorkItem* __restrict__ ring, unsigned int mask,
                                  unsigned int base, int n_items,
                                  unsigned int* __restrict__ counter, unsigned long long slice_ns,
                                  unsigned long long* __restrict__ t0,
                                  __grid_constant__ const ParkBufs pk)
{
    run_slice<true, false, true, kPotMolecule>(insts, ring, mask, base, n_items, counter, slice_ns,
                                              t0, &pk);
}
template <int MAXREG>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_slice_fixed(const DevInstance* __restrict__ insts,
                            const WorkItem* __restrict__ ring, unsigned int mask,
                            unsigned int base, int n_items, unsigned int* __restrict__ counter,
                            unsigned long long slice_ns, unsigned long long* __restrict__ t0,
                            __grid_constant__ const ParkBufs pk)
{
    run_slice<true, false, true, kPotMolecule>(insts, ring, mask, base, n_items, counter, slice_ns,
                                              t0, &pk);
}

template <bool MIXED>
__global__ void __launch_bounds__(128)
    k_propagate_slice_poly_nocap(const DevInstance* __restrict__ insts,
                                 const WorkItem* __restrict__ ring, unsigned int mask,
                                 unsigned int base, int n_items,
                                 unsigned int* __restrict__ counter, unsigned long long slice_ns,
                                 unsigned long long* __restrict__ t0,
                                 __grid_constant__ const ParkBufs pk, int slots)
{
    run_slice<MIXED, true>(insts, ring, mask, base, n_items, counter, slice_ns, t0, &pk, slots);
}
template <bool MIXED, int MAXREG>
__global__ void __launch_bounds__(128) __maxnreg__(MAXREG)
    k_propagate_slice_poly(const DevInstance* __restrict__ insts,
                           const WorkItem* __restrict__ ring, unsigned int mask,
                           unsigned int base, int n_items, unsigned int* __restrict__ counter,
                           unsigned long long slice_ns, unsigned long long* __restrict__ t0,
                           __grid_constant__ const ParkBufs pk, int slots)
{
    run_slice<MIXED, true>(insts, ring, mask, base, n_items, counter, slice_ns, t0, &pk, slots);
}

using KernelFn = void (*)(const DevInstance*, const WorkItem*, int, unsigned int*);
using PolyFn = void (*)(const DevInstance*, const WorkItem*, int, unsigned int*, int);
using SliceFn = void (*)(const DevInstance*, const WorkItem*, unsigned int, unsigned int, int,
                         unsigned int*, unsigned long long, unsigned long long*, const ParkBufs);
using SlicePolyFn = void (*)(const DevInstance*, const WorkItem*, unsigned int, unsigned int,
                             int, unsigned int*, unsigned long long, unsigned long long*,
                             const ParkBufs, int);

// variants: index 0 = no register cap, then at most 168, 152, 144, 136, 128
// registers per thread (12 to 16 resident warps per SM)
constexpr int kVariantMaxReg[kPropVariants] = {0, 168, 152, 144, 136, 128};

template <int PK>
KernelFn fixed_variant_pk(int v)
{
    static const KernelFn fn[kPropVariants] = {
        k_propagate_fixed_nocap<PK>, k_propagate_fixed<168, PK>, k_propagate_fixed<152, PK>,
        k_propagate_fixed<144, PK>, k_propagate_fixed<136, PK>, k_propagate_fixed<128, PK>};
    return fn[v];
}

// pk: the launch's potential form (kPotBare, kPotScreened or kPotMolecule)
KernelFn fixed_variant(int v, int pk)
{
    return pk == kPotBare       ? fixed_variant_pk<kPotBare>(v)
           : pk == kPotScreened ? fixed_variant_pk<kPotScreened>(v)
                                : fixed_variant_pk<kPotMolecule>(v);
}

KernelFn variant(int precision, int v)
{
    static const KernelFn mixed[kPropVariants] = {
        k_propagate_nocap<true>, k_propagate<true, 168>, k_propagate<true, 152>,
        k_propagate<true, 144>, k_propagate<true, 136>, k_propagate<true, 128>};
    static const KernelFn fp64[kPropVariants] = {
        k_propagate_nocap<false>, k_propagate<false, 168>, k_propagate<false, 152>,
        k_propagate<false, 144>, k_propagate<false, 136>, k_propagate<false, 128>};
    return precision == SFHK_MIXED ? mixed[v] : fp64[v];
}

// centre counts with a specialised (unrolled) polyatomic kernel
constexpr int kPolyNC[2] = {0, 3};

template <int NC>
PolyFn poly_variant_nc(int precision, int v)
{
    static const PolyFn mixed[kPropVariants] = {
        k_propagate_poly_nocap<true, NC>, k_propagate_poly<true, 168, NC>,
        k_propagate_poly<true, 152, NC>, k_propagate_poly<true, 144, NC>,
        k_propagate_poly<true, 136, NC>, k_propagate_poly<true, 128, NC>};
    static const PolyFn fp64[kPropVariants] = {
        k_propagate_poly_nocap<false, NC>, k_propagate_poly<false, 168, NC>,
        k_propagate_poly<false, 152, NC>, k_propagate_poly<false, 144, NC>,
        k_propagate_poly<false, 136, NC>, k_propagate_poly<false, 128, NC>};
    return precision == SFHK_MIXED ? mixed[v] : fp64[v];
}

// nc: the common centre count of the launch's targets (0 when they differ);
// fixed: every instance has FixedParams' values (used for three centres in
// mixed precision)
PolyFn poly_variant(int precision, int v, int nc, bool fixed = false)
{
    static const PolyFn fixed3[kPropVariants] = {
        k_propagate_poly_fixed_nocap, k_propagate_poly_fixed<168>, k_propagate_poly_fixed<152>,
        k_propagate_poly_fixed<144>, k_propagate_poly_fixed<136>, k_propagate_poly_fixed<128>};
    if (fixed && nc == 3 && precision == SFHK_MIXED) return fixed3[v];
    return nc == 3 ? poly_variant_nc<3>(precision, v) : poly_variant_nc<0>(precision, v);
}

SliceFn slice_variant(int precision, int v, bool fixed = false)
{
    static const SliceFn fixed_fn[kPropVariants] = {
        k_propagate_slice_fixed_nocap, k_propagate_slice_fixed<168>,
        k_propagate_slice_fixed<152>, k_propagate_slice_fixed<144>,
        k_propagate_slice_fixed<136>, k_propagate_slice_fixed<128>};
    if (fixed && precision == SFHK_MIXED) return fixed_fn[v];
    static const SliceFn mixed[kPropVariants] = {
        k_propagate_slice_nocap<true>, k_propagate_slice<true, 168>,
        k_propagate_slice<true, 152>, k_propagate_slice<true, 144>,
        k_propagate_slice<true, 136>, k_propagate_slice<true, 128>};
    static const SliceFn fp64[kPropVariants] = {
        k_propagate_slice_nocap<false>, k_propagate_slice<false, 168>,
        k_propagate_slice<false, 152>, k_propagate_slice<false, 144>,
        k_propagate_slice<false, 136>, k_propagate_slice<false, 128>};
    return precision == SFHK_MIXED ? mixed[v] : fp64[v];
}

SlicePolyFn slice_poly_variant(int precision, int v)
{
    static const SlicePolyFn mixed[kPropVariants] = {
        k_propagate_slice_poly_nocap<true>, k_propagate_slice_poly<true, 168>,
        k_propagate_slice_poly<true, 152>, k_propagate_slice_poly<true, 144>,
        k_propagate_slice_poly<true, 136>, k_propagate_slice_poly<true, 128>};
    static const SlicePolyFn fp64[kPropVariants] = {
        k_propagate_slice_poly_nocap<false>, k_propagate_slice_poly<false, 168>,
        k_propagate_slice_poly<false, 152>, k_propagate_slice_poly<false, 144>,
        k_propagate_slice_poly<false, 136>, k_propagate_slice_poly<false, 128>};
    return precision == SFHK_MIXED ? mixed[v] : fp64[v];
}

// dynamic shared memory of a block: one contribution buffer per warp
size_t red_bytes(int precision, int block_threads)
{
    const size_t elem = precision == SFHK_MIXED ? sizeof(float) : sizeof(double);
    return size_t(block_threads / kWarp) * kRedElems * elem;
}

}  // namespace

int launch_propagate_slice(int precision, int variant_index, const DevInstance* insts,
                           const WorkItem* ring, unsigned int mask, unsigned int base,
                           int n_items, unsigned int* counter, unsigned long long slice_ns,
                           unsigned long long* t0, int block_threads, int sm_count,
                           cudaStream_t s, const ParkBufs& park, int poly_slots, bool fixed)
{
    if (block_threads <= 0 || block_threads > 128 || block_threads % kWarp) return SFHK_E_INVAL;
    if (variant_index < 0 || variant_index >= kPropVariants || n_items < 0 || park.n_in < 0 ||
        park.n_in > park.cap || n_items + (long long)park.n_in <= 0 || !park.in_ctr ||
        !park.out_ctr || !park.out_work || !park.out_hdr || !park.out_state ||
        (park.n_in > 0 && !park.in_state))
        return SFHK_E_INVAL;
    if (poly_slots < 0 || poly_slots > SFHK_MAX_CENTRES + SFHK_MAX_PRIM) return SFHK_E_INVAL;
    const bool poly = poly_slots > 0;
    const bool mixed = precision == SFHK_MIXED;
    const size_t elem = mixed ? sizeof(float) : sizeof(double);
    // the polyatomic slices also hold every warp's centre table
    const size_t smem = red_bytes(precision, block_threads) +
                        (poly ? size_t(block_threads / kWarp) * poly_slots * (mixed ? 4 : 3) *
                                    kWarp * elem
                              : 0);
    int occ = 0;
    if (poly)
        SFHK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, slice_poly_variant(precision, variant_index), block_threads, smem));
    else
        SFHK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, slice_variant(precision, variant_index, fixed), block_threads, smem));
    if (occ < 1) occ = 1;
    const int warps_per_block = block_threads / kWarp;
    int grid = sm_count * occ;
    const int grid_cap = (int)((n_items + (long long)park.n_in + warps_per_block - 1) /
                               warps_per_block);
    if (grid > grid_cap) grid = grid_cap;
    // every warp of the launch can park one item at once
    if ((long long)grid * warps_per_block > park.cap) return SFHK_E_INVAL;
    SFHK_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
    SFHK_CUDA_TRY(cudaMemsetAsync(t0, 0, sizeof(unsigned long long), s));
    SFHK_CUDA_TRY(cudaMemsetAsync(park.in_ctr, 0, sizeof(unsigned int), s));
    SFHK_CUDA_TRY(cudaMemsetAsync(park.out_ctr, 0, sizeof(unsigned int), s));
    SFHK_CUDA_TRY(cudaMemsetAsync(park.out_work, 0, sizeof(unsigned long long), s));
    count_launch();
    if (poly)
        slice_poly_variant(precision, variant_index)<<<grid, block_threads, smem, s>>>(
            insts, ring, mask, base, n_items, counter, slice_ns, t0, park, poly_slots);
    else
        slice_variant(precision, variant_index, fixed)<<<grid, block_threads, smem, s>>>(
            insts, ring, mask, base, n_items, counter, slice_ns, t0, park);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

int slice_max_warps(int precision, int variant_index, int block_threads, int sm_count)
{
    if (variant_index < 0 || variant_index >= kPropVariants || block_threads <= 0 ||
        block_threads > 128 || block_threads % kWarp)
        return 0;
    const size_t smem = red_bytes(precision, block_threads);
    int best = 0;
    // the smallest shared memory of each kernel (a polyatomic slice adds its
    // centre tables), so the largest occupancy
    const void* fns[3] = {(const void*)slice_variant(precision, variant_index, false),
                          (const void*)slice_variant(precision, variant_index, true),
                          (const void*)slice_poly_variant(precision, variant_index)};
    for (const void* fn : fns) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block_threads, smem) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        best = std::max(best, occ);
    }
    return sm_count * best * (block_threads / kWarp);
}

int propagate_variant_maxreg(int v) { return (v >= 0 && v < kPropVariants) ? kVariantMaxReg[v] : 0; }

// the kernel of a diatomic launch: the FixedParams instantiation of the
// launch's potential form when every instance has those values (fixed, a
// kPot* form; mixed precision only), else the generic one
static KernelFn diatomic_kernel(int precision, int v, int fixed)
{
    return fixed != kPotAny && precision == SFHK_MIXED ? fixed_variant(v, fixed)
                                                      : variant(precision, v);
}

int propagate_occupancy(int precision, int variant_index, int block_threads, int* blocks_per_sm,
                        int fixed)
{
    if (variant_index < 0 || variant_index >= kPropVariants) return SFHK_E_INVAL;
    if (block_threads <= 0 || block_threads > 128 || block_threads % kWarp) return SFHK_E_INVAL;
    SFHK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, diatomic_kernel(precision, variant_index, fixed), block_threads,
        red_bytes(precision, block_threads)));
    return SFHK_OK;
}

bool fixed_params(const DevInstance& I)
{
    using F = FixedParams;
    return I.tgt.kind != SFHK_POT_HARMONIC && I.returns == nullptr && I.dt == F::dt &&
           I.gamma == F::gamma &&
           I.inv_gamma == 1.0 / F::gamma && I.cutoff2 == F::cutoff * F::cutoff &&
           I.stab_cut == F::stab && I.stab_hi == F::taper * F::stab;
}

namespace {

// Polyatomic launch: the reduction buffers plus every warp's centre table.
int launch_poly(int precision, int variant_index, const DevInstance* insts,
                const WorkItem* items, int n_items, unsigned int* item_counter,
                int block_threads, int blocks_per_sm, int sm_count, int slots, int nc,
                bool fixed, cudaStream_t s)
{
    if (slots < 1 || slots > SFHK_MAX_CENTRES + SFHK_MAX_PRIM) return SFHK_E_INVAL;
    const bool mixed = precision == SFHK_MIXED;
    const PolyFn fn = poly_variant(precision, variant_index, nc, fixed);
    const size_t elem = mixed ? sizeof(float) : sizeof(double);
    const size_t smem = red_bytes(precision, block_threads) +
                        size_t(block_threads / kWarp) * slots * (mixed ? 4 : 3) * kWarp * elem;
    // above 48 KB the kernels rely on the limit raised by configure_kernels()
    int occ = 0;
    SFHK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block_threads, smem));
    if (occ < 1) occ = 1;
    const int bps = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
    const int warps_per_block = block_threads / kWarp;
    int grid = sm_count * bps;
    const int grid_cap = (n_items + warps_per_block - 1) / warps_per_block;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    SFHK_CUDA_TRY(cudaMemsetAsync(item_counter, 0, sizeof(unsigned int), s));
    count_launch();
    fn<<<grid, block_threads, smem, s>>>(insts, items, n_items, item_counter, slots);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

}  // namespace

// Raise the dynamic shared-memory limit of the polyatomic kernels to their
// largest launch (128 threads, SFHK_MAX_CENTRES + SFHK_MAX_PRIM table rows),
// once per device at context creation, so that no launch (in a captured
// graph either) changes a function attribute.
int configure_kernels()
{
    for (int prec = 0; prec < 2; ++prec) {
        const size_t elem = prec == SFHK_MIXED ? sizeof(float) : sizeof(double);
        const size_t smem = red_bytes(prec, 128) + size_t(128 / kWarp) *
                                                       (SFHK_MAX_CENTRES + SFHK_MAX_PRIM) *
                                                       (prec == SFHK_MIXED ? 4 : 3) * kWarp * elem;
        for (int v = 0; v < kPropVariants; ++v) {
            for (int nc : kPolyNC)
                for (bool fixed : {false, true})
                    SFHK_CUDA_TRY(cudaFuncSetAttribute(poly_variant(prec, v, nc, fixed),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)smem));
            SFHK_CUDA_TRY(cudaFuncSetAttribute(slice_poly_variant(prec, v),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
        }
    }
    return SFHK_OK;
}

int launch_propagate(int precision, int variant_index, const DevInstance* insts,
                     const WorkItem* items, int n_items, unsigned int* item_counter,
                     int block_threads, int blocks_per_sm, int sm_count, cudaStream_t s,
                     int poly_slots, int poly_nc, int fixed)
{
    if (block_threads <= 0 || block_threads > 128 || block_threads % kWarp) return SFHK_E_INVAL;
    if (variant_index < 0 || variant_index >= kPropVariants) return SFHK_E_INVAL;
    if (poly_slots > 0)
        return launch_poly(precision, variant_index, insts, items, n_items, item_counter,
                           block_threads, blocks_per_sm, sm_count, poly_slots, poly_nc,
                           fixed != kPotAny, s);
    int occ = 0;
    int rc = propagate_occupancy(precision, variant_index, block_threads, &occ, fixed);
    if (rc) return rc;
    if (occ < 1) occ = 1;
    const int bps = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
    const int warps_per_block = block_threads / kWarp;
    int grid = sm_count * bps;
    const int grid_cap = (n_items + warps_per_block - 1) / warps_per_block;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    SFHK_CUDA_TRY(cudaMemsetAsync(item_counter, 0, sizeof(unsigned int), s));
    count_launch();
    diatomic_kernel(precision, variant_index, fixed)<<<grid, block_threads,
                                                       red_bytes(precision, block_threads), s>>>(
        insts, items, n_items, item_counter);
    SFHK_CUDA_TRY(cudaGetLastError());
    return SFHK_OK;
}

}  // namespace sfhk

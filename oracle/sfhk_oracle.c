/*
 * sfhk_oracle.c -- plain, slow, FP64 CPU oracle for the strong-field
 * Herman-Kluk (SFHK) high-harmonic path of "Strong-field Herman-Kluk
 * propagator method for high-harmonic generation in molecules"
 * (Tran, Truong, Goetz, Le).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links
 * or calls this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * Every routine follows the paper's statement of the method step by step,
 * in the paper's order and notation, in double precision, with no blocking,
 * fusion or reordering:
 *   - ionization step: saddle-point equation (Eq. 2), tunnel exit and
 *     tunnelling action (Sec. II.A, text after Eq. 2), ionization amplitude
 *     (second line of Eq. 1) with the initial orbital expanded in Gaussians
 *     (Sec. II.A, GTO paragraph);
 *   - continuum propagation: Hamilton's equations in the model potential of
 *     Eq. 7 plus the laser (length gauge), stability matrix, continuum action
 *     S = int (p.qdot - H) dt, Herman-Kluk prefactor (Sec. II.A);
 *   - recombination and dipole velocity (Eq. 4, and the approximation of
 *     v_z(t) before Eq. 1);
 *   - orientation sampled per trajectory (Eq. 6);
 *   - Hann-windowed Fourier transform and yield omega^2 |v(omega)|^2 (Eq. 3).
 * Where the paper is silent the reading is stated at the routine.
 *
 * Parity pinning: every function here is checked in tests/ against values
 * fixed by the mathematics (finite differences, closed forms, symplecticity,
 * energy balance, quadrature, exact Herman-Kluk results for quadratic
 * Hamiltonians).  Agreement with the paper's plotted spectra is
 * "parity unpinned": the figures are not printed, the fitted GTO coefficients
 * are not given and there is no TDSE data.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off -o liboracle.so
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Inputs (plain C structs; the Python side fills them with ctypes).    */
/* ------------------------------------------------------------------ */
typedef struct {
    double lambda_nm;   /* carrier wavelength                          */
    double intensity;   /* peak intensity, W/cm^2                      */
    double n_cycles;    /* sin^2 envelope: total duration in cycles    */
    double cep;         /* carrier-envelope phase (rad)                */
    double dt;          /* time step (a.u.)                            */
    double t_center;    /* time of the pulse centre (0: the centred     */
                        /* axis of the reading below); every time of    */
                        /* the method moves with it                     */
} or_pulse_in;

enum { OR_POT_MOLECULE = 0, OR_POT_HARMONIC = 1, OR_POT_POLY = 2 };
#define OR_MAX_CENTRES 8

typedef struct {
    int kind;           /* OR_POT_MOLECULE (Eq. 7) or OR_POT_HARMONIC (test) */
    int n_prim;         /* s-type Gaussian primitives per centre          */
    double R;           /* internuclear distance                          */
    double Zinf, Z0;    /* asymptotic and near-nucleus charges (Eq. 7)    */
    double alpha;       /* screening exponent (Eq. 7)                     */
    double soft_a;      /* softening length a: |r-R_i| -> sqrt(d^2+a^2)   */
    double Ip;          /* ionization potential                           */
    double ho_omega;    /* harmonic test potential V = w^2 r^2 / 2        */
    double pexp[8];     /* primitive exponents                            */
    double pcoef[8];    /* primitive coefficients (un-normalised)         */
    int ionization;     /* 0: SFA saddle (Eq. 2); 1: modified saddle      */
                        /* with -eta E(t_s).r0 (SFHK2, Sec. III.D)        */
    int sampling;       /* 0: proposal with weights a/pdf; 1: initial    */
                        /* points distributed ~ |a| (Sec. II.B)           */
    double sampling_factor; /* kappa of the |a| sampler (<= 0: 5)         */
    int pkind[8];       /* primitive k: 0 s-type e^{-a|x-A|^2}; 1 sigma    */
                        /* p-type s_c n.(x-A) e^{-a|x-A|^2}, s_c = +-1 for */
                        /* the centre at +-(R/2) n (gerade combination);  */
                        /* 2 pi p-type m.(x-A) e^{-a|x-A|^2} on both      */
                        /* centres with the same sign (1 pi_u, ungerade), */
                        /* m the unit vector perpendicular to n at        */
                        /* azimuth pi_azimuth (see pi_direction)          */
    double pi_azimuth;  /* chi: m = cos(chi) theta_hat + sin(chi) phi_hat */
    /* OR_POT_POLY: N centres at molecular-frame positions cpos, each    */
    /* with its own Eq. 7 charges; primitive k sits on centre pcentre[k] */
    /* only (kind 0 s-type, kind 3 p-type (u.(x-A)) e^{-a|x-A|^2} with u */
    /* the molecular-frame direction pdir[k] normalised, rotated with    */
    /* the molecule).  The orientation of a trajectory is then the ZYZ   */
    /* Euler triple (phi, theta, psi) in place of the axis n.            */
    int n_centres;
    double cpos[OR_MAX_CENTRES][3];
    double cZinf[OR_MAX_CENTRES], cZ0[OR_MAX_CENTRES], calpha[OR_MAX_CENTRES];
    int pcentre[8];
    double pdir[8][3];
    double proposal_mix;    /* eps in [0, 1): defensive share of the time   */
                            /* proposal, uniform over the grid              */
    double proposal_floor;  /* f in [0, 1]: the k_perp width is at least    */
                            /* sigma(f E0), the width for a field f E0      */
    double origin[3];       /* lab position of the molecule: every centre   */
                            /* and primitive moved by it, the tunnel exit   */
                            /* measured from it (0: the molecule at the     */
                            /* origin, as the paper places it)              */
} or_target_in;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, from its published            */
/* definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as */
/* easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with */
/* a Weyl-sequence key schedule.                                        */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two 32-bit words -> one uniform double in (0,1) with 53 random bits:
 * u = ((a >> 5) * 2^26 + (b >> 6) + 1/2) * 2^-53.                       */
static double or_u01(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5), lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0);
}

/* The uniforms of trajectory j of instance `instance`: counter
 * (j mod 2^32, j div 2^32, instance, draw), key (seed mod 2^32, seed div 2^32).
 * draw 0 -> (u_time, u_bm1), draw 1 -> (u_bm2, u_al1), draw 2 -> (u_al2, -). */
static void uniforms_at(uint64_t seed, uint32_t instance, uint64_t j, uint32_t d0, double u[6])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t d = 0; d < 3; ++d) {
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), instance, d0 + d};
        uint32_t r[4];
        or_philox4x32_10(ctr, key, r);
        u[2 * d] = or_u01(r[0], r[1]);
        u[2 * d + 1] = or_u01(r[2], r[3]);
    }
}

void or_uniforms(uint64_t seed, uint32_t instance, uint64_t j, double u[6])
{
    uniforms_at(seed, instance, j, 0u, u);
}

/* ------------------------------------------------------------------ */
/* Pulse.  The paper gives wavelength, intensity, cycles of a sin^2      */
/* envelope and CEP (Sec. II.D / III.A); the formulas are the reading:   */
/*   omega = 45.5633525 / lambda[nm],  E0 = sqrt(I / 3.50944758e16),     */
/*   Tp = N_c 2 pi / omega, time centred on the pulse, t in [-Tp/2,Tp/2],*/
/*   A(t) = -(E0/omega) cos^2(pi t/Tp) sin(omega t + cep), E = -dA/dt,   */
/*   linear polarisation along z.                                        */
/* Time grid t_n = -Tp/2 + n dt, n = 0..Nt-1, Nt = floor(Tp/dt) + 1.      */
/* A pulse centred at t_c instead (t_center; a test of the time-origin    */
/* invariance of the dipole) is A(t - t_c), E(t - t_c) on the grid         */
/* t_n = t_c - Tp/2 + n dt.                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    double omega, E0, Tp, cep, dt, t_origin, tc;
    int nt;
} or_pulse;

void or_pulse_derive(const or_pulse_in* in, double out[6], int* nt)
{
    double omega = 45.5633525 / in->lambda_nm;
    double E0 = sqrt(in->intensity / 3.50944758e16);
    double Tp = in->n_cycles * 2.0 * OR_PI / omega;
    out[0] = omega; out[1] = E0; out[2] = Tp; out[3] = in->cep; out[4] = in->dt;
    out[5] = in->t_center - 0.5 * Tp;
    *nt = (int)floor(Tp / in->dt * (1.0 + 1e-12)) + 1;
}

static or_pulse or_make_pulse(const or_pulse_in* in)
{
    double d[6]; int nt;
    or_pulse_derive(in, d, &nt);
    or_pulse P = {d[0], d[1], d[2], d[3], d[4], d[5], in->t_center, nt};
    return P;
}

/* A(tau) and E(tau) for complex tau, straight from the definition above.  */
static cplx pulse_A(const or_pulse* P, cplx tau)
{
    tau -= P->tc;
    cplx c = ccos(OR_PI * tau / P->Tp);
    return -(P->E0 / P->omega) * c * c * csin(P->omega * tau + P->cep);
}

static cplx pulse_E(const or_pulse* P, cplx tau)
{
    /* E = -dA/dtau, differentiated by hand:
     * dA/dtau = -(E0/w)[ -(pi/Tp) sin(2 pi tau/Tp) sin(w tau+cep)
     *                    + w cos^2(pi tau/Tp) cos(w tau+cep) ]              */
    tau -= P->tc;
    cplx c = ccos(OR_PI * tau / P->Tp);
    cplx s2 = csin(2.0 * OR_PI * tau / P->Tp);
    cplx ph = P->omega * tau + P->cep;
    return P->E0 * c * c * ccos(ph) - (P->E0 * OR_PI / (P->omega * P->Tp)) * s2 * csin(ph);
}

/* dE/dtau, differentiated by hand from pulse_E:
 *   -E0 w cos^2(pi tau/Tp) sin(ph) - 2 E0 (pi/Tp) sin(2 pi tau/Tp) cos(ph)
 *   - (2 pi^2 E0 / (w Tp^2)) cos(2 pi tau/Tp) sin(ph),  ph = w tau + cep.   */
static cplx pulse_Edot(const or_pulse* P, cplx tau)
{
    tau -= P->tc;
    cplx c = ccos(OR_PI * tau / P->Tp);
    cplx s2 = csin(2.0 * OR_PI * tau / P->Tp);
    cplx c2 = ccos(2.0 * OR_PI * tau / P->Tp);
    cplx ph = P->omega * tau + P->cep;
    return -P->E0 * P->omega * c * c * csin(ph) - 2.0 * P->E0 * (OR_PI / P->Tp) * s2 * ccos(ph)
           - (2.0 * OR_PI * OR_PI * P->E0 / (P->omega * P->Tp * P->Tp)) * c2 * csin(ph);
}

void or_pulse_Edot_complex(const or_pulse_in* in, double tr, double ti, double out[2])
{
    or_pulse P = or_make_pulse(in);
    cplx e = pulse_Edot(&P, tr + I * ti);
    out[0] = creal(e); out[1] = cimag(e);
}

double or_pulse_A_real(const or_pulse_in* in, double t)
{
    or_pulse P = or_make_pulse(in);
    if (fabs(t - P.tc) > 0.5 * P.Tp) return 0.0;
    return creal(pulse_A(&P, t));
}

double or_pulse_E_real(const or_pulse_in* in, double t)
{
    or_pulse P = or_make_pulse(in);
    if (fabs(t - P.tc) > 0.5 * P.Tp) return 0.0;
    return creal(pulse_E(&P, t));
}

void or_pulse_E_complex(const or_pulse_in* in, double tr, double ti, double out[2])
{
    or_pulse P = or_make_pulse(in);
    cplx e = pulse_E(&P, tr + I * ti);
    out[0] = creal(e); out[1] = cimag(e);
}

void or_pulse_A_complex(const or_pulse_in* in, double tr, double ti, double out[2])
{
    or_pulse P = or_make_pulse(in);
    cplx a = pulse_A(&P, tr + I * ti);
    out[0] = creal(a); out[1] = cimag(a);
}

static double pulse_E_real(const or_pulse* P, double t)
{
    if (fabs(t - P->tc) > 0.5 * P->Tp) return 0.0;
    return creal(pulse_E(P, t));
}

/* ------------------------------------------------------------------ */
/* Orientation of the molecule in the lab frame.  Diatomic targets: the  */
/* axis n, centres R_{1,2} = +-(R/2) n.  Polyatomic targets: the ZYZ     */
/* Euler angles (phi, theta, psi), rotation Rot = Rz(phi) Ry(theta)       */
/* Rz(psi), centres R_i = Rot x_i for the molecular-frame positions x_i; */
/* the molecular z axis goes to n = Rot z = (sin th cos ph, sin th sin ph, */
/* cos th), as for a diatomic.                                           */
/* ------------------------------------------------------------------ */
void or_euler_rotation(double ph, double th, double ps, double Rot[9])
{
    double Rz1[9] = {cos(ph), -sin(ph), 0.0, sin(ph), cos(ph), 0.0, 0.0, 0.0, 1.0};
    double Ry[9] = {cos(th), 0.0, sin(th), 0.0, 1.0, 0.0, -sin(th), 0.0, cos(th)};
    double Rz2[9] = {cos(ps), -sin(ps), 0.0, sin(ps), cos(ps), 0.0, 0.0, 0.0, 1.0};
    double T1[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T1[3 * i + j] = 0.0;
            for (int k = 0; k < 3; ++k) T1[3 * i + j] += Rz1[3 * i + k] * Ry[3 * k + j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Rot[3 * i + j] = 0.0;
            for (int k = 0; k < 3; ++k) Rot[3 * i + j] += T1[3 * i + k] * Rz2[3 * k + j];
        }
}

typedef struct {
    int nc;                          /* centres */
    double C[OR_MAX_CENTRES][3];     /* lab positions */
    double Zinf[OR_MAX_CENTRES], dZ[OR_MAX_CENTRES], alpha[OR_MAX_CENTRES];
    double nhat[3];                  /* molecular axis (diatomic) */
    double Rot[9];                   /* molecule -> lab (polyatomic) */
} or_frame;

/* orient: the axis n (diatomic) or the Euler angles (polyatomic) */
static void make_frame(const or_target_in* T, const double orient[3], or_frame* F)
{
    if (T->kind == OR_POT_POLY) {
        or_euler_rotation(orient[0], orient[1], orient[2], F->Rot);
        F->nc = T->n_centres;
        for (int i = 0; i < F->nc; ++i) {
            for (int a = 0; a < 3; ++a) {
                F->C[i][a] = 0.0;
                for (int b = 0; b < 3; ++b) F->C[i][a] += F->Rot[3 * a + b] * T->cpos[i][b];
            }
            F->Zinf[i] = T->cZinf[i];
            F->dZ[i] = T->cZ0[i] - T->cZinf[i];
            F->alpha[i] = T->calpha[i];
        }
        for (int a = 0; a < 3; ++a) F->nhat[a] = F->Rot[3 * a + 2];
        for (int i = 0; i < F->nc; ++i)
            for (int a = 0; a < 3; ++a) F->C[i][a] += T->origin[a];
        return;
    }
    F->nc = 2;
    for (int i = 0; i < 2; ++i) {
        double sign = (i == 0) ? 1.0 : -1.0;
        for (int a = 0; a < 3; ++a) F->C[i][a] = sign * 0.5 * T->R * orient[a] + T->origin[a];
        F->Zinf[i] = T->Zinf;
        F->dZ[i] = T->Z0 - T->Zinf;
        F->alpha[i] = T->alpha;
    }
    for (int a = 0; a < 3; ++a) F->nhat[a] = orient[a];
    for (int a = 0; a < 9; ++a) F->Rot[a] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Model potential, Eq. 7, for one electron in the field of the centres  */
/* R_i of the frame:                                                     */
/*   V(r) = - sum_i [Zinf_i + (Z0_i - Zinf_i) exp(-alpha_i s_i)] / s_i,  */
/* with the softening reading s_i = sqrt(|r - R_i|^2 + a^2).  Two        */
/* centres R_{1,2} = +-(R/2) n with common charges for a diatomic (the   */
/* paper's form); any number, each with its own charges, for the         */
/* polyatomic generalisation.                                            */
/* Gradient and Hessian are the analytic derivatives, written out:       */
/*   with f(s) = -(Zinf + dZ e^{-alpha s})/s,                            */
/*   f'(s)  = Zinf/s^2 + dZ e^{-alpha s}(alpha/s + 1/s^2),                */
/*   f''(s) = -2 Zinf/s^3 - dZ e^{-alpha s}(alpha^2/s + 2 alpha/s^2 + 2/s^3),*/
/*   grad V = f'(s) d/s,  Hess V = (f'/s) I + (f'' - f'/s) d d^T / s^2.   */
/* The harmonic test potential V = omega^2 |r|^2 / 2 has closed-form     */
/* classical and quantum solutions and pins the propagation.             */
/* ------------------------------------------------------------------ */
static void potential(const or_target_in* T, const double orient[3], const double q[3],
                      double* V, double grad[3], double hess[9])
{
    *V = 0.0;
    for (int a = 0; a < 3; ++a) grad[a] = 0.0;
    for (int a = 0; a < 9; ++a) hess[a] = 0.0;
    if (T->kind == OR_POT_HARMONIC) {
        double w2 = T->ho_omega * T->ho_omega;
        for (int a = 0; a < 3; ++a) {
            *V += 0.5 * w2 * q[a] * q[a];
            grad[a] = w2 * q[a];
            hess[4 * a] = w2;
        }
        return;
    }
    or_frame F;
    make_frame(T, orient, &F);
    for (int i = 0; i < F.nc; ++i) {
        double d[3], d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = q[a] - F.C[i][a];
            d2 += d[a] * d[a];
        }
        double Zinf = F.Zinf[i], dZ = F.dZ[i], alpha = F.alpha[i];
        double s = sqrt(d2 + T->soft_a * T->soft_a);
        double e = exp(-alpha * s);
        double f = -(Zinf + dZ * e) / s;
        double f1 = Zinf / (s * s) + dZ * e * (alpha / s + 1.0 / (s * s));
        double f2 = -2.0 * Zinf / (s * s * s)
                    - dZ * e * (alpha * alpha / s + 2.0 * alpha / (s * s) + 2.0 / (s * s * s));
        *V += f;
        for (int a = 0; a < 3; ++a) grad[a] += f1 * d[a] / s;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                hess[3 * a + b] += (a == b ? f1 / s : 0.0) + (f2 - f1 / s) * d[a] * d[b] / (s * s);
    }
}

void or_potential(const or_target_in* T, const double nhat[3], const double q[3],
                  double out[13])
{
    potential(T, nhat, q, &out[0], &out[1], &out[4]);
}

/* ------------------------------------------------------------------ */
/* Hamilton's equations (length gauge, electron charge -1, field along z)*/
/*   H = p^2/2 + V(q) + E(t) q_z,                                        */
/*   dq/dt = p,  dp/dt = -grad V - E(t) z^,                              */
/* the stability matrix M = d(q_t,p_t)/d(q_0,p_0) (6x6, row-major,       */
/* M(0) = identity):  dM_q./dt = M_p.,  dM_p./dt = -Hess V(q) M_q.,       */
/* and the continuum action S = int (p.qdot - H) dt:                     */
/*   dS/dt = p^2/2 - V(q) - E(t) q_z.                                    */
/* State layout y[43] = (q[3], p[3], M[36], S).                          */
/* ------------------------------------------------------------------ */
#define OR_NY 43

static void derivs(const or_target_in* T, const double nhat[3], double Ez,
                   const double* y, double* dy)
{
    double V, g[3], h[9];
    potential(T, nhat, y, &V, g, h);
    const double* p = y + 3;
    const double* M = y + 6;
    double* dM = dy + 6;
    for (int a = 0; a < 3; ++a) dy[a] = p[a];
    for (int a = 0; a < 3; ++a) dy[3 + a] = -g[a];
    dy[5] -= Ez;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c)
            dM[6 * r + c] = M[6 * (r + 3) + c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += h[3 * r + k] * M[6 * k + c];
            dM[6 * (r + 3) + c] = -acc;
        }
    double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    dy[42] = 0.5 * p2 - V - Ez * y[2];
}

/* Classical fourth-order Runge-Kutta step of the whole state from t to  */
/* t+h; the field is evaluated at t, t+h/2 and t+h.                      */
static void rk4_step(const or_target_in* T, const or_pulse* P, const double nhat[3],
                     double t, double h, double* y)
{
    double k1[OR_NY], k2[OR_NY], k3[OR_NY], k4[OR_NY], tmp[OR_NY];
    derivs(T, nhat, pulse_E_real(P, t), y, k1);
    for (int i = 0; i < OR_NY; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
    derivs(T, nhat, pulse_E_real(P, t + 0.5 * h), tmp, k2);
    for (int i = 0; i < OR_NY; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
    derivs(T, nhat, pulse_E_real(P, t + 0.5 * h), tmp, k3);
    for (int i = 0; i < OR_NY; ++i) tmp[i] = y[i] + h * k3[i];
    derivs(T, nhat, pulse_E_real(P, t + h), tmp, k4);
    for (int i = 0; i < OR_NY; ++i)
        y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Propagate one trajectory from grid point n0 over n_steps steps of +-dt
 * (dt may be negative for time reversal) and record the state after each
 * step: out[(k) * 43 + i], k = 0..n_steps (k = 0 is the start).          */
void or_trajectory(const or_target_in* T, const or_pulse_in* Pin, const double nhat[3],
                   const double y0[OR_NY], double t_start, double h, int n_steps, double* out)
{
    or_pulse P = or_make_pulse(Pin);
    double y[OR_NY];
    memcpy(y, y0, sizeof y);
    memcpy(out, y, sizeof y);
    for (int k = 0; k < n_steps; ++k) {
        double t = t_start + k * h;   /* time is computed, never accumulated */
        rk4_step(T, &P, nhat, t, h, y);
        memcpy(out + (size_t)(k + 1) * OR_NY, y, sizeof y);
    }
}

/* ------------------------------------------------------------------ */
/* Herman-Kluk prefactor (Sec. II.A, "pre-exponent factor ... fully      */
/* included"; standard HK form for coherent states of width gamma):      */
/*   C = sqrt( det[ (M_qq + M_pp - i gamma M_qp + (i/gamma) M_pq) / 2 ] ) */
/* with M_ab = d a_t / d b_0.  The square root follows a continuous      */
/* branch: theta_n = theta_{n-1} + arg(det_n / det_{n-1}),               */
/* C = |det|^(1/2) exp(i theta/2), starting from det = 1, theta = 0.     */
/* ------------------------------------------------------------------ */
static cplx det3(const cplx b[9])
{
    return b[0] * (b[4] * b[8] - b[5] * b[7])
         - b[1] * (b[3] * b[8] - b[5] * b[6])
         + b[2] * (b[3] * b[7] - b[4] * b[6]);
}

static cplx hk_det(const double* M, double gamma)
{
    cplx b[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double mqq = M[6 * r + c], mqp = M[6 * r + c + 3];
            double mpq = M[6 * (r + 3) + c], mpp = M[6 * (r + 3) + c + 3];
            b[3 * r + c] = 0.5 * (mqq + mpp - I * gamma * mqp + (I / gamma) * mpq);
        }
    return det3(b);
}

void or_hk_det(const double M[36], double gamma, double out[2])
{
    cplx d = hk_det(M, gamma);
    out[0] = creal(d); out[1] = cimag(d);
}

/* ------------------------------------------------------------------ */
/* Initial orbital psi0 (Sec. II.A, GTO expansion), a sum of Gaussian    */
/* primitives placed on the centres:                                     */
/*   psi0(r) = N sum_{placed i} coef_i f_i(r - A_i) exp(-a_i |r - A_i|^2) */
/* with f = 1 (s-type) or f(x) = s_i u_i.x (p-type).  Diatomic targets:  */
/* every primitive k sits on both centres (the sigma_g combination); a    */
/* sigma p-type one has u = n and s = +-1 on the centre at +-(R/2) n      */
/* (gerade), a pi p-type one u = m (pi_direction) and s = 1 (ungerade,   */
/* 1 pi_u).  Polyatomic targets: primitive k sits on centre pcentre[k]    */
/* only; a p-type one has u = Rot pdir[k]/|pdir[k]| and s = 1.            */
/* ------------------------------------------------------------------ */
/* Direction m of a pi p-type primitive: the unit vector perpendicular   */
/* to the axis n = (sin th cos ph, sin th sin ph, cos th) at azimuth chi  */
/* about n, m = cos(chi) theta_hat + sin(chi) phi_hat with the spherical  */
/* unit vectors theta_hat = (cos th cos ph, cos th sin ph, -sin th) and   */
/* phi_hat = (-sin ph, cos ph, 0); on the z axis ph = 0 is taken.  chi = 0 */
/* puts the lobe in the plane of n and the polarisation axis z, chi =    */
/* pi/2 perpendicular to that plane.                                      */
void or_pi_direction(const double nhat[3], double chi, double m[3])
{
    double rho = sqrt(nhat[0] * nhat[0] + nhat[1] * nhat[1]);
    double cp = 1.0, sp = 0.0;
    if (rho > 0.0) { cp = nhat[0] / rho; sp = nhat[1] / rho; }
    double th_hat[3] = {nhat[2] * cp, nhat[2] * sp, -rho};
    double ph_hat[3] = {-sp, cp, 0.0};
    for (int a = 0; a < 3; ++a) m[a] = cos(chi) * th_hat[a] + sin(chi) * ph_hat[a];
}

typedef struct {
    int c;           /* centre index in the frame */
    double a, coef;  /* exponent, coefficient */
    int p;           /* 0 s-type, 1 p-type */
    double u[3];     /* p-type direction (lab) */
    double s;        /* p-type sign */
} or_placed;

static int place_primitives(const or_target_in* T, const or_frame* F, or_placed* out)
{
    int m = 0;
    if (T->kind == OR_POT_POLY) {
        for (int k = 0; k < T->n_prim; ++k) {
            or_placed P = {T->pcentre[k], T->pexp[k], T->pcoef[k], 0, {0.0, 0.0, 0.0}, 1.0};
            if (T->pkind[k] == 3) {
                double len = sqrt(T->pdir[k][0] * T->pdir[k][0] + T->pdir[k][1] * T->pdir[k][1] +
                                  T->pdir[k][2] * T->pdir[k][2]);
                P.p = 1;
                for (int x = 0; x < 3; ++x) {
                    P.u[x] = 0.0;
                    for (int y = 0; y < 3; ++y) P.u[x] += F->Rot[3 * x + y] * T->pdir[k][y] / len;
                }
            }
            out[m++] = P;
        }
        return m;
    }
    for (int c = 0; c < 2; ++c) {
        double sign = (c == 0) ? 1.0 : -1.0;
        for (int k = 0; k < T->n_prim; ++k) {
            or_placed P = {c, T->pexp[k], T->pcoef[k], 0, {0.0, 0.0, 0.0}, 1.0};
            if (T->pkind[k] == 1) {
                P.p = 1;
                for (int x = 0; x < 3; ++x) P.u[x] = F->nhat[x];
                P.s = sign;
            } else if (T->pkind[k] == 2) {
                P.p = 1;
                or_pi_direction(F->nhat, T->pi_azimuth, P.u);
            }
            out[m++] = P;
        }
    }
    return m;
}

/* Normalisation: 1/sqrt(<psi|psi>) with the overlaps of placed          */
/* primitives, in the frame of a reference orientation (n = z, or the     */
/* identity rotation; the norm does not depend on the orientation).  Two  */
/* Gaussians at A, B with exponents a, b multiply to S0 e^{-p|x-P|^2} with */
/* p = a + b, P = (aA + bB)/p, S0 = e^{-ab/p |A-B|^2}; with y = x - P a    */
/* p-type factor is s (u.y + u.(P - A)), and int (u1.y + al1)(u2.y + al2)  */
/* e^{-p y^2} = [al1 al2 + u1.u2/(2p)] (pi/p)^{3/2} (one factor: al (pi/p)^{3/2}). */
static double orbital_norm(const or_target_in* T)
{
    const double ref[3] = {0.0, 0.0, T->kind == OR_POT_POLY ? 0.0 : 1.0};
    or_frame F;
    make_frame(T, ref, &F);
    or_placed L[16];
    int m = place_primitives(T, &F, L);
    double s = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            const double* A = F.C[L[i].c];
            const double* B = F.C[L[j].c];
            double a = L[i].a, b = L[j].a, pp = a + b;
            double P[3], AB2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                P[x] = (a * A[x] + b * B[x]) / pp;
                AB2 += (A[x] - B[x]) * (A[x] - B[x]);
            }
            double S0 = pow(OR_PI / pp, 1.5) * exp(-a * b / pp * AB2);
            double al1 = 0.0, al2 = 0.0, uu = 0.0;
            for (int x = 0; x < 3; ++x) {
                al1 += L[i].u[x] * (P[x] - A[x]);
                al2 += L[j].u[x] * (P[x] - B[x]);
                uu += L[i].u[x] * L[j].u[x];
            }
            double f;
            if (!L[i].p && !L[j].p) f = 1.0;
            else if (!L[i].p) f = L[j].s * al2;
            else if (!L[j].p) f = L[i].s * al1;
            else f = L[i].s * L[j].s * (al1 * al2 + uu / (2.0 * pp));
            s += L[i].coef * L[j].coef * f * S0;
        }
    return 1.0 / sqrt(s);
}

double or_orbital_norm(const or_target_in* T) { return orbital_norm(T); }

static double orbital_value_n(const or_target_in* T, double N, const double orient[3],
                              const double r[3])
{
    or_frame F;
    make_frame(T, orient, &F);
    or_placed L[16];
    int m = place_primitives(T, &F, L);
    double v = 0.0;
    for (int i = 0; i < m; ++i) {
        const double* A = F.C[L[i].c];
        double d2 = 0.0, ang = 1.0;
        for (int a = 0; a < 3; ++a) d2 += (r[a] - A[a]) * (r[a] - A[a]);
        if (L[i].p) {
            ang = 0.0;
            for (int a = 0; a < 3; ++a) ang += L[i].u[a] * (r[a] - A[a]);
            ang *= L[i].s;
        }
        v += L[i].coef * ang * exp(-L[i].a * d2);
    }
    return N * v;
}

double or_orbital_value(const or_target_in* T, const double orient[3], const double r[3])
{
    return orbital_value_n(T, orbital_norm(T), orient, r);
}

void or_orbital_values(const or_target_in* T, const double orient[3], const double* r, int64_t n,
                       double* out)
{
    double N = orbital_norm(T);
    for (int64_t i = 0; i < n; ++i) out[i] = orbital_value_n(T, N, orient, r + 3 * i);
}

/* ------------------------------------------------------------------ */
/* Recombination element <psi0| k_z |p,q> (Eq. 4) with the coherent       */
/* state <x|p,q> = (gamma/pi)^{3/4} exp(-gamma/2 |x-q|^2 + i p.(x-q))     */
/* and k_z = -i d/dz.  k_z acting on the coherent state gives            */
/* [p_z + i gamma (z - q_z)] <x|p,q>.  For one primitive e^{-a|x-A|^2},  */
/* shift x = A + y, d = q - A, b = gamma/2, c = a + b: the integrand is  */
/*   e^{-a y^2 - b (y-d)^2 + i p.(y-d)} = e^{-c (y-m)^2 + c m.m - b d.d - i p.d}, */
/*   m = (2 b d + i p) / (2c),                                           */
/* so I0 = (pi/c)^{3/2} e^{c m.m - b d.d - i p.d} and                    */
/* int (z - q_z) (...) = (m_z - d_z) I0.                                 */
/* ------------------------------------------------------------------ */
static cplx recomb(const or_target_in* T, double N, const double orient[3],
                   const double q[3], const double p[3], double gamma)
{
    or_frame F;
    make_frame(T, orient, &F);
    or_placed L[16];
    int np = place_primitives(T, &F, L);
    double b = 0.5 * gamma;
    cplx total = 0.0;
    for (int i = 0; i < np; ++i) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = q[a] - F.C[L[i].c][a];
        double a = L[i].a;
        double c = a + b;
        cplx m[3], mm = 0.0;
        double dd = 0.0, pd = 0.0;
        for (int x = 0; x < 3; ++x) {
            m[x] = (2.0 * b * d[x] + I * p[x]) / (2.0 * c);
            mm += m[x] * m[x];
            dd += d[x] * d[x];
            pd += p[x] * d[x];
        }
        cplx I0 = pow(OR_PI / c, 1.5) * cexp(c * mm - b * dd - I * pd);
        cplx I1 = (m[2] - d[2]) * I0;
        if (L[i].p) {
            /* p-type: extra factor s u.x' (x' = x - A):                */
            /* int u.x' e = (u.m) I0, int u.x' (x'_z - d_z) e =        */
            /* [(u.m)(m_z - d_z) + u_z/(2c)] I0                         */
            const double* u = L[i].u;
            cplx um = u[0] * m[0] + u[1] * m[1] + u[2] * m[2];
            cplx J0 = um * I0;
            cplx J1 = (um * (m[2] - d[2]) + u[2] / (2.0 * c)) * I0;
            total += L[i].s * L[i].coef * (p[2] * J0 + I * gamma * J1);
        } else {
            total += L[i].coef * (p[2] * I0 + I * gamma * I1);
        }
    }
    return N * pow(gamma / OR_PI, 0.75) * total;
}

void or_recomb(const or_target_in* T, const double orient[3], const double q[3],
               const double p[3], double gamma, double out[2])
{
    cplx r = recomb(T, orbital_norm(T), orient, q, p, gamma);
    out[0] = creal(r); out[1] = cimag(r);
}

/* ------------------------------------------------------------------ */
/* Ionization step (Sec. II.A, Eqs. 1-2).                                */
/* Plane-wave bra <kappa| = (2 pi)^{-3/2} e^{-i kappa.r}, continued to   */
/* complex kappa.  For one primitive centred at A:                       */
/*   int e^{-i kappa.r} e^{-a|r-A|^2} = (pi/a)^{3/2} e^{-i kappa.A - kappa.kappa/(4a)}, */
/*   int e^{-i kappa.r} z e^{-a|r-A|^2} = (A_z - i kappa_z/(2a)) x (above). */
/* ------------------------------------------------------------------ */
/* only: -1 every centre; else that centre alone (diatomic: 0 the centre  */
/* at +(R/2) n, 1 the one at -(R/2) n)                                   */
static void dipole_matrix_element(const or_target_in* T, double N, const double orient[3],
                                  const cplx kappa[3], int only, cplx* mz)
{
    or_frame F;
    make_frame(T, orient, &F);
    or_placed L[16];
    int np = place_primitives(T, &F, L);
    cplx kk = kappa[0] * kappa[0] + kappa[1] * kappa[1] + kappa[2] * kappa[2];
    cplx tot = 0.0;
    for (int i = 0; i < np; ++i) {
        if (only >= 0 && L[i].c != only) continue;
        const double* A = F.C[L[i].c];
        cplx kA = kappa[0] * A[0] + kappa[1] * A[1] + kappa[2] * A[2];
        double a = L[i].a;
        cplx G = pow(OR_PI / a, 1.5) * cexp(-I * kA - kk / (4.0 * a));
        if (L[i].p) {
            /* p-type: int e^{-i k.x} (x_z + A_z)(u.x) e^{-a x^2} =        */
            /* [u_z/(2a) - k_z (u.k)/(4a^2) - i A_z (u.k)/(2a)] G           */
            const double* u = L[i].u;
            cplx uk = u[0] * kappa[0] + u[1] * kappa[1] + u[2] * kappa[2];
            tot += L[i].s * L[i].coef *
                   (u[2] / (2.0 * a) - kappa[2] * uk / (4.0 * a * a) -
                    I * A[2] * uk / (2.0 * a)) * G;
        } else {
            tot += L[i].coef * (A[2] - I * kappa[2] / (2.0 * a)) * G;
        }
    }
    *mz = N * pow(2.0 * OR_PI, -1.5) * tot;
}

void or_dipole_matrix_element(const or_target_in* T, const double orient[3],
                              const double kre[3], const double kim[3], double out[2])
{
    cplx kap[3];
    for (int a = 0; a < 3; ++a) kap[a] = kre[a] + I * kim[a];
    cplx m;
    dipole_matrix_element(T, orbital_norm(T), orient, kap, -1, &m);
    out[0] = creal(m); out[1] = cimag(m);
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n,     */
/* nodes in descending order.                                            */
static void gauss_legendre(int n, double* xs, double* ws)
{
    for (int i = 0; i < n; ++i) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = pk;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* P_n'(x) at the converged node */
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = pk;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

#define OR_GL 64
static double gl_x[OR_GL], gl_w[OR_GL];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    gauss_legendre(OR_GL, gl_x, gl_w);
    gl_ready = 1;
}

/* K-node Gauss-Legendre rule on x = cos(theta) in [0, 1] (Eq. 5 with the  */
/* cylindrical and inversion symmetry of a homonuclear diatomic in a      */
/* linearly polarised field: the isotropic average over the axis reduces  */
/* to int_0^1 dx f(arccos x)); node k = 0..K-1 in descending x, weights    */
/* summing to 1.                                                          */
void or_quad_nodes(int K, double* x01, double* w01)
{
    gauss_legendre(K, x01, w01);
    for (int k = 0; k < K; ++k) {
        x01[k] = 0.5 * (x01[k] + 1.0);
        w01[k] = 0.5 * w01[k];
    }
}

/* Saddle point (Eq. 2) for t_s = t0 + i tt with given k_perp:           */
/*   [k + A(t_s) - A(t0)]^2 / 2 + Ip = 0.                                */
/* With A along z and A(t0) real, the imaginary part forces              */
/*   k_z = -Re[A(t0 + i tt) - A(t0)] and the real part gives             */
/*   (Im A(t0 + i tt))^2 = 2 Ip + k_perp^2.                              */
/* Reading: tt is the smallest positive root.  Found by marching s from  */
/* 0 in steps of s_qs/64 (s_qs = sqrt(2Ip+kp^2)/|E(t0)|, the quasi-static */
/* value) to the first sign change, then bisection to the last bit.      */
/* Returns 0 on success, -1 if no root below 64 s_qs.                     */
static int saddle(const or_pulse* P, double Ip, double t0, double kperp2,
                  double* tt_out, double* kz_out)
{
    double target = 2.0 * Ip + kperp2;
    double E0 = fabs(pulse_E_real(P, t0));
    if (!(E0 > 0.0)) return -1;
    double sqs = sqrt(target) / E0;
    double h = sqs / 64.0;
    double s_lo = 0.0, f_lo = -target, s_hi = 0.0, f_hi = -target;
    int found = 0;
    for (int k = 1; k <= 64 * 64; ++k) {
        double s = k * h;
        double y = cimag(pulse_A(P, t0 + I * s));
        double f = y * y - target;
        if (f >= 0.0) { s_hi = s; f_hi = f; found = 1; break; }
        s_lo = s; f_lo = f;
    }
    if (!found) return -1;
    (void)f_lo; (void)f_hi;
    for (int it = 0; it < 200; ++it) {
        double sm = 0.5 * (s_lo + s_hi);
        if (sm <= s_lo || sm >= s_hi) break;
        double y = cimag(pulse_A(P, t0 + I * sm));
        if (y * y - target >= 0.0) s_hi = sm; else s_lo = sm;
    }
    double tt = 0.5 * (s_lo + s_hi);
    *tt_out = tt;
    *kz_out = -(creal(pulse_A(P, t0 + I * tt)) - creal(pulse_A(P, t0)));
    return 0;
}

int or_saddle(const or_pulse_in* Pin, double Ip, double t0, double kperp2, double out[2])
{
    or_pulse P = or_make_pulse(Pin);
    return saddle(&P, Ip, t0, kperp2, &out[0], &out[1]);
}

/* Modified saddle point (SFHK2, Sec. III.D):                            */
/*   [k + A(t_s) - A(t0)]^2 / 2 + Ip - eta E(t_s).r0 = 0,  r0 = (R/2) n,  */
/* with E along z: c = eta (R/2) n_z.  With Y = Im A(t_s), E(t_s) =       */
/* E_r + i E_i, the imaginary part gives X = k_z + Re A(t_s) - A(t0)      */
/*   = c E_i / Y, and the real part                                      */
/*   F(tt) = Y^2 - X^2 - 2 Ip - k_perp^2 + 2 c E_r = 0.                  */
/* Reading: tt is the smallest positive root, found as in saddle() by    */
/* marching to the first sign change of F and bisecting.  c = 0 gives     */
/* the standard saddle.  Returns 0 on success, -1 if no root.            */
static int saddle_modified(const or_pulse* P, double Ip, double t0, double kperp2, double c,
                           double* tt_out, double* kz_out)
{
    double target = 2.0 * Ip + kperp2;
    double E0 = fabs(pulse_E_real(P, t0));
    if (!(E0 > 0.0)) return -1;
    double sqs = sqrt(target) / E0;
    double h = sqs / 64.0;
    double s_lo = 0.0, s_hi = 0.0;
    int found = 0;
#define OR_F_MOD(s_, f_)                                                       \
    do {                                                                       \
        cplx A_ = pulse_A(P, t0 + I * (s_));                                   \
        cplx E_ = pulse_E(P, t0 + I * (s_));                                   \
        double Y_ = cimag(A_), X_ = c * cimag(E_) / Y_;                        \
        (f_) = Y_ * Y_ - X_ * X_ - target + 2.0 * c * creal(E_);               \
    } while (0)
    for (int k = 1; k <= 64 * 64; ++k) {
        double s = k * h, f;
        OR_F_MOD(s, f);
        if (f >= 0.0) { s_hi = s; found = 1; break; }
        s_lo = s;
    }
    if (!found) return -1;
    for (int it = 0; it < 200; ++it) {
        double sm = 0.5 * (s_lo + s_hi), f;
        if (sm <= s_lo || sm >= s_hi) break;
        OR_F_MOD(sm, f);
        if (f >= 0.0) s_hi = sm; else s_lo = sm;
    }
#undef OR_F_MOD
    double tt = 0.5 * (s_lo + s_hi);
    cplx A = pulse_A(P, t0 + I * tt);
    cplx E = pulse_E(P, t0 + I * tt);
    *tt_out = tt;
    *kz_out = c * cimag(E) / cimag(A) - (creal(A) - creal(pulse_A(P, t0)));
    return 0;
}

int or_saddle_modified(const or_pulse_in* Pin, double Ip, double t0, double kperp2, double c,
                       double out[2])
{
    or_pulse P = or_make_pulse(Pin);
    return saddle_modified(&P, Ip, t0, kperp2, c, &out[0], &out[1]);
}

/* Tunnel exit q_{t0} = Re int_{t_s}^{t0} A(tau) dtau along tau = t0 + i s
 * (s from tt down to 0, dtau = i ds), and the tunnelling action
 *   S_down = Ip t_s - int_{t_s}^{t0} [k + A(tau) - A(t0)]^2 / 2 dtau,
 * both by 64-point Gauss-Legendre quadrature over s in [0, tt].          */
static void tunnel_exit_and_action(const or_pulse* P, double Ip, double t0, double tt,
                                   const double k[3], double* qz, cplx* Sdown)
{
    gl_init();
    double At0 = creal(pulse_A(P, t0));
    double kperp2 = k[0] * k[0] + k[1] * k[1];
    cplx intA = 0.0, intK = 0.0;
    for (int i = 0; i < OR_GL; ++i) {
        double s = 0.5 * tt * (gl_x[i] + 1.0);
        double w = 0.5 * tt * gl_w[i];
        cplx A = pulse_A(P, t0 + I * s);
        cplx kz = k[2] + A - At0;
        intA += w * A;
        intK += w * 0.5 * (kperp2 + kz * kz);
    }
    /* int_{t_s}^{t0} f dtau = int_{tt}^{0} f(t0+is) i ds = -i int_0^{tt} f ds */
    *qz = creal(-I * intA);
    *Sdown = Ip * (t0 + I * tt) - (-I * intK);
}

void or_tunnel(const or_pulse_in* Pin, double Ip, double t0, double tt, const double k[3],
               double out[3])
{
    or_pulse P = or_make_pulse(Pin);
    double qz; cplx S;
    tunnel_exit_and_action(&P, Ip, t0, tt, k, &qz, &S);
    out[0] = qz; out[1] = creal(S); out[2] = cimag(S);
}

/* The ionization step for one initial point (Sec. II.A, Eqs. 1-2):      */
/* the saddle t_s = t0 + i tt with k_z (Eq. 2; for SFHK2, target          */
/* ionization 1, the modified saddle of Sec. III.D with c = eta (R/2) n_z),*/
/* the tunnel exit q_z and the tunnelling action S_down (text after Eq. 2),*/
/* and the amplitude of the second line of Eq. 1,                         */
/*   a = side_w E(t_s) <kappa| z |psi0> / sqrt(curv) e^{i(S_down + k.q0)}, */
/* kappa = k + A(t_s) - A(t0), curv = E(t_s) kappa_z + c dE/dt(t_s) (the   */
/* curvature of the whole phase at the saddle; E kappa_z for SFHK1), the   */
/* principal square root (reading); q0 = origin + q_z z^, the exit lying   */
/* on the polarisation axis through the molecule's position (k.q0 = k_z q_z */
/* for a molecule at the origin).  `only` >= 0 keeps one centre's part of  */
/* the dipole element (SFHK2).  Returns 0, or 1 when the saddle has no root. */
typedef struct {
    double tt, kz, qz;
    cplx Sd, curv, mz, a;
} or_ionization;

static int ionization_step(const or_target_in* T, const or_pulse* Pp, double N,
                           const double orient[3], double t0, double kx, double ky, double cmod,
                           int only, double side_w, or_ionization* out)
{
    double tt = 0.0, kz = 0.0, qz = 0.0;
    cplx Sd = 0.0;
    int sok = (T->ionization == 1)
                  ? saddle_modified(Pp, T->Ip, t0, kx * kx + ky * ky, cmod, &tt, &kz)
                  : saddle(Pp, T->Ip, t0, kx * kx + ky * ky, &tt, &kz);
    memset(out, 0, sizeof *out);
    if (sok != 0) return 1;
    double k[3] = {kx, ky, kz};
    tunnel_exit_and_action(Pp, T->Ip, t0, tt, k, &qz, &Sd);
    cplx ts = t0 + I * tt;
    cplx Es = pulse_E(Pp, ts);
    cplx kap[3] = {kx, ky, kz + pulse_A(Pp, ts) - creal(pulse_A(Pp, t0))};
    cplx mz;
    dipole_matrix_element(T, N, orient, kap, only, &mz);
    cplx curv = Es * kap[2] + cmod * pulse_Edot(Pp, ts);
    out->tt = tt;
    out->kz = kz;
    out->qz = qz;
    out->Sd = Sd;
    out->curv = curv;
    out->mz = mz;
    const double kq = kx * T->origin[0] + ky * T->origin[1] + kz * (T->origin[2] + qz);
    out->a = side_w * Es * mz / csqrt(curv) * cexp(I * (Sd + kq));
    return 0;
}

/* The same for the tests: orient is the axis (or the Euler angles of a    */
/* polyatomic target); eta = +-1 picks the emitting centre of an SFHK2      */
/* target (weight 1), 0 for SFHK1.  out: tt, kz, qz, S_down (re, im),     */
/* curv (re, im), <kappa|z|psi0> (re, im), a (re, im).                    */
int or_ionization_step(const or_target_in* T, const or_pulse_in* Pin, const double orient[3],
                       double t0, double kx, double ky, int eta, double out[11])
{
    or_pulse P = or_make_pulse(Pin);
    double cmod = 0.0;
    int only = -1;
    if (T->ionization == 1) {
        if (eta != 1 && eta != -1) return -1;
        only = (eta > 0) ? 1 : 0;
        double nz = (T->kind == OR_POT_POLY) ? 0.0 : orient[2];
        cmod = eta * 0.5 * T->R * nz;
    }
    or_ionization ion;
    int rc = ionization_step(T, &P, orbital_norm(T), orient, t0, kx, ky, cmod, only, 1.0, &ion);
    double v[11] = {ion.tt, ion.kz, ion.qz, creal(ion.Sd), cimag(ion.Sd), creal(ion.curv),
                    cimag(ion.curv), creal(ion.mz), cimag(ion.mz), creal(ion.a), cimag(ion.a)};
    for (int i = 0; i < 11; ++i) out[i] = v[i];
    return rc;
}

/* ------------------------------------------------------------------ */
/* Initial ensemble (Sec. II.A sampling paragraph and Eq. 6), in the     */
/* proposal form: t0 drawn on the time grid with probability             */
/*   p_n = W_n / sum W,  W_n = exp(-2 (2Ip)^{3/2} / (3 |E(t_n)|)),       */
/* by inverse CDF (smallest n with CDF_n > u sum W, sequential sums);    */
/* k_x, k_y ~ N(0, sigma^2), sigma = sqrt(|E(t0)| / (2 sqrt(2 Ip))),     */
/* by Box-Muller; orientation per trajectory: fixed, isotropic           */
/* (cos th = 2u-1) or cos^2 (cos th = cbrt(2u-1)), phi = 2 pi u, or the   */
/* K-node quadrature of Eq. 5 (cos th = x_{j mod K}, phi = 2 pi u, weight */
/* times K W_{j mod K}; or_quad_nodes).  Returns -1 for a bad K.          */
/* The amplitude of the second line of Eq. 1,                            */
/*   a = <kappa| r.E(t_s) |psi0> / sqrt(E(t_s).kappa) e^{i(S_down + k.q0)}, */
/* kappa = k + A(t_s) - A(t0), principal square root (reading), and the  */
/* Monte Carlo weight w = a / pdf, pdf = (p_n / dt) N(kx) N(ky).          */
/* Output SoA, field-major: soa[f * n + j], fields                       */
/*   0 n0 | 1-3 q0 | 4-6 p0 | 7-9 nhat | 10-11 w (re, im).               */
/* A trajectory whose saddle has no root gets w = 0 (it still counts in N).*/
/* ------------------------------------------------------------------ */
enum { OR_ALIGN_FIXED = 0, OR_ALIGN_ISO = 1, OR_ALIGN_COS2 = 2, OR_ALIGN_QUAD = 3 };
#define OR_MAX_QUAD 64

void or_adk_table(const or_pulse_in* Pin, double Ip, double* W, double* cdf)
{
    or_pulse P = or_make_pulse(Pin);
    double acc = 0.0;
    double c = 2.0 * pow(2.0 * Ip, 1.5) / 3.0;
    for (int n = 0; n < P.nt; ++n) {
        double e = fabs(pulse_E_real(&P, P.t_origin + n * P.dt));
        W[n] = (e > 0.0) ? exp(-c / e) : 0.0;
        acc += W[n];
        cdf[n] = acc;
    }
}

/* Time table of the proposal.  Plain: the ADK weights (or_adk_table).    */
/* Defensive (proposal_mix = eps > 0, a reading): W_n = (1 - eps) e_n /     */
/* sum e + eps u_n, with u_n = 1 / N_u on the N_u grid points where |E(t_n)| */
/* >= OR_DEF_FIELD E0 and 0 elsewhere.  The ADK exponent falls much faster   */
/* than the SFA amplitude where the field is weak (Keldysh parameter above  */
/* 1), which gives w = a / pdf a heavy tail; the uniform share bounds the   */
/* time factor of 1/pdf there, and the floor on the k_perp width            */
/* (proposal_floor) keeps the momentum factor bounded.  Below OR_DEF_FIELD   */
/* E0 (the pulse's ends) both weights are zero in effect and the saddle's   */
/* imaginary time would overflow, so the share leaves those points out.     */
/* Any eps and floor leave every weighted mean unbiased, since w = a / pdf  */
/* uses the density actually sampled.                                       */
#define OR_DEF_FIELD 1e-2
static void defensive_table(const or_target_in* T, const or_pulse_in* Pin, double* W,
                            double* cdf)
{
    or_adk_table(Pin, T->Ip, W, cdf);
    double eps = T->proposal_mix;
    if (!(eps > 0.0)) return;
    or_pulse P = or_make_pulse(Pin);
    double sum = cdf[P.nt - 1], acc = 0.0;
    int nu = 0;
    for (int n = 0; n < P.nt; ++n)
        nu += fabs(pulse_E_real(&P, P.t_origin + n * P.dt)) >= OR_DEF_FIELD * P.E0;
    for (int n = 0; n < P.nt; ++n) {
        int in = fabs(pulse_E_real(&P, P.t_origin + n * P.dt)) >= OR_DEF_FIELD * P.E0;
        W[n] = (1.0 - eps) * W[n] / sum + (in ? eps / nu : 0.0);
        acc += W[n];
        cdf[n] = acc;
    }
}

/* One draw of the proposal and its amplitude: t0, k_perp, axis from the  */
/* six uniforms u, then saddle, exit, action, amplitude and the weight     */
/* w = a / pdf (node weight of the quadrature alignment included).         */
/* f receives the 12 SoA fields (w zero without a saddle root); returns 0, */
/* or 1 when the saddle has no root.                                       */
typedef struct {
    const or_target_in* T;
    or_pulse P;
    const double *W, *cdf;
    double total, N;
    int align_kind, n_nodes, eta_force;
    double theta, phi, psi;
    const double *qx, *qw;
} or_proposal;

static int propose(const or_proposal* Q, uint64_t j, const double u[6], double f[12],
                   double* tt_out, cplx* Sd_out)
{
    const or_target_in* T = Q->T;
    const or_pulse* Pp = &Q->P;
    /* time index */
    int n0 = Pp->nt - 1;
    double thr = u[0] * Q->total;
    for (int m = 0; m < Pp->nt; ++m)
        if (Q->cdf[m] > thr) { n0 = m; break; }
    double t0 = Pp->t_origin + n0 * Pp->dt;
    double Et0 = pulse_E_real(Pp, t0);
    double sigma = sqrt(fabs(Et0) / (2.0 * sqrt(2.0 * T->Ip)));
    if (T->proposal_floor > 0.0)      /* defensive floor on the k_perp width */
        sigma = fmax(sigma, sqrt(T->proposal_floor * Pp->E0 / (2.0 * sqrt(2.0 * T->Ip))));
    double r = sqrt(-2.0 * log(u[1]));
    double kx = sigma * r * cos(2.0 * OR_PI * u[2]);
    double ky = sigma * r * sin(2.0 * OR_PI * u[2]);
    /* orientation */
    double th = Q->theta, ph = Q->phi;
    if (Q->align_kind == OR_ALIGN_ISO) {
        th = acos(2.0 * u[3] - 1.0);
        ph = 2.0 * OR_PI * u[4];
    } else if (Q->align_kind == OR_ALIGN_COS2) {
        th = acos(cbrt(2.0 * u[3] - 1.0));
        ph = 2.0 * OR_PI * u[4];
    } else if (Q->align_kind == OR_ALIGN_QUAD) {
        /* Eq. 5 by quadrature: trajectory j sits at node j mod K */
        th = acos(Q->qx[j % (uint64_t)Q->n_nodes]);
        ph = 2.0 * OR_PI * u[4];
    }
    double nhat[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
    /* polyatomic: the orientation is the Euler triple (phi, theta, psi),  */
    /* psi uniform for the isotropic and cos^2 distributions (Eq. 6 over   */
    /* all three Euler angles); n = Rot z is the same axis as above        */
    double orient[3] = {nhat[0], nhat[1], nhat[2]};
    if (T->kind == OR_POT_POLY) {
        double ps = Q->psi;
        if (Q->align_kind == OR_ALIGN_ISO || Q->align_kind == OR_ALIGN_COS2)
            ps = 2.0 * OR_PI * u[5];
        orient[0] = ph;
        orient[1] = th;
        orient[2] = ps;
    }
    /* saddle, exit, action, amplitude.  SFHK2: the electron leaves     */
    /* from one centre, eta = +1 (the centre at -(R/2) n) or -1 (the     */
    /* centre at +(R/2) n) with probability 1/2 each (weight x 2), the   */
    /* modified saddle, that centre's part of the dipole element (its    */
    /* factor e^{-i kappa.R_c} is the phase whose t_s-derivative is the  */
    /* extra term), and the Gaussian-integration factor from the         */
    /* curvature of the whole phase, E kappa_z + c dE/dt.                */
    double tt = 0.0, kz = 0.0, qz = 0.0;
    cplx w = 0.0, Sd = 0.0;
    int only = -1;
    double cmod = 0.0, side_w = 1.0;
    if (T->ionization == 1) {
        /* eta_force = +-1 fixes the side (test hook, weight x 1) */
        double eta = Q->eta_force ? (double)Q->eta_force : ((u[5] < 0.5) ? 1.0 : -1.0);
        only = (eta > 0.0) ? 1 : 0;
        cmod = eta * 0.5 * T->R * cos(th);
        side_w = Q->eta_force ? 1.0 : 2.0;
    }
    or_ionization ion;
    int sok = ionization_step(T, Pp, Q->N, orient, t0, kx, ky, cmod, only, side_w, &ion);
    if (sok == 0) {
        tt = ion.tt;
        kz = ion.kz;
        qz = ion.qz;
        Sd = ion.Sd;
        cplx a = ion.a;
        double pdf = (Q->W[n0] / Q->total) / Pp->dt
                     * exp(-(kx * kx + ky * ky) / (2.0 * sigma * sigma))
                     / (2.0 * OR_PI * sigma * sigma);
        w = a / pdf;
        /* node weight, times K for the 1/N over all K nodes' trajectories */
        if (Q->align_kind == OR_ALIGN_QUAD) w *= Q->n_nodes * Q->qw[j % (uint64_t)Q->n_nodes];
        /* a birth where the field all but vanishes (reached only through   */
        /* the defensive share: the pulse's ends) has a saddle so far up    */
        /* the imaginary axis that it overflows; its amplitude is zero in   */
        /* effect, and it counts as a draw without a root                   */
        if (!isfinite(kz) || !isfinite(qz) || !isfinite(creal(w)) || !isfinite(cimag(w))) {
            sok = 1;
            kz = qz = 0.0;
            w = 0.0;
            Sd = 0.0;
            tt = 0.0;
        }
    }
    double g[12] = {(double)n0, T->origin[0], T->origin[1], T->origin[2] + qz, kx, ky, kz,
                    orient[0], orient[1], orient[2], creal(w), cimag(w)};
    for (int q = 0; q < 12; ++q) f[q] = g[q];
    *tt_out = tt;
    *Sd_out = Sd;
    return sok == 0 ? 0 : 1;
}

/* Initial points distributed ~ |a| (target sampling 1; Sec. II.B draws    */
/* the initial points, Euler angles included, with density proportional   */
/* to |sin(beta) <W| r.E(t_s) |psi0>|; here with the axis measure in the  */
/* proposal).  Exact rejection with weight correction on top of the        */
/* proposal: a draw with weight w is accepted with alpha = min(1, |w|/M)  */
/* and then carries the alpha-corrected weight                            */
/*   omega = P w / alpha,  P = E[alpha]  (= P M w/|w| whenever |w| <= M),   */
/* so that E[omega f] over accepted draws is the integral of a f for any  */
/* M.  M is kappa times the mean |w| over the first half of a pilot of     */
/* proposal draws (kappa = sampling_factor; M >= max |w| would give the   */
/* exact |a| distribution at a sampling cost of max/mean draws per point)  */
/* and P the mean alpha over its second half (independent of M).  Draws:   */
/* attempt k of trajectory j uses draws 3k..3k+2 (attempt 0 = the plain    */
/* sampler's), its acceptance uniform draw OR_ACC_BASE + k, pilot draw i   */
/* the trajectory index i with draws OR_PILOT_BASE.. .  A trajectory with */
/* no acceptance in K = OR_ATTEMPTS attempts gets w = 0 (invalid); as     */
/* every attempt is accepted with the same probability P, that happens    */
/* with probability (1 - P)^K, and the kept weights are divided by        */
/* 1 - (1 - P)^K so that the mean over all N trajectories (invalid ones    */
/* included, the 1/N of the dipole) stays unbiased for any kappa.         */
#define OR_PILOT 16384
#define OR_ATTEMPTS 256
#define OR_ACC_BASE (1u << 20)
#define OR_PILOT_BASE (1u << 24)

static double acc_uniform(uint64_t seed, uint32_t instance, uint64_t j, uint32_t k)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), instance, OR_ACC_BASE + k};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    return or_u01(r[0], r[1]);
}

/* M and P of the |a|-proportional sampler (out[0] = M, out[1] = P). */
static void abs_sampling_constants(const or_proposal* Q, uint64_t seed, uint32_t instance,
                                   double out[2])
{
    double u[6], f[12], tt, sum = 0.0;
    cplx Sd;
    for (uint64_t i = 0; i < OR_PILOT / 2; ++i) {
        uniforms_at(seed, instance, i, OR_PILOT_BASE, u);
        propose(Q, i, u, f, &tt, &Sd);
        sum += hypot(f[10], f[11]);
    }
    double kappa = Q->T->sampling_factor > 0.0 ? Q->T->sampling_factor : 5.0;
    double M = kappa * sum / (OR_PILOT / 2);
    double asum = 0.0;
    for (uint64_t i = OR_PILOT / 2; i < OR_PILOT; ++i) {
        uniforms_at(seed, instance, i, OR_PILOT_BASE, u);
        propose(Q, i, u, f, &tt, &Sd);
        double aw = hypot(f[10], f[11]);
        asum += (M > 0.0) ? fmin(1.0, aw / M) : 0.0;
    }
    out[0] = M;
    out[1] = asum / (OR_PILOT / 2);
}

void or_abs_sampling_constants(const or_target_in* T, const or_pulse_in* Pin, int align_kind,
                               double theta, double phi, double psi, int n_nodes, uint64_t seed,
                               uint32_t instance, double out[2]);

int or_sample(const or_target_in* T, const or_pulse_in* Pin, int align_kind,
              double theta, double phi, double psi, int n_nodes, int eta_force, uint64_t seed,
              uint32_t instance, uint64_t j_begin, uint64_t n, double* soa, double* aux)
{
    double qx[OR_MAX_QUAD], qw[OR_MAX_QUAD];
    /* polyatomic targets: no quadrature in cos theta (it relies on the    */
    /* symmetry of a homonuclear diatomic) and no modified saddle          */
    if (T->kind == OR_POT_POLY && (align_kind == OR_ALIGN_QUAD || T->ionization == 1))
        return -1;
    if (align_kind == OR_ALIGN_QUAD) {
        if (n_nodes < 1 || n_nodes > OR_MAX_QUAD) return -1;
        or_quad_nodes(n_nodes, qx, qw);
    }
    or_proposal Q;
    Q.T = T;
    Q.P = or_make_pulse(Pin);
    double* W = (double*)malloc(sizeof(double) * Q.P.nt);
    double* cdf = (double*)malloc(sizeof(double) * Q.P.nt);
    defensive_table(T, Pin, W, cdf);
    Q.W = W;
    Q.cdf = cdf;
    Q.total = cdf[Q.P.nt - 1];
    Q.N = orbital_norm(T);
    Q.align_kind = align_kind;
    Q.n_nodes = n_nodes;
    Q.eta_force = eta_force;
    Q.theta = theta;
    Q.phi = phi;
    Q.psi = psi;
    Q.qx = qx;
    Q.qw = qw;
    double MP[2] = {0.0, 0.0};
    double keep = 0.0;   /* weight factor of an accepted draw: P / (1 - (1-P)^K) */
    if (T->sampling == 1) {
        abs_sampling_constants(&Q, seed, instance, MP);
        if (MP[1] > 0.0) keep = MP[1] / -expm1(OR_ATTEMPTS * log1p(-MP[1]));
    }
    int bad = 0;
    for (uint64_t jj = 0; jj < n; ++jj) {
        uint64_t j = j_begin + jj;
        double u[6], f[12], tt = 0.0;
        cplx Sd = 0.0;
        int inval;
        if (T->sampling == 1) {
            inval = 1;
            for (uint32_t k = 0; k < OR_ATTEMPTS; ++k) {
                uniforms_at(seed, instance, j, 3u * k, u);
                if (propose(&Q, j, u, f, &tt, &Sd)) continue;
                double aw = hypot(f[10], f[11]);
                double alpha = (MP[0] > 0.0) ? fmin(1.0, aw / MP[0]) : 0.0;
                if (!(alpha > 0.0) || acc_uniform(seed, instance, j, k) >= alpha) continue;
                f[10] *= keep / alpha;
                f[11] *= keep / alpha;
                inval = 0;
                break;
            }
            if (inval) {
                f[10] = f[11] = 0.0;
                tt = 0.0;
                Sd = 0.0;
            }
        } else {
            or_uniforms(seed, instance, j, u);
            inval = propose(&Q, j, u, f, &tt, &Sd);
        }
        bad += inval;
        for (int q = 0; q < 12; ++q) soa[(size_t)q * n + jj] = f[q];
        if (aux) {
            aux[(size_t)0 * n + jj] = tt;
            aux[(size_t)1 * n + jj] = creal(Sd);
            aux[(size_t)2 * n + jj] = cimag(Sd);
        }
    }
    free(W);
    free(cdf);
    return bad;
}

void or_abs_sampling_constants(const or_target_in* T, const or_pulse_in* Pin, int align_kind,
                               double theta, double phi, double psi, int n_nodes, uint64_t seed,
                               uint32_t instance, double out[2])
{
    double qx[OR_MAX_QUAD], qw[OR_MAX_QUAD];
    if (align_kind == OR_ALIGN_QUAD) or_quad_nodes(n_nodes, qx, qw);
    or_proposal Q;
    Q.T = T;
    Q.P = or_make_pulse(Pin);
    double* W = (double*)malloc(sizeof(double) * Q.P.nt);
    double* cdf = (double*)malloc(sizeof(double) * Q.P.nt);
    defensive_table(T, Pin, W, cdf);
    Q.W = W;
    Q.cdf = cdf;
    Q.total = cdf[Q.P.nt - 1];
    Q.N = orbital_norm(T);
    Q.align_kind = align_kind;
    Q.n_nodes = n_nodes;
    Q.eta_force = 0;
    Q.theta = theta;
    Q.phi = phi;
    Q.psi = psi;
    Q.qx = qx;
    Q.qw = qw;
    abs_sampling_constants(&Q, seed, instance, out);
    free(W);
    free(cdf);
}

/* ------------------------------------------------------------------ */
/* Continuum propagation and dipole velocity (Eq. 4 and the v_z          */
/* approximation before Eq. 1):                                          */
/*   v_z(t_n) = -(2/N) sum_j Re[ w_j C_j(t_n) e^{i(S_j(t_n) - Ip t_n)}    */
/*                              <psi0^{(j)}| k_z |p_j(t_n), q_j(t_n)> ]   */
/* over trajectories with t_n >= t0_j.  Reading of the phase sign: the   */
/* bra <psi0 e^{i Ip t}| conjugates to e^{-i Ip t}.  Each trajectory     */
/* starts at grid point n0 with C = 1, S = 0, M = identity, contributes  */
/* at t_{n0}, then alternates one RK4 step and one contribution up to     */
/* t_{Nt-1}.  Optional filters (the paper is silent; both default off):  */
/* once |C| > cutoff (prefactor filter), or once the largest element of  */
/* the stability matrix exceeds stab_cutoff (stability filter: a chaotic */
/* trajectory), the trajectory contributes nothing from that step on.    */
/* The checks run in this order after each step: finiteness, |C|, |M|.   */
/* Tapered stability filter (stab_taper = r > 1; a reading, the paper is  */
/* silent): with Mhat_n the running maximum over steps k <= n of the     */
/* largest |M_ij(t_k)|, m0 = stab_cutoff and m1 = r m0, the contribution  */
/* at t_n is multiplied by g(Mhat_n) = 1 for Mhat <= m0,                   */
/* (1 + cos(pi x))/2 with x = ln(Mhat/m0)/ln r for m0 < Mhat < m1, and the */
/* trajectory stops (status 3) once Mhat >= m1.  The dipole is then a     */
/* continuous function of M, so a rounding-level change of M changes it   */
/* by a rounding-level amount (the hard filter, r = 0, can jump by a      */
/* whole step's contribution).                                            */
/* final_state (optional): per trajectory, field-major,                  */
/*   q[3] p[3] M[36] S C_re C_im theta status  (47 fields)                */
/* status: 0 ok, 1 prefactor-filtered, 2 non-finite, 3 stability-filtered.*/
/* ------------------------------------------------------------------ */
#define OR_NFINAL 47

/* First return (for the long/short trajectory analysis of Sec. III.D;    */
/* reading): the first grid step at which the electron is closer than     */
/* r_in to the molecular centre along the polarisation axis (|q_z| < r_in) */
/* after having been farther than r_out (|q_z| > r_out), and its kinetic  */
/* energy |p|^2/2 there.  returns[j] = step (-1: none), returns[n + j] =  */
/* energy.                                                                */
typedef struct {
    double r_out, r_in;
    double* returns;
} or_return_opts;

double or_stab_taper_weight(double Mhat, double m0, double r)
{
    if (Mhat <= m0) return 1.0;
    if (Mhat >= r * m0) return 0.0;
    return 0.5 * (1.0 + cos(OR_PI * log(Mhat / m0) / log(r)));
}

static void propagate_one(const or_target_in* T, const or_pulse* P, double Nnorm,
                          double gamma, double cutoff, double stab_cutoff, double stab_taper,
                          const double* soa, uint64_t n,
                          uint64_t j, double scale, double* vz, double* final_state,
                          const or_return_opts* ro)
{
    int left = 0, returned = 0;
    if (ro && ro->returns) {
        ro->returns[j] = -1.0;
        ro->returns[n + j] = 0.0;
    }
    int n0 = (int)soa[j];
    double nhat[3] = {soa[7 * n + j], soa[8 * n + j], soa[9 * n + j]};
    cplx w = soa[10 * n + j] + I * soa[11 * n + j];
    double y[OR_NY];
    for (int a = 0; a < 3; ++a) {
        y[a] = soa[(1 + a) * n + j];
        y[3 + a] = soa[(4 + a) * n + j];
    }
    for (int a = 0; a < 36; ++a) y[6 + a] = (a % 7 == 0) ? 1.0 : 0.0;
    y[42] = 0.0;
    double theta = 0.0, Mhat = 0.0;
    cplx det_prev = 1.0;
    cplx C = 1.0;
    int status = 0;
    for (int m = n0; m < P->nt; ++m) {
        double t = P->t_origin + m * P->dt;
        if (m > n0) {
            rk4_step(T, P, nhat, P->t_origin + (m - 1) * P->dt, P->dt, y);
            cplx det = hk_det(y + 6, gamma);
            theta += carg(det / det_prev);
            det_prev = det;
            C = sqrt(cabs(det)) * cexp(I * 0.5 * theta);
        }
        int finite = 1;
        for (int a = 0; a < OR_NY; ++a) if (!isfinite(y[a])) finite = 0;
        if (!finite) { status = 2; break; }
        if (cutoff > 0.0 && cabs(C) > cutoff) { status = 1; break; }
        double g = 1.0;
        if (stab_cutoff > 0.0) {
            double mmax = 0.0;
            for (int a = 0; a < 36; ++a) if (fabs(y[6 + a]) > mmax) mmax = fabs(y[6 + a]);
            if (stab_taper > 1.0) {
                if (mmax > Mhat) Mhat = mmax;
                if (Mhat >= stab_taper * stab_cutoff) { status = 3; break; }
                g = or_stab_taper_weight(Mhat, stab_cutoff, stab_taper);
            } else if (mmax > stab_cutoff) { status = 3; break; }
        }
        if (ro && ro->returns && !returned) {
            double az = fabs(y[2]);
            if (az > ro->r_out) left = 1;
            else if (left && az < ro->r_in) {
                returned = 1;
                ro->returns[j] = (double)m;
                ro->returns[n + j] = 0.5 * (y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
            }
        }
        cplx R = recomb(T, Nnorm, nhat, y, y + 3, gamma);
        cplx X = w * C * cexp(I * (y[42] - T->Ip * t)) * R;
        vz[m] += -2.0 * scale * g * creal(X);
    }
    if (final_state) {
        for (int a = 0; a < 42; ++a) final_state[(size_t)a * n + j] = y[a];
        final_state[(size_t)42 * n + j] = y[42];
        final_state[(size_t)43 * n + j] = creal(C);
        final_state[(size_t)44 * n + j] = cimag(C);
        final_state[(size_t)45 * n + j] = theta;
        final_state[(size_t)46 * n + j] = status;
    }
}

/* vz_out[nt] receives the dipole; n_norm is N of the 1/N normalisation
 * (0 -> n).  n_threads <= 0 uses all cores.  Returns the count of
 * trajectories that were filtered (either filter) or non-finite.        */
static int propagate_all(const or_target_in* T, const or_pulse_in* Pin, double gamma,
                         double cutoff, double stab_cutoff, double stab_taper, const double* soa,
                         uint64_t n, double n_norm, double* vz_out, double* final_state,
                         int n_threads, const or_return_opts* ro);

int or_propagate(const or_target_in* T, const or_pulse_in* Pin, double gamma, double cutoff,
                 double stab_cutoff, double stab_taper, const double* soa, uint64_t n,
                 double n_norm, double* vz_out, double* final_state, int n_threads)
{
    return propagate_all(T, Pin, gamma, cutoff, stab_cutoff, stab_taper, soa, n, n_norm, vz_out,
                         final_state, n_threads, NULL);
}

/* The same, also recording each trajectory's first return (returns: 2 x n). */
int or_propagate_returns(const or_target_in* T, const or_pulse_in* Pin, double gamma,
                         double cutoff, double stab_cutoff, const double* soa, uint64_t n,
                         double n_norm, double* vz_out, double r_out, double r_in,
                         double* returns, int n_threads)
{
    or_return_opts ro = {r_out, r_in, returns};
    return propagate_all(T, Pin, gamma, cutoff, stab_cutoff, 0.0, soa, n, n_norm, vz_out, NULL,
                         n_threads, &ro);
}

static int propagate_all(const or_target_in* T, const or_pulse_in* Pin, double gamma,
                         double cutoff, double stab_cutoff, double stab_taper, const double* soa,
                         uint64_t n, double n_norm, double* vz_out, double* final_state,
                         int n_threads, const or_return_opts* ro)
{
    or_pulse P = or_make_pulse(Pin);
    double Nnorm = orbital_norm(T);
    double scale = 1.0 / (n_norm > 0.0 ? n_norm : (double)n);
    for (int m = 0; m < P.nt; ++m) vz_out[m] = 0.0;
    int nthr = 1;
#ifdef _OPENMP
    nthr = (n_threads > 0) ? n_threads : omp_get_max_threads();
#endif
    double* part = (double*)calloc((size_t)nthr * P.nt, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
#endif
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        propagate_one(T, &P, Nnorm, gamma, cutoff, stab_cutoff, stab_taper, soa, n, (uint64_t)j,
                      scale, part + (size_t)tid * P.nt, final_state, ro);
    }
    for (int t = 0; t < nthr; ++t)
        for (int m = 0; m < P.nt; ++m) vz_out[m] += part[(size_t)t * P.nt + m];
    free(part);
    int bad = 0;
    if (final_state)
        for (uint64_t j = 0; j < n; ++j) bad += final_state[(size_t)46 * n + j] != 0.0;
    return bad;
}

/* ------------------------------------------------------------------ */
/* Spectrum (Eq. 3): v(omega) = sum_n v_z(t_n) W_H(t_n) e^{i omega t_n} dt */
/* with the Hann window W_H(t) = [1 + cos(pi t / tau_H)] / 2 (zero for   */
/* |t| > tau_H), yield = omega^2 |v(omega)|^2, phase = arg v(omega), on  */
/* omega_k = 2 pi k / (Nt dt), k = 0..n_out-1.  A naive DFT.              */
/* ------------------------------------------------------------------ */
void or_spectrum(const double* vz, int nt, double dt, double t_origin, double tau_H,
                 int n_out, double* omega, double* yield, double* phase, double* vre,
                 double* vim)
{
    for (int k = 0; k < n_out; ++k) {
        double w = 2.0 * OR_PI * k / (nt * dt);
        cplx acc = 0.0;
        for (int m = 0; m < nt; ++m) {
            double t = t_origin + m * dt;
            double win = (fabs(t) <= tau_H) ? 0.5 * (1.0 + cos(OR_PI * t / tau_H)) : 0.0;
            acc += vz[m] * win * cexp(I * w * t) * dt;
        }
        omega[k] = w;
        yield[k] = w * w * creal(acc * conj(acc));
        phase[k] = carg(acc);
        if (vre) vre[k] = creal(acc);
        if (vim) vim[k] = cimag(acc);
    }
}

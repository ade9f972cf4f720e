/*
 * sfhk.h -- C ABI of the B300 strong-field Herman-Kluk (SFHK) high-harmonic
 * library: Monte Carlo ensemble of classical trajectories launched at the
 * tunnel exit, propagated with their stability matrix, action and
 * Herman-Kluk prefactor through a two-centre molecular potential plus the
 * laser, and reduced on the GPU into the dipole velocity and its spectrum.
 *
 * Method: "Strong-field Herman-Kluk propagator method for high-harmonic
 * generation in molecules" (Tran, Truong, Goetz, Le).  Each entry point
 * cites the passage that defines what it computes.
 *
 * Conventions for every call
 *   - Return value: SFHK_OK (0) or a negative SFHK_E_* code;
 *     sfhk_strerror() gives its text.  On error no output is written and no
 *     handle is created; a handle passed in stays valid.
 *   - Atomic units throughout (time, length, momentum, energy); the laser is
 *     linearly polarised along z, time is centred on the pulse
 *     (t in [-Tp/2, Tp/2]) and sampled on t_n = -Tp/2 + n dt, n = 0..Nt-1,
 *     Nt = floor(Tp/dt) + 1.
 *   - Ownership: the library owns all device memory and all handles (freed by
 *     the matching sfhk_destroy_*); the caller owns every host buffer and
 *     passes its size explicitly.  Host pointers are only read or written
 *     during the call.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls that take a stream enqueue their device work on
 *     it and return without waiting unless stated otherwise.
 *   - A context is not thread-safe; use one per host thread, or the server
 *     (sfhk_server_*), which serialises its own calls.
 *   - There is no CPU fallback: every computing call needs a CUDA device with
 *     compute capability 10.3 and fails with SFHK_E_CUDA otherwise.
 */
#ifndef SFHK_H
#define SFHK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SFHK_API __attribute__((visibility("default")))
#else
#define SFHK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define SFHK_OK           0
#define SFHK_E_INVAL     -1  /* bad argument, size or descriptor            */
#define SFHK_E_NOMEM     -2  /* device-memory budget or allocation exceeded */
#define SFHK_E_CUDA      -3  /* CUDA runtime error or no suitable device    */
#define SFHK_E_TIMEOUT   -4  /* a bounded wait expired                      */
#define SFHK_E_NUMERIC   -5  /* non-finite trajectories above the limit     */
#define SFHK_E_BUSY      -6  /* result not ready yet                        */
#define SFHK_E_NOTFOUND  -7  /* unknown request id                          */
#define SFHK_E_CANCELLED -8  /* the request was cancelled                   */

#define SFHK_MAX_PRIM     8  /* Gaussian primitives per centre (diatomic) or */
                             /* in all (polyatomic)                          */
#define SFHK_MAX_CENTRES  8  /* centres of a polyatomic target               */

/* ---------------------------------------------------------------- handles */
typedef struct sfhk_ctx sfhk_ctx;
typedef struct sfhk_target sfhk_target;
typedef struct sfhk_pulse sfhk_pulse;
typedef struct sfhk_ensemble sfhk_ensemble;
typedef struct sfhk_server sfhk_server;

/* ---------------------------------------------------------------- descriptors */
enum { SFHK_POT_MOLECULE = 0, SFHK_POT_HARMONIC = 1, SFHK_POT_POLYATOMIC = 2 };
enum { SFHK_ALIGN_FIXED = 0, SFHK_ALIGN_ISOTROPIC = 1, SFHK_ALIGN_COS2 = 2,
       SFHK_ALIGN_QUADRATURE = 3 };
#define SFHK_MAX_QUAD_NODES 64
enum { SFHK_FP64 = 0, SFHK_MIXED = 1 };

/* Target (Eq. 7, Tables I-II): two centres at +-(R/2) n, n the molecular axis,
 * V(r) = -sum_i [Z_inf + (Z0 - Z_inf) exp(-alpha s_i)] / s_i with the softened
 * distance s_i = sqrt(|r - R_i|^2 + soft_a^2).  The initial orbital is the
 * sigma_g combination  N sum_centres sum_k prim_coef[k] exp(-prim_exp[k] |r-R_c|^2)
 * (normalised by the library).  kind = SFHK_POT_HARMONIC replaces V by the
 * test potential ho_omega^2 |r|^2 / 2 (closed-form checks).
 * kind = SFHK_POT_POLYATOMIC is the N-centre generalisation of Eq. 7 (the
 * potential summed over the centres): n_centres centres at the
 * molecular-frame positions centre_pos (bohr), each with its own
 * centre_Z_inf, centre_Z0, centre_alpha, the common softening soft_a, and
 * the molecule turned by the ZYZ Euler angles (phi, theta, psi) of each
 * trajectory, Rot = Rz(phi) Ry(theta) Rz(psi), lab position = Rot x (the
 * molecular z axis goes to n(theta, phi), as for a diatomic).  The orbital
 * is N sum_k prim_coef[k] f_k exp(-prim_exp[k] |r - R_{c_k}|^2) with each
 * primitive on its own centre c_k = prim_centre[k]: f = 1 (SFHK_PRIM_S) or
 * f = u.(r - R_c) (SFHK_PRIM_P_DIR) with u = Rot d/|d|, d = prim_dir[k]
 * given in the molecular frame.  R, Z_inf, Z0, alpha, the sigma/pi kinds
 * and pi_azimuth are not used; ionization must be SFHK_IONIZE_SFA.
 * ionization selects the ionization step of the sampler: SFHK_IONIZE_SFA is
 * the saddle point of Eq. 2 (SFHK1); SFHK_IONIZE_MODIFIED is SFHK2
 * (Sec. III.D): each trajectory leaves from one centre, eta = +1 (the centre
 * at -(R/2) n) or -1 (at +(R/2) n) with probability 1/2 each and weight x 2,
 * through the saddle [k + A(t_s) - A(t0)]^2/2 + Ip - eta E(t_s).(R/2) n = 0,
 * with that centre's part of the dipole element and the Gaussian-integration
 * factor 1/sqrt(E(t_s) kappa_z + eta (R/2) n_z dE/dt(t_s)).
 * sampling selects how the initial points are drawn: SFHK_SAMPLE_PROPOSAL
 * draws them from the ADK-time x Gaussian-k_perp x alignment proposal with
 * weight w = a/pdf; SFHK_SAMPLE_ABS_AMPLITUDE distributes them ~ |a|
 * (Sec. II.B) by exact rejection with weight correction on that proposal: a
 * draw is kept with probability alpha = min(1, |w|/M) and weighs
 * P w / (alpha (1 - (1-P)^256)), M = sampling_factor x mean |w| and P = mean
 * alpha from a pilot of 16384 draws; a trajectory not accepted within 256
 * draws gets weight 0 (it happens with probability (1-P)^256, which the
 * factor 1/(1 - (1-P)^256) of the kept weights makes up for), so every
 * weighted mean stays unbiased for any factor.  Larger factors give more
 * nearly equal weights (lower variance per propagated trajectory) at about
 * 1/P proposal draws per point.
 * prim_kind[k] selects the angular part of primitive k: SFHK_PRIM_S is the
 * s-type exp(-a |r-R_c|^2); SFHK_PRIM_P_SIGMA is the sigma p-type
 * s_c n.(r-R_c) exp(-a |r-R_c|^2), s_c = +1 at +(R/2) n and -1 at -(R/2) n,
 * so that every primitive stays gerade (the 2p_sigma character of the N2
 * 3 sigma_g orbital, Sec. III.B); SFHK_PRIM_P_PI is the pi p-type
 * m.(r-R_c) exp(-a |r-R_c|^2) with the same sign on both centres (the N2
 * HOMO-1 1 pi_u of Table II, ungerade), m the unit vector perpendicular to n
 * at azimuth pi_azimuth about n: m = cos(chi) theta_hat + sin(chi) phi_hat,
 * theta_hat = (cos th cos ph, cos th sin ph, -sin th), phi_hat =
 * (-sin ph, cos ph, 0) for n = (sin th cos ph, sin th sin ph, cos th) (ph = 0
 * on the z axis); chi = 0 puts the lobe in the plane of n and the
 * polarisation axis.  The normalisation, the dipole element of the sampler
 * and the recombination element take the p-type factor in closed form.
 * Errors: SFHK_E_INVAL for any other kind, a non-finite pi_azimuth, or an
 * orbital of zero norm. */
enum { SFHK_IONIZE_SFA = 0, SFHK_IONIZE_MODIFIED = 1 };
enum { SFHK_PRIM_S = 0, SFHK_PRIM_P_SIGMA = 1, SFHK_PRIM_P_PI = 2, SFHK_PRIM_P_DIR = 3 };
enum { SFHK_SAMPLE_PROPOSAL = 0, SFHK_SAMPLE_ABS_AMPLITUDE = 1 };
typedef struct {
    int kind;
    int n_prim;                       /* 1..SFHK_MAX_PRIM */
    double R, Z_inf, Z0, alpha, soft_a;
    double Ip;                        /* ionization potential (> 0 for sampling) */
    double ho_omega;
    double prim_exp[SFHK_MAX_PRIM];   /* > 0 */
    double prim_coef[SFHK_MAX_PRIM];
    int ionization;                   /* SFHK_IONIZE_SFA or SFHK_IONIZE_MODIFIED */
    int sampling;                     /* SFHK_SAMPLE_PROPOSAL or SFHK_SAMPLE_ABS_AMPLITUDE */
    double sampling_factor;           /* kappa of the |a| sampler (<= 0: 5) */
    int prim_kind[SFHK_MAX_PRIM];     /* SFHK_PRIM_S, _P_SIGMA or _P_PI */
    double pi_azimuth;                /* chi of the SFHK_PRIM_P_PI lobe (rad) */
    /* SFHK_POT_POLYATOMIC only */
    int n_centres;                                /* 1..SFHK_MAX_CENTRES */
    double centre_pos[SFHK_MAX_CENTRES][3];       /* molecular frame, bohr */
    double centre_Z_inf[SFHK_MAX_CENTRES], centre_Z0[SFHK_MAX_CENTRES];
    double centre_alpha[SFHK_MAX_CENTRES];        /* >= 0 */
    int prim_centre[SFHK_MAX_PRIM];               /* 0..n_centres-1 */
    double prim_dir[SFHK_MAX_PRIM][3];            /* SFHK_PRIM_P_DIR: nonzero */
} sfhk_target_desc;

/* Pulse (Sec. II.D / III.A): wavelength (nm), peak intensity (W/cm^2),
 * number of cycles of the sin^2 envelope, CEP (rad), time step (a.u.).
 * omega = 45.5633525/lambda_nm, E0 = sqrt(I/3.50944758e16),
 * Tp = n_cycles 2 pi / omega, A(t) = -(E0/omega) cos^2(pi t/Tp) sin(omega t + cep),
 * E = -dA/dt.  n_cycles >= 1.5. */
typedef struct {
    double lambda_nm, intensity_Wcm2, n_cycles, cep, dt;
} sfhk_pulse_desc;

/* Orientation distribution (Eqs. 5-6): FIXED axis n(theta, phi); ISOTROPIC
 * (the joint Monte Carlo over the axis of Eq. 6, one axis per trajectory);
 * COS2 = axis density proportional to cos^2 theta (<cos^2> = 3/5);
 * QUADRATURE = the isotropic average done as Eq. 5 with n_nodes fixed
 * angles: trajectory j sits at cos theta = x_{j mod K}, the K-node
 * Gauss-Legendre rule on [0, 1] with nodes in descending x (by the
 * cylindrical and inversion symmetry of a homonuclear diatomic in a linearly
 * polarised field the average over the axis is int_0^1 f(arccos x) dx), phi
 * uniform, and its weight is multiplied by K W_{j mod K} (weights summing to
 * 1), so that the ensemble dipole is sum_k W_k <v_z>_k.
 * Polyatomic targets take the full orientation, the Euler angles
 * (phi, theta, psi): FIXED uses psi below; ISOTROPIC and COS2 draw psi
 * uniform in [0, 2 pi) (the Haar measure for ISOTROPIC); QUADRATURE is
 * refused (SFHK_E_INVAL), as it rests on the diatomic's symmetry. */
typedef struct {
    int kind;
    double theta, phi;                /* radians, FIXED only */
    int n_nodes;                      /* QUADRATURE only: 1..SFHK_MAX_QUAD_NODES */
    double psi;                       /* radians, FIXED polyatomic only */
} sfhk_align_desc;

/* Propagation options.
 *   precision        SFHK_FP64: every step in double precision.
 *                    SFHK_MIXED: position, momentum and stability matrix in
 *                    single precision with compensated (two-float) state
 *                    updates; action, phase reduction, prefactor branch and
 *                    the dipole reduction in two-float / double.
 *   gamma            coherent-state width (Sec. II.A; the paper uses 1).
 *   prefactor_cutoff 0 = off; else a trajectory stops contributing from the
 *                    first step with |C| > cutoff (the paper is silent).
 *   dump_final       keep each trajectory's final state for sfhk_final_state.
 *   block_threads    threads per block of the integrator (32, 64 or 128);
 *                    0 = the context's tuned choice (see sfhk_autotune).
 *   blocks_per_sm    resident blocks per SM to launch; 0 = as many as fit.
 *   stability_cutoff 0 = off; else a trajectory stops contributing from the
 *                    first step at which the largest element of its
 *                    stability matrix exceeds the cutoff (chaotic
 *                    trajectories; the paper is silent).
 * The per-step checks run in the order: finiteness, prefactor, stability.
 */
typedef struct {
    int precision;
    double gamma;
    double prefactor_cutoff;
    int dump_final;
    int block_threads;
    int blocks_per_sm;
    double stability_cutoff;
    int kernel_variant;               /* register-cap variant 1..6 (no cap, then at
                                         most 168, 152, 144, 136, 128 registers per
                                         thread); 0 = the context's tuned choice */
    int record_returns;               /* keep each trajectory's first return for
                                         sfhk_returns (long/short trajectories,
                                         Sec. III.D) */
    double return_r_out, return_r_in; /* the return: first step with |q_z| <
                                         r_in after one with |q_z| > r_out
                                         (0 < r_in < r_out) */
    double stability_taper;           /* 0: the stability filter is a hard cut.
                                         r > 1: a taper (a reading, the paper
                                         is silent): with Mhat the running
                                         maximum of max |M_ij| over the steps so
                                         far and m0 = stability_cutoff, each
                                         contribution is weighted by 1 for
                                         Mhat <= m0, (1 + cos(pi x))/2 with
                                         x = ln(Mhat/m0)/ln r up to r m0, and
                                         the trajectory stops once Mhat >= r m0.
                                         The dipole is then continuous in M, so
                                         FP32 rounding of M moves it by a
                                         rounding-level amount instead of a
                                         whole step's contribution. */
    int check_nonfinite;              /* 1: the synchronising calls on the
                                         ensemble (sfhk_dipole, sfhk_stats_get)
                                         return SFHK_E_NUMERIC when more than
                                         max_nonfinite trajectories stopped on a
                                         non-finite state or prefactor; 0 (the
                                         default): no limit, the count is only
                                         reported.  A non-finite trajectory
                                         stops contributing at that step either
                                         way, so the dipole itself stays finite;
                                         the limit tells a caller that the
                                         estimate lost more trajectories to
                                         overflow than it accepts. */
    uint64_t max_nonfinite;           /* the count tolerated when checking */
} sfhk_run_opts;

/* Per-ensemble counters of the last propagation. */
typedef struct {
    uint64_t n_traj;          /* trajectories in the ensemble                 */
    uint64_t n_invalid;       /* saddle without root: weight 0                */
    uint64_t n_filtered;      /* stopped by the prefactor filter              */
    uint64_t n_nonfinite;     /* stopped on a non-finite state or prefactor   */
    uint64_t n_unstable;      /* stopped by the stability filter              */
    uint64_t traj_steps;      /* RK4 steps actually integrated                */
    int nt;                   /* time-grid length                             */
    float kernel_ms;          /* duration of the propagation kernel (events)  */
    uint64_t recomb_evals;    /* trajectory-steps at which the recombination  */
                              /* element was evaluated (its Gaussian overlaps */
                              /* above e^-30 of their peak in FP32, e^-200 in */
                              /* FP64) and the contribution formed; the other */
                              /* steps contribute zero without that work      */
    int fixed_params;         /* 1: the launch ran the integrator compiled    */
                              /* with the method's dt = 0.05, gamma = 0.5 and */
                              /* the filters |C| <= 1e4, stability taper      */
                              /* 1e3..2e3 as constants (mixed precision,      */
                              /* molecular diatomic or three-centre targets,  */
                              /* the diatomic potential's screening compiled  */
                              /* in too when all instances agree; chosen when */
                              /* every instance of the launch has exactly     */
                              /* these values and no first returns are        */
                              /* recorded)                                    */
} sfhk_stats;

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device` that may hold at most
 * `device_mem_budget` bytes of library allocations (0 = no limit).
 * Errors: SFHK_E_INVAL (null out), SFHK_E_CUDA (no such device, or not
 * compute capability 10.3). */
SFHK_API int sfhk_create(sfhk_ctx** out, int device, size_t device_mem_budget);
SFHK_API int sfhk_destroy(sfhk_ctx* ctx);
/* Bytes of device memory the context holds now. */
SFHK_API int sfhk_mem_used(const sfhk_ctx* ctx, size_t* bytes);

/* Target descriptor -> device-resident target (Eq. 7, Tables I-II, Sec. II.A
 * GTO expansion).  Errors: SFHK_E_INVAL (n_prim outside 1..8, non-positive
 * exponent, negative softening, unknown kind). */
SFHK_API int sfhk_create_target(sfhk_ctx* ctx, const sfhk_target_desc* desc, sfhk_target** out);
SFHK_API int sfhk_destroy_target(sfhk_target* t);

/* Pulse descriptor -> device tables of E(t) at every half step and the time
 * grid (Sec. III.A laser; Eq. 3 window uses tau_H = Tp/2).  Runs a kernel
 * on the legacy default stream and waits for it.
 * Errors: SFHK_E_INVAL (non-positive lambda/dt, n_cycles < 1.5, negative
 * intensity, more than 2^26 steps). */
SFHK_API int sfhk_set_pulse(sfhk_ctx* ctx, const sfhk_pulse_desc* desc, sfhk_pulse** out);
SFHK_API int sfhk_destroy_pulse(sfhk_pulse* p);
/* Time grid of a pulse: Nt, t_0 = -Tp/2, dt, Tp (any output may be NULL). */
SFHK_API int sfhk_pulse_grid(const sfhk_pulse* p, int* nt, double* t_origin, double* dt, double* Tp);

/* Initial ensemble (Sec. II.A, Eqs. 1-2, 6), sampled on the device:
 * t0 on the time grid with probability p_n proportional to
 * exp(-2 (2 Ip)^{3/2} / (3 |E(t_n)|)), k_x, k_y ~ N(0, |E(t0)| / (2 sqrt(2 Ip))),
 * the molecular axis from `align`; then per trajectory the saddle point
 * t_s = t0 + i t_t of Eq. 2 (smallest positive root), k_z, the tunnel exit
 * q0 = Re int_{t_s}^{t0} A, the tunnelling action S_down, the amplitude
 * a = <kappa| z E(t_s) |psi0> / sqrt(E(t_s) kappa_z) e^{i(S_down + k.q0)}
 * and the weight w = a / pdf.  Random numbers: Philox4x32-10 with key = seed
 * and counter (j, instance, draw), so every trajectory is reproducible on its
 * own.  Trajectories whose saddle has no root get w = 0.  The ensemble keeps
 * references to `target` and `pulse`, which must outlive it.
 * Errors: SFHK_E_INVAL (n_traj = 0 or > 2^31-1, Ip <= 0, zero field),
 * SFHK_E_NOMEM. */
SFHK_API int sfhk_sample_initial(sfhk_ctx* ctx, const sfhk_target* target, const sfhk_pulse* pulse,
                        const sfhk_align_desc* align, uint64_t n_traj, uint64_t seed,
                        uint32_t instance, sfhk_ensemble** out, void* stream);

/* Re-draw the initial points of an existing sampled ensemble in place (same
 * target, pulse and size; new alignment, seed and instance), reusing its
 * device buffers: no allocation, asynchronous on `stream`.  Same method and
 * errors as sfhk_sample_initial. */
SFHK_API int sfhk_sample_into(sfhk_ctx* ctx, sfhk_ensemble* e, const sfhk_align_desc* align,
                              uint64_t seed, uint32_t instance, void* stream);

/* Ensemble from caller-given initial points (tests, external samplers).
 * soa_host: 12 x n_traj doubles, field-major (soa[f * n_traj + j]):
 *   0 grid index n0 of t0 (integer valued, 0..Nt-1) | 1-3 q0 | 4-6 p0 |
 *   7-9 molecular axis n (unit; for a polyatomic target the Euler angles
 *   phi, theta, psi) | 10-11 weight w (re, im).
 * n_norm: N of the 1/N normalisation of the dipole (0 = n_traj).
 * Errors: SFHK_E_INVAL (n0 out of range, non-finite entries), SFHK_E_NOMEM. */
SFHK_API int sfhk_load_ensemble(sfhk_ctx* ctx, const sfhk_target* target, const sfhk_pulse* pulse,
                       const double* soa_host, uint64_t n_traj, double n_norm,
                       sfhk_ensemble** out);
/* Copy the initial points (same 12-field layout) to the host; synchronous. */
SFHK_API int sfhk_ensemble_read(sfhk_ensemble* e, double* soa_host, uint64_t n_traj);
SFHK_API int sfhk_destroy_ensemble(sfhk_ensemble* e);

/* Continuum propagation and dipole (Sec. II.A, Eq. 4): every trajectory runs
 * from its grid point n0 to Nt-1 with RK4 through Hamilton's equations in
 * V + z E(t), with its 6x6 stability matrix, action S = int (p.qdot - H) and
 * prefactor C = sqrt(det[(M_qq + M_pp - i gamma M_qp + (i/gamma) M_pq)/2])
 * on a continuous branch; the GPU reduces
 *   v_z(t_n) = -(2/N) sum_j Re[w_j C_j e^{i(S_j - Ip t_n)} <psi0^{(j)}|k_z|p_j,q_j>]
 * over trajectories with n >= n0_j, without writing any per-trajectory time
 * series.  Overwrites the ensemble's dipole accumulator.  Asynchronous.
 * Errors: SFHK_E_INVAL (gamma <= 0, bad precision), SFHK_E_NOMEM (dump). */
SFHK_API int sfhk_propagate(sfhk_ctx* ctx, sfhk_ensemble* e, const sfhk_run_opts* opts, void* stream);

/* The same for several ensembles (any mix of targets, pulses, sizes and
 * alignments) in ONE persistent launch: the warps pull work items of 32
 * trajectories, longest first, from a shared queue; each ensemble gets its
 * own dipole.  Asynchronous. */
SFHK_API int sfhk_propagate_batch(sfhk_ctx* ctx, sfhk_ensemble* const* ens, int n_ens,
                         const sfhk_run_opts* opts, void* stream);

/* A prepared batch: the instance table and the work-item buffers of a fixed
 * set of ensembles, built once, so that each launch only enqueues device
 * work (zeroing the dipoles, rebuilding and sorting the work items from the
 * ensembles' current samples, one persistent propagation launch) -- no host
 * synchronisation, allocation or host-to-device copy.  A step made of
 * sfhk_sample_into, sfhk_batch_launch and the device-pointer sfhk_spectrum can
 * therefore be captured once in a CUDA graph and replayed.  The ensembles must
 * outlive the batch and keep their sizes; opts are fixed at creation
 * (dump_final is ignored).  Errors: as sfhk_propagate_batch. */
typedef struct sfhk_batch sfhk_batch;
SFHK_API int sfhk_batch_create(sfhk_ctx* ctx, sfhk_ensemble* const* ens, int n_ens,
                               const sfhk_run_opts* opts, sfhk_batch** out);
SFHK_API int sfhk_batch_launch(sfhk_batch* b, void* stream);
SFHK_API int sfhk_batch_destroy(sfhk_batch* b);

/* Autotuner of the integrator's launch shape (block size x register-cap
 * variant), run on the caller's ensemble: every candidate propagates the
 * first `max_items` work items of 32 trajectories (0 = all) twice, the second
 * launch is timed with CUDA events, and the fastest becomes the context's
 * default for `opts->precision` (used whenever block_threads or
 * kernel_variant is 0).  choice (may be NULL) receives
 * {block_threads, kernel_variant, register cap of that variant (0 = none)}.
 * Synchronous, on the legacy default stream; the ensemble's dipole is
 * overwritten.  Not a method step: launch configuration only. */
SFHK_API int sfhk_autotune(sfhk_ctx* ctx, sfhk_ensemble* e, const sfhk_run_opts* opts,
                           int max_items, int* choice);

/* Dipole v_z(t_n), n = 0..Nt-1, of the last propagation, copied to the host
 * after waiting for it.  nt must equal the pulse's Nt.  Also returns the
 * grid origin and step (either may be NULL).  Errors: SFHK_E_INVAL;
 * SFHK_E_NUMERIC (nothing written) when that propagation ran with
 * check_nonfinite and more than max_nonfinite trajectories went non-finite.
 * sfhk_propagate itself is asynchronous and cannot see the count; the check
 * happens here and in sfhk_stats_get. */
SFHK_API int sfhk_dipole(sfhk_ctx* ctx, sfhk_ensemble* e, double* vz_host, size_t nt,
                double* t_origin, double* dt);
/* Device pointer of the same dipole (valid until the ensemble is destroyed or
 * propagated again). */
SFHK_API int sfhk_dipole_device(sfhk_ensemble* e, const double** vz_dev, size_t* nt);
/* Counters of the last propagation (waits for it).  Returns SFHK_E_NUMERIC
 * under the same condition as sfhk_dipole, and in that case, unlike other
 * errors, still fills *out, so that the caller sees the counts. */
SFHK_API int sfhk_stats_get(sfhk_ensemble* e, sfhk_stats* out);
/* Final per-trajectory state of the last propagation run with dump_final,
 * 47 x n_traj doubles, field-major: q[3] p[3] M[36] (6x6 row-major,
 * M_ab = d a_t / d b_0 for (q,p)) S C_re C_im n_state status, where n_state is
 * the time index of the stored state and status is 0 ok, 1 prefactor-filtered,
 * 2 non-finite, 3 stability-filtered.  For a stopped trajectory the state is the
 * one at the step where it stopped (n_state = that step).  Synchronous.
 * Errors: SFHK_E_INVAL (no dump taken). */
SFHK_API int sfhk_final_state(sfhk_ensemble* e, double* host, uint64_t n_traj);

/* First returns of the last propagation run with record_returns: 2 x n_traj
 * doubles, host[j] = the grid step of trajectory j's first return (-1: none),
 * host[n_traj + j] = its kinetic energy |p|^2/2 there.  The return is the
 * first step at which the electron is closer than r_in to the molecular
 * centre along the polarisation axis (|q_z| < r_in) after one with
 * |q_z| > r_out, while the trajectory is alive (not filtered).  Histograms of
 * birth step against return step separate the long and short trajectories of
 * Sec. III.D.  Synchronous.  Errors: SFHK_E_INVAL (not recorded, wrong n). */
SFHK_API int sfhk_returns(sfhk_ensemble* e, double* host, uint64_t n_traj);

/* Spectrum (Eq. 3): v(omega_k) = sum_n v_z(t_n) W_H(t_n) e^{i omega_k t_n} dt,
 * W_H(t) = [1 + cos(pi t / tau_H)]/2 for |t| <= tau_H (else 0),
 * omega_k = 2 pi k / (Nt dt), k = 0..n_out-1; yield = omega^2 |v|^2,
 * phase = arg v.  Computed by a DFT kernel on the GPU.  device_ptrs = 0: all
 * arrays are host memory and the call is synchronous; 1: all are device
 * memory and the call is asynchronous on `stream`.  Any output may be NULL.
 * Errors: SFHK_E_INVAL (nt < 2, n_out > nt, dt <= 0). */
SFHK_API int sfhk_spectrum(const double* vz, size_t nt, double dt, double t_origin, double tau_H,
                  double* omega_out, double* yield_out, double* phase_out, size_t n_out,
                  int device_ptrs, void* stream);

/* Gabor time-frequency map of the dipole velocity (the analysis of Sec. III.D):
 *   G(t_m, w_k) = | sum_n v_z(t_n) exp(-(t_n - t_m)^2 / (2 sigma^2)) e^{i w_k t_n} dt |^2,
 * t_n = t_origin + n dt (n < nt), t_m = t_first + m t_step (m < n_t),
 * w_k = omega_first + k omega_step (k < n_w); out[m * n_w + k].  Samples with
 * |t_n - t_m| > 8.6 sigma (window factor below 1e-16) are skipped.  The paper
 * does not give sigma; 1/(3 omega_0) is the usual choice.  device_ptrs = 1:
 * vz and out are device pointers and the call is asynchronous on `stream`;
 * 0: host buffers, synchronous.  FP64.
 * Errors: SFHK_E_INVAL (null pointer, nt, n_t or n_w = 0 or too large,
 * dt <= 0, sigma <= 0, a non-finite argument), SFHK_E_CUDA. */
SFHK_API int sfhk_gabor(const double* vz, size_t nt, double dt, double t_origin, double sigma,
                        double t_first, double t_step, size_t n_t, double omega_first,
                        double omega_step, size_t n_w, double* out, int device_ptrs,
                        void* stream);

/* ---------------------------------------------------------------- serving */
/* A spectrum server with continuous batching (not in the paper, which runs
 * its trajectories as independent CPU jobs).  A host thread owned by the
 * server admits submitted requests (one target, pulse, alignment and
 * trajectory count each) in arrival order while its device-memory budget,
 * its instance slots, its work rings and its admission horizon have room,
 * samples each admitted request on the device, and appends its work items
 * (32 trajectories, longest first) to a device ring: one for diatomic
 * targets, one for polyatomic ones.  The GPU runs the integrator as a
 * sequence of persistent slices over those rings (each slice launches the
 * diatomic and then the polyatomic integrator over the rings that have
 * work): once `slice_ms` has passed, a warp takes no new item and parks the
 * one it runs at its next 32-step chunk boundary (the state of its
 * trajectories goes to a device buffer; the next slice resumes parked items
 * before it takes new ones, with the same arithmetic), so a slice ends
 * within one chunk of its deadline, and every request that arrived
 * meanwhile joins the next slice, so the work of
 * requests of different sizes, targets and pulses runs on the device
 * together.  A request is done when all its items are; the server then
 * copies its dipole (and spectrum) to host memory and frees its device state,
 * which admits the next requests.  No kernel ever waits on another thread.
 * The server owns its own context on `device`; all calls are thread-safe. */
typedef struct {
    size_t device_mem_budget;   /* bytes of device state it may hold (0 = no limit) */
    int max_pending;            /* queued, not yet admitted requests (0 = 4096)     */
    int max_active;             /* requests resident at once (0 = 512)              */
    int precision;              /* SFHK_FP64 | SFHK_MIXED                          */
    double gamma, prefactor_cutoff, stability_cutoff;   /* as in sfhk_run_opts     */
    double slice_ms;            /* slice length (0 = 50 ms)                         */
    int spectrum;               /* also compute yield and phase of each result      */
    int fifo;                   /* 1: work items in arrival order; 0 (default): a
                                   request whose work (items x Nt) is smaller than
                                   the work still queued goes to the front of the
                                   ring, so short requests overtake long ones      */
    double stability_taper;     /* as in sfhk_run_opts                              */
    int check_nonfinite;        /* as in sfhk_run_opts, per request: a request     */
    uint64_t max_nonfinite;     /* with more non-finite trajectories ends with     */
                                /* status SFHK_E_NUMERIC and no dipole             */
    double max_reorder_s;       /* age limit of short-first (0 = none): while an   */
                                /* admitted request of the same kind (diatomic or  */
                                /* polyatomic) has waited longer than this since   */
                                /* its admission, new requests go to the tail, so  */
                                /* that under overload the largest requests are    */
                                /* not overtaken without bound                     */
    double max_queued_s;        /* admission horizon (0 = none): a request is      */
                                /* admitted only while the work queued on its ring */
                                /* is below this many seconds at the rate the      */
                                /* server measured over its last slices (any       */
                                /* request is admitted before the first slice, and */
                                /* into an empty ring); the rest wait in the       */
                                /* pending queue, bounded by max_pending, so that  */
                                /* under overload latency stays near the horizon   */
                                /* plus the pending queue's wait instead of the    */
                                /* whole resident backlog                          */
} sfhk_server_opts;

typedef struct {
    sfhk_target_desc target;
    sfhk_pulse_desc pulse;
    sfhk_align_desc align;
    uint64_t n_traj, seed;
    uint32_t instance;          /* Philox counter word: the same (seed, instance)
                                   gives the same ensemble as sfhk_sample_initial */
} sfhk_request;

/* Result of a finished request.  The caller sets vz / yield / phase (host
 * buffers, may be NULL) and their capacities; sfhk_poll / sfhk_wait fill them
 * (vz: nt values; yield, phase: n_out = nt/2 values; truncated to capacity)
 * and every other field.  Times are seconds on the server's clock. */
typedef struct {
    int status;                 /* SFHK_OK, SFHK_E_CANCELLED or the failing code */
    int nt;
    double t_origin, dt;
    size_t n_out;
    double* vz;
    size_t vz_capacity;
    double* yield;
    double* phase;
    size_t spec_capacity;
    double t_submit, t_admit, t_done;
    uint64_t traj_steps, n_filtered, n_unstable;
    uint64_t n_nonfinite;       /* trajectories stopped on a non-finite state      */
    uint64_t recomb_evals;      /* as sfhk_stats.recomb_evals, for the request     */
} sfhk_result;

typedef struct {
    uint64_t submitted, completed, rejected, cancelled, failed, slices;
    uint64_t traj_steps;
    int pending, active;
    double gpu_busy_s, uptime_s;
    uint64_t device_bytes;      /* device memory the server holds now */
    uint64_t parked;            /* work items a slice stopped at a chunk boundary */
                                /* when its time was up (the next slice resumes   */
                                /* them), counted each time                       */
} sfhk_server_stats;

/* Errors: SFHK_E_INVAL (bad options), SFHK_E_CUDA (device). */
SFHK_API int sfhk_server_create(int device, const sfhk_server_opts* opts, sfhk_server** out);
/* Stops the server thread after its current slice; unfinished requests are dropped. */
SFHK_API int sfhk_server_destroy(sfhk_server* s);
/* Queue a request; returns at once with its id.  Diatomic and polyatomic
 * targets are both served: their work items go to two device rings, and each
 * slice runs the diatomic and the polyatomic integrator in turn over them.
 * Errors: SFHK_E_INVAL (bad descriptor; for a polyatomic target also a
 * quadrature alignment or the modified saddle, which rest on the diatomic's
 * symmetry), SFHK_E_NOMEM (admission refused: the queue is full, or the
 * request alone needs more than the device-memory budget). */
SFHK_API int sfhk_submit(sfhk_server* s, const sfhk_request* req, uint64_t* req_id);
/* SFHK_E_BUSY while the request is queued or running; once it has ended,
 * fills *result, forgets the request and returns SFHK_OK (result->status says
 * how it ended).  SFHK_E_NOTFOUND for an unknown (or already polled) id. */
SFHK_API int sfhk_poll(sfhk_server* s, uint64_t req_id, sfhk_result* result);
/* As sfhk_poll, but blocks up to timeout_s seconds; SFHK_E_TIMEOUT if it has
 * not ended by then. */
SFHK_API int sfhk_wait(sfhk_server* s, uint64_t req_id, double timeout_s, sfhk_result* result);
/* Cancel a queued or running request (a running one stops at its next work
 * items).  SFHK_E_NOTFOUND if unknown or already ended. */
SFHK_API int sfhk_cancel(sfhk_server* s, uint64_t req_id);
SFHK_API int sfhk_server_stats_get(sfhk_server* s, sfhk_server_stats* out);

/* Spectrum without allocation.  No counterpart in the paper: a variant of
 * sfhk_spectrum with device pointers for callers that must not allocate
 * device memory during the call -- for instance a latency-bound serving loop
 * that cannot take the device synchronisation an allocation may cause, or a
 * process whose device memory is reserved up front by another framework's
 * caching allocator.  Same computation and outputs as sfhk_spectrum
 * (device_ptrs = 1); the caller passes device buffers for vz (nt doubles) and
 * for every output it wants (n_out doubles each; NULL skips one).
 * Scratch: a fixed file-scope device array of SFHK_NOALLOC_MAX_NT x 24 bytes
 * (768 KiB), held on every GPU that loads the library until the process
 * exits.  Every call looks up that array's device address on the current
 * device (cudaGetSymbolAddress, which allocates nothing), so an address is
 * never reused across a reset of the device's context; the first call on a
 * device may also load the library's device code there, so make that first
 * call before any stream capture.  It calls no allocator.  Every call
 * shares the one array, so calls that overlap on the GPU (different
 * streams, or other host threads) race on it; serialise them.  Each call
 * overwrites all the scratch it reads, so no state carries over.
 * Asynchronous on `stream`.  Errors: SFHK_E_INVAL (nt < 2,
 * nt > SFHK_NOALLOC_MAX_NT, n_out = 0 or > nt, dt or tau_H <= 0),
 * SFHK_E_CUDA. */
#define SFHK_NOALLOC_MAX_NT 32768
SFHK_API int sfhk_spectrum_noalloc(const double* vz_dev, size_t nt, double dt, double t_origin,
                                   double tau_H, double* omega_dev, double* yield_dev,
                                   double* phase_dev, size_t n_out, void* stream);

SFHK_API const char* sfhk_strerror(int code);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts).  For accounting of launches in a timed region. */
SFHK_API int sfhk_launch_count(uint64_t* out);

/* Throughput of the device's FMA pipes: the measured denominators of the
 * integrators' rooflines (a measurement utility, not a step of the method).
 * kind 0 = FP32 FMA, 1 = packed FP32 FMA pairs (one f32x2 instruction, two
 * FMAs), 2 = FP64 FMA.  One warm-up and one timed launch, each thread
 * running 8 independent FMA recurrences for `iters` rounds, 4 blocks of 256
 * threads per SM, timed with CUDA events on a private stream.  *tflops
 * receives 2 x FMAs / duration (an FMA counts 2 flops); *ms the duration
 * (may be NULL).  Synchronous; allocates (and frees) SMs x 8 KiB of device
 * memory for the result sink.  The clock is whatever the GPU runs at
 * meanwhile: sample it beside the call.  Errors: SFHK_E_INVAL (kind outside
 * 0..2, iters < 1, null tflops), SFHK_E_CUDA. */
SFHK_API int sfhk_fma_peak(int device, int kind, int iters, double* tflops, float* ms);

#ifdef __cplusplus
}
#endif
#endif /* SFHK_H */

"""Work per trajectory-step of the SFHK integrator, for the roofline of the
propagation kernel.  An FMA counts 2 flops, an add or multiply 1; the
special-function operations (rsqrt, exp, sincos) are listed, not counted.

Algorithmic count (the roofline's numerator)
-------------------------------------------
The method's own formulation, item by item: classical RK4 on the whole
43-component state y = (q, p, M, S) of Hamilton's equations, the
stability-matrix equations and the action, with the derivative evaluated
four times per step; the Herman-Kluk determinant and its continuous root
every step; the recombination element, the phase and the per-step
contribution where the trajectory overlaps the orbital.

  derivative of y at one point, diatomic (two centres)
    potential, gradient, Hessian: per centre 15 (difference 3,
      |d|^2 + a^2 6, u^2 u^3 2, V 1, g1 1, g2 2), screened centres
      15 more (s = s^2 u, the exponential's argument and factor,
      V, g1, g2 terms); sum over the centres 38 (V 1, force 9,
      sum of g1 1, g2 d 6, Hessian 21)            2 x 15 (+ 2 x 15) + 38
    dp/dt = F - E z 1, dS/dt = p^2/2 - V - z E 9                        10
    dM_p/dt = -Hess V M_q (3x3 by 3x6, 2 m n k)                          108
                                                   H2: 186, N2: 216 (x 4)
  RK4 combination on 43 components: three stage points y + c k (2 each)
    and y + h/6 (k1 + 2 k2 + 2 k3 + k4) (6)                     43 x 12 = 516
  prefactor: B (9 x 4), complex 3x3 determinant by cofactors 64, scale 2,
    |det| 3, root 6, branch 3                                             114
  per recombination evaluation (the steps counted by the kernel, see
    sfhk_stats.recomb_evals): |p|^2 5; per centre d 3, |d|^2 5, p.d 5;
    per primitive and centre: exponent 3, magnitude 1, phase 1,
    (p_z - i g d_z) 3, complex accumulate 8 = 16, a p-type factor 18
    more; then the phase and contribution 27 (S mod 2 pi 5, w C 6,
    e^{iS} 6, e^{-i Ip t} 6, Re[. R] 3, scale 1)
                             H2 (2 s): 5 + 26 + 64 + 27 = 122; N2_sp 258

  per trajectory-step: 4 derivatives + 516 + 114, plus the recombination
  work times the fraction of steps that evaluate it.

  Polyatomic targets (N screened centres): the potential at one point is
  30 N + 23 N + 3 (per-centre terms, accumulation, diagonal), the
  derivative 53 N + 3 + 118; recombination per primitive (on its own
  centre) 29 (+18 p-type), plus |p|^2 5 and the 27 of the contribution.

Executed count (for comparison)
-------------------------------
The kernel does less than the method's plain form: the stability matrix
advances with collapsed RK4 sums (Mq' = Mq + h Mp - h^2/6 sum a, Mp' = Mp -
h/6 sum a: 684 flops for the six columns, against 4 x 108 + 36 x 12 = 864
in the plain form) and the overlaps are skipped, after a 43-flop far-field
test, where they are below e^-30 of their peak.  Counted from the kernel's own
arithmetic, without the recombination work:

  potential at one point, two centres 68 (x 4 = 272); stage points,
  derivatives, actions, RK4 sums 111; two-float updates of q, p, S 70;
  stability matrix 684; prefactor 119; recombination far-field test 43
                                                 H2 1299, N2 1419 (+30 x 4)
"""

# ---------------------------------------------------------------- algorithmic
_DERIV_COMMON = 10 + 108          # dp/dt, dS/dt; -Hess V M_q
_RK4_PLAIN = 43 * 12              # stage points and the final combination
_PREFACTOR = 114
_PHASE_COMBINE = 27


def _diatomic_base(screened: bool) -> int:
    per_centre = 15 + (15 if screened else 0)
    deriv = 2 * per_centre + 38 + _DERIV_COMMON
    return 4 * deriv + _RK4_PLAIN + _PREFACTOR


def _diatomic_recomb(n_s: int, n_p: int) -> int:
    return 5 + 2 * 13 + 2 * (16 * n_s + 34 * n_p) + _PHASE_COMBINE


def _poly_base(n_centres: int) -> int:
    deriv = 53 * n_centres + 3 + _DERIV_COMMON
    return 4 * deriv + _RK4_PLAIN + _PREFACTOR


def _poly_recomb(n_s: int, n_p: int) -> int:
    return 5 + 29 * n_s + 47 * n_p + _PHASE_COMBINE


# per target: (flops every trajectory-step, flops per recombination evaluation)
ALGORITHMIC = {
    "H2": (_diatomic_base(False), _diatomic_recomb(2, 0)),
    "N2": (_diatomic_base(True), _diatomic_recomb(2, 0)),
    "N2_sp": (_diatomic_base(True), _diatomic_recomb(2, 2)),
    "N2_pi": (_diatomic_base(True), _diatomic_recomb(0, 2)),
    "H2O": (_poly_base(3), _poly_recomb(0, 2)),
    "H2O_3a1": (_poly_base(3), _poly_recomb(2, 2)),
}


def algorithmic_flops(target: str, traj_steps: int, recomb_evals: int) -> float:
    """The method's flops for a launch that integrated `traj_steps`
    trajectory-steps and evaluated the recombination element `recomb_evals`
    times (both from sfhk_stats)."""
    base, rec = ALGORITHMIC[target]
    return float(base) * traj_steps + float(rec) * recomb_evals


# ---------------------------------------------------------------- executed
EXECUTED_FLOPS_PER_STEP = {"H2": 1299, "N2": 1419, "N2_sp": 1431, "N2_pi": 1419, "H2O": 1659,
                           "H2O_3a1": 1681}

# FP32 FMA pipe of a B300 from its unit counts (148 SMs x 128 lanes x 2 flops
# at the maximum SM clock): context beside the measured peak (sfhk_fma_peak)
SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2032.0


def fp32_peak_tflops(sm_mhz: float = MAX_SM_MHZ) -> float:
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# dram__bytes_read.sum + dram__bytes_write.sum per full-size launch of the
# dominant kernel, keyed by (workload, kernel variant), from an ncu capture of
# the current kernel, scaled by the trajectories to the full size (the
# traffic is the initial-point SoA read once, about 100 B per trajectory):
# H2 0/45/90 deg captured at 3 x 5e4 trajectories with the fixed-parameter
# integrator of the unscreened two-centre potential (no first-return record)
# in 32-thread blocks, uncapped (variant 1: 14.86 MB read, 0 written) and at
# 168 registers (variant 2: 14.85 MB), the autotuner's two choices, scaled to
# 3 x 1e6; H2O 1b1 isotropic (three-centre fixed-parameter kernel) captured
# at 1e5 trajectories with the 168-register variant (2) in 64-thread blocks
# (9.90 MB read), scaled to 1e6; N2 cos^2 (fixed-parameter integrator of the
# screened two-centre potential) captured at 1e5 trajectories with the
# 168-register variant (2) in 128-thread blocks, the shape its bench line runs
# (10.24 MB read, 0 written), scaled to 1e7.
TRAFFIC = {("h2-angles", 1): 297.1e6, ("h2-angles", 2): 297.1e6, ("h2o-iso", 2): 99.0e6,
           ("n2-cos2", 2): 1024.1e6}

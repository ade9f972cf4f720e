"""Algorithmic work per trajectory-step of the SFHK integrator, used for the
roofline of the propagation kernel.

One trajectory-step = one RK4 step of (q, p, S) with the four stage
potential/gradient/Hessian evaluations, the six stability-matrix columns
advanced with the stage Hessians, the Herman-Kluk determinant and its
continuous square root, and the far-field test of the recombination element.
Counted from the arithmetic the method needs (FMA = 2 flops, add/mul = 1;
rsqrt/exp/sincos/sqrt on the special-function unit not counted):

  potential at one point, two centres            2 x 40 =  80  (x4 stages = 320)
    (difference 3, |d|^2 + a^2 6, u^2 u^3 2, V 2, g1 1, g2 2, force 6,
     g2 d_x, g2 d_y 2, diagonal Hessian 10, off-diagonal 6)
  stage points, derivatives, actions, RK4 sums               111
  two-float (compensated) updates of q, p, S: 7 x 10           70
  stability matrix: 6 columns x (4 Hessian products 60,
     stage vectors 36, RK4 sums 36)                          792
  prefactor: B (9 x 6), complex 3x3 determinant 64, root
     and branch test 9, filter test 4                        131
  recombination far-field test (|p|^2, d, |d|^2, p.d per
     centre, exponent per primitive)                          43
  ---------------------------------------------------------------
  H2 (unscreened centres)                                   1467
  N2 (screened centres: exp(-alpha s) terms, +30 per point)  1587

Steps near a nucleus also evaluate the Gaussian overlaps, the phase and the
warp reduction; they are not counted, so the figure is a lower bound.
"""

FLOPS_PER_STEP = {"H2": 1467, "N2": 1587}

# FP32 FMA pipe of a B300: 148 SMs x 128 lanes x 2 flops x 2.032 GHz (max SM clock)
SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2032.0


def fp32_peak_tflops(sm_mhz: float = MAX_SM_MHZ) -> float:
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# dram__bytes_read.sum + dram__bytes_write.sum per full-size launch of the
# dominant kernel, keyed by (workload, kernel variant), from an ncu capture of
# the current kernel: H2 0/45/90 deg captured at 3 x 2e5 trajectories (80.5 MB
# read + 6.8 MB written) and scaled by trajectories to 3 x 1e6.
TRAFFIC = {("h2-angles", 4): 437.0e6}

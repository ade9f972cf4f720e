"""Algorithmic work per trajectory-step of the SFHK integrator, used for the
roofline of the propagation kernel.

One trajectory-step = one RK4 step of (q, p, S) with the four stage
potential/gradient/Hessian evaluations, the six stability-matrix columns
advanced with the stage Hessians, the Herman-Kluk determinant and its
continuous square root, and the far-field test of the recombination element.
Counted from the arithmetic of the formulation the kernel uses (FMA = 2
flops, add/mul = 1; rsqrt/exp/sincos on the special-function unit and the
Newton step that refines rsqrt are not counted):

  potential at one point, two centres                              68  (x4 stages = 272)
    per centre 15: difference 3, |d|^2 + a^2 6, u^2 u^3 2, V 1, g1 1, g2 2;
    sum over centres 38: V 1, force 9, sum of g1 1, g2 d 6,
    diagonal Hessian 12, off-diagonal 9
  stage points, derivatives, actions, RK4 sums                    111
  two-float (compensated) updates of q, p, S: 7 x 10                70
  stability matrix, 6 columns x 114: stage points 12, four
    Hessian products 60, stage corrections 12, the two RK4
    sums 30 (Mq' = Mq + h Mp - h^2/6 sum a, Mp' = Mp - h/6 sum a)  684
  prefactor: B (9 x 4), complex 3x3 determinant 64 and scale 2,
    |det| 4, root and branch test 9, filter test 4                 119
  recombination far-field test (|p|^2, d, |d|^2, p.d per
    centre, exponent per primitive)                                 43
  ---------------------------------------------------------------
  H2 (unscreened centres)                                         1299
  N2 (screened centres: exp(-alpha s) terms, +30 per point)       1419

Steps near a nucleus also evaluate the Gaussian overlaps, the phase and the
per-step contribution; they are not counted, so the figure is a lower bound.

Polyatomic targets (N centres, each with its own screened charge), same
counting:

  potential at one point, per centre: the 15 above plus the screening
    term 15; accumulation 23: V 1, force 6, sum of g1 1, g2 d 3,
    Hessian 12; then 3 for the diagonal                     30 N + 23 N + 3
  stage points, two-float updates, stability matrix, prefactor
    (as above)                                                      984
  recombination test per primitive (d 3, |d|^2 5, exponent 3) 11 per
    primitive, |p|^2 5                                        11 n_prim + 5
  ---------------------------------------------------------------
  H2O (3 centres, 2 primitives): 4 x 162 + 984 + 27              1659
  H2O_3a1 (3 centres, 4 primitives): 4 x 162 + 984 + 49          1681

Diatomic targets with more primitives add the per-primitive exponent of the
recombination test (3 per primitive and centre): N2_sp (4 primitives, two of
them p-type) 1419 + 2 x 2 x 3 = 1431; N2_pi (2 primitives) 1419.
"""

FLOPS_PER_STEP = {"H2": 1299, "N2": 1419, "N2_sp": 1431, "N2_pi": 1419, "H2O": 1659,
                  "H2O_3a1": 1681}

# FP32 FMA pipe of a B300: 148 SMs x 128 lanes x 2 flops x 2.032 GHz (max SM clock)
SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2032.0


def fp32_peak_tflops(sm_mhz: float = MAX_SM_MHZ) -> float:
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# dram__bytes_read.sum + dram__bytes_write.sum per full-size launch of the
# dominant kernel, keyed by (workload, kernel variant), from an ncu capture of
# the current kernel: H2 0/45/90 deg captured at 3 x 2e5 trajectories with the
# 168-register variant in 32-thread blocks (63.3 MB read + 3.0 MB written) and
# scaled by trajectories to 3 x 1e6.
# H2O 1b1 isotropic: captured at 2e5 trajectories with the 128-register
# variant in 64-thread blocks (19.8 MB read + 0.19 MB written), scaled to 1e6.
TRAFFIC = {("h2-angles", 2): 331.0e6, ("h2o-iso", 6): 100.0e6}

"""The modified saddle point of SFHK2 (Sec. III.D) in the oracle:

    [k + A(t_s) - A(t0)]^2 / 2 + Ip - eta E(t_s).r0 = 0,   r0 = (R/2) n.

Pinned by the complex residual of that equation at the returned (t_s, k_z),
by its reduction to the standard saddle at c = eta (R/2) n_z = 0, by a finite
difference of the field derivative it uses, and, at 90 deg where E.r0 = 0,
by the sum over the two emitting centres reproducing the standard weight
(the dipole element is linear in the centres)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

P = W.PULSE_1200


def test_field_derivative_matches_finite_difference():
    d = O.pulse_derived(P)
    for tau in (0.3 * d["Tp"] * 0.5 + 4.0j, -40.0 + 11.0j, 17.0 + 0.5j):
        h = 1e-4
        fd = (O.pulse_E_complex(P, tau + h) - O.pulse_E_complex(P, tau - h)) / (2 * h)
        an = O.pulse_Edot_complex(P, tau)
        assert abs(an - fd) <= 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("t0,kperp2,c", [(-30.0, 0.01, 0.8), (-30.0, 0.01, -0.8),
                                          (12.5, 0.09, 1.03), (55.0, 0.0, -0.4)])
def test_modified_saddle_solves_the_complex_equation(t0, kperp2, c):
    Ip = W.TARGETS["N2"]["Ip"]
    rc, tt, kz = O.saddle_modified(P, Ip, t0, kperp2, c)
    assert rc == 0 and tt > 0.0
    ts = t0 + 1j * tt
    kap_z = kz + O.pulse_A_complex(P, ts) - O.pulse_A_complex(P, complex(t0))
    res = 0.5 * (kperp2 + kap_z * kap_z) + Ip - c * O.pulse_E_complex(P, ts)
    assert abs(res) <= 1e-10


def test_zero_offset_is_the_standard_saddle():
    Ip = W.TARGETS["N2"]["Ip"]
    for t0, kp2 in ((-30.0, 0.01), (12.5, 0.09), (55.0, 0.0)):
        rc0, tt0, kz0 = O.saddle(P, Ip, t0, kp2)
        rc1, tt1, kz1 = O.saddle_modified(P, Ip, t0, kp2, 0.0)
        assert rc0 == rc1 == 0 and tt0 == tt1 and kz0 == kz1


def test_both_centres_sum_to_the_standard_weight_at_ninety_degrees():
    t = W.TARGETS["N2"]
    al = W.fixed(90.0)
    s1, _, _ = O.sample(t, P, al, seed=3, n=50)
    sp, _, _ = O.sample(W.sfhk2(t), P, al, seed=3, n=50, eta_force=1)
    sm, _, _ = O.sample(W.sfhk2(t), P, al, seed=3, n=50, eta_force=-1)
    # same saddle, exit and momentum (E.r0 = 0), weights add up
    assert np.allclose(sp[0:10], s1[0:10], rtol=0, atol=1e-13)
    assert np.allclose(sm[0:10], s1[0:10], rtol=0, atol=1e-13)
    w1 = s1[10] + 1j * s1[11]
    wsum = (sp[10] + 1j * sp[11]) + (sm[10] + 1j * sm[11])
    assert np.all(np.abs(wsum - w1) <= 1e-10 * np.abs(w1).max())


def test_drawn_side_weighs_twice_the_forced_one():
    t = W.sfhk2(W.TARGETS["N2"])
    al = W.fixed(0.0)
    s, _, _ = O.sample(t, P, al, seed=8, n=40)
    sp, _, _ = O.sample(t, P, al, seed=8, n=40, eta_force=1)
    sm, _, _ = O.sample(t, P, al, seed=8, n=40, eta_force=-1)
    u = np.array([O.uniforms(8, 0, j)[5] for j in range(40)])
    pick = np.where(u[None, :] < 0.5, sp, sm)
    assert np.array_equal(s[0:10], pick[0:10])
    assert np.allclose(s[10:12], 2.0 * pick[10:12], rtol=1e-15, atol=0)
    # at 0 deg the two sides have different saddles
    assert np.any(sp[3] != sm[3])

"""Tapered stability filter in the oracle (a reading; the paper gives no
filter): with Mhat_n the running maximum of max|M_ij| up to step n, the
contribution at t_n is weighted by g = 1 below m0, (1 + cos(pi x))/2 with
x = ln(Mhat/m0)/ln r in between, and the trajectory stops once Mhat >= r m0.

Pins: the weight's values and symmetry; the special cases that reduce to the
unfiltered and to the empty sum; the hard filter as the limit r -> 1; and the
continuity that motivates it (the dipole changes linearly with m0)."""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

T, P = W.TARGETS["H2"], W.PULSE_800


def test_weight_function():
    m0, r = 1000.0, 2.0
    assert O.stab_taper_weight(500.0, m0, r) == 1.0
    assert O.stab_taper_weight(m0, m0, r) == 1.0
    assert O.stab_taper_weight(r * m0, m0, r) == 0.0
    assert abs(O.stab_taper_weight(np.sqrt(r) * m0, m0, r) - 0.5) <= 1e-15
    xs = np.linspace(0.0, 1.0, 41)
    g = np.array([O.stab_taper_weight(m0 * r ** x, m0, r) for x in xs])
    assert np.all(np.diff(g) <= 0.0)
    assert np.allclose(g + g[::-1], 1.0, atol=1e-14)        # odd about the midpoint
    assert np.allclose(g, 0.5 * (1 + np.cos(np.pi * xs)), atol=1e-14)


@pytest.fixture(scope="module")
def ens():
    soa, _, _ = O.sample(T, P, W.fixed(0.0), seed=4, n=300)
    return soa


def test_reduces_to_no_filter_and_to_nothing(ens):
    v0, fin, _ = O.propagate(T, P, ens, 0.5, want_final=True)
    Mmax = np.abs(fin[6:42]).max()
    # cutoff above every |M| the ensemble reaches at its final step, and far
    # above: nothing is tapered
    big = 1e6 * max(Mmax, 1.0)
    v1, f1, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=big, stab_taper=2.0, want_final=True)
    # (the threads' partial sums are added in a run-dependent order)
    assert np.all(f1[46] == 0) and np.linalg.norm(v1 - v0) <= 1e-13 * np.linalg.norm(v0)
    # m0 r < 1 = max|M(t0)|: every trajectory stops at birth
    v2, f2, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=0.4, stab_taper=2.0, want_final=True)
    assert np.all(f2[46] == 3) and np.all(v2 == 0.0)


def test_hard_filter_is_the_limit(ens):
    vh, fh, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=1e3, want_final=True)
    vt, ft, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=1e3, stab_taper=1.0 + 1e-12,
                            want_final=True)
    assert (fh[46] == 3).sum() > 0 and np.array_equal(fh[46], ft[46])
    assert np.linalg.norm(vt - vh) <= 1e-12 * np.linalg.norm(vh)


def test_dipole_is_continuous_in_the_cutoff(ens):
    """With the taper the dipole moves linearly with m0 (no jumps): the
    change for 2 delta is twice the change for delta."""
    base, _, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=1e3, stab_taper=2.0)
    d1, _, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=1e3 * (1 + 1e-6), stab_taper=2.0)
    d2, _, _ = O.propagate(T, P, ens, 0.5, stab_cutoff=1e3 * (1 + 2e-6), stab_taper=2.0)
    a, b = np.linalg.norm(d1 - base), np.linalg.norm(d2 - base)
    assert a > 0.0                           # some trajectory is in the taper
    assert a <= 1e-4 * np.linalg.norm(base)
    assert 1.8 <= b / a <= 2.2

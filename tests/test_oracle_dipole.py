"""Symmetry and additivity pins of the oracle's dipole sum (CPU only).

* Rotating the molecular axis and the transverse momenta together about the
  polarisation axis z leaves every contribution unchanged (the laser and the
  dipole component are along z).
* Swapping the two centres (n -> -n) leaves a sigma_g orbital, and hence every
  contribution, unchanged.
* The estimator is additive over any partition of the ensemble.
The symmetry checks run with the prefactor filter at |C| > 1e4: beyond it
trajectories are chaotic (|M| > ~1e3), and there a last-bit rounding
difference (the rotated arithmetic) grows to O(1).
"""
import math

import numpy as np

import oracle as O
from paper_2608_13686_b300 import workloads as W

CUT = 1e4


def _ensemble(n=48, seed=4):
    t, p = W.TARGETS["N2"], W.pulse(800.0, 1.5e14, 2)
    soa, _, bad = O.sample(t, p, W.fixed(35.0, 20.0), seed=seed, n=n)
    assert bad == 0
    return t, p, soa


def test_rotation_about_polarisation_axis():
    t, p, soa = _ensemble()
    vz, _, _ = O.propagate(t, p, soa, 0.5, cutoff=CUT, n_threads=4)
    a = 0.9
    rot = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    s2 = soa.copy()
    s2[4:6] = rot @ soa[4:6]
    s2[1:3] = rot @ soa[1:3]
    s2[7:9] = rot @ soa[7:9]
    vz2, _, _ = O.propagate(t, p, s2, 0.5, cutoff=CUT, n_threads=4)
    assert np.max(np.abs(vz2 - vz)) < 1e-9 * np.max(np.abs(vz))
    assert np.max(np.abs(vz)) > 0


def test_centre_swap():
    t, p, soa = _ensemble()
    vz, _, _ = O.propagate(t, p, soa, 0.5, cutoff=CUT, n_threads=4)
    s2 = soa.copy()
    s2[7:10] = -soa[7:10]
    vz2, _, _ = O.propagate(t, p, s2, 0.5, cutoff=CUT, n_threads=4)
    assert np.max(np.abs(vz2 - vz)) < 1e-9 * np.max(np.abs(vz))


def test_additive_over_partitions():
    t, p, soa = _ensemble(n=60)
    vz, _, _ = O.propagate(t, p, soa, 0.5, n_threads=4)
    va, _, _ = O.propagate(t, p, np.ascontiguousarray(soa[:, :25]), 0.5, n_norm=60, n_threads=2)
    vb, _, _ = O.propagate(t, p, np.ascontiguousarray(soa[:, 25:]), 0.5, n_norm=60, n_threads=3)
    assert np.max(np.abs(va + vb - vz)) < 1e-12 * np.max(np.abs(vz))


def test_contribution_starts_at_birth():
    t, p, soa = _ensemble(n=1)
    vz, _, _ = O.propagate(t, p, soa, 0.5)
    n0 = int(soa[0, 0])
    assert np.all(vz[:n0] == 0.0)
    assert vz[n0] != 0.0


def test_prefactor_filter_drops_from_threshold_on():
    t, p, soa = _ensemble(n=16)
    _, fin, bad0 = O.propagate(t, p, soa, 0.5, want_final=True)
    cmax = np.abs(fin[43] + 1j * fin[44])
    cut = float(np.median(cmax)) * 0.999
    vz_f, fin_f, bad = O.propagate(t, p, soa, 0.5, cutoff=cut, want_final=True)
    assert bad >= 1 and np.all(fin_f[46][fin_f[46] != 0] == 1)


def _dt_change(t, p, al, n, seed, **filt):
    """Relative change of the n-trajectory dipole when dt is halved (the same
    births on the finer grid, the finer dipole read at the coarser times)."""
    p2 = dict(p, dt=0.5 * p["dt"])
    soa, _, _ = O.sample(t, p, al, seed=seed, n=n)
    soa2 = soa.copy()
    soa2[0] = 2 * soa[0]
    v1, _, _ = O.propagate(t, p, soa, W.GAMMA, **filt)
    v2, _, _ = O.propagate(t, p2, soa2, W.GAMMA, **filt)
    b = v2[::2][: len(v1)]
    return float(np.linalg.norm(v1 - b) / np.linalg.norm(b))


def _study():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "dt_resolution.json")))["cases"]


FILT = dict(cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF, stab_taper=W.STAB_TAPER)


def test_filtered_n2_dipole_is_resolved_at_the_prescribed_step():
    """N2 (1200 nm, cos^2 axis) with the workloads' filters: halving dt moves
    a 1000-trajectory dipole by less than 2 % of its Monte Carlo noise at that
    size (c_noise / sqrt(N), c_noise from the 2e4-trajectory oracle study in
    tests/golden/dt_resolution.json, where the change was 1.6e-3 of the
    noise).  With the prefactor filter only, the unresolved chaotic
    trajectories move it by a sizeable fraction of the noise."""
    n = 1000
    c_noise = _study()["N2"]["workloads"]["c_noise"]
    noise = c_noise / np.sqrt(n)
    t, p, al = W.TARGETS["N2"], W.PULSE_1200, W.COS2
    assert _dt_change(t, p, al, n, 12, **FILT) <= 0.02 * noise
    assert _dt_change(t, p, al, n, 12, cutoff=W.CUTOFF) >= 0.3 * noise


def test_stability_filter_removes_unresolved_trajectories():
    """H2 along the field: the trajectories beyond the stability filter
    (max|M| > 1e3) are not resolved by RK4 at dt = 0.05, and halving dt
    moves the prefactor-filtered dipole several-fold.  With the workloads'
    filters the change is much smaller but, per trajectory, of the size of
    the Monte Carlo spread (head-on passes through the softened nuclei are
    under-resolved without a large |M|; the 2e4-trajectory study measured a
    change of 0.9 times the sample noise, consistent with zero in the mean):
    it stays below 1.5 times the noise at N = 1000."""
    n = 1000
    study = _study()["H2"]
    noise = study["workloads"]["c_noise"] / np.sqrt(n)
    t, p, al = W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0)
    unfiltered = _dt_change(t, p, al, n, 12, cutoff=W.CUTOFF)
    filtered = _dt_change(t, p, al, n, 12, **FILT)
    assert unfiltered > 1.0
    assert filtered < 0.25 * unfiltered
    assert filtered <= 1.5 * noise

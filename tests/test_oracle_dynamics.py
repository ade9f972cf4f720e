"""Pins of the oracle's classical propagation: trajectory, stability matrix,
action and Herman-Kluk prefactor (CPU only).

Closed forms: free particle and isotropic harmonic oscillator (exact classical
motion, M, S = (p_t q_t - p_0 q_0)/2, prefactor with its continuous branch);
invariants: energy conservation with the field off, the energy balance
dH/dt = z dE/dt with the field on, symplecticity M^T J M = J, det M = 1,
time reversal, and M against finite differences of whole trajectories.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

NOFIELD = W.pulse(800.0, 0.0, 3, dt=0.05)
J6 = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])


def _M(y):
    return y[6:42].reshape(6, 6)


def test_free_particle_exact():
    t = W.harmonic_target(0.0)
    q0, p0 = np.array([1.0, -2.0, 0.5]), np.array([0.3, 0.2, -0.7])
    out = O.trajectory(t, NOFIELD, [0, 0, 1], O.initial_state(q0, p0), -10.0, 0.05, 200)
    tau = 0.05 * np.arange(201)
    assert np.max(np.abs(out[:, 0:3] - (q0 + np.outer(tau, p0)))) < 1e-12
    assert np.max(np.abs(out[:, 3:6] - p0)) < 1e-15
    Mexp = np.block([[np.eye(3), tau[-1] * np.eye(3)], [np.zeros((3, 3)), np.eye(3)]])
    assert np.max(np.abs(_M(out[-1]) - Mexp)) < 1e-12
    assert np.max(np.abs(out[:, 42] - 0.5 * p0 @ p0 * tau)) < 1e-12


def test_volkov_momentum_in_field():
    # free electron in the laser: p(t) = p0 + A(t) - A(t0) (E = -dA/dt)
    t = W.harmonic_target(0.0)
    p = W.PULSE_800
    q0, p0 = np.array([0.0, 0.0, -5.0]), np.array([0.1, 0.0, 0.4])
    t0 = -30.0
    out = O.trajectory(t, p, [0, 0, 1], O.initial_state(q0, p0), t0, 0.05, 1200)
    times = t0 + 0.05 * np.arange(1201)
    pz = p0[2] + O.pulse_A(p, times) - O.pulse_A(p, [t0])[0]
    assert np.max(np.abs(out[:, 5] - pz)) < 1e-10


def _ho_errors(dt, omega=0.8, T=12.0):
    t = W.harmonic_target(omega)
    q0, p0 = np.array([1.0, 0.5, -0.3]), np.array([0.2, -0.4, 0.9])
    n = int(round(T / dt))
    y = O.trajectory(t, NOFIELD, [0, 0, 1], O.initial_state(q0, p0), 0.0, dt, n)[-1]
    c, s = math.cos(omega * T), math.sin(omega * T)
    q = q0 * c + p0 / omega * s
    pp = -q0 * omega * s + p0 * c
    M = np.block([[c * np.eye(3), s / omega * np.eye(3)], [-omega * s * np.eye(3), c * np.eye(3)]])
    S = 0.5 * (pp @ q - p0 @ q0)
    return (np.max(np.abs(y[0:3] - q)), np.max(np.abs(y[3:6] - pp)),
            np.max(np.abs(_M(y) - M)), abs(y[42] - S))


def test_harmonic_oscillator_closed_form_fourth_order():
    e1 = _ho_errors(0.05)
    e2 = _ho_errors(0.025)
    for a, b in zip(e1, e2):
        assert a < 1e-6
        assert 12.0 < a / b < 20.0       # RK4: error ~ dt^4


def test_energy_conservation_field_off_fourth_order():
    t = W.TARGETS["N2"]
    nhat = np.array([0.6, 0.0, 0.8])
    # unbound, impact parameter 4: stays where dt = 0.05 resolves the motion
    q0, p0 = np.array([4.0, 0.3, -10.0]), np.array([0.0, 0.1, 1.0])

    def drift(dt, T=20.0):
        n = int(round(T / dt))
        out = O.trajectory(t, NOFIELD, nhat, O.initial_state(q0, p0), 0.0, dt, n)
        H = [0.5 * y[3:6] @ y[3:6] + O.potential(t, nhat, y[0:3])[0] for y in out]
        return np.max(np.abs(np.array(H) - H[0]))

    d1, d2 = drift(0.05), drift(0.025)
    assert d1 < 1e-5
    assert 10.0 < d1 / d2 < 22.0


def test_energy_balance_with_field():
    # dH/dt = dH/dt|explicit = z dE/dt  =>  H(T) - H(t0) = int z Edot dt
    t = W.TARGETS["H2"]
    p = W.PULSE_800
    nhat = np.array([0.0, 0.0, 1.0])
    t0, dt, n = -20.0, 0.025, 1600
    q0, p0 = np.array([0.5, 0.0, -7.0]), np.array([0.05, 0.02, 0.1])
    out = O.trajectory(t, p, nhat, O.initial_state(q0, p0), t0, dt, n)
    times = t0 + dt * np.arange(n + 1)
    E = O.pulse_E(p, times)
    H = np.array([0.5 * y[3:6] @ y[3:6] + O.potential(t, nhat, y[0:3])[0] + y[2] * e
                  for y, e in zip(out, E)])
    h = 1e-5
    Edot = (O.pulse_E(p, times + h) - O.pulse_E(p, times - h)) / (2 * h)
    f = out[:, 2] * Edot
    integ = dt / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    assert abs((H[-1] - H[0]) - integ) < 1e-7 * max(1.0, abs(integ))


def test_symplectic_and_unit_determinant():
    # RK4 is not symplectic: M^T J M - J and det M - 1 are O(dt^4) errors, so
    # check both their size and their fourth-order shrinkage with dt.
    t = W.TARGETS["N2"]
    p = W.PULSE_1200
    nhat = np.array([math.sin(0.4), 0.0, math.cos(0.4)])

    # a scattering trajectory that dt = 0.05 resolves (core-penetrating ones
    # with Z0 = 7 and softening 0.1 are not resolved by RK4 at this step)
    def errs(dt, T=40.0):
        n = int(round(T / dt))
        out = O.trajectory(t, p, nhat, O.initial_state([4.0, 0.3, -10.0], [0.0, 0.1, 1.0]),
                           -40.0, dt, n)
        es, ed = 0.0, 0.0
        for y in out[:: n // 12]:
            M = _M(y)
            sc = max(1.0, np.abs(M).max() ** 2)
            es = max(es, np.max(np.abs(M.T @ J6 @ M - J6)) / sc)
            ed = max(ed, abs(np.linalg.det(M) - 1.0) / sc)
        return es, ed

    (s1, d1), (s2, d2) = errs(0.05), errs(0.025)
    assert s1 < 1e-4 and d1 < 1e-4
    assert s2 < s1 / 10 and d2 < d1 / 10


def test_stability_matrix_against_finite_differences():
    t = W.TARGETS["H2"]
    p = W.PULSE_800
    nhat = np.array([0.0, math.sin(1.0), math.cos(1.0)])
    y0 = O.initial_state([0.2, 0.0, -6.0], [0.1, 0.05, 0.3])
    n = 400
    M = _M(O.trajectory(t, p, nhat, y0, -10.0, 0.05, n)[-1])
    h = 1e-6
    Mfd = np.zeros((6, 6))
    for c in range(6):
        yp, ym = y0.copy(), y0.copy()
        yp[c] += h
        ym[c] -= h
        fp = O.trajectory(t, p, nhat, yp, -10.0, 0.05, n)[-1][0:6]
        fm = O.trajectory(t, p, nhat, ym, -10.0, 0.05, n)[-1][0:6]
        Mfd[:, c] = (fp - fm) / (2 * h)
    assert np.max(np.abs(M - Mfd)) < 1e-6 * max(1.0, np.abs(M).max())


def test_time_reversal():
    t = W.TARGETS["N2"]
    p = W.PULSE_1200
    nhat = np.array([0.0, 0.0, 1.0])
    y0 = O.initial_state([0.3, 0.0, -7.0], [0.0, 0.1, 0.05])
    fwd = O.trajectory(t, p, nhat, y0, -30.0, 0.05, 600)[-1]
    back = O.trajectory(t, p, nhat, fwd, 0.0, -0.05, 600)[-1]
    assert np.max(np.abs(back[0:6] - y0[0:6])) < 1e-8
    assert abs(back[42]) < 1e-8                 # the action integral returns to zero
    assert np.max(np.abs(_M(back) - np.eye(6))) < 1e-7


# ----------------------------------------------------------------- prefactor
def _prefactor_run(target, gamma, taus, dt=0.05):
    d = O.pulse_derived(NOFIELD)
    nt = d["nt"]
    n = len(taus)
    soa = np.zeros((O.NFIELDS, n))
    for j, tau in enumerate(taus):
        soa[0, j] = nt - 1 - int(round(tau / dt))
        soa[1:4, j] = [0.3, -0.2, 0.5]
        soa[4:7, j] = [0.1, 0.2, -0.1]
        soa[9, j] = 1.0
        soa[10, j] = 1.0
    _, fin, bad = O.propagate(target, NOFIELD, soa, gamma, want_final=True, n_threads=4)
    assert bad == 0
    return fin[43] + 1j * fin[44]


def test_prefactor_free_particle_continuous_branch():
    gamma = 0.5
    taus = np.array([1.0, 5.0, 6.5, 7.5, 20.0, 100.0])   # branch point of principal sqrt at 2 sqrt(3)/gamma
    C = _prefactor_run(W.harmonic_target(0.0), gamma, taus)
    z = 1 - 0.5j * gamma * taus
    expect = np.abs(z) ** 1.5 * np.exp(-1.5j * np.arctan(0.5 * gamma * taus))
    assert np.max(np.abs(C - expect) / np.abs(expect)) < 1e-12
    # the principal root of det would flip sign past the branch point
    principal = np.sqrt(z ** 3)
    assert np.any(np.abs(principal - expect) > 0.5 * np.abs(expect))


def test_prefactor_harmonic_coherent_width_winds():
    # gamma = omega: C = exp(-3 i omega t / 2), winding many times
    w = 0.4
    taus = np.array([2.0, 11.0, 40.0, 150.0, 300.0])
    C = _prefactor_run(W.harmonic_target(w), w, taus)
    expect = np.exp(-1.5j * w * taus)
    assert np.max(np.abs(C - expect)) < 1e-6


def test_prefactor_harmonic_general_width():
    # C = [cos wt - (i/2)(g/w + w/g) sin wt]^{3/2} on the continuous branch
    w, g = 0.3, 0.5
    taus = np.array([3.0, 17.0, 60.0, 123.0])
    C = _prefactor_run(W.harmonic_target(w), g, taus)
    grid = np.linspace(0, taus.max(), 200001)
    z = np.cos(w * grid) - 0.5j * (g / w + w / g) * np.sin(w * grid)
    arg = np.unwrap(np.angle(z))
    zt = np.cos(w * taus) - 0.5j * (g / w + w / g) * np.sin(w * taus)
    near = np.interp(taus, grid, arg)                      # picks the branch
    argt = np.angle(zt) + 2 * np.pi * np.round((near - np.angle(zt)) / (2 * np.pi))
    expect = np.abs(zt) ** 1.5 * np.exp(1.5j * argt)
    assert np.max(np.abs(C - expect) / np.abs(expect)) < 1e-5


def test_prefactor_formula_on_hand_built_matrix():
    # det[(Mqq + Mpp - i g Mqp + (i/g) Mpq)/2] for a block-diagonal M
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6))
    g = 0.7
    B = 0.5 * (A[:3, :3] + A[3:, 3:] - 1j * g * A[:3, 3:] + 1j / g * A[3:, :3])
    assert abs(O.hk_det(A, g) - np.linalg.det(B)) < 1e-12 * max(1, abs(np.linalg.det(B)))

"""First returns of the trajectories (the long/short trajectory analysis of
Sec. III.D) in the oracle, pinned against exact field-driven trajectories:
with the potential switched off, p(t) = k + A(t) - A(t0) and
q(t) = q0 + (k - A(t0))(t - t0) + int_{t0}^t A, with A written as its three
sinusoids, so the first return step and energy follow in closed form."""
import math

import numpy as np

import oracle as O
from paper_2608_13686_b300 import workloads as W


def _free_target():
    t = dict(W.TARGETS["H2"])
    t["Zinf"] = 0.0
    t["Z0"] = 0.0
    return t


def _closed_form(p, soa, j, r_out, r_in):
    d = O.pulse_derived(p)
    w, E0, Tp, dt, t_or, nt = d["omega"], d["E0"], d["Tp"], d["dt"], d["t_origin"], d["nt"]
    Wn = 2.0 * math.pi / Tp
    a = (-E0 / (2 * w), -E0 / (4 * w), -E0 / (4 * w))
    k = (w, w + Wn, w - Wn)
    cep = p.get("cep", 0.0)
    A = lambda t: sum(ai * math.sin(ki * t + cep) for ai, ki in zip(a, k))
    IA = lambda t: sum(-ai / ki * math.cos(ki * t + cep) for ai, ki in zip(a, k))
    n0 = int(soa[0, j])
    t0 = t_or + n0 * dt
    q0 = soa[1:4, j]
    k0 = soa[4:7, j]
    left = False
    for n in range(n0, nt):
        t = t_or + n * dt
        q = q0 + k0 * (t - t0)
        q[2] += -A(t0) * (t - t0) + IA(t) - IA(t0)
        az = abs(q[2])
        if az > r_out:
            left = True
        elif left and az < r_in:
            pz = k0[2] + A(t) - A(t0)
            return n, 0.5 * (k0[0] ** 2 + k0[1] ** 2 + pz * pz)
    return -1, 0.0


def test_first_returns_match_field_driven_trajectories():
    t, p = _free_target(), W.PULSE_800
    soa, _, _ = O.sample(t, p, W.fixed(0.0), seed=2, n=120)
    _, steps, energies = O.propagate_returns(t, p, soa, W.GAMMA, r_out=6.0, r_in=2.0)
    n_ret = 0
    for j in range(soa.shape[1]):
        n_ref, e_ref = _closed_form(p, soa, j, 6.0, 2.0)
        assert steps[j] == n_ref, j
        if n_ref >= 0:
            n_ret += 1
            assert abs(energies[j] - e_ref) <= 1e-8 * max(1.0, e_ref)
    assert n_ret >= 10          # enough returning trajectories to mean something


def test_highest_return_energy_is_the_classical_cutoff():
    # the textbook result for field-driven returns: electrons starting at rest
    # at the origin come back with at most 3.17 Up (Up = E0^2 / (4 w^2)); a
    # 20-cycle pulse, births over its central optical cycle
    t, p = _free_target(), W.pulse(800.0, 1.5e14, 20)
    d = O.pulse_derived(p)
    c, per = d["nt"] // 2, int(2.0 * math.pi / d["omega"] / d["dt"])
    n0 = np.arange(c - per, c, 3)
    soa = np.zeros((12, len(n0)))
    soa[0] = n0
    soa[9] = 1.0            # axis along z (irrelevant without a potential)
    soa[10] = 1.0           # unit weight
    _, steps, energies = O.propagate_returns(t, p, soa, W.GAMMA, r_out=0.5, r_in=0.05)
    Up = d["E0"] ** 2 / (4.0 * d["omega"] ** 2)
    top = energies[steps >= 0].max() / Up
    assert 3.12 <= top <= 3.18, top

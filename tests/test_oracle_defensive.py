"""Defensive proposal in the oracle's sampler (a reading, not the paper's):
the time proposal mixes the ADK weights with a uniform share eps over the
grid, and the k_perp width has a floor sigma(f E0).  The weights stay
w = a / pdf with the density actually sampled, so every weighted mean is
unchanged in expectation while the weights of weak-field births are bounded.

The uniform share covers the grid points where |E(t_n)| >= 1e-2 E0 (below
that both weights vanish in effect).  Pins: eps = f = 0 is the plain sampler,
bit for bit; w * pdf equals the amplitude assembled from the separately
pinned pieces, with the mixture density written out here; weighted means
agree with the plain sampler within their statistical error; the uniform
share shows up in the birth times and never below the field threshold."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

T, P = W.TARGETS["H2"], W.PULSE_800
EPS, FLOOR = 0.05, 0.3


def _defensive(t):
    return dict(t, proposal_mix=EPS, proposal_floor=FLOOR)


def test_zero_share_and_floor_is_the_plain_sampler():
    a, _, _ = O.sample(T, P, W.ISO, seed=2, n=300)
    b, _, _ = O.sample(dict(T, proposal_mix=0.0, proposal_floor=0.0), P, W.ISO, seed=2, n=300)
    assert np.array_equal(a, b)


def test_weight_is_amplitude_over_the_mixture_density():
    from test_oracle_ionization import _amplitude
    t = _defensive(T)
    d = O.pulse_derived(P)
    Wt, cdf = O.adk_table(P, t["Ip"])
    Eg = np.abs(O.pulse_E(P, d["t_origin"] + np.arange(len(Wt)) * d["dt"]))
    inside = Eg >= 1e-2 * d["E0"]
    soa, _, bad = O.sample(t, P, W.fixed(30.0, 10.0), seed=11, n=200)
    assert bad == 0
    s_floor2 = FLOOR * d["E0"] / (2 * math.sqrt(2 * t["Ip"]))
    for j in range(200):
        n0 = int(soa[0, j])
        kx, ky = soa[4, j], soa[5, j]
        a, _, _ = _amplitude(t, P, soa[7:10, j], n0, kx, ky)
        E = abs(O.pulse_E(P, [d["t_origin"] + n0 * d["dt"]])[0])
        sig2 = max(E / (2 * math.sqrt(2 * t["Ip"])), s_floor2)
        p_t = (1 - EPS) * Wt[n0] / cdf[-1] + (EPS / inside.sum() if inside[n0] else 0.0)
        pdf = p_t / d["dt"] * math.exp(-(kx * kx + ky * ky) / (2 * sig2)) / (2 * math.pi * sig2)
        w = soa[10, j] + 1j * soa[11, j]
        assert abs(w * pdf - a) <= 1e-12 * abs(a)     # (a = 0 at the pulse's ends)


def test_unbiased_against_the_plain_sampler():
    n = 60000
    sd, _, _ = O.sample(_defensive(T), P, W.fixed(0.0), seed=21, n=n)
    sp, _, _ = O.sample(T, P, W.fixed(0.0), seed=22, n=n)
    funcs = [lambda s: np.ones(s.shape[1]), lambda s: s[6], lambda s: s[3],
             lambda s: s[4] ** 2 + s[5] ** 2]
    for g in funcs:
        xd = (sd[10] + 1j * sd[11]) * g(sd)
        xp = (sp[10] + 1j * sp[11]) * g(sp)
        se = np.hypot(np.std(xd) / np.sqrt(n), np.std(xp) / np.sqrt(n))
        assert abs(xd.mean() - xp.mean()) <= 5.0 * se


def test_uniform_share_in_the_birth_times():
    """Births where the ADK weight is below 1e-9 of its peak come only from
    the uniform share: their fraction is eps times the fraction of such grid
    points."""
    n = 20000
    d = O.pulse_derived(P)
    Wt, _ = O.adk_table(P, T["Ip"])
    Eg = np.abs(O.pulse_E(P, d["t_origin"] + np.arange(len(Wt)) * d["dt"]))
    inside = Eg >= 1e-2 * d["E0"]
    weak = (Wt < 1e-9 * Wt.max()) & inside
    sd, _, bad = O.sample(_defensive(T), P, W.fixed(0.0), seed=5, n=n)
    born = sd[0].astype(int)
    got = weak[born].mean()
    expect = EPS * weak.sum() / inside.sum()
    assert abs(got - expect) <= 5 * math.sqrt(expect * (1 - expect) / n)
    assert np.all(inside[born]) and bad == 0
    sp, _, _ = O.sample(T, P, W.fixed(0.0), seed=5, n=n)
    assert weak[sp[0].astype(int)].mean() == 0.0

"""Pins of the oracle's generator, pulse and potential (CPU only).

Each check compares the oracle with something other than itself: published
known-answer vectors, numbers printed in the paper's text, finite differences
and closed-form limits.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

EV = W.EV
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    # Known-answer vectors of Philox4x32-10 distributed with Random123
    # (Salmon et al., SC'11): zero, all-ones and pi-digit counters/keys.
    assert O.philox([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert O.philox([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert O.philox([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                    [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_uniforms_open_interval_and_moments():
    u = np.array([O.uniforms(7, 3, j) for j in range(4000)])
    assert np.all(u > 0.0) and np.all(u < 1.0)
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.01


# ----------------------------------------------------------------- pulse
def test_paper_laser_numbers():
    """Sec. III.A: 1200 nm, 1.5e14 W/cm^2 give a Keldysh parameter near 0.6
    and, for H2 (15.4 eV), a cutoff near 80 eV, i.e. harmonic ~77."""
    g = GOLD["laser_sec3A"]
    p = W.pulse(g["lambda_nm"], g["intensity_Wcm2"], g["n_cycles"])
    d = O.pulse_derived(p)
    Up = d["E0"] ** 2 / (4 * d["omega"] ** 2)
    Ip = GOLD["h2_cutoff"]["threshold_eV"] / EV
    keldysh = math.sqrt(Ip / (2 * Up))
    cutoff_ev = (Ip + 3.17 * Up) * EV
    assert abs(keldysh - g["keldysh_near"]) < 0.05
    assert abs(cutoff_ev - GOLD["h2_cutoff"]["cutoff_eV_near"]) < 2.5
    assert abs(cutoff_ev / (d["omega"] * EV) - GOLD["h2_cutoff"]["cutoff_harmonic"]) < 2
    # photon energy of 1200 nm: 1.0332 eV; period 165.5 a.u.
    assert abs(d["omega"] * EV - 1239.84198 / 1200) < 1e-4
    assert abs(2 * math.pi / d["omega"] - 165.48) < 0.01
    # the workload targets carry Table I / Table II where they are the paper's
    t1 = W.TARGETS["N2_table1"]
    assert (t1["Zinf"], t1["Z0"], t1["alpha"], t1["R"]) == tuple(
        GOLD["table1"]["N2"][k] for k in ("Zinf", "Z0", "alpha", "R"))
    assert t1["Ip"] * EV == pytest.approx(GOLD["table2"]["N2_3sigma_g"])
    # the HOMO-1 target binds with Table II's 1 pi_u energy
    assert W.TARGETS["N2_pi"]["Ip"] * EV == pytest.approx(GOLD["table2"]["N2_1pi_u"])


def test_time_grid():
    d = O.pulse_derived(W.PULSE_800)
    assert d["nt"] == 6620
    assert d["t_origin"] == pytest.approx(-0.5 * d["Tp"])
    assert d["t_origin"] + (d["nt"] - 1) * d["dt"] <= 0.5 * d["Tp"] + 1e-9
    d2 = O.pulse_derived(W.PULSE_1200)
    assert d2["nt"] == 9929


@pytest.mark.parametrize("p", [W.PULSE_800, W.PULSE_1200, W.pulse(1000, 1e14, 2, cep=0.7)])
def test_field_is_minus_dA_dt(p):
    d = O.pulse_derived(p)
    t = np.linspace(-0.45 * d["Tp"], 0.45 * d["Tp"], 37)
    h = 1e-4
    fd = -(O.pulse_A(p, t + h) - O.pulse_A(p, t - h)) / (2 * h)
    assert np.max(np.abs(fd - O.pulse_E(p, t))) < 1e-9
    # also at complex times (the saddle lives there): dA/dtau along i
    for tau in (3.0 + 10.0j, -40.0 + 25.0j):
        dA = (O.pulse_A_complex(p, tau + h) - O.pulse_A_complex(p, tau - h)) / (2 * h)
        assert abs(-dA - O.pulse_E_complex(p, tau)) < 1e-8 * max(1.0, abs(dA))
        dAi = (O.pulse_A_complex(p, tau + 1j * h) - O.pulse_A_complex(p, tau - 1j * h)) / (2j * h)
        assert abs(dAi - dA) < 1e-7 * max(1.0, abs(dA))  # analytic (Cauchy-Riemann)


def test_vector_potential_vanishes_at_pulse_edges():
    d = O.pulse_derived(W.PULSE_800)
    assert abs(O.pulse_A(W.PULSE_800, [0.5 * d["Tp"]])[0]) < 1e-15
    assert abs(O.pulse_A(W.PULSE_800, [-0.5 * d["Tp"]])[0]) < 1e-15
    # int E dt = A(-Tp/2) - A(Tp/2) = 0 (Simpson on a fine grid)
    t = np.linspace(-0.5 * d["Tp"], 0.5 * d["Tp"], 20001)
    E = O.pulse_E(W.PULSE_800, t)
    integ = (t[1] - t[0]) / 3 * (E[0] + E[-1] + 4 * E[1:-1:2].sum() + 2 * E[2:-1:2].sum())
    assert abs(integ) < 1e-10
    # peak field ~ E0 at the centre (cos carrier, CEP 0)
    assert O.pulse_E(W.PULSE_800, [0.0])[0] == pytest.approx(d["E0"], rel=1e-12)


# ----------------------------------------------------------------- potential
def _fd_check(t, nhat, q, h=1e-5):
    V, g, H = O.potential(t, nhat, q)
    gfd = np.zeros(3)
    Hfd = np.zeros((3, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        gfd[a] = (O.potential(t, nhat, q + e)[0] - O.potential(t, nhat, q - e)[0]) / (2 * h)
        Hfd[a] = (O.potential(t, nhat, q + e)[1] - O.potential(t, nhat, q - e)[1]) / (2 * h)
    return V, g, H, gfd, Hfd


@pytest.mark.parametrize("name", ["H2", "N2", "H2_table1", "N2_table1"])
def test_potential_gradient_hessian_finite_differences(name):
    t = W.TARGETS[name]
    rng = np.random.default_rng(1)
    for _ in range(12):
        th, ph = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        nhat = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        q = rng.normal(0, 1.5, 3)
        V, g, H, gfd, Hfd = _fd_check(t, nhat, q)
        scale = max(1.0, np.abs(g).max())
        assert np.max(np.abs(g - gfd)) < 1e-6 * scale
        assert np.max(np.abs(H - Hfd)) < 1e-5 * max(1.0, np.abs(H).max())
        assert np.max(np.abs(H - H.T)) < 1e-14 * max(1.0, np.abs(H).max())


def test_potential_limits():
    # Eq. 7: Coulombic -(2 Zinf)/r far away (total asymptotic charge 1)
    t = W.TARGETS["N2"]
    nhat = np.array([0.0, 0.6, 0.8])
    for r in (60.0, 200.0):
        q = r * np.array([0.48, -0.6, 0.64])
        V = O.potential(t, nhat, q)[0]
        assert V == pytest.approx(-1.0 / r, rel=2e-4 * (60 / r) ** 2 + 1e-9)
    # at a nucleus (softening a): V = -Z(a)/a - Z(s2)/s2, s2 = sqrt(R^2 + a^2),
    # with the screened charge Z(s) = Zinf + (Z0 - Zinf) exp(-alpha s)
    a, R = t["soft_a"], t["R"]
    q = 0.5 * R * nhat
    s2 = math.sqrt(R * R + a * a)
    Z = lambda s: t["Zinf"] + (t["Z0"] - t["Zinf"]) * math.exp(-t["alpha"] * s)
    expect = -Z(a) / a - Z(s2) / s2
    # unsoftened Table I form: Z -> Z0 near a nucleus (Eq. 7 limit)
    t1 = W.TARGETS["N2_table1"]
    eps = 1e-7
    qn = 0.5 * t1["R"] * nhat + np.array([eps, 0, 0])
    assert O.potential(t1, nhat, qn)[0] * eps == pytest.approx(-t1["Z0"], rel=1e-5)
    assert O.potential(t, nhat, q)[0] == pytest.approx(expect, rel=1e-13)
    # H2 (Z0 = Zinf): plain soft-core charges 0.5, symmetric under r -> -r
    h = W.TARGETS["H2"]
    q = np.array([0.3, -0.2, 0.9])
    assert O.potential(h, nhat, q)[0] == pytest.approx(O.potential(h, nhat, -q)[0], rel=1e-15)
    d1 = np.linalg.norm(q - 0.7 * nhat)
    d2 = np.linalg.norm(q + 0.7 * nhat)
    expect = -0.5 / math.sqrt(d1 ** 2 + 0.01) - 0.5 / math.sqrt(d2 ** 2 + 0.01)
    assert O.potential(h, nhat, q)[0] == pytest.approx(expect, rel=1e-14)


def test_harmonic_test_potential():
    t = W.harmonic_target(0.7)
    q = np.array([0.5, -1.0, 2.0])
    V, g, H = O.potential(t, [0, 0, 1], q)
    assert V == pytest.approx(0.5 * 0.49 * q @ q)
    assert np.allclose(g, 0.49 * q)
    assert np.allclose(H, 0.49 * np.eye(3))

"""Pins of the oracle's ionization step, Gaussian-orbital integrals, sampler
and spectrum (CPU only).

References used: the residual of the saddle-point equation (Eq. 2) itself,
the static-field limit (closed forms for tunnelling time, exit and action),
closed-form antiderivatives of the sin^2 pulse, 1-D numerical quadrature of
the Gaussian integrals, sampling statistics against the stated proposal, and
numpy's FFT for the discrete Fourier sum.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W


# ----------------------------------------------------------------- saddle
@pytest.mark.parametrize("p", [W.PULSE_800, W.PULSE_1200, W.PULSE_PAPER])
def test_saddle_residual(p):
    Ip = 0.567
    d = O.pulse_derived(p)
    rng = np.random.default_rng(5)
    tested = 0
    for t0 in rng.uniform(-0.3 * d["Tp"], 0.3 * d["Tp"], 40):
        if abs(O.pulse_E(p, [t0])[0]) < 0.3 * d["E0"]:
            continue
        kx, ky = rng.normal(0, 0.3, 2)
        rc, tt, kz = O.saddle(p, Ip, t0, kx * kx + ky * ky)
        assert rc == 0 and tt > 0
        ts = t0 + 1j * tt
        kap = np.array([kx, ky, kz + O.pulse_A_complex(p, ts) - O.pulse_A(p, [t0])[0]])
        resid = 0.5 * np.sum(kap * kap) + Ip
        assert abs(resid) < 1e-12
        tested += 1
    assert tested > 10


def test_static_field_limit():
    # very long wavelength: near t0 = 0 the field is E0 and constant, so
    # tt = sqrt(2Ip + k^2)/E0, exit z = -(2Ip + k^2)/(2 E0),
    # Im S_down = (2Ip + k^2)^{3/2} / (3 E0), Re S_down = Ip t0 = 0.
    p = W.pulse(4.0e5, 1.5e14, 3)
    d = O.pulse_derived(p)
    E0, Ip = d["E0"], 0.567
    for kp2 in (0.0, 0.04, 0.1):
        rc, tt, kz = O.saddle(p, Ip, 0.0, kp2)
        assert rc == 0
        assert tt == pytest.approx(math.sqrt(2 * Ip + kp2) / E0, rel=1e-5)
        assert abs(kz) < 1e-6
        qz, Sd = O.tunnel(p, Ip, 0.0, tt, [math.sqrt(kp2), 0.0, kz])
        assert qz == pytest.approx(-(2 * Ip + kp2) / (2 * E0), rel=1e-5)
        assert Sd.imag == pytest.approx((2 * Ip + kp2) ** 1.5 / (3 * E0), rel=1e-5)
        assert abs(Sd.real) < 1e-4


def _sin2_terms(p):
    """A(t) = sum_m a_m sin(k_m t + cep): cos^2 envelope written as three
    sinusoids (cos^2 x = (1 + cos 2x)/2 and product-to-sum)."""
    d = O.pulse_derived(p)
    w, E0, Om = d["omega"], d["E0"], 2 * math.pi / d["Tp"]
    return [(-E0 / (2 * w), w), (-E0 / (4 * w), w + Om), (-E0 / (4 * w), w - Om)], d["cep"]


def test_tunnel_exit_and_action_against_closed_forms():
    p = W.PULSE_800
    Ip = 0.567
    terms, cep = _sin2_terms(p)
    for t0, k in ((-10.0, (0.1, -0.05)), (44.0, (0.0, 0.2)), (3.0, (0.3, 0.1))):
        kp2 = k[0] ** 2 + k[1] ** 2
        rc, tt, kz = O.saddle(p, Ip, t0, kp2)
        assert rc == 0
        # int_0^tt Im A(t0 + is) ds with Im sin(th + iks) = cos th sinh(ks)
        qz_exact = sum(a * math.cos(km * t0 + cep) * (math.cosh(km * tt) - 1) / km
                       for a, km in terms)
        qz, Sd = O.tunnel(p, Ip, t0, tt, [k[0], k[1], kz])
        assert qz == pytest.approx(qz_exact, rel=1e-12, abs=1e-12)
        # S_down = Ip t_s + (i/2) int_0^tt [k^2 + (kz + A(t0+is) - A(t0))^2] ds
        s = np.linspace(0, tt, 40001)
        A0 = O.pulse_A(p, [t0])[0]
        f = np.array([kp2 + (kz + O.pulse_A_complex(p, t0 + 1j * x) - A0) ** 2 for x in s])
        h = s[1] - s[0]
        integ = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        S_ref = Ip * (t0 + 1j * tt) + 0.5j * integ
        assert abs(Sd - S_ref) < 1e-9 * abs(S_ref)


# ----------------------------------------------------------------- orbital integrals
def _trap(f, h):
    return h * (f.sum() - 0.5 * (f[0] + f[-1]))


def _prims(t, nhat):
    R = t["R"]
    out = []
    for sgn in (1.0, -1.0):
        A = sgn * 0.5 * R * np.asarray(nhat, float)
        for a, c in zip(t["pexp"], t["pcoef"]):
            out.append((a, c, A))
    return out


@pytest.mark.parametrize("name", ["H2", "N2"])
def test_orbital_normalised(name):
    t = W.TARGETS[name]
    nhat = np.array([0.0, 0.6, 0.8])
    x = np.linspace(-12, 12, 2401)
    h = x[1] - x[0]
    N = O.orbital_norm(t)
    tot = 0.0
    for a1, c1, A1 in _prims(t, nhat):
        for a2, c2, A2 in _prims(t, nhat):
            f = 1.0
            for dd in range(3):
                f *= _trap(np.exp(-a1 * (x - A1[dd]) ** 2 - a2 * (x - A2[dd]) ** 2), h)
            tot += c1 * c2 * f
    assert N * N * tot == pytest.approx(1.0, rel=1e-12)
    # value function agrees with the primitive sum
    r = np.array([0.1, -0.4, 0.7])
    v = N * sum(c * math.exp(-a * np.sum((r - A) ** 2)) for a, c, A in _prims(t, nhat))
    assert O.orbital_value(t, nhat, r) == pytest.approx(v, rel=1e-14)


@pytest.mark.parametrize("name,gamma", [("H2", 0.5), ("N2", 1.0)])
def test_recombination_element_against_quadrature(name, gamma):
    """<psi0| k_z |p,q> = int psi0(x) [p_z + i gamma (z - q_z)] <x|p,q> dx with
    <x|p,q> = (gamma/pi)^{3/4} exp(-gamma/2 |x-q|^2 + i p.(x-q)); each primitive
    term factorises into three 1-D integrals done by the trapezoid rule."""
    t = W.TARGETS[name]
    nhat = np.array([0.48, 0.0, 0.877])
    nhat /= np.linalg.norm(nhat)
    x = np.linspace(-16, 16, 6401)
    h = x[1] - x[0]
    N = O.orbital_norm(t)
    for q, p in (([0.3, -0.2, 1.1], [0.4, 0.1, -0.9]), ([2.0, 0.5, -3.0], [-1.2, 0.3, 1.5]),
                 ([0.0, 0.0, 0.0], [0.0, 0.0, 0.0])):
        q, p = np.array(q), np.array(p)
        ref = 0.0
        for a, c, A in _prims(t, nhat):
            fac = []
            for dd in range(3):
                g = np.exp(-a * (x - A[dd]) ** 2 - 0.5 * gamma * (x - q[dd]) ** 2
                           + 1j * p[dd] * (x - q[dd]))
                fac.append((_trap(g, h), _trap((x - q[dd]) * g, h)))
            I0 = fac[0][0] * fac[1][0] * fac[2][0]
            Iz = fac[0][0] * fac[1][0] * fac[2][1]
            ref += c * (p[2] * I0 + 1j * gamma * Iz)
        ref *= N * (gamma / math.pi) ** 0.75
        got = O.recomb(t, nhat, q, p, gamma)
        assert abs(got - ref) < 1e-11 * max(1e-3, abs(ref))


def test_dipole_matrix_element_against_quadrature():
    """<kappa| z |psi0> = (2pi)^{-3/2} int e^{-i kappa.r} z psi0(r) dr, with
    complex kappa (analytic continuation) as at the saddle point."""
    t = W.TARGETS["N2"]
    nhat = np.array([0.6, 0.0, 0.8])
    x = np.linspace(-14, 14, 5601)
    h = x[1] - x[0]
    N = O.orbital_norm(t)
    for kap in ([0.2, -0.1, 0.3], [0.1, 0.05, 0.4 + 0.9j], [0.0, 0.0, 1.066j]):
        kap = np.array(kap, complex)
        ref = 0.0
        for a, c, A in _prims(t, nhat):
            f = [np.exp(-1j * kap[dd] * x - a * (x - A[dd]) ** 2) for dd in range(3)]
            ref += c * _trap(f[0], h) * _trap(f[1], h) * _trap(x * f[2], h)
        ref *= N * (2 * math.pi) ** -1.5
        got = O.dipole_matrix_element(t, nhat, kap)
        assert abs(got - ref) < 1e-11 * max(1e-3, abs(ref))


# ----------------------------------------------------------------- sampler
def _amplitude(t, p, nhat, n0, kx, ky):
    """The second line of Eq. 1 assembled from the separately pinned pieces."""
    d = O.pulse_derived(p)
    t0 = d["t_origin"] + n0 * d["dt"]
    rc, tt, kz = O.saddle(p, t["Ip"], t0, kx * kx + ky * ky)
    qz, Sd = O.tunnel(p, t["Ip"], t0, tt, [kx, ky, kz])
    ts = t0 + 1j * tt
    Es = O.pulse_E_complex(p, ts)
    kap = np.array([kx, ky, kz + O.pulse_A_complex(p, ts) - O.pulse_A(p, [t0])[0]])
    mz = O.dipole_matrix_element(t, nhat, kap)
    return Es * mz / np.sqrt(Es * kap[2]) * np.exp(1j * (Sd + kz * qz)), qz, kz


def test_sample_weight_is_amplitude_over_pdf():
    t, p = W.TARGETS["H2"], W.PULSE_800
    d = O.pulse_derived(p)
    Wt, cdf = O.adk_table(p, t["Ip"])
    soa, aux, bad = O.sample(t, p, W.fixed(30.0, 10.0), seed=11, n=64)
    assert bad == 0
    for j in range(64):
        n0 = int(soa[0, j])
        kx, ky = soa[4, j], soa[5, j]
        nhat = soa[7:10, j]
        a, qz, kz = _amplitude(t, p, nhat, n0, kx, ky)
        E = abs(O.pulse_E(p, [d["t_origin"] + n0 * d["dt"]])[0])
        sig2 = E / (2 * math.sqrt(2 * t["Ip"]))
        pdf = Wt[n0] / cdf[-1] / d["dt"] * math.exp(-(kx * kx + ky * ky) / (2 * sig2)) / (
            2 * math.pi * sig2)
        w = soa[10, j] + 1j * soa[11, j]
        assert abs(w * pdf - a) < 1e-12 * abs(a)
        assert soa[3, j] == pytest.approx(qz, rel=1e-14) and soa[6, j] == pytest.approx(kz, rel=1e-14)
        assert np.all(soa[1:3, j] == 0.0)
        assert nhat == pytest.approx([math.sin(math.radians(30)) * math.cos(math.radians(10)),
                                      math.sin(math.radians(30)) * math.sin(math.radians(10)),
                                      math.cos(math.radians(30))], abs=1e-15)


def test_sampler_statistics():
    t, p = W.TARGETS["N2"], W.PULSE_1200
    d = O.pulse_derived(p)
    n = 40000
    soa, _, bad = O.sample(t, p, W.COS2, seed=3, instance=2, n=n)
    assert bad == 0
    Wt, cdf = O.adk_table(p, t["Ip"])
    prob = Wt / cdf[-1]
    # time index drawn from p_n: chi-square over 40 equal-probability bins
    edges = np.searchsorted(np.cumsum(prob), np.linspace(0, 1, 41)[1:-1])
    counts = np.bincount(np.searchsorted(edges, soa[0].astype(int), side="right"), minlength=40)
    expect = np.array([prob[a:b].sum() for a, b in zip(np.r_[0, edges], np.r_[edges, len(prob)])]) * n
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < 39 + 6 * math.sqrt(2 * 39)
    # k_perp / sigma(t0) standard normal
    E = np.abs(O.pulse_E(p, d["t_origin"] + soa[0] * d["dt"]))
    sig = np.sqrt(E / (2 * math.sqrt(2 * t["Ip"])))
    z = np.concatenate([soa[4] / sig, soa[5] / sig])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # cos^2 axis distribution: <cos^2 theta> = 3/5, <cos^4> = 3/7, phi uniform
    c = soa[9]
    assert abs(np.mean(c * c) - 0.6) < 5 * math.sqrt((3 / 7 - 0.36) / n)
    assert abs(np.mean(np.arctan2(soa[8], soa[7]))) < 5 * math.pi / math.sqrt(3 * n)
    assert np.allclose(np.sum(soa[7:10] ** 2, axis=0), 1.0)
    # isotropic: <cos^2> = 1/3
    soa_i, _, _ = O.sample(t, p, W.ISO, seed=3, n=20000)
    assert abs(np.mean(soa_i[9] ** 2) - 1 / 3) < 5 * math.sqrt((1 / 5 - 1 / 9) / 20000)


def test_sample_is_partition_independent():
    t, p = W.TARGETS["H2"], W.PULSE_800
    whole, _, _ = O.sample(t, p, W.COS2, seed=9, n=300)
    a, _, _ = O.sample(t, p, W.COS2, seed=9, j_begin=0, n=100)
    b, _, _ = O.sample(t, p, W.COS2, seed=9, j_begin=100, n=200)
    assert np.array_equal(whole, np.concatenate([a, b], axis=1))


# ----------------------------------------------------------------- spectrum
def test_spectrum_is_a_windowed_dft():
    rng = np.random.default_rng(2)
    nt, dt, t0 = 1000, 0.05, -24.975
    vz = rng.normal(size=nt)
    tau = 0.5 * nt * dt
    om, y, ph, v = O.spectrum(vz, dt, t0, tau, 300)
    t = t0 + dt * np.arange(nt)
    win = np.where(np.abs(t) <= tau, 0.5 * (1 + np.cos(np.pi * t / tau)), 0.0)
    # sum_n f_n e^{i w_k t_n} dt = dt e^{i w_k t0} * nt * ifft(f)_k
    ref = dt * np.exp(1j * om * t0) * nt * np.fft.ifft(vz * win)[:300]
    assert np.max(np.abs(v - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.allclose(om, 2 * np.pi * np.arange(300) / (nt * dt))
    assert np.allclose(y, om ** 2 * np.abs(ref) ** 2, rtol=1e-10, atol=1e-300)
    assert np.allclose(np.exp(1j * ph), ref / np.abs(ref), atol=1e-9)


def test_spectrum_of_windowed_cosine():
    # a harmonic on the DFT grid lands in its own bin, with the Hann window's
    # two neighbours at -1/2 of the peak
    nt, dt = 2000, 0.05
    t0 = -0.5 * (nt - 1) * dt
    K = 37
    w = 2 * np.pi * K / (nt * dt)
    t = t0 + dt * np.arange(nt)
    vz = np.cos(w * t)
    om, y, ph, v = O.spectrum(vz, dt, t0, 0.5 * nt * dt, 80)
    mag = np.abs(v)
    assert np.argmax(mag) == K
    assert mag[K] == pytest.approx(0.25 * nt * dt, rel=2e-3)
    assert mag[K + 1] == pytest.approx(0.125 * nt * dt, rel=2e-2)
    assert mag[K + 5] < 1e-2 * mag[K]

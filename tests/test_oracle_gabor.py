"""The oracle's Gabor time-frequency map (Sec. III.D), pinned by a closed form
(a Gaussian-enveloped cosine, whose windowed transform is a Gaussian
integral) and, for a window much wider than the signal, by numpy's FFT."""
import numpy as np

import oracle as O


def _closed_form(a, tau, Om, sigma, tm, w):
    # exp(-(t-a)^2/(2 tau^2)) exp(-(t-tm)^2/(2 sigma^2)) = A exp(-(t-c)^2/(2 s^2))
    s2 = sigma ** 2 * tau ** 2 / (sigma ** 2 + tau ** 2)
    c = (a * sigma ** 2 + tm * tau ** 2) / (sigma ** 2 + tau ** 2)
    A = np.exp(-(a - tm) ** 2 / (2.0 * (sigma ** 2 + tau ** 2)))
    f = lambda x: np.sqrt(2.0 * np.pi * s2) * np.exp(1j * x * c - 0.5 * s2 * x * x)
    return np.abs(0.5 * A * (f(w + Om) + f(w - Om))) ** 2


def test_gaussian_enveloped_cosine_closed_form():
    dt, t0, nt = 0.05, -200.0, 8001
    t = t0 + dt * np.arange(nt)
    a, tau, Om = 15.0, 25.0, 0.9
    vz = np.exp(-(t - a) ** 2 / (2 * tau ** 2)) * np.cos(Om * t)
    sigma = 1.0 / (3 * 0.057)
    tc = np.array([-60.0, 0.0, 15.0, 42.5, 90.0])
    om = np.linspace(0.2, 2.0, 37)
    G = O.gabor(vz, dt, t0, sigma, tc, om)
    ref = np.array([[_closed_form(a, tau, Om, sigma, tm, w) for w in om] for tm in tc])
    assert np.max(np.abs(G - ref)) <= 1e-12 * ref.max()


def test_wide_window_is_the_fourier_transform():
    # a window far wider than the signal: G(t_m, w_k) = |sum v e^{i w t} dt|^2,
    # here on the FFT grid w_k = 2 pi k / (N dt), from numpy's inverse FFT
    rng = np.random.default_rng(3)
    dt, t0, nt = 0.05, -10.0, 400
    vz = rng.standard_normal(nt) * np.hanning(nt)
    k = np.arange(0, 60, 7)
    om = 2 * np.pi * k / (nt * dt)
    G = O.gabor(vz, dt, t0, 1e7, [0.0], om)[0]
    # sum_n v_n e^{i w_k t_n} dt = e^{i w_k t0} sum_n v_n e^{2 pi i k n / N} dt; the
    # phase e^{i w_k t0} drops out of |.|^2
    V = np.fft.ifft(vz) * nt * dt
    ref = np.abs(V[k]) ** 2
    assert np.max(np.abs(G - ref)) <= 1e-10 * ref.max()


def test_map_is_nonnegative_and_shift_covariant():
    # shifting the signal by s grid points shifts the map in time by s dt
    rng = np.random.default_rng(5)
    dt, t0, nt, s = 0.05, 0.0, 3000, 100
    v = np.zeros(nt + s)
    v[:nt] = rng.standard_normal(nt) * np.hanning(nt)
    w = np.roll(v, s)
    om = np.linspace(0.1, 3.0, 11)
    G1 = O.gabor(v, dt, t0, 4.0, [40.0, 70.0], om)
    G2 = O.gabor(w, dt, t0, 4.0, [40.0 + s * dt, 70.0 + s * dt], om)
    assert np.all(G1 >= 0.0)
    assert np.allclose(G1, G2, rtol=1e-10, atol=1e-14 * G1.max())

"""Herman-Kluk exactness pin of the oracle's whole continuum leg (CPU only).

For a Hamiltonian at most quadratic in (q, p) the Herman-Kluk propagator is
exact.  A free electron in the laser field (length gauge, H = p^2/2 + z E(t))
is such a case.  Feeding the oracle's dipole sum an "ensemble" that is a
Gauss-Hermite grid over the initial phase space, weighted by
(2 pi)^-3 <p0,q0|g_a>, turns it into the HK approximation of

    D(t) = <psi0| k_z exp(-i H (t - t0)) |g_a>,

with g_a a coherent state.  The exact D(t) is computed here independently in
momentum space, where the length-gauge evolution is
psi(k,t) = g_a(k - Delta(t)) exp(-i int_{t0}^t (k - Delta(t) + Delta(t'))^2/2 dt'),
Delta(t) = A(t) - A(t0), by 1-D quadratures.  This pins at once the action
(sign and convention), the prefactor, the coherent-state phase convention and
the recombination element k_z.
"""
import math

import numpy as np

import oracle as O
from paper_2608_13686_b300 import workloads as W


def _exact_D(pa, qa, gamma, a, pulse, t0, times):
    k = np.linspace(-12, 12, 24001)
    hk = k[1] - k[0]
    psi0 = (1 / (2 * math.pi * a)) ** 0.25 * np.exp(-k * k / (4 * a))

    def ga(kk, d):
        return (1 / (math.pi * gamma)) ** 0.25 * np.exp(-(kk - pa[d]) ** 2 / (2 * gamma)
                                                        - 1j * kk * qa[d])

    A0 = O.pulse_A(pulse, [t0])[0]
    out = []
    for t in times:
        tau = t - t0
        ts = np.linspace(t0, t, 4001)
        Delta = O.pulse_A(pulse, ts) - A0
        Dt = Delta[-1]
        h = ts[1] - ts[0]

        def simpson(f):
            return h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())

        B = simpson(Delta - Dt) if tau > 0 else 0.0
        c = simpson(0.5 * (Delta - Dt) ** 2) if tau > 0 else 0.0
        fx = psi0 * ga(k, 0) * np.exp(-0.5j * k * k * tau)
        fy = psi0 * ga(k, 1) * np.exp(-0.5j * k * k * tau)
        fz = psi0 * k * ga(k - Dt, 2) * np.exp(-1j * (0.5 * k * k * tau + k * B + c))
        out.append(hk * fx.sum() * hk * fy.sum() * hk * fz.sum())
    return np.array(out)


def test_herman_kluk_exact_for_free_electron_in_laser():
    gamma, a = 1.0, 0.6
    pa, qa = np.array([0.2, -0.1, 0.5]), np.array([0.3, 0.1, -1.0])
    # a one-cycle 100 nm pulse at 5e15 W/cm^2, dt = 0.25: the trajectories
    # start near the pulse centre, where the field changes D(t) by ~50%
    pulse = W.pulse(100.0, 5e15, 1, dt=0.25)
    d = O.pulse_derived(pulse)
    n0, ncmp = 24, 4
    t0 = d["t_origin"] + n0 * d["dt"]
    target = W.harmonic_target(0.0, prims=((a, 1.0),))      # psi0: one Gaussian at 0
    target["R"] = 0.0

    ng = 8
    x, wgh = np.polynomial.hermite.hermgauss(ng)
    # q0 = qa + (2/sqrt(g)) x, p0 = pa + 2 sqrt(g) x: Gauss-Hermite against
    # exp(-g/4 (q0-qa)^2 - (p0-pa)^2/(4g)), the modulus of <p0,q0|g_a>
    grids = np.meshgrid(*([np.arange(ng)] * 6), indexing="ij")
    idx = [g.ravel() for g in grids]
    n = idx[0].size
    q0 = np.stack([qa[i] + 2 / math.sqrt(gamma) * x[idx[i]] for i in range(3)])
    p0 = np.stack([pa[i] + 2 * math.sqrt(gamma) * x[idx[3 + i]] for i in range(3)])
    wq = np.prod([wgh[idx[i]] for i in range(6)], axis=0) * 4.0 ** 3
    # <p0,q0|g_a> = exp(-g/4|q0-qa|^2 - |p0-pa|^2/(4g) + (i/2)(p0+pa).(q0-qa))
    phase = np.exp(0.5j * np.sum((p0 + pa[:, None]) * (q0 - qa[:, None]), axis=0))
    w = (2 * math.pi) ** -3 * wq * phase

    soa = np.zeros((O.NFIELDS, n))
    soa[0] = n0
    soa[1:4] = q0
    soa[4:7] = p0
    soa[9] = 1.0
    soa[10], soa[11] = w.real, w.imag
    vre, _, bad = O.propagate(target, pulse, soa, gamma, n_norm=1.0)
    assert bad == 0
    wi = -1j * w
    soa[10], soa[11] = wi.real, wi.imag
    vim, _, _ = O.propagate(target, pulse, soa, gamma, n_norm=1.0)
    D_hk = -0.5 * (vre[n0:n0 + ncmp + 1] + 1j * vim[n0:n0 + ncmp + 1])   # vz = -2 Re(...)

    times = t0 + d["dt"] * np.arange(ncmp + 1)
    D_ex = _exact_D(pa, qa, gamma, a, pulse, t0, times)
    scale = np.abs(D_ex).max()
    # the residual is the 8-node Gauss-Hermite error (it falls with more nodes)
    err = np.abs(D_hk - D_ex) / scale
    assert err.max() < 1e-2, err
    # the field matters here: the field-free answer is far off
    D_free = _exact_D(pa, qa, gamma, a, W.pulse(100.0, 0.0, 1, dt=0.25), t0, times)
    assert np.abs(D_free - D_ex).max() / scale > 0.2

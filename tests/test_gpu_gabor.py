"""Gabor time-frequency map on the GPU (sfhk_gabor) against the oracle's
definition, host and device buffers, several tiles of frequencies and a
window wider than one staged chunk, and the degenerate cases."""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk
    return sfhk


def _signal(nt, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(nt)
    return (rng.standard_normal(nt) * np.hanning(nt) + np.sin(0.9 * 0.05 * t)
            * np.exp(-((t - nt / 2) / (nt / 6)) ** 2))


@pytest.mark.parametrize("nt,sigma,n_t,n_w", [
    (6620, 1.0 / (3 * 0.057), 33, 70),     # the H2 grid, sigma = 1/(3 w0)
    (2001, 40.0, 5, 300),                  # window wider than a staged chunk, >1 tile of w
    (17, 0.3, 4, 1),                       # tiny
])
def test_gabor_matches_oracle(S, nt, sigma, n_t, n_w):
    dt, t0 = 0.05, -0.5 * 0.05 * (nt - 1)
    vz = _signal(nt, nt)
    t_first, t_step = t0 - 3.0, (2 * abs(t0) + 6.0) / max(n_t - 1, 1)
    w_first, w_step = 0.05, 3.5 / max(n_w, 1)
    G = S.sfhk_gabor(vz, dt, t0, sigma, t_first, t_step, n_t, w_first, w_step, n_w)
    tc = t_first + t_step * np.arange(n_t)
    om = w_first + w_step * np.arange(n_w)
    ref = O.gabor(vz, dt, t0, sigma, tc, om)
    assert G.shape == ref.shape
    assert np.max(np.abs(G - ref)) <= 1e-10 * ref.max()


def test_gabor_of_an_oracle_dipole_device_buffers(S):
    import torch
    t, p = W.TARGETS["H2"], W.PULSE_800
    soa, _, _ = O.sample(t, p, W.fixed(0.0), seed=4, n=64)
    vz, _, _ = O.propagate(t, p, soa, W.GAMMA, cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF)
    d = O.pulse_derived(p)
    w0 = 45.5633525 / p["lambda_nm"]
    sigma = 1.0 / (3.0 * w0)
    n_t, n_w = 48, 96
    t_first, t_step = d["t_origin"], d["Tp"] / (n_t - 1)
    w_first, w_step = w0, 30.0 * w0 / n_w
    dvz = torch.tensor(vz, dtype=torch.float64, device="cuda")
    out = torch.zeros((n_t, n_w), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    S.sfhk_gabor_device(dvz.data_ptr(), len(vz), d["dt"], d["t_origin"], sigma, t_first, t_step,
                        n_t, w_first, w_step, n_w, out.data_ptr(), s.cuda_stream)
    s.synchronize()
    ref = O.gabor(vz, d["dt"], d["t_origin"], sigma, t_first + t_step * np.arange(n_t),
                  w_first + w_step * np.arange(n_w))
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-10 * ref.max()


def test_window_outside_the_signal_is_zero_and_bad_arguments_are_refused(S):
    vz = _signal(500, 1)
    G = S.sfhk_gabor(vz, 0.05, 0.0, 1.0, 1e6, 1.0, 3, 0.1, 0.1, 5)
    assert np.all(G == 0.0)
    G = S.sfhk_gabor(vz, 0.05, 0.0, 1.0, -1e300, 0.0, 2, 0.1, 0.1, 5)
    assert np.all(G == 0.0)
    for bad in (dict(dt=0.0), dict(sigma=-1.0), dict(n_t=0), dict(n_w=0),
                dict(t_step=float("nan"))):
        a = dict(dt=0.05, t_origin=0.0, sigma=1.0, t_first=0.0, t_step=1.0, n_t=2,
                 omega_first=0.1, omega_step=0.1, n_w=2)
        a.update(bad)
        with pytest.raises(RuntimeError):
            S.sfhk_gabor(vz, a["dt"], a["t_origin"], a["sigma"], a["t_first"], a["t_step"],
                         a["n_t"], a["omega_first"], a["omega_step"], a["n_w"])

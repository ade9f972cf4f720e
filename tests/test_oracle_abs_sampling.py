"""Initial points distributed ~ |a| (Sec. II.B: the initial points are drawn
according to |sin(beta) <W| r.E |psi0>|) in the oracle's sampler, done as
rejection with weight correction on top of the ADK/Gaussian proposal:
accept a draw of weight w with alpha = min(1, |w|/M), give it P w / alpha.

Pinned by: unbiasedness (weighted means of several functions of the initial
point agree with those of the plain importance-sampled ensemble within their
statistical error), the weight rule on every trajectory whose first attempt
was accepted (it is then the plain sampler's trajectory), the bound
|omega| >= P M on all weights, and the variance reduction the scheme exists
for."""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

T, P_ = W.TARGETS["H2"], W.PULSE_800


def _w(s):
    return s[10] + 1j * s[11]


def test_weight_rule_and_bound():
    ta = W.abs_sampled(T, 5.0)
    n = 600
    sa, _, bad = O.sample(ta, P_, W.fixed(0.0), seed=4, n=n)
    sp, _, _ = O.sample(T, P_, W.fixed(0.0), seed=4, n=n)
    M, P = O.abs_sampling_constants(ta, P_, W.fixed(0.0), seed=4)
    assert bad == 0 and 0.0 < P < 1.0 and M > 0.0
    wa, wp = _w(sa), _w(sp)
    assert np.all(np.abs(wa) >= P * M * (1.0 - 1e-12))
    first = np.all(sa[0:10] == sp[0:10], axis=0)          # attempt 0 accepted
    assert first.sum() > 0.05 * n
    alpha = np.minimum(1.0, np.abs(wp[first]) / M)
    keep = P / (1.0 - (1.0 - P) ** 256)
    assert np.allclose(wa[first], keep * wp[first] / alpha, rtol=1e-13, atol=0.0)


@pytest.mark.parametrize("align,kappa", [(W.fixed(0.0), 5.0), (W.ISO, 2.0)])
def test_unbiased_against_the_plain_sampler(align, kappa):
    na, npl = 12000, 60000
    sa, _, _ = O.sample(W.abs_sampled(T, kappa), P_, align, seed=21, n=na)
    sp, _, _ = O.sample(T, P_, align, seed=22, n=npl)
    funcs = [lambda s: np.ones(s.shape[1]), lambda s: s[6], lambda s: s[3],
             lambda s: s[4] ** 2 + s[5] ** 2]
    for g in funcs:
        xa, xp = _w(sa) * g(sa), _w(sp) * g(sp)
        se = np.hypot(np.std(xa) / np.sqrt(na), np.std(xp) / np.sqrt(npl))
        assert abs(xa.mean() - xp.mean()) <= 5.0 * se


def test_variance_per_point_is_lower():
    n = 8000
    sa, _, _ = O.sample(W.abs_sampled(T, 5.0), P_, W.fixed(0.0), seed=31, n=n)
    sp, _, _ = O.sample(T, P_, W.fixed(0.0), seed=32, n=n)
    assert np.var(_w(sa)) < 0.5 * np.var(_w(sp))


def test_unbiased_at_a_large_factor_with_the_attempt_cap():
    """At kappa = 150 an attempt is accepted with P ~ 0.0064, so about 19 % of
    the trajectories exhaust their 256 attempts and get weight 0.  Every
    attempt has the same acceptance probability, so the invalid count is
    binomial with q = (1 - P)^256, and the kept weights must carry the factor
    1 / (1 - q) for the mean over all N trajectories to stay unbiased.

    The means compared are of |w| g (the phase of an accepted weight is the
    proposal's, so E[|omega| g] = int |a| g under both samplers), which have
    a definite sign and resolve the factor: dropping it (the planted mistake,
    applied here as the multiplication by 1 - q) moves the g = 1 mean by
    about 16 standard errors."""
    kappa, na, npl = 150.0, 3000, 200000
    ta = W.abs_sampled(T, kappa)
    _, P = O.abs_sampling_constants(ta, P_, W.fixed(0.0), seed=21)
    q = (1.0 - P) ** 256
    assert 0.1 < q < 0.3
    sa, _, bad = O.sample(ta, P_, W.fixed(0.0), seed=21, n=na)
    sp, _, _ = O.sample(T, P_, W.fixed(0.0), seed=22, n=npl)
    assert abs(bad - na * q) <= 5.0 * np.sqrt(na * q * (1.0 - q))
    funcs = [lambda s: np.ones(s.shape[1]), lambda s: np.abs(s[6]), lambda s: np.abs(s[3])]
    for i, g in enumerate(funcs):
        xa, xp = np.abs(_w(sa)) * g(sa), np.abs(_w(sp)) * g(sp)
        se = np.hypot(np.std(xa) / np.sqrt(na), np.std(xp) / np.sqrt(npl))
        assert abs(xa.mean() - xp.mean()) <= 4.0 * se
        if i == 0:
            assert abs((1.0 - q) * xa.mean() - xp.mean()) >= 8.0 * se

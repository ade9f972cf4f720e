"""p-type Gaussian primitives in the oracle's orbital.  Sigma p-type (the N2
HOMO, 3 sigma_g, has p character): phi_{c,k}(x) = s_c n.(x - A_c)
e^{-a|x - A_c|^2}, s_c = +-1 for the centre at +-(R/2) n, so that the sum is
gerade.  Pi p-type (the N2 HOMO-1, 1 pi_u, Table II): m.(x - A_c)
e^{-a|x - A_c|^2} on both centres with the same sign (ungerade), m the unit
vector perpendicular to n at the target's azimuth.

Pinned by brute force on a 3D grid (the trapezoid rule is spectrally
accurate for Gaussians): the normalisation, the inversion symmetry, the
ionization dipole element <kappa| z |psi0> (Eq. 1) and the recombination
element <psi0| k_z |p, q> (Eq. 4) against their closed forms."""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

T = W.TARGETS["N2_sp"]
NH = np.array([np.sin(0.6) * np.cos(0.3), np.sin(0.6) * np.sin(0.3), np.cos(0.6)])
H = 0.15
G = np.arange(-10.5, 10.5 + H / 2, H)


TPI = W.pi_component(W.TARGETS["N2_pi"], 0.7)


@pytest.fixture(scope="module")
def rgrid():
    X, Y, Z = np.meshgrid(G, G, G, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


@pytest.fixture(scope="module")
def grid(rgrid):
    return rgrid, O.orbital_values(T, NH, rgrid)


@pytest.fixture(scope="module")
def pigrid(rgrid):
    return rgrid, O.orbital_values(TPI, NH, rgrid)


def test_normalised_and_gerade(grid):
    r, v = grid
    assert abs((v * v).sum() * H ** 3 - 1.0) <= 1e-8
    assert np.max(np.abs(v - O.orbital_values(T, NH, -r))) <= 1e-14
    # the p primitives matter: without them the orbital differs
    ts = dict(T, pkind=[0, 0, 0, 0])
    assert abs(O.orbital_norm(ts) - O.orbital_norm(T)) > 1e-3


@pytest.mark.parametrize("kappa", [(0.3, -0.2, 0.5), (0.0, 0.1, -0.9), (0.6, 0.4, 0.2 + 0.15j)])
def test_dipole_element_against_the_integral(grid, kappa):
    r, v = grid
    k = np.asarray(kappa, complex)
    num = (np.exp(-1j * (r @ k)) * r[:, 2] * v).sum() * H ** 3 * (2 * np.pi) ** -1.5
    ref = O.dipole_matrix_element(T, NH, k)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("q,p", [((0.4, -0.3, 1.1), (0.2, 0.1, -0.7)),
                                 ((-1.5, 0.2, -0.6), (0.0, -0.4, 1.3)),
                                 ((0.1, 0.9, 2.4), (0.5, 0.3, 0.8))])
def test_recombination_element_against_the_integral(grid, q, p):
    r, v = grid
    g = 0.5
    q, p = np.asarray(q), np.asarray(p)
    d = r - q
    cs = (g / np.pi) ** 0.75 * np.exp(-0.5 * g * (d * d).sum(1) + 1j * (d @ p))
    num = (v * (p[2] + 1j * g * d[:, 2]) * cs).sum() * H ** 3
    ref = O.recomb(T, NH, q, p, g)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))


# ------------------------------------------------------------------ pi p-type
def test_pi_direction():
    """m is a unit vector perpendicular to n; chi = 0 lies in the plane of n
    and z, chi = pi/2 is perpendicular to it; on the z axis m(chi = 0) = x."""
    zhat = np.array([0.0, 0.0, 1.0])
    for chi in (0.0, 0.7, np.pi / 2, 2.5):
        m = O.pi_direction(NH, chi)
        assert abs(m @ m - 1.0) <= 1e-15 and abs(m @ NH) <= 1e-15
    assert abs(O.pi_direction(NH, 0.0) @ np.cross(NH, zhat)) <= 1e-15
    assert abs(O.pi_direction(NH, np.pi / 2) @ zhat) <= 1e-15
    assert np.allclose(O.pi_direction(zhat, 0.0), [1.0, 0.0, 0.0], atol=1e-15)
    assert np.allclose(O.pi_direction(zhat, np.pi / 2), [0.0, 1.0, 0.0], atol=1e-15)


def test_pi_normalised_ungerade_and_degenerate_pair(pigrid):
    r, v = pigrid
    assert abs((v * v).sum() * H ** 3 - 1.0) <= 1e-8
    assert np.max(np.abs(v + O.orbital_values(TPI, NH, -r))) <= 1e-14
    # the two components at chi and chi + pi/2 are orthogonal, and
    # orthogonal to the sigma_g orbital
    v2 = O.orbital_values(W.pi_component(TPI, 0.7 + np.pi / 2), NH, r)
    assert abs((v * v2).sum() * H ** 3) <= 1e-10
    vs = O.orbital_values(T, NH, r)
    assert abs((v * vs).sum() * H ** 3) <= 1e-10
    # the orbital changes sign under a rotation by pi about n (m -> -m)
    v3 = O.orbital_values(W.pi_component(TPI, 0.7 + np.pi), NH, r)
    assert np.max(np.abs(v + v3)) <= 1e-14


@pytest.mark.parametrize("kappa", [(0.3, -0.2, 0.5), (0.6, 0.4, 0.2 + 0.15j)])
def test_pi_dipole_element_against_the_integral(pigrid, kappa):
    r, v = pigrid
    k = np.asarray(kappa, complex)
    num = (np.exp(-1j * (r @ k)) * r[:, 2] * v).sum() * H ** 3 * (2 * np.pi) ** -1.5
    ref = O.dipole_matrix_element(TPI, NH, k)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("q,p", [((0.4, -0.3, 1.1), (0.2, 0.1, -0.7)),
                                 ((-1.5, 0.2, -0.6), (0.0, -0.4, 1.3))])
def test_pi_recombination_element_against_the_integral(pigrid, q, p):
    r, v = pigrid
    g = 0.5
    q, p = np.asarray(q), np.asarray(p)
    d = r - q
    cs = (g / np.pi) ** 0.75 * np.exp(-0.5 * g * (d * d).sum(1) + 1j * (d @ p))
    num = (v * (p[2] + 1j * g * d[:, 2]) * cs).sum() * H ** 3
    ref = O.recomb(TPI, NH, q, p, g)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))


def test_pi_parallel_axis_has_no_dipole_along_z():
    """With the axis along the field (n = z) a pi_u orbital is odd under the
    reflection through the plane perpendicular to m, so <kappa|z|psi> vanishes
    for kappa in that plane, and so does <psi|k_z|p,q> for q, p in it."""
    z = np.array([0.0, 0.0, 1.0])
    t = W.pi_component(W.TARGETS["N2_pi"], 0.0)     # m = x
    assert abs(O.dipole_matrix_element(t, z, np.array([0.0, 0.3, 0.5 + 0.2j]))) <= 1e-16
    assert abs(O.recomb(t, z, np.array([0.0, 0.4, -1.0]), np.array([0.0, -0.2, 0.9]), 0.5)) <= 1e-16
    assert abs(O.dipole_matrix_element(t, z, np.array([0.2, 0.3, 0.5 + 0.2j]))) > 1e-4

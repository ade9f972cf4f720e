"""Polyatomic targets in the oracle: the model potential of Eq. 7 summed over N
centres, each with its own charges, the molecule turned by the ZYZ Euler
angles (phi, theta, psi) (the orientation of Eq. 6 in full), and an orbital
of Gaussian primitives each on its own centre (s-type, or p-type along a
molecular-frame direction).

Pins that do not use the oracle against itself:
  * the Euler rotation is orthonormal with det 1 and carries z to the axis
    n(theta, phi);
  * force and Hessian are the finite differences of V (bent triatomic);
  * V, the orbital, the dipole element and the recombination element are
    covariant under rotation: turning the molecule equals turning the
    evaluation point (and kappa, p) the other way;
  * a diatomic written as a two-centre polyatomic reproduces the diatomic
    (itself pinned elsewhere) in V, orbital, both elements, the sampler and
    the propagated dipole;
  * the normalisation, the dipole element and the recombination element of a
    bent molecule against brute-force 3D grid integrals;
  * isotropic sampling is uniform over the rotation group (moments of the
    rotation matrix entries)."""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

T_B1 = W.TARGETS["H2O"]
T_A1 = W.TARGETS["H2O_3a1"]
ANG = (0.4, 1.1, -0.7)          # (phi, theta, psi)


def _n(theta, phi):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def test_euler_rotation():
    R = O.euler_rotation(*ANG)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(R) - 1.0) <= 1e-14
    assert np.allclose(R @ [0.0, 0.0, 1.0], _n(ANG[1], ANG[0]), atol=1e-15)
    # psi turns the molecule about its own axis first
    Rz = O.euler_rotation(0.0, 0.0, ANG[2])
    assert np.allclose(Rz, [[np.cos(ANG[2]), -np.sin(ANG[2]), 0], [np.sin(ANG[2]), np.cos(ANG[2]), 0],
                            [0, 0, 1]], atol=1e-15)


@pytest.mark.parametrize("q", [(0.3, -0.8, 0.5), (1.2, 0.4, 1.9), (-0.2, 0.1, -1.3)])
def test_force_and_hessian_are_derivatives(q):
    q = np.asarray(q, float)
    V, g, H = O.potential(T_A1, ANG, q)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Vp, gp, _ = O.potential(T_A1, ANG, q + e)
        Vm, gm, _ = O.potential(T_A1, ANG, q - e)
        assert abs((Vp - Vm) / (2 * h) - g[a]) <= 1e-7 * max(1.0, abs(g[a]))
        assert np.allclose((gp - gm) / (2 * h), H[:, a], rtol=1e-6, atol=1e-7)
    assert np.allclose(H, H.T, atol=1e-14)


def test_potential_is_the_sum_over_centres_and_rotates():
    """V at a lab point equals the sum of the single-centre soft-core terms at
    the rotated centres; and is unchanged when the molecule and the point turn
    together."""
    q = np.array([0.7, -0.4, 0.9])
    R = O.euler_rotation(*ANG)
    a2 = T_A1["soft_a"] ** 2
    ref = 0.0
    for c in T_A1["centres"]:
        s = np.sqrt(np.sum((q - R @ np.asarray(c[:3])) ** 2) + a2)
        ref -= (c[3] + (c[4] - c[3]) * np.exp(-c[5] * s)) / s
    V, g, H = O.potential(T_A1, ANG, q)
    assert abs(V - ref) <= 1e-13 * abs(ref)
    V0, g0, H0 = O.potential(T_A1, (0.0, 0.0, 0.0), R.T @ q)
    assert abs(V - V0) <= 1e-13 * abs(V)
    assert np.allclose(g, R @ g0, atol=1e-13)
    assert np.allclose(H, R @ H0 @ R.T, atol=1e-12)


def test_elements_rotate_with_the_molecule():
    """The z-dipole and k_z-recombination elements single out the lab z axis,
    so the covariance check turns the molecule about z only (phi), with the
    point, kappa, q and p turned the same way."""
    a1 = (0.3, 0.9, 0.5)
    d = 0.8
    a2 = (0.3 + d, 0.9, 0.5)
    Rz = O.euler_rotation(d, 0.0, 0.0)
    for t in (T_B1, T_A1):
        r = np.array([0.4, -0.2, 0.7])
        assert abs(O.orbital_value(t, a2, Rz @ r) - O.orbital_value(t, a1, r)) <= 1e-14
        k = np.array([0.3, -0.5, 0.2 + 0.4j])
        kr = np.concatenate([Rz[:2, :2] @ k[:2].real, [k[2]]]).astype(complex)
        m1 = O.dipole_matrix_element(t, a1, k)
        m2 = O.dipole_matrix_element(t, a2, kr)
        assert abs(m1 - m2) <= 1e-13 * max(1.0, abs(m1))
        q, p = np.array([0.5, 1.1, -0.6]), np.array([-0.3, 0.2, 0.9])
        r1 = O.recomb(t, a1, q, p, 0.5)
        r2 = O.recomb(t, a2, Rz @ q, Rz @ p, 0.5)
        assert abs(r1 - r2) <= 1e-13 * max(1.0, abs(r1))


# ------------------------------------------------------------------ diatomic as polyatomic
@pytest.mark.parametrize("name", ["N2", "N2_sp", "H2"])
def test_diatomic_written_as_polyatomic(name):
    t = W.TARGETS[name]
    tp = W.diatomic_as_poly(t)
    th, ph, ps = 0.8, -0.6, 1.3
    n = _n(th, ph)
    ang = (ph, th, ps)
    assert abs(O.orbital_norm(tp) - O.orbital_norm(t)) <= 1e-14 * O.orbital_norm(t)
    q, p = np.array([0.6, -0.9, 1.4]), np.array([0.2, 0.7, -0.4])
    V1, g1, H1 = O.potential(t, n, q)
    V2, g2, H2 = O.potential(tp, ang, q)
    assert abs(V1 - V2) <= 1e-14 * abs(V1)
    assert np.allclose(g1, g2, atol=1e-14) and np.allclose(H1, H2, atol=1e-13)
    assert abs(O.orbital_value(t, n, q) - O.orbital_value(tp, ang, q)) <= 1e-14
    k = np.array([0.3, -0.2, 0.4 + 0.6j])
    m1, m2 = O.dipole_matrix_element(t, n, k), O.dipole_matrix_element(tp, ang, k)
    assert abs(m1 - m2) <= 1e-13 * abs(m1)
    r1, r2 = O.recomb(t, n, q, p, 0.5), O.recomb(tp, ang, q, p, 0.5)
    assert abs(r1 - r2) <= 1e-13 * abs(r1)


def test_diatomic_as_polyatomic_sampler_and_dipole():
    """Same draws: t0, exit, momentum and weight agree with the diatomic
    sampler; the orientation fields hold (phi, theta, psi) with n(theta, phi)
    the diatomic's axis; the propagated dipoles agree."""
    t = W.TARGETS["N2_sp"]
    tp = W.diatomic_as_poly(t)
    pulse = W.PULSE_1200
    s1, _, b1 = O.sample(t, pulse, W.ISO, seed=3, n=64)
    s2, _, b2 = O.sample(tp, pulse, W.ISO, seed=3, n=64)
    assert b1 == b2
    assert np.array_equal(s1[0], s2[0])
    for f in (1, 2, 3, 4, 5, 6):
        assert np.allclose(s1[f], s2[f], rtol=1e-13, atol=1e-13)
    w1, w2 = s1[10] + 1j * s1[11], s2[10] + 1j * s2[11]
    assert np.all(np.abs(w1 - w2) <= 1e-12 * np.abs(w1) + 1e-300)
    n2 = np.stack([_n(s2[8][i], s2[7][i]) for i in range(64)], 1)
    assert np.allclose(n2, s1[7:10], atol=1e-14)
    assert np.all((s2[9] >= 0) & (s2[9] < 2 * np.pi))
    v1, _, _ = O.propagate(t, pulse, s1[:, :16], 0.5, cutoff=1e4, stab_cutoff=1e3)
    v2, _, _ = O.propagate(tp, pulse, s2[:, :16], 0.5, cutoff=1e4, stab_cutoff=1e3)
    assert np.linalg.norm(v1 - v2) <= 1e-9 * np.linalg.norm(v1)


def test_polyatomic_refuses_quadrature_and_sfhk2():
    with pytest.raises(ValueError):
        O.sample(T_A1, W.PULSE_800, W.quadrature(4), n=4)
    with pytest.raises(ValueError):
        O.sample(W.sfhk2(T_A1), W.PULSE_800, W.ISO, n=4)


def test_isotropic_rotations_are_uniform():
    """Haar measure on SO(3): every entry of the rotation matrix has mean 0
    and mean square 1/3."""
    s, _, _ = O.sample(T_A1, W.PULSE_800, W.ISO, seed=5, n=20000)
    Rs = np.stack([O.euler_rotation(*s[7:10, i]) for i in range(4000)])
    m1, m2 = Rs.mean(0), (Rs ** 2).mean(0)
    se = np.sqrt(1.0 / 3.0 / 4000)
    assert np.all(np.abs(m1) <= 5 * se)
    assert np.all(np.abs(m2 - 1.0 / 3.0) <= 5 * 0.3 / np.sqrt(4000))


# ------------------------------------------------------------------ grid integrals
H = 0.15
G = np.arange(-10.5, 10.5 + H / 2, H)


@pytest.fixture(scope="module")
def rgrid():
    X, Y, Z = np.meshgrid(G, G, G, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


@pytest.fixture(scope="module", params=["H2O", "H2O_3a1"])
def orb(request, rgrid):
    t = W.TARGETS[request.param]
    return t, rgrid, O.orbital_values(t, ANG, rgrid)


def test_normalised(orb):
    t, r, v = orb
    assert abs((v * v).sum() * H ** 3 - 1.0) <= 1e-8


def test_b1_is_odd_under_the_molecular_plane():
    """1b1 changes sign under reflection through the molecular (xz) plane,
    3a1 does not (molecular frame, identity rotation)."""
    r = np.array([[0.3, 0.7, 0.2], [-0.5, 1.1, 0.9], [0.1, 0.4, -0.6]])
    rr = r * [1.0, -1.0, 1.0]
    for x, y in zip(r, rr):
        assert abs(O.orbital_value(T_B1, (0, 0, 0), x) + O.orbital_value(T_B1, (0, 0, 0), y)) <= 1e-15
        assert abs(O.orbital_value(T_A1, (0, 0, 0), x) - O.orbital_value(T_A1, (0, 0, 0), y)) <= 1e-15


@pytest.mark.parametrize("kappa", [(0.3, -0.2, 0.5), (0.6, 0.4, 0.2 + 0.15j)])
def test_dipole_element_against_the_integral(orb, kappa):
    t, r, v = orb
    k = np.asarray(kappa, complex)
    num = (np.exp(-1j * (r @ k)) * r[:, 2] * v).sum() * H ** 3 * (2 * np.pi) ** -1.5
    ref = O.dipole_matrix_element(t, ANG, k)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("q,p", [((0.4, -0.3, 1.1), (0.2, 0.1, -0.7)),
                                 ((-1.5, 0.2, -0.6), (0.0, -0.4, 1.3))])
def test_recombination_element_against_the_integral(orb, q, p):
    t, r, v = orb
    g = 0.5
    q, p = np.asarray(q), np.asarray(p)
    d = r - q
    cs = (g / np.pi) ** 0.75 * np.exp(-0.5 * g * (d * d).sum(1) + 1j * (d @ p))
    num = (v * (p[2] + 1j * g * d[:, 2]) * cs).sum() * H ** 3
    ref = O.recomb(t, ANG, q, p, g)
    assert abs(num - ref) <= 1e-9 * max(1.0, abs(ref))

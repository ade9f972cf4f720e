"""Sigma p-type Gaussian primitives in the oracle's orbital (the N2 HOMO,
3 sigma_g, has p character): phi_{c,k}(x) = s_c n.(x - A_c) e^{-a|x - A_c|^2},
s_c = +-1 for the centre at +-(R/2) n, so that the sum is gerade.

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


@pytest.fixture(scope="module")
def grid():
    X, Y, Z = np.meshgrid(G, G, G, indexing="ij")
    r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    return r, O.orbital_values(T, NH, r)


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

"""Pins of the oracle's final synthesis (Sect. 2.5, last paragraphs; CPU only): the k-d tree
two-nearest search equals brute force (periodic sides, ragged site density), the inverse-distance
weights reproduce site values on sites and constants everywhere, and the vertical emergent
intensity equals the closed-form column integral for a constant source function."""
import numpy as np

from oracle.synthesis import (emergent_mu1, idw_weights, interpolate, mesh_points,
                              two_nearest, two_nearest_bruteforce)


def _sites(rng, n):
    # denser towards the bottom, like the |dtau/dz| densities
    xyz = rng.random((n, 3))
    xyz[:, 2] = xyz[:, 2] ** 3
    return xyz


def test_two_nearest_kdtree_equals_bruteforce():
    rng = np.random.default_rng(5)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    sites = _sites(rng, 700)
    targets = np.concatenate([rng.random((500, 3)), mesh_points(8, 8, 0.125, 0.125,
                                                               np.linspace(0.01, 0.99, 7))])
    k1, d1 = two_nearest(sites, targets, box)
    k2, d2 = two_nearest_bruteforce(sites, targets, box)
    np.testing.assert_allclose(d1, d2, rtol=1e-12)
    np.testing.assert_array_equal(k1, k2)


def test_idw_on_sites_and_constants():
    rng = np.random.default_rng(6)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    sites = _sites(rng, 300)
    vals = rng.random((3, 300))
    k, d = two_nearest(sites, sites[:50], box)
    np.testing.assert_allclose(interpolate(vals, k, idw_weights(d)), vals[:, :50], rtol=0,
                               atol=0)
    targets = rng.random((200, 3))
    k, d = two_nearest(sites, targets, box)
    w = idw_weights(d)
    np.testing.assert_allclose(w.sum(1), 1.0, rtol=1e-14)
    assert np.all(w[:, 0] >= w[:, 1])            # the nearer site weighs more
    np.testing.assert_allclose(interpolate(np.full((1, 300), 2.5), k, w), 2.5, rtol=1e-14)


def test_emergent_mu1_constant_source_closed_form():
    nx, ny, nz = 4, 3, 12
    z = np.cumsum(np.r_[0.0, np.linspace(0.1, 0.6, nz - 1)])
    a = np.full((2, nx * ny * nz), 0.7)
    S = np.full((2, nx * ny * nz), 1.3)
    I = emergent_mu1(nx, ny, nz, 0.5, 0.5, z, a, S, bc=1)   # no inflow
    np.testing.assert_allclose(I, 1.3 * (1.0 - np.exp(-0.7 * (z[-1] - z[0]))), rtol=1e-13)

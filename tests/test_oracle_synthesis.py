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


def test_regular_maps_converge_to_the_fine_reference():
    """The mu = 1 map of the LTE continuum (500 nm) on regular grids of 32 x 32 x 64 and
    64 x 64 x 128 points approaches that of the 128 x 128 x 256 reference at the shared pixels,
    at close to second order (linear S across each interval, Eq. 2): the RMS relative difference
    falls by more than a factor 3 when the cells halve."""
    from oracle.physics import lte_alpha_S
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)

    def mu1_map(n):
        f, (x, y, z, dx, dy) = regular_fields(n, n, 2 * n, atm)
        a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
        return emergent_mu1(n, n, 2 * n, dx, dy, z, a[None], s[None])[0].reshape(n, n)
    fine = mu1_map(128)
    err = [np.sqrt(np.mean((mu1_map(n) / fine[::128 // n, ::128 // n] - 1.0) ** 2))
           for n in (32, 64)]
    assert err[0] / err[1] > 3.0, err


def test_top_sites_are_the_top_layer_of_a_lattice():
    """The emergent layer (sites with a mirror in the top wall) of a lattice of sites is exactly
    its top layer of sites."""
    from helpers import lattice_grid
    from oracle.synthesis import top_sites
    g = lattice_grid(4, 5)
    np.testing.assert_array_equal(top_sites(g["nbr_off"], g["nbr_idx"]), np.arange(64, 80))

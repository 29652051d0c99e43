"""Pins of the oracle's rejection sampling of Voronoi sites (Sect. 2.4; CPU only).

* Its Philox4x64-10 blocks equal numpy's own implementation of the generator (a separate code
  base), for keys and counters that exercise every word, the counter's carry included.
* A constant target accepts every proposal: the sites are the proposals themselves.
* The trilinear interpolation reproduces a trilinear function exactly (non-uniform z) and equals
  scipy's interpolator on a random mesh padded with its periodic images (clamped beyond the end
  planes).
* The accepted sites follow the target: for f linear in z the heights pass a Kolmogorov-Smirnov
  test against the exact distribution, x and y against the uniform one, and the acceptance rate
  is mean f / max f within five standard deviations.
"""
import numpy as np
import pytest
from scipy import stats

from oracle.sampling import interpolate, philox4x64, proposals, rejection_sample, uniform53

BOX = (0.0, 6.0, 0.0, 6.0, -0.5, 2.5)


def _split(v):
    return [(v >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]


@pytest.mark.parametrize("key,counter", [((12345, 0), (0, 0, 0, 0)),
                                         ((2 ** 63 + 7, 99), (2 ** 64 - 2, 3, 7, 11)),
                                         ((1, 2 ** 64 - 1), (5, 2 ** 64 - 1, 0, 2 ** 40))])
def test_philox_blocks_equal_numpy(key, counter):
    n = 6
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(counter, dtype=np.uint64))
    ref = bg.random_raw(4 * n).reshape(n, 4)            # numpy steps the counter, then draws
    c = sum(int(w) << (64 * i) for i, w in enumerate(counter))
    ctr = np.array([_split((c + s) % 2 ** 256) for s in range(1, n + 1)], dtype=np.uint64)
    np.testing.assert_array_equal(philox4x64(ctr, key), ref)


def test_uniform53_is_exact():
    w = np.array([0, 2 ** 11 - 1, 2 ** 11, 2 ** 64 - 1], dtype=np.uint64)
    np.testing.assert_array_equal(uniform53(w), [0.0, 0.0, 2.0 ** -53, 1.0 - 2.0 ** -53])


def test_constant_target_keeps_every_proposal():
    f = np.full((5, 4, 6), 3.0)
    z = np.linspace(-0.5, 2.5, 5)
    xyz, nprop = rejection_sample(f, z, BOX, 1000, seed=7)
    pos, _ = proposals(7, 0, 1000, BOX)
    assert nprop == 1000
    np.testing.assert_array_equal(xyz, pos)


def test_trilinear_interpolation_is_exact_for_trilinear_functions():
    nx, ny = 12, 10
    z = np.sort(np.r_[-0.5, 2.5, np.random.default_rng(1).uniform(-0.5, 2.5, 7)])
    g = lambda x, y, zz: (1.0 + 0.3 * x) * (2.0 - 0.1 * y) * (0.5 + zz)   # noqa: E731
    X = np.arange(nx) * 6.0 / nx
    Y = np.arange(ny) * 6.0 / ny
    Z, YY, XX = np.meshgrid(z, Y, X, indexing="ij")
    f = g(XX, YY, Z)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(0, X[-1], 500), rng.uniform(0, Y[-1], 500),
                    rng.uniform(z[0], z[-1], 500)], axis=1)       # away from the periodic seam
    np.testing.assert_allclose(interpolate(f, z, BOX, pts), g(*pts.T), rtol=1e-12)
    mesh = np.stack([XX.ravel(), YY.ravel(), Z.ravel()], axis=1)
    np.testing.assert_allclose(interpolate(f, z, BOX, mesh), f.ravel(), rtol=1e-14)


def test_interpolation_equals_scipy_on_a_random_periodic_mesh():
    """Against scipy's RegularGridInterpolator on the mesh padded with its periodic images: the
    bracketing plane, the periodic seam and the weights, everywhere inside [z_0, z_{nz-1}]."""
    from scipy.interpolate import RegularGridInterpolator
    nx, ny, nz = 9, 7, 8
    rng = np.random.default_rng(3)
    z = np.sort(np.r_[-0.4, 2.3, rng.uniform(-0.4, 2.3, nz - 2)])
    f = rng.uniform(0.0, 5.0, (nz, ny, nx))
    X = np.arange(nx + 1) * 6.0 / nx
    Y = np.arange(ny + 1) * 6.0 / ny
    fp = np.concatenate([f, f[:, :1, :]], axis=1)
    fp = np.concatenate([fp, fp[:, :, :1]], axis=2)
    ref = RegularGridInterpolator((z, Y, X), fp, method="linear")
    pts = np.stack([rng.uniform(0, 6, 4000), rng.uniform(0, 6, 4000),
                    rng.uniform(z[0], z[-1], 4000)], axis=1)
    np.testing.assert_allclose(interpolate(f, z, BOX, pts), ref(pts[:, ::-1]), rtol=1e-12,
                               atol=1e-12)
    # below z_0 and above z_{nz-1}: the values of the end planes
    lo = pts.copy()
    lo[:, 2] = -0.5
    hi = pts.copy()
    hi[:, 2] = 2.5
    end = pts.copy()
    end[:, 2] = z[0]
    np.testing.assert_allclose(interpolate(f, z, BOX, lo), interpolate(f, z, BOX, end), rtol=0)
    end[:, 2] = z[-1]
    np.testing.assert_allclose(interpolate(f, z, BOX, hi), interpolate(f, z, BOX, end), rtol=0)


def test_sites_follow_the_target():
    n = 20000
    z = np.linspace(-0.5, 2.5, 13)
    s = (z - z[0]) / (z[-1] - z[0])
    f = np.broadcast_to((1.0 + 9.0 * s)[:, None, None], (13, 8, 8)).copy()
    xyz, nprop = rejection_sample(f, z, BOX, n, seed=11)
    assert xyz.shape == (n, 3)
    sz = (xyz[:, 2] - z[0]) / (z[-1] - z[0])
    cdf = lambda t: (t + 4.5 * t * t) / 5.5            # noqa: E731  (density 1 + 9 t, normalised)
    crit = 1.95 / np.sqrt(n)                            # Kolmogorov-Smirnov, alpha = 1e-3
    assert stats.kstest(sz, cdf).statistic < crit
    assert stats.kstest(xyz[:, 0] / 6.0, "uniform").statistic < crit
    assert stats.kstest(xyz[:, 1] / 6.0, "uniform").statistic < crit
    p = 5.5 / 10.0                                       # mean f / max f
    rate = n / nprop
    assert abs(rate - p) < 5.0 * np.sqrt(p * (1 - p) / nprop)

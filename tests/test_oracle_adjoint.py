"""Pins of the oracle's hand-derived adjoint sweeps (Eq. 2 differentiated): central finite
differences in FP64 and the exact linearity of I in S (CPU only)."""
import numpy as np
import pytest

import oracle
from synth import delaunay_neighbours, s4_quadrature


def _reg_setup(seed=0):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 6, 5, 10
    z = np.cumsum(np.r_[0.0, 0.5 + rng.random(nz - 1)]) * 0.1
    al = rng.uniform(0.5, 8.0, (2, nx * ny * nz))
    S = rng.uniform(0.5, 2.0, (2, nx * ny * nz))
    return nx, ny, nz, 0.13, 0.11, z, al, S


def _reg_loss(setup, mu, al, S, g, bc):
    nx, ny, nz, dx, dy, z, _, _ = setup
    _, I = oracle.sc_regular(nx, ny, nz, dx, dy, z, mu[None], np.ones(1), al, S, bc=bc,
                             want_I=True)
    return float((I[0] * g).sum())


@pytest.mark.parametrize("mu", [(0.0, 0.0, 1.0), (0.3500212, -0.3500212, 0.8688903),
                                (-0.8688903, 0.3500212, -0.3500212)])
def test_regular_adjoint_matches_fd(mu):
    st = _reg_setup()
    nx, ny, nz, dx, dy, z, al, S = st
    mu = np.array(mu)
    rng = np.random.default_rng(1)
    g = rng.standard_normal(al.shape)
    ga, gs = oracle.sc_regular_adjoint(nx, ny, nz, dx, dy, z, mu, al, S, g, bc=0)
    for _ in range(32):
        l, p = rng.integers(al.shape[0]), rng.integers(al.shape[1])
        for arr, grad in ((al, ga), (S, gs)):
            h = 1e-6 * arr[l, p]
            ap, am = arr.copy(), arr.copy()
            ap[l, p] += h
            am[l, p] -= h
            if arr is al:
                fd = (_reg_loss(st, mu, ap, S, g, 0) - _reg_loss(st, mu, am, S, g, 0)) / (2 * h)
            else:
                fd = (_reg_loss(st, mu, al, ap, g, 0) - _reg_loss(st, mu, al, am, g, 0)) / (2 * h)
            assert grad[l, p] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(grad).max())


def test_regular_adjoint_dot_product_in_S():
    """I is linear in S, so <I(S + dS) - I(S), g> = <dS, g_S> holds to rounding."""
    st = _reg_setup(2)
    nx, ny, nz, dx, dy, z, al, S = st
    mu = np.array([0.3500212, 0.8688903, 0.3500212])
    rng = np.random.default_rng(3)
    g = rng.standard_normal(al.shape)
    dS = rng.standard_normal(al.shape)
    _, gs = oracle.sc_regular_adjoint(nx, ny, nz, dx, dy, z, mu, al, S, g, bc=0)
    lhs = _reg_loss(st, mu, al, S + dS, g, 0) - _reg_loss(st, mu, al, S, g, 0)
    assert lhs == pytest.approx(float((dS * gs).sum()), rel=1e-12)


def _vor_setup():
    rng = np.random.default_rng(9)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((200, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    dirs, _ = s4_quadrature()
    dirs = np.vstack([dirs, [[0.0, 0.0, 1.0]]])
    tab = oracle.voronoi_tables(xyz, off, code, shift, box, dirs, 7.0)
    al = rng.uniform(1.0, 30.0, (2, 200))
    S = rng.uniform(0.5, 2.0, (2, 200))
    return tab, dirs, al, S


@pytest.mark.parametrize("d", [24, 3, 17])
def test_voronoi_adjoint_matches_fd(d):
    tab, dirs, al, S = _vor_setup()
    up = dirs[d, 2] > 0
    rng = np.random.default_rng(4)
    g = rng.standard_normal(al.shape)

    def loss(a, s):
        _, I = oracle.voronoi_fs(tab, dirs, np.full(len(dirs), 1.0), a, s, bc=0, want_I=True)
        return float((I[d] * g).sum())

    ga, gs = oracle.voronoi_adjoint(tab, d, up, al, S, g, bc=0)
    for _ in range(32):
        l, p = rng.integers(2), rng.integers(200)
        for which in (0, 1):
            arr = al if which == 0 else S
            h = 1e-6 * arr[l, p]
            ap, am = arr.copy(), arr.copy()
            ap[l, p] += h
            am[l, p] -= h
            fd = ((loss(ap, S) - loss(am, S)) if which == 0 else
                  (loss(al, ap) - loss(al, am))) / (2 * h)
            grad = ga if which == 0 else gs
            assert grad[l, p] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(grad).max())

"""Pins of the oracle's accelerated Lambda iteration (CPU only).

* Lambda* is checked against dJ_p/dS_p measured with the formal solution itself (J is linear in
  S for fixed opacities, so a unit bump of S at one point gives the diagonal exactly), on the
  regular grid (periodic and closed sides, inflow and interior planes) and on a Voronoi grid
  (sites with wall neighbours included).
* The local update reduces to the plain Lambda update when Lambda* = 0, and solves its own
  equation n = SE(J + Lambda* (S(n) - S_old)) to the precision of Newton's method.
* The accelerated iteration converges to the populations of the Lambda iteration, in fewer
  iterations.
"""
import numpy as np
import pytest

import oracle
from oracle.ali import _local_update, ali_iterate, lambda_star_probe
from oracle.physics import Atom
from oracle.solve import RegularGrid, VoronoiGrid, lambda_iterate
from synth import delaunay_neighbours, make_atmosphere, model_atom, s4_quadrature
from synth.atmosphere import regular_fields


@pytest.mark.parametrize("periodic", [True, False])
def test_lambda_star_regular_is_the_diagonal(periodic):
    rng = np.random.default_rng(3)
    nx, ny, nz, nlam = 7, 6, 9, 2
    z = np.cumsum(np.r_[0.0, 0.3 + rng.random(nz - 1)])
    dirs, w = s4_quadrature()
    g = RegularGrid(nx, ny, nz, 0.7, 0.9, z, dirs, w, periodic=periodic)
    npt = nx * ny * nz
    a = 10.0 ** rng.uniform(-3, 1.5, (nlam, npt))
    s = rng.uniform(0.5, 2.0, (nlam, npt))
    L = g.lambda_star(a)
    pts = [(0, 0), (1, 5), (0, nx * ny + 3), (1, 4 * nx * ny + 11), (0, npt - 1), (1, npt - 7)]
    pts += [(int(rng.integers(nlam)), int(rng.integers(npt))) for _ in range(10)]
    probe = lambda_star_probe(lambda al, S: g.formal_solution(al, S), a, s, pts)
    np.testing.assert_allclose([L[l, p] for l, p in pts], probe, rtol=1e-9, atol=1e-12)
    assert np.all(L > 0) and np.all(L < 1)


def test_lambda_star_voronoi_is_the_diagonal():
    rng = np.random.default_rng(4)
    n, nlam = 300, 2
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((n, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    dirs, w = s4_quadrature()
    g = VoronoiGrid(dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box), dirs, w)
    a = 10.0 ** rng.uniform(-2, 1.5, (nlam, n))
    s = rng.uniform(0.5, 2.0, (nlam, n))
    L = g.lambda_star(a)
    walls = np.nonzero((g.tab["k"] < 0).any(axis=(0, 2)))[0]      # sites with a wall neighbour
    pts = [(0, int(i)) for i in walls[:8]] + [(1, int(i)) for i in rng.integers(n, size=8)]
    probe = lambda_star_probe(lambda al, S: g.formal_solution(al, S), a, s, pts)
    np.testing.assert_allclose([L[l, p] for l, p in pts], probe, rtol=1e-9, atol=1e-12)
    assert len(walls) > 0


def _small_nlte(nx=6, ny=6, nz=20):
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    A = Atom(model_atom(np.min(f["ne"] / np.sqrt(f["T"]))), atm.kappa0)
    dirs, w = s4_quadrature()
    return A, f, RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)


def test_local_update_reduces_to_lambda_and_solves_its_equation():
    A, f, g = _small_nlte()
    T, rho, ne, nH = f["T"], f["rho"], f["ne"], f["nH"]
    pops = A.lte_pops(T, ne, nH)
    alpha, S = A.alpha_S(T, rho, ne, pops)
    J = g.formal_solution(alpha, S)
    plain = A.statistical_equilibrium(A.rate_matrix(T, ne, J), nH)
    zero = _local_update(A, T, rho, ne, nH, pops, J, np.zeros_like(J), S, newton=2)
    np.testing.assert_allclose(zero, plain, rtol=1e-6)
    L = g.lambda_star(alpha)
    n = _local_update(A, T, rho, ne, nH, pops, J, L, S, newton=6)
    _, Sn = A.alpha_S(T, rho, ne, n)
    back = A.statistical_equilibrium(A.rate_matrix(T, ne, J + L * (Sn - S)), nH)
    np.testing.assert_allclose(back, n, rtol=1e-6)
    np.testing.assert_allclose(n.sum(0), nH, rtol=1e-12)


def test_ali_reaches_the_lambda_fixed_point_in_fewer_iterations():
    A, f, g = _small_nlte()
    args = (g, A, f["T"], f["rho"], f["ne"], f["nH"])
    ref, it_l, _ = lambda_iterate(*args, max_iter=300, tol=1e-7)
    ali, it_a, hist = ali_iterate(*args, max_iter=300, tol=1e-7)
    assert it_a < it_l / 2, (it_a, it_l)
    np.testing.assert_allclose(ali, ref, rtol=2e-5)
    assert hist[-1] < 1e-7
    # Lambda* of the starting opacities held fixed, one Newton step: the same fixed point
    fx, it_f, _ = ali_iterate(*args, max_iter=300, tol=1e-7, newton=1, fixed_lstar=True)
    assert it_f < it_l / 2, (it_f, it_l)
    np.testing.assert_allclose(fx, ref, rtol=2e-5)

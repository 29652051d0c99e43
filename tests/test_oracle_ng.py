"""Pins of the oracle's Ng extrapolation (CPU only).

* For a linear fixed-point iteration whose error lives in a two-dimensional invariant subspace
  (two eigenvalues), the second-order extrapolation from four iterates is the fixed point, to
  rounding.
  That holds for any positive weights.
* Applied every few Lambda iterations on a small NLTE problem, it reaches the Lambda iteration's
  fixed point in fewer iterations.
"""
import numpy as np

from oracle.ng import ng_extrapolate
from oracle.physics import Atom
from oracle.solve import RegularGrid, lambda_iterate
from synth import make_atmosphere, model_atom, s4_quadrature
from synth.atmosphere import regular_fields


def _linear_iteration(eigs, n=40, seed=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.zeros(n)
    lam[:len(eigs)] = eigs
    M = Q @ np.diag(lam) @ Q.T
    xstar = 1.0 + rng.random(n)
    c = xstar - M @ xstar
    x = xstar + Q[:, :len(eigs)] @ rng.normal(size=len(eigs))   # error in the invariant subspace
    xs = [x]
    for _ in range(3):
        xs.append(M @ xs[-1] + c)
    return xstar, xs


def test_ng_exact_for_two_eigenvalues():
    xstar, xs = _linear_iteration([0.9, -0.5])
    x = ng_extrapolate(xs[3], xs[2], xs[1], xs[0])
    np.testing.assert_allclose(x, xstar, rtol=1e-11)


def test_ng_exact_for_two_eigenvalues_with_any_weights():
    xstar, xs = _linear_iteration([0.97, 0.3], seed=2)
    w = np.random.default_rng(3).uniform(0.1, 10.0, xstar.size)
    x = ng_extrapolate(xs[3], xs[2], xs[1], xs[0], weights=w)
    np.testing.assert_allclose(x, xstar, rtol=1e-11)


def test_ng_accelerates_the_lambda_iteration():
    atm = make_atmosphere(0)
    nx, ny, nz = 6, 6, 20
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    A = Atom(model_atom(np.min(f["ne"] / np.sqrt(f["T"]))), atm.kappa0)
    dirs, w = s4_quadrature()
    g = RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    args = (g, A, f["T"], f["rho"], f["ne"], f["nH"])
    ref, it_plain, _ = lambda_iterate(*args, max_iter=300, tol=1e-7)
    hist = []
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    for it in range(1, 300):
        alpha, S = A.alpha_S(f["T"], f["rho"], f["ne"], pops)
        new = A.statistical_equilibrium(A.rate_matrix(f["T"], f["ne"], g.formal_solution(alpha, S)),
                                        f["nH"])
        d = np.max(np.abs(new - pops) / new)
        pops = new
        hist.append(pops.copy())
        if d < 1e-7:
            break
        if len(hist) >= 4 and it % 3 == 0:
            x = ng_extrapolate(hist[-1], hist[-2], hist[-3], hist[-4])
            if np.all(x > 0):
                pops = x
                hist[-1] = x
    assert it < 0.7 * it_plain, (it, it_plain)
    np.testing.assert_allclose(pops, ref, rtol=1e-5)

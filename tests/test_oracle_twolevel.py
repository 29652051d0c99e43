"""The sqrt(epsilon) surface law of the two-level atom (Sect. 2.1, Eq. 3 and 4).

For S = (1 - eps) J + eps B in an isothermal, semi-infinite, horizontally homogeneous medium the
surface value is S(0) = sqrt(eps) B.  The oracle's regular-grid solver (nx = ny = 1, periodic, so
the in-plane interpolation is exact) builds the Lambda operator column by column, and the
two-level problem (I - (1 - eps) Lambda) S = eps B is solved directly.  The depth discretisation
error must shrink under refinement and the Richardson-extrapolated value must meet sqrt(eps).
"""
import numpy as np
import pytest

import oracle
from synth import s4_quadrature


def surface_source(eps, per_decade, lo=1e-4, hi=1e4):
    n = int(round(np.log10(hi / lo) * per_decade)) + 1
    tau = np.logspace(np.log10(lo), np.log10(hi), n)
    z = (tau[-1] - tau)[::-1]                 # height increases upward; z[-1] is the surface
    dirs, w = s4_quadrature()
    Lam = np.empty((n, n))
    al = np.ones((n, n))
    S = np.eye(n)                             # one unit source vector per column ... per lambda
    J = oracle.sc_regular(1, 1, n, 1.0, 1.0, z, dirs, w, al, S, bc=0)
    Lam[:, :] = J.T                           # J[m] = Lambda e_m  -> column m
    A = np.eye(n) - (1.0 - eps) * Lam
    Ssol = np.linalg.solve(A, eps * np.ones(n))
    return Ssol[-1]


@pytest.mark.parametrize("eps", [0.1, 0.05])
def test_sqrt_eps_law(eps):
    s10 = surface_source(eps, 10)
    s20 = surface_source(eps, 20)
    s40 = surface_source(eps, 40)
    target = np.sqrt(eps)
    e10, e20, e40 = abs(s10 - target), abs(s20 - target), abs(s40 - target)
    assert e20 / target < 0.02                  # 2 % at 20 points per decade
    assert e40 < e20 < e10                      # the discretisation error shrinks
    rich = s40 + (s40 - s20) / 3.0              # second-order Richardson extrapolation
    assert abs(rich - target) / target < 2e-3

"""Oracle Lambda iteration (Sect. 2.1, Eq. 3-4 and the loop of Sect. 2.5/2.6):
populations -> alpha, S -> formal solution -> J -> rates -> statistical equilibrium -> populations,
repeated until the largest relative population change falls below ``tol``.
TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import lib
from .physics import Atom


class RegularGrid:
    """scheme: "plane" (plane-to-plane short characteristics) or "face" (face hitting, periodic
    sides only); lambda_star is the plane-to-plane one for both."""

    def __init__(self, nx, ny, nz, dx, dy, z, dirs, wdir, periodic=True, scheme="plane"):
        self.nx, self.ny, self.nz, self.dx, self.dy = nx, ny, nz, dx, dy
        self.z = np.asarray(z, float)
        self.dirs = np.asarray(dirs, float)
        self.wdir = np.asarray(wdir, float)
        self.periodic = periodic
        if scheme not in ("plane", "face") or (scheme == "face" and not periodic):
            raise ValueError("scheme must be 'plane', or 'face' with periodic sides")
        self.scheme = scheme

    def lambda_star(self, alpha, bc=0):
        from .ali import lambda_star_regular
        return lambda_star_regular(self.nx, self.ny, self.nz, self.dx, self.dy, self.z, self.dirs,
                                   self.wdir, alpha, bc=bc, periodic=self.periodic)

    def formal_solution(self, alpha, S, bc=0, ibc=None, want_I=False):
        if self.scheme == "face":
            return lib.sc_regular_face(self.nx, self.ny, self.nz, self.dx, self.dy, self.z,
                                       self.dirs, self.wdir, alpha, S, bc=bc, ibc=ibc,
                                       want_I=want_I)
        return lib.sc_regular(self.nx, self.ny, self.nz, self.dx, self.dy, self.z, self.dirs,
                              self.wdir, alpha, S, bc=bc, ibc=ibc, periodic=self.periodic,
                              want_I=want_I)


class VoronoiGrid:
    def __init__(self, grid, dirs, wdir, r_exp=7.0):
        self.dirs = np.asarray(dirs, float)
        self.wdir = np.asarray(wdir, float)
        self.tab = lib.voronoi_tables(grid["xyz"], grid["nbr_off"], grid["nbr_idx"],
                                      grid["nbr_shift"], grid["box"], self.dirs, r_exp)
        self.order = lib.voronoi_order(self.tab["level"])

    def lambda_star(self, alpha, bc=0):
        from .ali import lambda_star_voronoi
        return lambda_star_voronoi(self.tab, self.dirs, self.wdir, alpha, bc=bc)

    def formal_solution(self, alpha, S, bc=0, ibc=None, want_I=False):
        return lib.voronoi_fs(self.tab, self.dirs, self.wdir, alpha, S, bc=bc, ibc=ibc,
                              order=self.order, want_I=want_I)


def lambda_iterate(grid, atom: Atom, T, rho, ne, nH, pops0=None, max_iter=300, tol=1e-3,
                   callback=None):
    """Returns (pops [3][npt], iterations, history of max relative change)."""
    pops = atom.lte_pops(T, ne, nH) if pops0 is None else np.array(pops0, float)
    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        alpha, S = atom.alpha_S(T, rho, ne, pops)
        J = grid.formal_solution(alpha, S, bc=0)
        P = atom.rate_matrix(T, ne, J)
        new = atom.statistical_equilibrium(P, nH)
        dmax = float(np.max(np.abs(new - pops) / new))
        hist.append(dmax)
        pops = new
        if callback is not None:
            callback(it, pops, dmax)
        if dmax < tol:
            break
    return pops, it, np.array(hist)

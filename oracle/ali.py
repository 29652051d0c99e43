"""Oracle of the accelerated Lambda iteration (ALI).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper iterates plain Lambda (Sect. 2.1: populations -> source functions -> formal solution ->
J -> statistical equilibrium) and notes there that accelerated schemes converge much faster.  This module states the accelerated scheme used here, in FP64:

Lambda* [nlam][npt]
    dJ_p / dS_p with the opacities fixed: the diagonal of the linear map S -> J of the formal
    solution.  With S linear across every interval (Eq. 2) the source function of point p enters
    the intensity at p only through the weight w1 of the interval that ends at p -- or, where the
    ray starts at p, through the inflow rule (thermal inflow I = S at the bottom wall).  On a
    Voronoi grid a wall neighbour stands in with the site's own S, so it adds w0 (and e^-d under
    thermal inflow) to the site's own weight.  ``lambda_star_*`` write this out; the tests check
    it against dJ_p/dS_p measured with the formal solution itself.

One iteration
    alpha_old, S_old from the current populations; J from the formal solution; then at every
    point the populations n that solve
        n = SE( J + Lambda* (S(n) - S_old) )
    (statistical equilibrium with the point's own source function updated inside its J), found
    by Newton's method on the logarithms of the two smaller populations (the largest follows
    from n1 + n2 + np = nH without cancellation), with a forward-difference Jacobian.  When the
    iteration has converged, S(n) = S_old and J is the formal solution of the final state: the
    fixed point is the Lambda iteration's.
"""
from __future__ import annotations

import numpy as np


def w1_weight(d):
    """The interval weight of the downstream end, w1 = (d - (1 - e^-d)) / d (Eq. 2), with the
    Taylor series below d = 1e-6; also returns e^-d and w0."""
    d = np.asarray(d, float)
    small = d < 1e-6
    ds = np.where(small, 1.0, d)
    e0 = -np.expm1(-ds)
    w1 = np.where(small, d * (0.5 - d * (1.0 / 6.0 - d / 24.0)), (ds - e0) / ds)
    w0 = np.where(small, d * (0.5 - d * (1.0 / 3.0 - d / 8.0)), e0 - (ds - e0) / ds)
    return np.exp(-d), w0, w1


def lambda_star_regular(nx, ny, nz, dx, dy, z, dirs, wdir, alpha, bc=0, periodic=True):
    """Diagonal of the regular-grid Lambda operator [nlam][npt] (plane-to-plane short
    characteristics: the upwind point of plane k on plane k -/+ 1, alpha interpolated
    bilinearly there, periodic or edge-clamped)."""
    alpha = np.asarray(alpha, float)
    nlam = alpha.shape[0]
    al = alpha.reshape(nlam, nz, ny, nx)
    L = np.zeros_like(al)
    z = np.asarray(z, float)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for mu, w in zip(np.asarray(dirs, float), np.asarray(wdir, float)):
        up = mu[2] > 0.0
        k0 = 0 if up else nz - 1
        if bc == 0 and up:
            L[:, k0] += w          # I = S on the inflow plane
        for s in range(1, nz):
            k = s if up else nz - 1 - s
            ku = k - 1 if up else k + 1
            ds = abs(z[k] - z[ku]) / abs(mu[2])
            fx = ii - ds * mu[0] / dx
            fy = jj - ds * mu[1] / dy
            i0, j0 = np.floor(fx).astype(int), np.floor(fy).astype(int)
            tx, ty = fx - i0, fy - j0
            a_up = np.zeros((nlam, ny, nx))
            for b, wy in ((0, 1.0 - ty), (1, ty)):
                for a, wx in ((0, 1.0 - tx), (1, tx)):
                    xi, yj = i0 + a, j0 + b
                    if periodic:
                        xi, yj = xi % nx, yj % ny
                    else:
                        xi, yj = np.clip(xi, 0, nx - 1), np.clip(yj, 0, ny - 1)
                    a_up += (wx * wy) * al[:, ku, yj, xi]
            _, _, w1 = w1_weight(0.5 * (a_up + al[:, k]) * ds)
            L[:, k] += w * w1
    return L.reshape(nlam, -1)


def lambda_star_voronoi(tab, dirs, wdir, alpha, bc=0):
    """Diagonal of the Voronoi Lambda operator [nlam][n] from the upwind tables of
    ``lib.voronoi_tables`` (two upwind neighbours per site and direction, Eq. 5)."""
    alpha = np.asarray(alpha, float)
    L = np.zeros_like(alpha)
    for d, (mu, wd) in enumerate(zip(np.asarray(dirs, float), np.asarray(wdir, float))):
        up = mu[2] > 0.0
        for c in range(2):
            kc = tab["k"][d, :, c]
            wc = tab["w"][d, :, c]
            real = kc >= 0
            a_k = np.where(real, alpha[:, np.where(real, kc, 0)], alpha)
            ex, w0, w1 = w1_weight(0.5 * (a_k + alpha) * tab["len"][d, :, c])
            inflow = (bc == 0 and up) & (kc == -1)
            own = np.where(real, w1, w0 + w1 + np.where(inflow, ex, 0.0))
            L += wd * np.where(wc != 0.0, wc, 0.0) * own
    return L


def _local_update(atom, T, rho, ne, nH, pops, J, Lst, S_old, newton):
    """n = SE(J + Lambda* (S(n) - S_old)) at every point, by ``newton`` Newton steps from
    ``pops`` (0: the plain update SE(J))."""
    def G(n):
        _, S = atom.alpha_S(T, rho, ne, n)
        P = atom.rate_matrix(T, ne, J + Lst * (S - S_old))
        return atom.statistical_equilibrium(P, nH)

    if newton == 0:            # the plain update
        return G(pops)
    npt = nH.size
    idx = np.arange(npt)
    big = np.argmax(pops, axis=0)
    small = np.array([[j for j in range(3) if j != b] for b in range(3)])[big].T   # [2][npt]

    def full(x):
        n = np.empty((3, npt))
        n[small[0], idx] = x[0]
        n[small[1], idx] = x[1]
        n[big, idx] = nH - x[0] - x[1]
        return n

    # Newton on u = log(x), the logarithms of the two smaller populations: positivity is kept
    # and the relative changes of a first iteration far from equilibrium stay well scaled
    x = np.stack([pops[small[0], idx], pops[small[1], idx]])
    for _ in range(newton):
        g = G(full(x))
        gx = np.stack([g[small[0], idx], g[small[1], idx]])
        H0 = np.log(gx) - np.log(x)
        Jm = np.empty((2, 2, npt))
        for c in range(2):
            h = 1e-6
            xp = x.copy()
            xp[c] *= np.exp(h)
            gp = G(full(xp))
            Hp = np.log(np.stack([gp[small[0], idx], gp[small[1], idx]])) - np.log(xp)
            Jm[:, c] = (Hp - H0) / h
        det = Jm[0, 0] * Jm[1, 1] - Jm[0, 1] * Jm[1, 0]
        step0 = (Jm[1, 1] * H0[0] - Jm[0, 1] * H0[1]) / det
        step1 = (-Jm[1, 0] * H0[0] + Jm[0, 0] * H0[1]) / det
        xn = x * np.exp(-np.stack([step0, step1]))
        # a step that is not finite or leaves no room for the largest population falls back to
        # the plain update G(x)
        bad = ~np.isfinite(xn).all(axis=0) | (xn.sum(axis=0) >= nH)
        x = np.where(bad, gx, xn)
    return full(x)


def ali_iterate(grid, atom, T, rho, ne, nH, pops0=None, max_iter=300, tol=1e-3, newton=3,
                fixed_lstar=False):
    """Accelerated Lambda iteration.  ``grid`` is an ``oracle.solve`` grid.  ``fixed_lstar``:
    Lambda* of the starting populations' opacities held fixed (the fixed point does not depend
    on it).  Returns (pops, iterations, history of the largest relative population change)."""
    pops = atom.lte_pops(T, ne, nH) if pops0 is None else np.array(pops0, float)
    hist = []
    it = 0
    Lst = None
    for it in range(1, max_iter + 1):
        alpha, S = atom.alpha_S(T, rho, ne, pops)
        J = grid.formal_solution(alpha, S, bc=0)
        if Lst is None or not fixed_lstar:
            Lst = grid.lambda_star(alpha, bc=0)
        new = _local_update(atom, T, rho, ne, nH, pops, J, Lst, S, newton)
        dmax = float(np.max(np.abs(new - pops) / new))
        hist.append(dmax)
        pops = new
        if dmax < tol:
            break
    return pops, it, np.array(hist)


def lambda_star_probe(formal_solution, alpha, S, points, eps=1.0):
    """dJ_p/dS_p measured with the formal solution itself: J(S + eps e_p) - J(S) at p (J is
    linear in S for fixed alpha).  ``points``: list of (wavelength, point)."""
    J0 = formal_solution(alpha, S)
    out = []
    for l, p in points:
        S1 = np.array(S, float)
        S1[l, p] += eps
        out.append((formal_solution(alpha, S1)[l, p] - J0[l, p]) / eps)
    return np.array(out)


__all__ = ["w1_weight", "lambda_star_regular", "lambda_star_voronoi", "ali_iterate",
           "lambda_star_probe"]

"""Oracle of the final synthesis on a Voronoi grid (Sect. 2.5, last paragraphs).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper does not take the emergent intensity from the irregular grid (its upper layers hold few
sites): it interpolates the converged level populations back to the original mesh with inverse
distance weighting over the two nearest sites, recomputes opacity and source function there, and
integrates a formal solution along vertical long characteristics (mu = 1).

Reading taken here: "inverse distance" weights 1/d (power 1), d the Euclidean distance with the
minimum-image convention in the periodic x and y; a target that coincides with a site takes that
site's value.  The mesh point (i, j, k) sits at (i dx, j dy, z_k) in the sites' frame.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from . import lib


def mesh_points(nx, ny, dx, dy, z):
    """Mesh positions [npt][3], x fastest (index (k ny + j) nx + i)."""
    Z, Y, X = np.meshgrid(np.asarray(z, float), np.arange(ny) * dy, np.arange(nx) * dx,
                          indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def two_nearest_bruteforce(sites, targets, box):
    """Indices [m][2] and distances [m][2] of the two nearest sites, by brute force (min image
    in x and y)."""
    Lx, Ly = box[1] - box[0], box[3] - box[2]
    k = np.empty((len(targets), 2), np.int64)
    d = np.empty((len(targets), 2))
    for s in range(0, len(targets), 256):
        t = targets[s:s + 256]
        dv = sites[None, :, :] - t[:, None, :]
        dv[..., 0] -= Lx * np.round(dv[..., 0] / Lx)
        dv[..., 1] -= Ly * np.round(dv[..., 1] / Ly)
        r = np.sqrt((dv ** 2).sum(-1))
        idx = np.argsort(r, axis=1, kind="stable")[:, :2]
        k[s:s + 256] = idx
        d[s:s + 256] = np.take_along_axis(r, idx, axis=1)
    return k, d


def two_nearest(sites, targets, box):
    """The same with a k-d tree (periodic in x, y; z shifted into a box large enough that it
    never wraps)."""
    Lx, Ly = box[1] - box[0], box[3] - box[2]
    zspan = max(sites[:, 2].max(), targets[:, 2].max()) - min(sites[:, 2].min(),
                                                                targets[:, 2].min())
    big = 4.0 * zspan + 1.0
    z0 = min(sites[:, 2].min(), targets[:, 2].min())

    def wrap(p):
        q = np.array(p, float)
        q[:, 0] = np.mod(q[:, 0] - box[0], Lx)
        q[:, 1] = np.mod(q[:, 1] - box[2], Ly)
        q[:, 2] = q[:, 2] - z0 + zspan
        return q

    tree = cKDTree(wrap(sites), boxsize=[Lx, Ly, big])
    d, k = tree.query(wrap(targets), k=2)
    return k, d


def idw_weights(d):
    """Weights [m][2] of the two nearest sites: 1/d normalised; (1, 0) on a site."""
    d = np.asarray(d, float)
    on = d[:, 0] == 0.0
    inv = 1.0 / np.where(d == 0.0, 1.0, d)
    w = inv / inv.sum(axis=1, keepdims=True)
    w[on] = [1.0, 0.0]
    return w


def interpolate(values, k, w):
    """values [nf][nsites] -> [nf][m]."""
    values = np.asarray(values, float)
    return values[:, k[:, 0]] * w[:, 0] + values[:, k[:, 1]] * w[:, 1]


def emergent_mu1(nx, ny, nz, dx, dy, z, alpha, S, bc=0):
    """Vertical (mu = 1) emergent intensity [nlam][nx ny] of the mesh: the regular-grid sweep of
    the single direction (0, 0, 1), whose rays run along the mesh columns."""
    I = lib.sc_regular(nx, ny, nz, dx, dy, z, np.array([[0.0, 0.0, 1.0]]), np.array([1.0]),
                       alpha, S, bc=bc)
    return I[:, (nz - 1) * nx * ny:]


def final_synthesis(atom, site_pops, sites, box, mesh, mesh_fields):
    """I_top [nlam][nx ny] of the mesh from the converged site populations [3][nsites].
    ``mesh`` = (nx, ny, nz, dx, dy, z); ``mesh_fields``: T, rho, ne on the mesh."""
    nx, ny, nz, dx, dy, z = mesh
    k, d = two_nearest(sites, mesh_points(nx, ny, dx, dy, z), box)
    pops = interpolate(site_pops, k, idw_weights(d))
    alpha, S = atom.alpha_S(mesh_fields["T"], mesh_fields["rho"], mesh_fields["ne"], pops)
    return emergent_mu1(nx, ny, nz, dx, dy, z, alpha, S)


def top_sites(nbr_off, nbr_idx):
    """Sites of the emergent layer: those whose neighbour list holds a mirror in the top wall
    (neighbour code -2 - 2k), in increasing site order."""
    off = np.asarray(nbr_off)
    code = np.asarray(nbr_idx)
    row = np.repeat(np.arange(len(off) - 1), np.diff(off))
    top_mirror = (code < 0) & (((-code - 1) & 1) == 1)
    return np.unique(row[top_mirror])


def resample_map(sites_xy, values, npx, npy, box):
    """Emergent intensities at the top sites ([nf][ntop], positions [ntop][2]) on an npx x npy
    pixel grid [nf][npy npx]: pixel (i, j) at (x0 + i Lx / npx, y0 + j Ly / npy), two nearest
    sites in (x, y) with the minimum image in x and y (brute force, ties to the smaller index),
    weights 1/d normalised, (1, 0) on a site."""
    Lx, Ly = box[1] - box[0], box[3] - box[2]
    J, I = np.meshgrid(np.arange(npy), np.arange(npx), indexing="ij")
    px = np.stack([box[0] + I.ravel() * Lx / npx, box[2] + J.ravel() * Ly / npy,
                   np.zeros(npx * npy)], axis=1)
    sites = np.column_stack([np.asarray(sites_xy, float)[:, :2], np.zeros(len(sites_xy))])
    k, d = two_nearest_bruteforce(sites, px, box)
    return interpolate(values, k, idw_weights(d))

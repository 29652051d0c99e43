"""Irregular-grid inputs: sites by rejection sampling (Sect. 2.4) and Delaunay neighbour lists.

Rejection sampling follows the paper's four steps (Sect. 2.4): a proposal uniform in the box, its
target density normalised by the maximum, a uniform rejection level, accept when the proposal is
at least the level; repeat until the requested number of sites is reached.

The paper obtains neighbour lists from voro++ (Sect. 2.4).  Here the Delaunay tessellation comes
from scipy (Qhull), which yields the same neighbour relation (two sites are Voronoi neighbours
exactly when they share a Delaunay edge).  Boundaries:

* x and y are periodic: sites within a margin of a side are replicated by +-Lx, +-Ly;
* the walls z = zmin and z = zmax get mirror ghosts (sites and images within the margin,
  reflected in the wall), so that cells touching a wall have a neighbour beyond it.

A neighbour is returned as (code, shift): code >= 0 is a real site; code = -1 - 2k is the mirror
of site k in the bottom wall and code = -2 - 2k its mirror in the top wall; shift = (sx+1)*3 +
(sy+1) says which periodic image (sx, sy in {-1, 0, 1}) of that site or ghost is the neighbour.
The margin is doubled until every Delaunay tetrahedron that touches a real site has its
circumsphere inside the replicated region, which makes the lists exact.
"""
from __future__ import annotations

import os

import numpy as np
from scipy.spatial import Delaunay

from .atmosphere import Atmosphere


def rejection_sample(f, n, lo, hi, seed, fmax, batch=1 << 18):
    """``n`` sites in the box [lo, hi) (3-vectors) with density proportional to f(x, y, z).

    ``fmax`` is the normalisation of the target density (its maximum over the box).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    out = []
    have = 0
    while have < n:
        p = lo + (hi - lo) * rng.random((batch, 3))
        dens = f(p[:, 0], p[:, 1], p[:, 2]) / fmax
        rej = rng.random(batch)
        acc = p[dens >= rej]
        out.append(acc)
        have += len(acc)
    return np.concatenate(out)[:n]


def _circumsphere(pts, simp):
    a = pts[simp[:, 0]]
    b = pts[simp[:, 1]] - a
    c = pts[simp[:, 2]] - a
    d = pts[simp[:, 3]] - a
    bb = (b * b).sum(1)
    cc = (c * c).sum(1)
    dd = (d * d).sum(1)
    cxd = np.cross(c, d)
    dxb = np.cross(d, b)
    bxc = np.cross(b, c)
    den = 2.0 * (b * cxd).sum(1)
    num = bb[:, None] * cxd + cc[:, None] * dxb + dd[:, None] * bxc
    with np.errstate(divide="ignore", invalid="ignore"):
        off = num / den[:, None]
    r = np.linalg.norm(off, axis=1)
    # slivers: a site, a neighbour and their two mirror images are coplanar up to rounding
    scale = np.maximum(np.maximum(bb, cc), dd) ** 1.5
    bad = ~np.isfinite(r) | (np.abs(den) < 1e-9 * scale)
    r[bad] = np.inf
    off[bad] = 0.0
    return a + off, r


def _local_spacing(z, z0, z1, nbin=60):
    """Mean inter-site spacing per height bin (bin edges, spacing per bin), smoothed upward."""
    edges = np.linspace(z0, z1, nbin + 1)
    cnt, _ = np.histogram(z, bins=edges)
    cnt = np.convolve(cnt, np.ones(3), mode="same") / 3.0
    return edges, cnt


def delaunay_neighbours(xyz, box, periodic_xy=True, grow=4.5):
    """Neighbour CSR (off int64[N+1], code int32[M], shift int8[M]) of sites ``xyz`` [N, 3].

    ``box`` = (x0, x1, y0, y1, z0, z1).  Images and mirror ghosts are generated within a
    height-dependent margin (``grow`` times the local site spacing), grown until certified.
    """
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = len(xyz)
    x0, x1, y0, y1, z0, z1 = box
    Lx, Ly, Lz = x1 - x0, y1 - y0, z1 - z0
    edges, cnt = _local_spacing(xyz[:, 2], z0, z1)
    bin_vol = Lx * Ly * (edges[1] - edges[0])
    spacing = (bin_vol / np.maximum(cnt, 0.5)) ** (1.0 / 3.0)
    zs = np.sort(xyz[:, 2])
    k = min(64, n - 1)
    # spacing among the sites nearest each wall, from the height span of the k nearest
    s_bot = (Lx * Ly * max(zs[k] - zs[0], 1e-9 * Lz) / k) ** (1.0 / 3.0)
    s_top = (Lx * Ly * max(zs[-1] - zs[-1 - k], 1e-9 * Lz) / k) ** (1.0 / 3.0)
    gap_bot = zs[0] - z0
    gap_top = z1 - zs[-1]
    fac = grow
    while True:
        m_bin = np.minimum(fac * spacing, max(Lx, Ly))
        # a margin may only shrink slowly with height so that big cells above dense layers are
        # still covered: take the running maximum over a window of neighbouring bins
        m_bin = np.maximum.reduce([np.roll(m_bin, k) for k in (-2, -1, 0, 1, 2)])
        m_bot = gap_bot + fac * s_bot
        m_top = gap_top + fac * s_top
        b = np.clip(((xyz[:, 2] - z0) / (edges[1] - edges[0])).astype(int), 0, len(m_bin) - 1)
        m_pt = m_bin[b]
        pts = [xyz]
        orig = [np.arange(n)]
        sh = [np.full(n, 4, np.int8)]
        if periodic_xy:
            for sx in (-1, 0, 1):
                for sy in (-1, 0, 1):
                    if sx == 0 and sy == 0:
                        continue
                    q = xyz + np.array([sx * Lx, sy * Ly, 0.0])
                    keep = ((q[:, 0] > x0 - m_pt) & (q[:, 0] < x1 + m_pt) &
                            (q[:, 1] > y0 - m_pt) & (q[:, 1] < y1 + m_pt))
                    pts.append(q[keep])
                    orig.append(np.nonzero(keep)[0])
                    sh.append(np.full(keep.sum(), (sx + 1) * 3 + (sy + 1), np.int8))
        P = np.concatenate(pts)
        O = np.concatenate(orig)
        S = np.concatenate(sh)
        gp, go, gs = [P], [O.astype(np.int64)], [S]
        for zw, tag, mw in ((z0, 1, m_bot), (z1, 2, m_top)):
            keep = np.abs(P[:, 2] - zw) < mw
            q = P[keep].copy()
            q[:, 2] = 2.0 * zw - q[:, 2]
            gp.append(q)
            go.append(-tag - 2 * O[keep].astype(np.int64))
            gs.append(S[keep])
        P = np.concatenate(gp)
        C = np.concatenate(go)
        S = np.concatenate(gs)
        tri = Delaunay(P)
        simp = tri.simplices
        real_simp = (simp < n).any(axis=1)
        cen, r = _circumsphere(P, simp[real_simp])
        # certified when each circumsphere stays inside the region where every image and ghost
        # exists: above z0 - m_bot, below z1 + m_top, and horizontally within the smallest
        # margin of the heights it spans
        fin = np.isfinite(r)
        cen, r = cen[fin], r[fin]
        ok = (cen[:, 2] - r > z0 - m_bot) & (cen[:, 2] + r < z1 + m_top)
        if periodic_xy:
            zlo = np.clip(((cen[:, 2] - r - z0) / (edges[1] - edges[0])).astype(int), 0,
                          len(m_bin) - 1)
            zhi = np.clip(((cen[:, 2] + r - z0) / (edges[1] - edges[0])).astype(int), 0,
                          len(m_bin) - 1)
            mmin = _range_min(m_bin, zlo, zhi)
            ok &= ((cen[:, 0] - r > x0 - mmin) & (cen[:, 0] + r < x1 + mmin) &
                   (cen[:, 1] - r > y0 - mmin) & (cen[:, 1] + r < y1 + mmin))
        if ok.all():
            break
        fac *= 1.5
        if fac > 50.0:
            raise RuntimeError("Delaunay margin exceeded the box: too few sites")
    indptr, indices = tri.vertex_neighbor_vertices
    cnt_nb = np.diff(indptr[:n + 1])
    row = np.repeat(np.arange(n), cnt_nb)
    nb = indices[:indptr[n]]
    c = C[nb]
    s = S[nb]
    order = np.lexsort((s, c, row))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(cnt_nb)
    return off, c[order].astype(np.int32), s[order].astype(np.int8)


def _range_min(a, lo, hi):
    """min(a[lo[i]:hi[i]+1]) for every i (a is short)."""
    m = len(a)
    table = np.full((m, m), np.inf)
    for i in range(m):
        table[i, i:] = np.minimum.accumulate(a[i:])
    return table[lo, hi]


def site_density(atm: Atmosphere, kind: str):
    """Target site densities of the irregular-grid recipes.

    * ``"dtau"``: proportional to |d tau_500 / dz| = alpha_500 of the recipe, capped at the
      horizontal mean of alpha_500 where the mean optical depth reaches 3 (deeper layers, where
      every wavelength is thermalised, are sampled uniformly at that cap);
    * ``"rho03"``: proportional to rho^0.3.
    """
    if kind == "rho03":
        return (lambda x, y, z: atm.rho(z) ** 0.3), atm.rho(atm.zmin) ** 0.3
    if kind == "dtau":
        zs = np.linspace(atm.zmax, atm.zmin, 30001)
        a_mean = atm.kappa0 * atm.rho(zs) * (atm.T0(zs) / 5000.0) ** 9
        tau = np.concatenate([[0.0], np.cumsum(0.5 * (a_mean[1:] + a_mean[:-1]) * -np.diff(zs))])
        cap = np.interp(3.0, tau, a_mean)

        def f(x, y, z):
            T = atm.T(x, y, z)
            return np.minimum(atm.kappa0 * atm.rho(z) * (T / 5000.0) ** 9, cap)
        return f, cap
    raise ValueError(kind)


def _cache_path(key):
    root = os.environ.get("RT_SYNTH_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                         "rt_synth"))
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, key + ".npz")


def make_voronoi_grid(atm: Atmosphere, nsites: int, kind: str, seed: int, uniform_frac=0.0,
                      cache=True):
    """Sites plus neighbour CSR for the synthetic box of ``atm`` (cached on disk by key)."""
    key = f"vor_a{atm.seed}_n{nsites}_{kind}_s{seed}_u{uniform_frac:g}_v1"
    if cache:
        path = _cache_path(key)
        if os.path.exists(path):
            z = np.load(path)
            return dict(xyz=z["xyz"], nbr_off=z["nbr_off"], nbr_idx=z["nbr_idx"],
                        nbr_shift=z["nbr_shift"], box=tuple(z["box"]))
    lo = (0.0, 0.0, atm.zmin)
    hi = (atm.Lx, atm.Ly, atm.zmax)
    n_uni = int(round(uniform_frac * nsites))
    f, fmax = site_density(atm, kind)
    xyz = rejection_sample(f, nsites - n_uni, lo, hi, seed, fmax)
    if n_uni:
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        xyz = np.concatenate([xyz, np.asarray(lo) + (np.asarray(hi) - np.asarray(lo)) *
                              rng.random((n_uni, 3))])
    box = (0.0, atm.Lx, 0.0, atm.Ly, atm.zmin, atm.zmax)
    off, code, shift = delaunay_neighbours(xyz, box, periodic_xy=True)
    out = dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)
    if cache:
        tmp = _cache_path(key + f".tmp{os.getpid()}")
        np.savez(tmp, xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=np.array(box))
        os.replace(tmp, _cache_path(key))
    return out

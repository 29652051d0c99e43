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


def rejection_sample(f, n, lo, hi, seed, fmax, batch=1 << 18, f_upper=None):
    """``n`` sites in the box [lo, hi) (3-vectors) with density proportional to f(x, y, z).

    ``fmax`` is the normalisation of the target density (its maximum over the box).  ``f_upper``
    (optional, a function of z alone with f_upper(z) >= f(x, y, z) everywhere) only saves work:
    a proposal whose level already exceeds f_upper / fmax is rejected without evaluating f, which
    takes the same decision.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    out = []
    have = 0
    while have < n:
        p = lo + (hi - lo) * rng.random((batch, 3))
        rej = rng.random(batch)
        if f_upper is None:
            keep = f(p[:, 0], p[:, 1], p[:, 2]) / fmax >= rej
        else:
            keep = f_upper(p[:, 2]) / fmax >= rej
            c = np.nonzero(keep)[0]
            keep[c] = f(p[c, 0], p[c, 1], p[c, 2]) / fmax >= rej[c]
        acc = p[keep]
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

    ``box`` = (x0, x1, y0, y1, z0, z1).  Periodic images and wall mirrors are generated within a
    height-dependent margin (``grow`` times the local site spacing at the point's height, and for
    the mirrors at least the gap between the wall and its nearest site), grown until certified:
    every Delaunay tetrahedron touching a real site must have its circumsphere inside the region
    where no image or mirror is missing.  The margin grows only in the height bins that a failing
    circumsphere spans.
    """
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = len(xyz)
    x0, x1, y0, y1, z0, z1 = box
    Lx, Ly, Lz = x1 - x0, y1 - y0, z1 - z0
    edges, cnt = _local_spacing(xyz[:, 2], z0, z1)
    hb = edges[1] - edges[0]
    nbin = len(edges) - 1
    bin_vol = Lx * Ly * hb
    spacing = (bin_vol / np.maximum(cnt, 0.5)) ** (1.0 / 3.0)
    zs = np.sort(xyz[:, 2])
    gap_bot = zs[0] - z0
    gap_top = z1 - zs[-1]

    def bin_of(z):
        return np.clip(((z - z0) / hb).astype(int), 0, nbin - 1)

    fac = np.full(nbin, float(grow))
    # the sparsest height bins, holding together at most 0.5 % of the sites, are replicated in
    # full from the start: their big cells would fail the certification of any local margin, and
    # replicating them costs little
    raw, _ = np.histogram(xyz[:, 2], bins=edges)
    by_count = np.argsort(raw, kind="stable")
    fac[by_count[np.cumsum(raw[by_count]) <= 0.005 * n]] = np.inf
    while True:
        m_bin = np.minimum(fac * spacing, max(Lx, Ly, Lz))
        # a margin may only shrink slowly with height so that big cells above dense layers are
        # still covered: take the running maximum over a window of neighbouring bins
        # (the window does not wrap around: the sparse top must not widen the dense bottom's)
        mp = np.pad(m_bin, 2, mode="edge")
        m_bin = np.maximum.reduce([mp[k:k + nbin] for k in range(5)])
        m_pt = m_bin[bin_of(xyz[:, 2])]
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
        mP = m_bin[bin_of(P[:, 2])]
        gp, go, gs = [P], [O.astype(np.int64)], [S]
        depth = {}
        for zw, tag, gap in ((z0, 1, gap_bot), (z1, 2, gap_top)):
            dist = np.abs(P[:, 2] - zw)
            keep = dist < gap + mP
            # the nearest missing mirror lies this far beyond the wall
            depth[tag] = dist[~keep].min() if (~keep).any() else np.inf
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
        fin = np.isfinite(r)
        cen, r = cen[fin], r[fin]
        zl, zh = cen[:, 2] - r, cen[:, 2] + r
        ok = (zl > z0 - depth[1]) & (zh < z1 + depth[2])
        # images exist within the margin of their real site's height; a mirror beyond a wall
        # stands for a point at the reflected height
        lo = np.minimum(np.maximum(zl, z0), np.where(zh > z1, 2 * z1 - zh, np.inf))
        hi = np.maximum(np.minimum(zh, z1), np.where(zl < z0, 2 * z0 - zl, -np.inf))
        blo, bhi = bin_of(np.maximum(lo, z0)), bin_of(np.minimum(hi, z1))
        if periodic_xy:
            mmin = _range_min(m_bin, blo, bhi)
            ok &= ((cen[:, 0] - r > x0 - mmin) & (cen[:, 0] + r < x1 + mmin) &
                   (cen[:, 1] - r > y0 - mmin) & (cen[:, 1] + r < y1 + mmin))
        if ok.all():
            break
        grow_bin = np.zeros(nbin + 1, np.int64)
        np.add.at(grow_bin, blo[~ok], 1)
        np.add.at(grow_bin, bhi[~ok] + 1, -1)
        fac[np.cumsum(grow_bin)[:nbin] > 0] *= 1.5
        if fac[np.isfinite(fac)].max(initial=0.0) > 50.0:
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


def site_density_envelope(atm: Atmosphere, kind: str):
    """A function of z alone bounding the target of ``site_density`` from above (None where the
    target depends on z only).  For "dtau": |g| <= sum of the absolute Fourier coefficients, so
    T <= T0(z) (1 + amp G), and the opacity grows with T; a relative margin of 1e-9 covers the
    rounding of both evaluations."""
    if kind != "dtau":
        return None
    f, cap = site_density(atm, kind)
    G = float(np.abs(atm._ca).sum() + np.abs(atm._sa).sum())

    def f_upper(z):
        Tu = atm.T0(z) * (1.0 + atm.amp * G)
        return np.minimum(atm.kappa0 * atm.rho(z) * (Tu / 5000.0) ** 9, cap) * (1.0 + 1e-9)
    return f_upper


def _cache_path(key):
    root = os.environ.get("RT_SYNTH_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                         "rt_synth"))
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, key + ".npz")


def make_voronoi_grid(atm: Atmosphere, nsites: int, kind: str, seed: int, uniform_frac=0.0,
                      cache=True):
    """Sites plus neighbour CSR for the synthetic box of ``atm`` (cached on disk by key)."""
    key = f"vor_a{atm.seed}_n{nsites}_{kind}_s{seed}_u{uniform_frac:g}_v2"
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
    xyz = rejection_sample(f, nsites - n_uni, lo, hi, seed, fmax,
                           f_upper=site_density_envelope(atm, kind))
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

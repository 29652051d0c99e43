"""Pins of the oracle's irregular-grid transport (Sect. 2.5, Eq. 5 and the weight formula after
it) and of the neighbour generator (CPU only)."""
import functools
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import delaunay_neighbours, s4_quadrature

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _uniform_grid(n, seed, box=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0)):
    rng = np.random.default_rng(seed)
    lo = np.array(box[0::2])
    hi = np.array(box[1::2])
    xyz = lo + (hi - lo) * rng.random((n, 3))
    off, code, shift = delaunay_neighbours(xyz, box, periodic_xy=True)
    return dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)


@functools.lru_cache(maxsize=None)
def _small():
    return _uniform_grid(300, 1)


def test_poisson_mean_neighbour_count():
    """Sites from a 3D Poisson process have 15.54 Delaunay neighbours on average (Sect. 2.5)."""
    g = _uniform_grid(6000, 2)
    z = g["xyz"][:, 2]
    cnt = np.diff(g["nbr_off"])
    interior = (z > 0.25) & (z < 0.75)           # away from the mirror walls
    assert cnt[interior].mean() == pytest.approx(GOLD["mean_neighbours_poisson"]["value"], abs=0.3)


def _brute_tables(g, dirs, r):
    """Direct restatement of the upwind choice: candidates with v > 0 that lie upwind in height,
    the two largest v, weights v^r / sum v^r; ghosts stand for their wall."""
    xyz, off, code, shift, box = (g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"])
    n = len(xyz)
    L = np.array([box[1] - box[0], box[3] - box[2]])
    out = {}
    for d, u in enumerate(dirs):
        for i in range(n):
            cands = []
            for e in range(off[i], off[i + 1]):
                c, s = int(code[e]), int(shift[e])
                sx, sy = s // 3 - 1, s % 3 - 1
                if c >= 0:
                    k, wall = c, 0
                elif (-c - 1) % 2 == 0:
                    k, wall = (-c - 1) // 2, 1
                else:
                    k, wall = (-c - 2) // 2, 2
                p = xyz[k] + np.array([sx * L[0], sy * L[1], 0.0])
                if wall == 1:
                    p[2] = 2 * box[4] - p[2]
                if wall == 2:
                    p[2] = 2 * box[5] - p[2]
                dv = xyz[i] - p
                ln = np.linalg.norm(dv)
                if (xyz[i][2] - p[2]) * np.sign(u[2]) <= 0:
                    continue
                v = float(u @ dv) / ln
                if v <= 0:
                    continue
                seg = ln if wall == 0 else ln * (xyz[i][2] - box[4 if wall == 1 else 5]) / (
                    xyz[i][2] - p[2])
                cands.append((-v, c, s, k if wall == 0 else -wall, seg, v))
            cands.sort()
            if len(cands) >= 2:
                a, b = cands[0][5] ** r, cands[1][5] ** r
                out[(d, i)] = ((cands[0][3], cands[1][3]), (a / (a + b), b / (a + b)),
                               (cands[0][4], cands[1][4]))
            elif len(cands) == 1:
                out[(d, i)] = ((cands[0][3], cands[0][3]), (1.0, 0.0), (cands[0][4], cands[0][4]))
            else:
                out[(d, i)] = None
    return out


def test_tables_match_bruteforce():
    g = _small()
    dirs, _ = s4_quadrature()
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    ref = _brute_tables(g, dirs, 7.0)
    nfb = 0
    for (d, i), v in ref.items():
        if v is None:
            nfb += 1
            continue
        (k1, k2), (w1, w2), (l1, l2) = v
        assert tuple(tab["k"][d, i]) == (k1, k2)
        np.testing.assert_allclose(tab["w"][d, i], (w1, w2), rtol=1e-12)
        np.testing.assert_allclose(tab["len"][d, i], (l1, l2), rtol=1e-12)
    assert nfb == tab["n_fallback"]
    # levels: 0 when only walls are upwind, else one more than the deepest upwind site
    for d in range(len(dirs)):
        lv = tab["level"][d]
        for i in range(len(g["xyz"])):
            ks = [k for k, w in zip(tab["k"][d, i], tab["w"][d, i]) if k >= 0 and w > 0]
            assert lv[i] == (1 + max(lv[k] for k in ks) if ks else 0)


def _dfs_intensity(tab, d, alpha, S, up):
    """Memoised recursion over upwind sites (no level schedule), Eq. 5 with linear S."""
    k, w, ln = tab["k"][d], tab["w"][d], tab["len"][d]

    @functools.lru_cache(maxsize=None)
    def I(i):
        acc = 0.0
        for c in range(2):
            if w[i, c] == 0.0:
                continue
            kk = int(k[i, c])
            if kk >= 0:
                Ik, Sk, ak = I(kk), S[kk], alpha[kk]
            else:
                Sk, ak = S[i], alpha[i]
                Ik = S[i] if (up and kk == -1) else 0.0
            t = 0.5 * (ak + alpha[i]) * ln[i, c]
            ex = math.exp(-t)
            w1 = (t - (1 - ex)) / t
            acc += w[i, c] * (Ik * ex + ((1 - ex) - w1) * Sk + w1 * S[i])
        return acc
    return np.array([I(i) for i in range(len(S))])


def test_level_sweep_matches_recursion():
    g = _small()
    dirs, wd = s4_quadrature()
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    rng = np.random.default_rng(3)
    n = len(g["xyz"])
    alpha = rng.uniform(0.5, 20.0, n)
    S = rng.uniform(0.5, 2.0, n)
    J, I = oracle.voronoi_fs(tab, dirs, wd, alpha[None], S[None], bc=0, want_I=True)
    for d in range(len(dirs)):
        ref = _dfs_intensity(tab, d, alpha, S, dirs[d, 2] > 0)
        np.testing.assert_allclose(I[d, 0], ref, rtol=1e-13)
    np.testing.assert_allclose(J[0], np.einsum("d,dn->n", wd, I[:, 0]), rtol=1e-13)


def test_constant_source_with_matching_inflow():
    """S constant and inflow I = S on both walls: I = S at every site (the interval weights
    plus exp(-dtau) sum to one and the two-line weights sum to one)."""
    g = _small()
    dirs, wd = s4_quadrature()
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    n = len(g["xyz"])
    alpha = np.random.default_rng(4).uniform(0.1, 30.0, (1, n))
    S = np.full((1, n), 1.7)
    ibc = np.full((len(dirs), 1, n), 1.7)
    J, I = oracle.voronoi_fs(tab, dirs, wd, alpha, S, bc=2, ibc=ibc, want_I=True)
    np.testing.assert_allclose(I, 1.7, rtol=1e-13)


def test_linear_source_deep_interior():
    """S = a + b z in a homogeneous, very thick medium.  Each upwind segment integrates the
    linear source exactly along its own Delaunay line e, whose particular solution is
    S - b e_z / alpha; with segments many optical depths long the memory of the upwind value is
    lost (exp(-dtau) < 1e-12), so I_i = S_i - (b / alpha) sum_c w_c e_z(k_c -> i) exactly."""
    g = _small()
    dirs, wd = s4_quadrature()
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    n = len(g["xyz"])
    a0, A, B = 2000.0, 3.0, 1.5
    z = g["xyz"][:, 2]
    S = (A + B * z)[None]
    alpha = np.full((1, n), a0)
    J, I = oracle.voronoi_fs(tab, dirs, wd, alpha, S, bc=1, want_I=True)
    checked = 0
    for d in range(len(dirs)):
        k, w, ln = tab["k"][d], tab["w"][d], tab["len"][d]
        for i in range(n):
            if np.any(k[i] < 0) or a0 * ln[i][w[i] > 0].min() < 28.0:
                continue
            ez = sum(w[i, c] * (z[i] - z[k[i, c]]) / ln[i, c] for c in range(2) if w[i, c] > 0)
            assert I[d, 0, i] == pytest.approx(S[0, i] - B * ez / a0, rel=1e-12)
            checked += 1
    assert checked > 1000


# ---- worked example of the upwind choice with closed-form weights (Sect. 2.5, Eq. 5) -----------
def _frame(u):
    """Orthonormal a (towards +z, perpendicular to u) and b = u x a."""
    a = np.array([0.0, 0.0, 1.0]) - u[2] * u
    a /= np.linalg.norm(a)
    return a, np.cross(u, a)


def _line(u, theta_deg, phi_deg):
    """Unit vector at angle theta from u, azimuth phi about u (phi = 0 towards +z)."""
    a, b = _frame(u)
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    return math.cos(t) * u + math.sin(t) * (math.cos(p) * a + math.sin(p) * b)


def test_upwind_choice_worked_example():
    """A hand-built site set whose Delaunay lines make chosen angles with the ray, so that every
    v = cos(angle) is known in closed form (the paper's two-line figure of Sect. 2.5):

    * site 0 has upwind lines at 10, 25 and 40 degrees, one line pointing downwind, and one line
      with v = 0.917 (more aligned than 25 degrees) whose far end lies above site 0, i.e. not
      upwind in height.  Expected: the 10 and 25 degree lines, weights cos^7 / sum cos^7, their
      lengths; the line from above is not a candidate;
    * site 6 sees only the mirror of site 7 in the bottom wall, at 15 degrees: one candidate, the
      bottom wall with weight 1; the segment runs from the wall crossing, length z_6 / e_z;
    * site 8 has no line with v > 0 that is upwind in height: the most nearly vertical upwind
      neighbour, weight 1 (the fallback reading);
    * sites without neighbours start at the wall (level 0); site 0 is one level above its
      upwind sites and site 8 one above site 10.
    """
    u = np.array([0.8688903, 0.3500212, 0.3500212])       # an S4 direction, mu_z = mu_1
    u /= np.linalg.norm(u)
    P = {0: np.array([0.5, 0.5, 0.6])}
    lines = {1: (10.0, 90.0, 0.10), 2: (25.0, 270.0, 0.12), 3: (40.0, 0.0, 0.08)}
    for k, (th, ph, dist) in lines.items():
        P[k] = P[0] - dist * _line(u, th, ph)
    P[4] = P[0] + 0.09 * _line(u, 30.0, 90.0)            # downwind: v = -cos 30 deg
    e5 = np.array([u[0], u[1], -0.05])                    # v > 0 but the far end is higher
    e5 /= np.linalg.norm(e5)
    P[5] = P[0] - 0.1 * e5
    v5 = float(u @ e5)
    assert v5 > math.cos(math.radians(25.0)) and P[5][2] > P[0][2]
    P[6] = np.array([0.3, 0.7, 0.05])
    e6 = _line(u, 15.0, 90.0)
    ghost7 = P[6] - 0.2 * e6                              # below the wall z = 0
    assert ghost7[2] < 0.0
    P[7] = np.array([ghost7[0], ghost7[1], -ghost7[2]])
    P[8] = np.array([0.8, 0.2, 0.5])
    e9 = np.array([-0.9, -0.3, 0.3]) / np.linalg.norm([-0.9, -0.3, 0.3])
    e10 = np.array([-0.5, -0.5, 0.7]) / np.linalg.norm([-0.5, -0.5, 0.7])
    assert u @ e9 < 0 and u @ e10 < 0
    P[9] = P[8] - 0.1 * e9
    P[10] = P[8] - 0.15 * e10
    n = 11
    xyz = np.array([P[i] for i in range(n)])
    nb = {0: [(1, 4), (2, 4), (3, 4), (4, 4), (5, 4)], 6: [(-1 - 2 * 7, 4)], 8: [(9, 4), (10, 4)]}
    off, code, shift = [0], [], []
    for i in range(n):
        for c, s in nb.get(i, []):
            code.append(c)
            shift.append(s)
        off.append(len(code))
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    tab = oracle.voronoi_tables(xyz, np.array(off, np.int64), np.array(code, np.int32),
                                np.array(shift, np.int8), box, u[None], 7.0)
    k, w, ln, lv = tab["k"][0], tab["w"][0], tab["len"][0], tab["level"][0]
    c10, c25 = math.cos(math.radians(10.0)) ** 7, math.cos(math.radians(25.0)) ** 7
    assert tuple(k[0]) == (1, 2)
    np.testing.assert_allclose(w[0], (c10 / (c10 + c25), c25 / (c10 + c25)), rtol=1e-12)
    np.testing.assert_allclose(ln[0], (0.10, 0.12), rtol=1e-12)
    assert tuple(k[6]) == (-1, -1) and tuple(w[6]) == (1.0, 0.0)
    np.testing.assert_allclose(ln[6], P[6][2] / e6[2], rtol=1e-12)
    assert tuple(k[8]) == (10, 10) and tuple(w[8]) == (1.0, 0.0)
    np.testing.assert_allclose(ln[8], 0.15, rtol=1e-12)
    for i in (1, 2, 3, 4, 5, 7, 9, 10):       # no neighbours: the bottom wall, vertical distance
        assert tuple(k[i]) == (-1, -1) and lv[i] == 0
        np.testing.assert_allclose(ln[i, 0], xyz[i, 2] / u[2], rtol=1e-12)
    assert lv[0] == 1 and lv[6] == 0 and lv[8] == 1
    # sites 1-5, 7, 9, 10 (no neighbours) and site 8 (no candidate) fall back
    assert tab["n_fallback"] == 9


# ---- mirror symmetry of the tables and the transport (x -> -x) --------------------------------
def test_mirror_symmetry_tables_and_intensity():
    """Mirroring the site set in x (x -> 1 - x) and every direction (u_x -> -u_x) maps the tables
    of direction d onto those of its mirror image d' site by site (same upwind sites, weights and
    lengths), and with the same alpha and S at every site the intensities of d and d' agree; J,
    a sum over a mirror-symmetric quadrature, is unchanged."""
    g = _small()
    dirs, wd = s4_quadrature()
    xm = g["xyz"].copy()
    xm[:, 0] = 1.0 - xm[:, 0]
    # the mirrored site set keeps each site's neighbours; a periodic image sx becomes -sx
    # (the Delaunay relation is mirror symmetric; rebuilding it would only differ where wall
    # mirrors make the triangulation degenerate)
    off, code = g["nbr_off"], g["nbr_idx"]
    s = g["nbr_shift"].astype(np.int64)
    shift = ((2 - s // 3) * 3 + s % 3).astype(np.int8)
    mir = np.array([int(np.argmin(np.abs(dirs - d * np.array([-1, 1, 1])).sum(1))) for d in dirs])
    np.testing.assert_allclose(dirs[mir], dirs * np.array([-1, 1, 1]), atol=1e-15)
    t0 = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                               dirs, 7.0)
    t1 = oracle.voronoi_tables(xm, off, code, shift, g["box"], dirs, 7.0)
    np.testing.assert_array_equal(t1["k"][mir], t0["k"])
    np.testing.assert_array_equal(t1["level"][mir], t0["level"])
    np.testing.assert_allclose(t1["w"][mir], t0["w"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(t1["len"][mir], t0["len"], rtol=1e-12)
    rng = np.random.default_rng(9)
    n = len(xm)
    alpha = 10.0 ** rng.uniform(-2, 1.5, (2, n))
    S = rng.uniform(0.5, 2.0, (2, n))
    J0, I0 = oracle.voronoi_fs(t0, dirs, wd, alpha, S, bc=0, want_I=True)
    J1, I1 = oracle.voronoi_fs(t1, dirs, wd, alpha, S, bc=0, want_I=True)
    np.testing.assert_allclose(I1[mir], I0, rtol=1e-12)
    np.testing.assert_allclose(J1, J0, rtol=1e-12)


# ---- searchlight beam on the Voronoi grid (Sect. 3.1) -----------------------------------------
def _numpy_tables(xyz, off, code, shift, box, u, rule):
    """Upwind tables of one direction built with a deliberately wrong rule (planted mistakes for
    the searchlight pins): "smallest" ranks the candidates by the smallest v, "inverse" weights
    by v^-7, "top1" keeps only the best line."""
    n = len(xyz)
    row = np.repeat(np.arange(n), np.diff(off))
    c = code.astype(np.int64)
    s = shift.astype(np.int64)
    wall = np.where(c >= 0, 0, np.where(((-c - 1) & 1) == 0, 1, 2))
    k = np.where(c >= 0, c, np.where(wall == 1, (-c - 1) // 2, (-c - 2) // 2))
    p = xyz[k].copy()
    p[:, 0] += (s // 3 - 1) * (box[1] - box[0])
    p[:, 1] += (s % 3 - 1) * (box[3] - box[2])
    p[wall == 1, 2] = 2 * box[4] - p[wall == 1, 2]
    p[wall == 2, 2] = 2 * box[5] - p[wall == 2, 2]
    dv = xyz[row] - p
    ln = np.linalg.norm(dv, axis=1)
    v = dv @ u / ln
    cand = (dv[:, 2] * np.sign(u[2]) > 0) & (v > 0)
    seg = np.where(wall == 1, ln * (xyz[row, 2] - box[4]) / dv[:, 2],
                   np.where(wall == 2, ln * (xyz[row, 2] - box[5]) / dv[:, 2], ln))
    kk = np.where(wall == 0, k, -wall)
    order = np.lexsort((np.where(cand, v if rule == "smallest" else -v, np.inf), row))
    cnt = np.bincount(row[cand], minlength=n)
    assert (cnt > 0).all()
    o1 = order[off[:-1]]
    o2 = order[np.minimum(off[:-1] + 1, off[1:] - 1)]
    two = (cnt >= 2) & (rule != "top1")
    e = -7.0 if rule == "inverse" else 7.0
    a, b = v[o1] ** e, v[o2] ** e
    K = np.stack([kk[o1], np.where(two, kk[o2], kk[o1])], 1).astype(np.int32)
    W = np.stack([np.where(two, a / (a + b), 1.0), np.where(two, b / (a + b), 0.0)], 1)
    L = np.stack([seg[o1], np.where(two, seg[o2], seg[o1])], 1)
    lv = np.zeros(n, np.int32)
    for i in np.argsort(xyz[:, 2] * np.sign(u[2]), kind="stable"):
        up = [lv[K[i, q]] + 1 for q in range(2) if K[i, q] >= 0 and W[i, q] > 0]
        lv[i] = max(up) if up else 0
    return dict(k=K[None], w=W[None], len=L[None], level=lv[None])


@functools.lru_cache(maxsize=None)
def _searchlight_box():
    """51^3 sites uniform in a 1 m box (Sect. 3.1: uniform sampling for this test only)."""
    m = 51
    xyz = np.random.default_rng(51).random((m ** 3, 3))
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    off, code, shift = delaunay_neighbours(xyz, box, periodic_xy=True)
    top = np.zeros(len(xyz), bool)
    for i in range(len(xyz)):
        cc = code[off[i]:off[i + 1]]
        top[i] = np.any((cc < 0) & (((-cc - 1) & 1) == 1))
    return m, xyz, off, code, shift, box, top


def _walk_moments(tab, u, xyz, sel):
    """alpha = S = 0 makes every site the weighted mean of its upwind sites, so with the inflow
    at the bottom wall set to x_b, y_b, x_b^2, y_b^2 of the ray's wall crossing each site returns
    the mean and second moment of where its intensity came from.  Returns the mean drift bias
    (x, y) against the straight ray and the mean lateral variance (x, y) over the sites ``sel``."""
    n = len(xyz)
    t = u[0] / u[2], u[1] / u[2]
    cx = xyz[:, 0] - xyz[:, 2] * t[0]
    cy = xyz[:, 1] - xyz[:, 2] * t[1]
    ibc = np.stack([cx, cy, cx * cx, cy * cy])[None]
    z4 = np.zeros((4, n))
    _, I = oracle.voronoi_fs(tab, u[None], np.array([1.0]), z4, z4, bc=2, ibc=ibc, want_I=True)
    Ex, Ey, Exx, Eyy = I[0]
    return ((Ex - cx)[sel].mean(), (Ey - cy)[sel].mean(), (Exx - Ex ** 2)[sel].mean(),
            (Eyy - Ey ** 2)[sel].mean())


@pytest.mark.slow
def test_searchlight_voronoi():
    """Sect. 3.1: a beam at theta = 20 deg through a 1 m box of 51^3 sites with alpha = S = 0.

    * Direction: the weighted pairs of Delaunay lines carry the beam along the ray; the mean
      arrival point of the top-layer sites lies within one site spacing h of the straight ray.
    * Diffusion: the paper finds the irregular grid's diffusion comparable with short
      characteristics with linear interpolation.  The regular grid's lateral variance after the
      50 plane steps is exactly 50 t (1 - t) h^2 (t = tan 20 deg, the bilinear weight); the
      Voronoi grid's total lateral variance must lie within a factor 2 of it.
    * Peak: with the beam of 0.2 m diameter (the reading taken, see the design notes; a 0.2 m
      radius keeps the peak at 1.00 on both grids), the peak at the top falls to 0.6-0.9 on both
      grids (the paper: about 70 % on both).
    * Planted mistakes: ranking by the smallest v, x and y of the ray swapped, and the sign of v
      flipped each move the beam by many h; weights v^-7 or one line instead of two put the
      variance outside the factor 2.  (The exponent r itself is pinned by the worked example:
      the paper notes the results are not very sensitive to it.)
    """
    m, xyz, off, code, shift, box, top = _searchlight_box()
    h = 1.0 / m
    th = math.radians(20.0)
    u = np.array([math.sin(th), 0.0, math.cos(th)])
    tant = math.tan(th)
    # the regular grid: exact bilinear random walk, with its closed-form variance
    zc = (np.arange(m) + 0.5) * h
    X, Y = np.meshgrid(zc, zc, indexing="xy")
    inflow = np.stack([X, Y, X * X, Y * Y]).reshape(1, 4, -1)
    z4 = np.zeros((4, m ** 3))
    _, Ir = oracle.sc_regular(m, m, m, h, h, zc, u[None], np.array([1.0]), z4, z4, bc=2,
                              ibc=inflow, want_I=True)
    Ex, Ey, Exx, Eyy = (Ir[0, q, -m * m:].reshape(m, m) for q in range(4))
    win = (X > 0.6) & (X < 0.95) & (Y > 0.25) & (Y < 0.75)     # away from the periodic seam
    var_reg = (Exx - Ex ** 2)[win].mean() + (Eyy - Ey ** 2)[win].mean()
    # (exact but for the walk's far tail, which reaches the periodic seam with weight < 1e-4)
    assert abs((Ex - (X - (m - 1) * h * tant))[win].mean()) < 1e-3 * h
    assert var_reg == pytest.approx((m - 1) * (tant % 1) * (1 - tant % 1) * h * h, rel=1e-3)
    sel = top & (xyz[:, 0] > 0.6) & (xyz[:, 0] < 0.95) & (xyz[:, 1] > 0.25) & (xyz[:, 1] < 0.75)
    assert sel.sum() > 300

    def moments(tab):
        bx, by, vx, vy = _walk_moments(tab, u, xyz, sel)
        return bx / h, by / h, (vx + vy) / var_reg

    tab = oracle.voronoi_tables(xyz, off, code, shift, box, u[None], 7.0)
    bx, by, ratio = moments(tab)
    assert abs(bx) < 1.0 and abs(by) < 1.0, (bx, by)
    assert 0.5 < ratio < 2.0, ratio

    # beam of 0.1 m radius from the centre of the bottom; peak near the axis in the top 5 %
    R = 0.1
    n = len(xyz)
    x0 = (xyz[:, 0] - xyz[:, 2] * tant) % 1.0
    beam = (((x0 - 0.5) ** 2 + (xyz[:, 1] - 0.5) ** 2) <= R * R).astype(float)[None, None]
    zero = np.zeros((1, n))
    _, Iv = oracle.voronoi_fs(tab, u[None], np.array([1.0]), zero, zero, bc=2, ibc=beam,
                              want_I=True)
    lay = xyz[:, 2] > 0.95
    dxa = (xyz[:, 0] - (0.5 + xyz[:, 2] * tant) + 0.5) % 1.0 - 0.5
    near = lay & (np.hypot(dxa, xyz[:, 1] - 0.5) < 0.03)
    peak_vor = Iv[0, 0, near].mean()
    xr0 = (X - zc[0] * tant) % 1.0
    beam_r = (((xr0 - 0.5) ** 2 + (Y - 0.5) ** 2) <= R * R).astype(float).reshape(1, 1, -1)
    _, Ib = oracle.sc_regular(m, m, m, h, h, zc, u[None], np.array([1.0]), zero, zero, bc=2,
                              ibc=beam_r, want_I=True)
    Ib = Ib[0, 0].reshape(m, m, m)
    ZZ, YY, XX = np.meshgrid(zc, zc, zc, indexing="ij")
    dxr = (XX - (0.5 + ZZ * tant) + 0.5) % 1.0 - 0.5
    near_r = (ZZ > 0.95) & (np.hypot(dxr, YY - 0.5) < 0.03)
    peak_reg = Ib[near_r].mean()
    assert 0.6 < peak_vor < 0.9 and 0.6 < peak_reg < 0.9, (peak_vor, peak_reg)
    assert Ib[-1].sum() == pytest.approx(beam_r.sum(), rel=1e-12)    # flux kept (periodic)

    # planted mistakes
    for rule in ("smallest",):
        bx, by, _ = moments(_numpy_tables(xyz, off, code, shift, box, u, rule))
        assert max(abs(bx), abs(by)) > 3.0, (rule, bx, by)
    for bad_u in (np.array([u[1], u[0], u[2]]), np.array([-u[0], -u[1], u[2]])):
        bx, by, _ = moments(oracle.voronoi_tables(xyz, off, code, shift, box, bad_u[None], 7.0))
        assert max(abs(bx), abs(by)) > 3.0, (bad_u, bx, by)
    for rule in ("inverse", "top1"):
        _, _, r_bad = moments(_numpy_tables(xyz, off, code, shift, box, u, rule))
        assert not 0.5 < r_bad < 2.0, (rule, r_bad)
    # the numpy restatement with the right rule reproduces the oracle's moments
    assert moments(_numpy_tables(xyz, off, code, shift, box, u, "ok")) == pytest.approx(
        moments(tab), rel=1e-9, abs=1e-9)

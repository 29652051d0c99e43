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

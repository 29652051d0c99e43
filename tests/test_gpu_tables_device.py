"""Voronoi upwind tables and dependency levels built on the GPU (rt_grid_build_tables_device)
against the host build and the FP64 oracle: the choices (upwind sites, levels, fallbacks) must be
identical, the FP32 weights and lengths equal to rounding; the formal solution on the rebuilt
tables keeps its parity."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, lattice_grid, tie_directions, to_gpu, voronoi_grid
from synth import delaunay_neighbours, s4_quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def _unit_box(seed=1, n=400):
    rng = np.random.default_rng(seed)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((n, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    return dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)


def _check(rt, g, dirs=None, w=None):
    """A grid created with the host table build (RT_VORONOI_TABLES=host), its tables rebuilt on
    the device in place: both against the oracle; and a grid created with the default build."""
    import os
    if dirs is None:
        dirs, w = s4_quadrature()
    os.environ["RT_VORONOI_TABLES"] = "host"
    try:
        G = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs,
                           w)
    finally:
        del os.environ["RT_VORONOI_TABLES"]
    default = rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs,
                             w).tables()
    host = G.tables()
    ml, nfb = G.max_levels, G.n_fallback
    G.build_tables_device()
    dev = G.tables()
    ref = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    np.testing.assert_array_equal(dev["k"], ref["k"])
    np.testing.assert_array_equal(dev["level"], ref["level"])
    np.testing.assert_allclose(dev["w"], ref["w"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(dev["len"], ref["len"], rtol=1e-6)
    np.testing.assert_array_equal(dev["k"], host["k"])
    np.testing.assert_array_equal(dev["level"], host["level"])
    for key in ("k", "w", "len", "level"):
        np.testing.assert_array_equal(default[key], dev[key])
    assert G.n_fallback == ref["n_fallback"] == nfb
    assert G.max_levels == ref["level"].max() + 1 == ml
    return G, dirs, w, ref


def test_unit_box_grid(rt):
    _check(rt, _unit_box())


def test_lattice_grid_with_exact_ties(rt):
    """Two neighbours tie exactly for second place for every direction: the tie rules decide (by
    neighbour code on the lattice); in a one-site-wide column every lateral neighbour is a periodic
    image of the site above or below."""
    _check(rt, lattice_grid(4), *tie_directions())
    _check(rt, lattice_grid(1, 4), *tie_directions())


def test_atmosphere_grid_and_formal_solution(rt):
    """A 3000-site grid sampled from |dtau/dz| of the synthetic atmosphere; the formal solution
    of three wavelengths on the rebuilt tables against the oracle, thermal and zero inflow."""
    atm, g, f = voronoi_grid(3000, "dtau", 4)
    G, dirs, w, tab = _check(rt, g)
    rng = np.random.default_rng(5)
    n = len(g["xyz"])
    a = 10.0 ** rng.uniform(-4, 1, (3, n)) / 1e5
    s = rng.uniform(0.5, 2.0, (3, n))
    for bc in (0, 1):
        J = rt.formal_solution(G, to_gpu(a), to_gpu(s), bc=bc).cpu().numpy()
        Jr = oracle.voronoi_fs(tab, dirs, w, a, s, bc=bc)
        assert_parity(J, Jr, what=f"J bc={bc}")

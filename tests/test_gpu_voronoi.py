"""GPU parity of the Voronoi-grid transport (Sect. 2.5, Eq. 5 and the weight formula after it) and
of its upwind tables and dependency levels against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, to_gpu, voronoi_grid
from synth import delaunay_neighbours, s4_quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def _small(seed=1, n=400):
    rng = np.random.default_rng(seed)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((n, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    return dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)


def _grid(rt, g, dirs, w):
    return rt.VoronoiGrid(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"], dirs,
                          w)


def test_tables_and_levels_match_oracle(rt):
    g = _small()
    dirs, w = s4_quadrature()
    G = _grid(rt, g, dirs, w)
    tab = G.tables()
    ref = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    np.testing.assert_array_equal(tab["k"], ref["k"])
    np.testing.assert_array_equal(tab["level"], ref["level"])
    np.testing.assert_allclose(tab["w"], ref["w"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(tab["len"], ref["len"], rtol=1e-6)
    assert G.n_fallback == ref["n_fallback"]
    assert G.max_levels == ref["level"].max() + 1


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_small_grid_multi_lambda(rt, bc):
    g = _small(2, 500)
    dirs, w = s4_quadrature()
    n, nlam = len(g["xyz"]), 5
    rng = np.random.default_rng(5)
    a = 10.0 ** rng.uniform(-4, 2, (nlam, n))
    s = rng.uniform(0.5, 2.0, (nlam, n))
    ibc = rng.uniform(0, 2, (24, nlam, n)) if bc == 2 else None
    G = _grid(rt, g, dirs, w)
    J, I = rt.formal_solution(G, to_gpu(a), to_gpu(s), bc=bc,
                              I_bc=to_gpu(ibc) if ibc is not None else None, want_I=True)
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    Jr, Ir = oracle.voronoi_fs(tab, dirs, w, a, s, bc=bc, ibc=ibc, want_I=True)
    assert_parity(J.cpu().numpy(), Jr, what="J")
    assert_parity(I.cpu().numpy(), Ir, what="I")


def test_constant_source_matching_inflow(rt):
    g = _small(3)
    dirs, w = s4_quadrature()
    n = len(g["xyz"])
    G = _grid(rt, g, dirs, w)
    a = np.random.default_rng(1).uniform(0.1, 50.0, (1, n))
    s = np.full((1, n), 1.7)
    ibc = np.full((24, 1, n), 1.7)
    _, I = rt.formal_solution(G, to_gpu(a), to_gpu(s), bc=2, I_bc=to_gpu(ibc), want_I=True)
    np.testing.assert_allclose(I.cpu().numpy(), 1.7, rtol=2e-6)


def test_lte_continuum_20k_sites(rt):
    """The 20k-site irregular LTE continuum workload (density from |dtau/dz|)."""
    from oracle.physics import lte_alpha_S
    atm, g, f = voronoi_grid(20000, "dtau", 0)
    dirs, w = s4_quadrature()
    a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    G = _grid(rt, g, dirs, w)
    alpha, S = rt.source_terms_lte(to_gpu(f["T"]), to_gpu(f["rho"]), atm.kappa0, 500e-9)
    J = rt.formal_solution(G, alpha[None], S[None])
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    Jr = oracle.voronoi_fs(tab, dirs, w, a[None], s[None])
    assert_parity(J.cpu().numpy(), Jr, what="J 20k")


@pytest.mark.parametrize("bc,nlam,n", [(0, 5, 500), (1, 7, 1500), (1, 52, 800)])
def test_persistent_sweep_equals_level_launches(rt, monkeypatch, bc, nlam, n):
    """The default J-only formal solution runs every direction of the grid in one persistent
    launch (per-direction intensities, J reduced in direction order); it equals the per-direction,
    per-level launches bit for bit and matches the oracle."""
    import torch
    g = _small(7, n)
    dirs, w = s4_quadrature()
    rng = np.random.default_rng(9)
    a = 10.0 ** rng.uniform(-4, 2, (nlam, n))
    s = rng.uniform(0.5, 2.0, (nlam, n))
    G = _grid(rt, g, dirs, w)
    out = {}
    for mode in ("persistent", "levels"):
        if mode == "levels":
            monkeypatch.setenv("RT_VORONOI_SWEEP", "levels")
        else:
            monkeypatch.delenv("RT_VORONOI_SWEEP", raising=False)
        n0 = rt.kernel_launches()
        out[mode] = rt.formal_solution(G, to_gpu(a), to_gpu(s), bc=bc).cpu()
        launched = rt.kernel_launches() - n0
        if mode == "persistent":   # (S, alpha) packing, sweep, J reduction into [nlam][n]
            assert launched == 3, launched
        torch.cuda.synchronize()
    assert torch.equal(out["persistent"], out["levels"])
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    Jr = oracle.voronoi_fs(tab, dirs, w, a, s, bc=bc)
    assert_parity(out["persistent"].numpy(), Jr, what="J persistent")


def test_wavelength_chunks_give_the_same_J(rt, monkeypatch):
    """When the per-direction intensities of all wavelengths exceed the device-memory budget, the
    single-grid sweep runs the wavelengths in equal chunks (a divisor of their count): J is bit
    for bit the one pass's, and matches the oracle."""
    import torch
    g = _small(4, 3000)
    dirs, w = s4_quadrature()
    n, nlam = len(g["xyz"]), 12
    rng = np.random.default_rng(8)
    a = 10.0 ** rng.uniform(-3, 2, (nlam, n))
    s = rng.uniform(0.5, 2.0, (nlam, n))
    ag, sg = to_gpu(a), to_gpu(s)
    monkeypatch.delenv("RT_VORONOI_BATCH_MB", raising=False)
    J1 = rt.formal_solution(_grid(rt, g, dirs, w), ag, sg)
    # 26 floats per site and padded wavelength (a multiple of 8): 3000 sites x 8 is 2.5 MB, so a
    # 3 MB budget allows chunks of 6 (two chunks); below 2.5 MB single wavelengths remain
    for mb in ("3", "1"):
        monkeypatch.setenv("RT_VORONOI_BATCH_MB", mb)
        Jc = rt.formal_solution(_grid(rt, g, dirs, w), ag, sg)
        torch.cuda.synchronize()
        assert torch.equal(Jc, J1), mb
    tab = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    Jr = oracle.voronoi_fs(tab, dirs, w, a, s)
    assert_parity(J1.cpu().numpy(), Jr, what="J")

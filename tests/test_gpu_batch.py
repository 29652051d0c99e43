"""The batched persistent sweep over several Voronoi grids of uneven size must equal the plain
per-direction, per-level launches, and CUDA-graph replay must equal eager execution."""
import numpy as np
import pytest

from helpers import assert_parity, to_gpu
from synth import delaunay_neighbours, s4_quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def _grids(rt, sizes, seed=0):
    rng = np.random.default_rng(seed)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    dirs, w = s4_quadrature()
    out = []
    for n in sizes:
        xyz = rng.random((n, 3))
        off, code, shift = delaunay_neighbours(xyz, box)
        out.append(rt.VoronoiGrid(xyz, off, code, shift, box, dirs, w))
    return out


@pytest.mark.parametrize("lam_chunk", [None, [1, 2, 7]])
def test_batch_equals_plain(rt, lam_chunk):
    grids = _grids(rt, [300, 700, 1500])
    nlam = 7
    rng = np.random.default_rng(1)
    alphas = [to_gpu(10.0 ** rng.uniform(-3, 2, (nlam, g.npt))) for g in grids]
    Ss = [to_gpu(rng.uniform(0.5, 2.0, (nlam, g.npt))) for g in grids]
    batch = rt.Batch(grids, nlam, lam_chunk=lam_chunk)
    Jb = batch.formal_solution(alphas, Ss)
    for g, a, s, jb in zip(grids, alphas, Ss, Jb):
        jp = rt.formal_solution(g, a, s)
        assert_parity(jb.cpu().numpy(), jp.cpu().numpy().astype(np.float64), rel=1e-6,
                      what="batch vs plain")


def test_graph_replay_equals_eager(rt):
    import torch
    grids = _grids(rt, [400, 900], seed=2)
    nlam = 4
    rng = np.random.default_rng(3)
    alphas = [to_gpu(10.0 ** rng.uniform(-2, 1, (nlam, g.npt))) for g in grids]
    Ss = [to_gpu(rng.uniform(0.5, 2.0, (nlam, g.npt))) for g in grids]
    batch = rt.Batch(grids, nlam)
    Js = [torch.empty_like(a) for a in alphas]
    eager = [j.clone() for j in batch.formal_solution(alphas, Ss, Js=Js)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.formal_solution(alphas, Ss, Js=Js, stream=s)   # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            batch.formal_solution(alphas, Ss, Js=Js, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for j in Js:
        j.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for e, j in zip(eager, Js):
        assert torch.equal(e, j)


def test_autotuner_choice_is_correct_and_cached(rt, tmp_path, monkeypatch):
    import importlib
    monkeypatch.setenv("RT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    import paper_2306_01041_gb300.autotune as at
    at = importlib.reload(at)
    grids = _grids(rt, [300, 900], seed=5)
    nlam = 5
    rng = np.random.default_rng(6)
    alphas = [to_gpu(10.0 ** rng.uniform(-2, 1, (nlam, g.npt))) for g in grids]
    Ss = [to_gpu(rng.uniform(0.5, 2.0, (nlam, g.npt))) for g in grids]
    batch, choice = at.tune_batch(grids, alphas, Ss, nlam, candidates=[(1.0, 256), (2.0, 512)])
    assert (tmp_path / "tune.json").exists() and len(choice["lam_chunk"]) == 2
    Jb = batch.formal_solution(alphas, Ss)
    for g, a, s, jb in zip(grids, alphas, Ss, Jb):
        assert_parity(jb.cpu().numpy(), rt.formal_solution(g, a, s).cpu().numpy().astype(np.float64),
                      rel=1e-6, what="tuned batch")
    _, again = at.tune_batch(grids, alphas, Ss, nlam)
    assert again == choice


# ---- the batch against the FP64 oracle ---------------------------------------------------------
def _atm_grid(rt, n, kind, seed, atm_seed):
    from helpers import voronoi_grid
    atm, vg, f = voronoi_grid(n, kind, seed, atm_seed)
    dirs, w = s4_quadrature()
    G = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"], dirs,
                       w)
    return atm, vg, f, G


def _lte_fields(atm, f, data):
    """alpha, S [52][n] of the NLTE atom at its LTE populations (FP64, the oracle's physics)."""
    from oracle.physics import Atom
    A = Atom(data, atm.kappa0)
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    return A.alpha_S(f["T"], f["rho"], f["ne"], pops)


@pytest.mark.parametrize("lam_chunk", [None, [4, 13, 52]])
def test_batch_uneven_grids_match_oracle(rt, lam_chunk):
    """Three atmosphere grids of uneven size (1500, 4000, 9000 sites; rho^0.3 and |dtau/dz|
    sampling), the 52 wavelengths of the atom and 24 directions in one batched launch, with the
    built-in wavelength chunks and with chunks of 4, 13 and 52: J of every grid against the
    oracle's level sweep (Sect. 2.5, Eq. 5)."""
    import oracle
    from synth import model_atom
    specs = [(1500, "rho03", 21), (4000, "dtau", 22), (9000, "rho03", 23)]
    grids, fields, vgs = [], [], []
    for n, kind, seed in specs:
        atm, vg, f, G = _atm_grid(rt, n, kind, seed, 0)
        data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
        fields.append(_lte_fields(atm, f, data))
        grids.append(G)
        vgs.append(vg)
    batch = rt.Batch(grids, 52, lam_chunk=lam_chunk)
    Jb = batch.formal_solution([to_gpu(a) for a, s in fields], [to_gpu(s) for a, s in fields])
    dirs, w = s4_quadrature()
    for vg, (a, s), jb in zip(vgs, fields, Jb):
        tab = oracle.voronoi_tables(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"],
                                    vg["box"], dirs, 7.0)
        assert_parity(jb.cpu().numpy(), oracle.voronoi_fs(tab, dirs, w, a, s), what="batched J")


def test_batch_with_a_deep_grid_matches_oracle(rt):
    """The 160 000-site rho^0.3 atmosphere of the 8-atmosphere workload (more than 100 dependency
    levels in its deepest directions) batched with a 20 000-site |dtau/dz| grid, 52 wavelengths:
    J at a line-core, a line-wing and a continuum wavelength against the oracle, at every site."""
    import oracle
    from synth import model_atom
    dirs, w = s4_quadrature()
    specs = [(160000, "rho03", 5, 5), (20000, "dtau", 10, 0)]
    grids, fields, vgs = [], [], []
    for n, kind, seed, atm_seed in specs:
        atm, vg, f, G = _atm_grid(rt, n, kind, seed, atm_seed)
        data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
        fields.append(_lte_fields(atm, f, data))
        grids.append(G)
        vgs.append(vg)
    assert grids[0].max_levels > 100
    batch = rt.Batch(grids, 52)
    Jb = batch.formal_solution([to_gpu(a) for a, s in fields], [to_gpu(s) for a, s in fields])
    pick = [25, 40, 50]
    for vg, (a, s), jb in zip(vgs, fields, Jb):
        tab = oracle.voronoi_tables(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"],
                                    vg["box"], dirs, 7.0)
        ref = oracle.voronoi_fs(tab, dirs, w, a[pick], s[pick])
        assert_parity(jb.cpu().numpy()[pick], ref, what="deep-grid batched J")


@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_lambda_iteration_matches_oracle(rt, use_graph):
    """Three Lambda iterations (Sect. 2.1, Eq. 3-4) of two atmospheres' grids together
    (rt_batch_lambda_iterate, one CUDA graph per iteration or eager launches) against the
    oracle's iteration of each grid on its own: populations after every grid's third update."""
    from oracle.physics import Atom
    from oracle.solve import VoronoiGrid as OrcVoronoi
    from oracle.solve import lambda_iterate as orc_lambda_iterate
    from synth import model_atom
    dirs, w = s4_quadrature()
    specs = [(2000, "rho03", 31), (3500, "dtau", 32)]
    grids, fs, vgs = [], [], []
    for n, kind, seed in specs:
        atm, vg, f, G = _atm_grid(rt, n, kind, seed, 0)
        grids.append(G)
        fs.append(f)
        vgs.append(vg)
    data = model_atom(min(np.min(f["ne"] / np.sqrt(f["T"])) for f in fs))
    A = Atom(data, atm.kappa0)
    ga = rt.Atom(data, atm.kappa0)
    atms = [rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))
            for f in fs]
    pops = [rt.lte_populations(G, ga, M) for G, M in zip(grids, atms)]
    batch = rt.Batch(grids, len(data["lam"]))
    its, hist, conv = batch.lambda_iterate(ga, atms, pops, max_iter=3, tol=0.0,
                                           use_graph=use_graph)
    assert its == 3 and not conv
    hmax = np.zeros(3)
    for vg, f, p in zip(vgs, fs, pops):
        ref, it, h = orc_lambda_iterate(OrcVoronoi(vg, dirs, w), A, f["T"], f["rho"], f["ne"],
                                        f["nH"], max_iter=3, tol=0.0)
        assert_parity(p.cpu().numpy(), ref, rel=1e-4, floor=0.0, what="batched iteration pops")
        hmax = np.maximum(hmax, h)
    np.testing.assert_allclose(hist, hmax, rtol=2e-2)

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

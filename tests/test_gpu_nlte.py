"""GPU parity of the atom kernels (opacity and source function, rates and statistical
equilibrium; Sect. 2.1-2.2) and of the Lambda iteration (Eq. 3-4) against the FP64 oracle."""
import functools

import numpy as np
import pytest

from helpers import assert_parity, to_gpu
from oracle.physics import Atom
from oracle.solve import RegularGrid as OrcRegular
from oracle.solve import VoronoiGrid as OrcVoronoi
from oracle.solve import lambda_iterate as orc_lambda_iterate
from synth import make_atmosphere, model_atom, s4_quadrature
from synth.atmosphere import regular_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


@functools.lru_cache(maxsize=None)
def _setup(nx, ny, nz, n_line=50):
    atm = make_atmosphere(0)
    f, ax = regular_fields(nx, ny, nz, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])), n_line=n_line)
    return atm, f, ax, data


def _gpu_atm(rt, f):
    return rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))


def test_lte_populations(rt):
    atm, f, (x, y, z, dx, dy), data = _setup(12, 10, 24)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(12, 10, 24, dx, dy, z, dirs, w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    assert_parity(pops.cpu().numpy(), A.lte_pops(f["T"], f["ne"], f["nH"]), rel=1e-5,
                  floor=0.0, what="LTE pops")


# (grid, line nodes): 52 nodes on 2880 points (a whole number of 32-point blocks), and 112 nodes
# (four per lane of a warp) on 2990 points (a ragged last block)
ATOM_CASES = [((12, 10, 24), 50), ((13, 10, 23), 110)]


@pytest.mark.parametrize("shape,n_line", ATOM_CASES)
@pytest.mark.parametrize("perturb", [0.0, 0.3])
def test_source_terms(rt, perturb, shape, n_line):
    """alpha, S at every node (Voigt line profile on the GPU vs scipy's in the oracle)."""
    atm, f, (x, y, z, dx, dy), data = _setup(*shape, n_line)
    A = Atom(data, atm.kappa0)
    rng = np.random.default_rng(2)
    pops = A.lte_pops(f["T"], f["ne"], f["nH"]) * np.exp(perturb * rng.standard_normal((3, f["T"].size)))
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(*shape, dx, dy, z, dirs, w)
    alpha, S = rt.source_terms(g, rt.Atom(data, atm.kappa0), _gpu_atm(rt, f), to_gpu(pops))
    ar, sr = A.alpha_S(f["T"], f["rho"], f["ne"], pops.astype(np.float32).astype(np.float64))
    assert_parity(alpha.cpu().numpy(), ar, rel=2e-5, floor=0.0, what="alpha")
    assert_parity(S.cpu().numpy(), sr, rel=2e-5, floor=0.0, what="S")


@pytest.mark.parametrize("shape,n_line", ATOM_CASES)
def test_statistical_equilibrium(rt, shape, n_line):
    atm, f, (x, y, z, dx, dy), data = _setup(*shape, n_line)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    alpha, S = A.alpha_S(f["T"], f["rho"], f["ne"], pops)
    J = OrcRegular(*shape, dx, dy, z, dirs, w).formal_solution(alpha, S)
    new = A.statistical_equilibrium(A.rate_matrix(f["T"], f["ne"], J), f["nH"])
    g = rt.RegularGrid(*shape, dx, dy, z, dirs, w)
    p = to_gpu(pops)
    dmax = rt.statistical_equilibrium(g, rt.Atom(data, atm.kappa0), _gpu_atm(rt, f), to_gpu(J), p)
    assert_parity(p.cpu().numpy(), new, rel=5e-5, floor=0.0, what="pops")
    ref_d = np.max(np.abs(new - pops.astype(np.float32)) / new)
    assert float(dmax.item()) == pytest.approx(ref_d, rel=1e-3)


@pytest.mark.parametrize("use_graph", [False, True])
def test_lambda_iteration_regular(rt, use_graph):
    """Eight Lambda iterations on a 20 x 20 x 32 grid (52 wavelengths, 24 directions)."""
    nx, ny, nz, nit = 20, 20, 32, 8
    atm, f, (x, y, z, dx, dy), data = _setup(nx, ny, nz)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    ref, it, hist = orc_lambda_iterate(OrcRegular(nx, ny, nz, dx, dy, z, dirs, w), A, f["T"],
                                       f["rho"], f["ne"], f["nH"], max_iter=nit, tol=0.0)
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    its, ghist, conv = rt.lambda_iterate(g, ga, gm, pops, max_iter=nit, tol=0.0,
                                         use_graph=use_graph)
    assert its == nit and not conv
    assert_parity(pops.cpu().numpy(), ref, rel=1e-4, floor=0.0, what="pops after 8 iterations")
    np.testing.assert_allclose(ghist, hist, rtol=2e-2)


def test_lambda_iteration_voronoi(rt):
    from helpers import voronoi_grid
    atm, vg, f = voronoi_grid(3000, "rho03", 3)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    ref, it, hist = orc_lambda_iterate(OrcVoronoi(vg, dirs, w), A, f["T"], f["rho"], f["ne"],
                                       f["nH"], max_iter=5, tol=0.0)
    g = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"], dirs,
                       w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    rt.lambda_iterate(g, ga, gm, pops, max_iter=5, tol=0.0)
    assert_parity(pops.cpu().numpy(), ref, rel=1e-4, floor=0.0, what="Voronoi pops")


def test_lambda_iteration_converges(rt):
    """Run to the paper's tolerance (max relative change 1e-3) on a 16 x 16 x 32 grid."""
    nx, ny, nz = 16, 16, 32
    atm, f, (x, y, z, dx, dy), data = _setup(nx, ny, nz)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    its, hist, conv = rt.lambda_iterate(g, ga, gm, pops, max_iter=300, tol=1e-3)
    assert conv and hist[-1] < 1e-3 and its < 300
    n = pops.cpu().double().numpy()
    np.testing.assert_allclose(n.sum(0), f["nH"], rtol=1e-5)


def test_one_iteration_at_the_benchmark_size(rt):
    """One Lambda iteration from LTE populations on the benchmark's 128^3 grid with the atom's 52
    wavelengths and 24 directions (source terms, formal solution, rates, statistical
    equilibrium): the GPU's populations against the oracle's at every point."""
    from oracle.physics import Atom
    n = 128
    atm, f, (x, y, z, dx, dy), data = _setup(n, n, n)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    f32 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in f.items()}
    pops0 = A.lte_pops(f32["T"], f32["ne"], f32["nH"])
    alpha, S = A.alpha_S(f32["T"], f32["rho"], f32["ne"], pops0)
    J = OrcRegular(n, n, n, dx, dy, z, dirs, w).formal_solution(alpha, S)
    del alpha, S
    ref = A.statistical_equilibrium(A.rate_matrix(f32["T"], f32["ne"], J), f32["nH"])
    del J
    g = rt.RegularGrid(n, n, n, dx, dy, z, dirs, w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    its, hist, conv = rt.lambda_iterate(g, ga, gm, pops, max_iter=1, tol=0.0)
    assert its == 1
    assert_parity(pops.cpu().numpy(), ref, rel=1e-4, floor=0.0, what="128^3 iteration pops")

"""GPU parity of the accelerated Lambda iteration against the FP64 oracle, through the C ABI:
Lambda* (the diagonal of the Lambda operator) on both grids, one accelerated statistical-
equilibrium update, and the iteration's fixed point (that of the Lambda iteration) reached in
fewer iterations."""
import functools

import numpy as np
import pytest

from helpers import assert_parity, to_gpu, voronoi_grid
from oracle.ali import _local_update, ali_iterate
from oracle.physics import Atom
from oracle.solve import RegularGrid as OrcRegular
from oracle.solve import VoronoiGrid as OrcVoronoi
from oracle.solve import lambda_iterate as orc_lambda_iterate
from synth import delaunay_neighbours, make_atmosphere, model_atom, s4_quadrature
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
def _setup(nx, ny, nz):
    atm = make_atmosphere(0)
    f, ax = regular_fields(nx, ny, nz, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    return atm, f, ax, data


def _gpu_atm(rt, f):
    return rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))


@pytest.mark.parametrize("periodic,bc", [(True, 0), (False, 0), (True, 1)])
def test_lambda_star_regular(rt, periodic, bc):
    rng = np.random.default_rng(11)
    nx, ny, nz, nlam = 37, 23, 17, 3
    z = np.cumsum(np.r_[0.0, 0.3 + rng.random(nz - 1)])
    dirs, w = s4_quadrature()
    a = 10.0 ** rng.uniform(-4, 2, (nlam, nx * ny * nz))
    ref = OrcRegular(nx, ny, nz, 0.7, 0.9, z, dirs, w, periodic=periodic).lambda_star(a, bc=bc)
    g = rt.RegularGrid(nx, ny, nz, 0.7, 0.9, z, dirs, w, periodic=periodic)
    got = rt.lambda_star(g, to_gpu(a), bc=bc)
    assert_parity(got.cpu().numpy(), ref, what="Lambda* regular")


@pytest.mark.parametrize("bc", [0, 1])
def test_lambda_star_voronoi(rt, bc):
    rng = np.random.default_rng(12)
    n, nlam = 900, 4
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((n, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    gd = dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)
    dirs, w = s4_quadrature()
    a = 10.0 ** rng.uniform(-3, 2, (nlam, n))
    ref = OrcVoronoi(gd, dirs, w).lambda_star(a, bc=bc)
    g = rt.VoronoiGrid(xyz, off, code, shift, box, dirs, w)
    got = rt.lambda_star(g, to_gpu(a), bc=bc)
    assert_parity(got.cpu().numpy(), ref, what="Lambda* Voronoi")


def test_accelerated_update_matches_oracle(rt):
    """One accelerated update from LTE populations (the most nonlinear one), with the oracle's
    J, Lambda* and S_old as inputs; both sides run 6 Newton steps."""
    nx, ny, nz = 12, 10, 24
    atm, f, (x, y, z, dx, dy), data = _setup(nx, ny, nz)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    og = OrcRegular(nx, ny, nz, dx, dy, z, dirs, w)
    T, rho, ne, nH = f["T"], f["rho"], f["ne"], f["nH"]
    pops = A.lte_pops(T, ne, nH)
    alpha, S = A.alpha_S(T, rho, ne, pops)
    J = og.formal_solution(alpha, S)
    L = og.lambda_star(alpha)
    ref = _local_update(A, T, rho, ne, nH, pops, J, L, S, newton=6)
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    p = to_gpu(pops)
    rt.statistical_equilibrium_ali(g, rt.Atom(data, atm.kappa0), _gpu_atm(rt, f), to_gpu(J),
                                   to_gpu(L), to_gpu(S), p, newton=6)
    assert_parity(p.cpu().numpy(), ref, rel=1e-3, floor=0.0, what="accelerated update")
    # no Newton step: the plain update of rt_statistical_equilibrium
    p0 = to_gpu(pops)
    rt.statistical_equilibrium_ali(g, rt.Atom(data, atm.kappa0), _gpu_atm(rt, f), to_gpu(J),
                                   to_gpu(L), to_gpu(S), p0, newton=0)
    p1 = to_gpu(pops)
    rt.statistical_equilibrium(g, rt.Atom(data, atm.kappa0), _gpu_atm(rt, f), to_gpu(J), p1)
    # the accelerated kernel forms J from J_eff + Lambda* S(n) with S(n) from linear opacity
    # coefficients: equal to J up to FP32 rounding
    assert_parity(p0.cpu().numpy(), p1.cpu().numpy().astype(np.float64), rel=2e-5, floor=0.0,
                  what="newton=0 vs plain")


@pytest.mark.parametrize("use_graph", [False, True])
def test_accelerated_iteration_regular(rt, use_graph):
    """Three accelerated iterations on 20 x 20 x 32 against the oracle's, then convergence to the
    Lambda iteration's fixed point in fewer iterations than the Lambda iteration on the GPU."""
    nx, ny, nz = 20, 20, 32
    atm, f, (x, y, z, dx, dy), data = _setup(nx, ny, nz)
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    og = OrcRegular(nx, ny, nz, dx, dy, z, dirs, w)
    args = (og, A, f["T"], f["rho"], f["ne"], f["nH"])
    ref3, _, _ = ali_iterate(*args, max_iter=3, tol=0.0, newton=3)
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pops = rt.lte_populations(g, ga, gm)
    its, hist, conv = rt.lambda_iterate_ali(g, ga, gm, pops, max_iter=3, tol=0.0, newton=3,
                                            fixed_lstar=False, use_graph=use_graph)
    assert its == 3
    assert_parity(pops.cpu().numpy(), ref3, rel=2e-3, floor=0.0, what="3 accelerated iterations")
    fixed, _, _ = orc_lambda_iterate(*args, max_iter=300, tol=1e-7)
    pa = rt.lte_populations(g, ga, gm)
    it_a, _, conv_a = rt.lambda_iterate_ali(g, ga, gm, pa, max_iter=300, tol=1e-4,
                                            use_graph=use_graph)
    pl = rt.lte_populations(g, ga, gm)
    it_l, _, conv_l = rt.lambda_iterate(g, ga, gm, pl, max_iter=300, tol=1e-4)
    assert conv_a and conv_l and it_a < it_l, (it_a, it_l)
    assert_parity(pa.cpu().numpy(), fixed, rel=2e-3, floor=0.0, what="accelerated fixed point")


def test_accelerated_iteration_voronoi(rt):
    atm, vg, f = voronoi_grid(3000, "rho03", 3)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    fixed, _, _ = orc_lambda_iterate(OrcVoronoi(vg, dirs, w), A, f["T"], f["rho"], f["ne"],
                                     f["nH"], max_iter=300, tol=1e-7)
    g = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"], dirs,
                       w)
    ga, gm = rt.Atom(data, atm.kappa0), _gpu_atm(rt, f)
    pa = rt.lte_populations(g, ga, gm)
    it_a, _, conv_a = rt.lambda_iterate_ali(g, ga, gm, pa, max_iter=300, tol=1e-4)
    pl = rt.lte_populations(g, ga, gm)
    it_l, _, conv_l = rt.lambda_iterate(g, ga, gm, pl, max_iter=300, tol=1e-4)
    assert conv_a and conv_l and it_a < it_l, (it_a, it_l)
    assert_parity(pa.cpu().numpy(), fixed, rel=2e-3, floor=0.0, what="Voronoi fixed point")

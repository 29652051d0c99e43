"""GPU adjoint of the emergent intensity (Eq. 2 differentiated): against the FP64 oracle's own
adjoint, against central finite differences of the GPU forward pass, across checkpoint strides,
through the torch.autograd.Function, and the temperature chain rule."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, lte_regular, to_gpu
from synth import delaunay_neighbours, s4_quadrature

pytestmark = pytest.mark.gpu
MU1 = (0.0, 0.0, 1.0)
OBLIQUE = (0.3500212, -0.3500212, 0.8688903)


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def f32(x):
    """The FP32 values the GPU receives, for the oracle to receive the same inputs."""
    return np.asarray(x, np.float32).astype(np.float64)


def _reg_problem(seed=0):
    rng = np.random.default_rng(seed)
    nx, ny, nz, nlam = 21, 17, 24, 3
    z = np.cumsum(np.r_[0.0, 0.5 + rng.random(nz - 1)]) * 0.05
    npt = nx * ny * nz
    a = f32(10.0 ** rng.uniform(-1, 1.5, (nlam, npt)))
    s = f32(rng.uniform(0.5, 2.0, (nlam, npt)))
    g = f32(rng.standard_normal((nlam, nx * ny)))
    return nx, ny, nz, z, a, s, g


@pytest.mark.parametrize("mu", [MU1, OBLIQUE])
@pytest.mark.parametrize("bc", [0, 1])
def test_regular_adjoint_vs_oracle(rt, mu, bc):
    nx, ny, nz, z, a, s, gtop = _reg_problem()
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(nx, ny, nz, 0.11, 0.13, z, dirs, w)
    I_top = rt.emergent_intensity(G, mu, to_gpu(a), to_gpu(s), bc=bc)
    _, Ir = oracle.sc_regular(nx, ny, nz, 0.11, 0.13, z, np.array([mu]), np.ones(1), a, s, bc=bc,
                              want_I=True)
    assert_parity(I_top.cpu().numpy(), Ir[0].reshape(3, nz, -1)[:, -1], what="I_top")
    ga, gs = rt.formal_solution_adjoint(G, mu, to_gpu(a), to_gpu(s), to_gpu(gtop), bc=bc,
                                        ckpt_stride=5)
    gI = np.zeros((3, nx * ny * nz))
    gI[:, -nx * ny:] = gtop
    gar, gsr = oracle.sc_regular_adjoint(nx, ny, nz, 0.11, 0.13, z, np.array(mu), a, s, gI, bc=bc)
    assert_parity(ga.cpu().numpy(), gar, rel=1e-4, floor=1e-6, what="g_alpha")
    assert_parity(gs.cpu().numpy(), gsr, rel=1e-4, floor=1e-6, what="g_S")


def test_checkpoint_strides_identical(rt):
    nx, ny, nz, z, a, s, gtop = _reg_problem(1)
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(nx, ny, nz, 0.11, 0.13, z, dirs, w)
    outs = [rt.formal_solution_adjoint(G, OBLIQUE, to_gpu(a), to_gpu(s), to_gpu(gtop),
                                       ckpt_stride=k) for k in (1, 4, 5, 23, 24)]
    for ga, gs in outs[1:]:
        assert np.array_equal(ga.cpu().numpy(), outs[0][0].cpu().numpy())
        assert np.array_equal(gs.cpu().numpy(), outs[0][1].cpu().numpy())


def test_regular_adjoint_vs_finite_differences(rt):
    """64 random points: the GPU adjoint against central differences (relative step 1e-6) of
    the FP64 forward model of the same discretisation."""
    nx, ny, nz, z, a, s, gtop = _reg_problem(2)
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(nx, ny, nz, 0.11, 0.13, z, dirs, w)
    ga, gs = rt.formal_solution_adjoint(G, OBLIQUE, to_gpu(a), to_gpu(s), to_gpu(gtop))
    ga, gs = ga.cpu().double().numpy(), gs.cpu().double().numpy()
    mu = np.array([OBLIQUE])

    def loss(aa, ss):
        _, I = oracle.sc_regular(nx, ny, nz, 0.11, 0.13, z, mu, np.ones(1), aa, ss, want_I=True)
        return float((I[0].reshape(3, nz, -1)[:, -1] * gtop).sum())
    rng = np.random.default_rng(3)
    scale = max(np.abs(ga).max(), np.abs(gs).max())
    for _ in range(64):
        l = int(rng.integers(3))
        p = int(rng.integers(nx * ny * nz))
        for which in (0, 1):
            base = a if which == 0 else s
            h = 1e-6 * base[l, p]
            bp, bm = base.copy(), base.copy()
            bp[l, p] += h
            bm[l, p] -= h
            fd = ((loss(bp, s) - loss(bm, s)) if which == 0 else
                  (loss(a, bp) - loss(a, bm))) / (2 * h)
            adj = (ga if which == 0 else gs)[l, p]
            assert abs(adj - fd) <= 1e-3 * max(abs(fd), 1e-3 * scale), (which, l, p, adj, fd)


def test_autograd_function(rt):
    import torch
    nx, ny, nz, z, a, s, gtop = _reg_problem(4)
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(nx, ny, nz, 0.11, 0.13, z, dirs, w)
    A = to_gpu(a).requires_grad_(True)
    S = to_gpu(s).requires_grad_(True)
    I = rt.EmergentIntensity.apply(A, S, G, MU1, 0, 3)
    (I * to_gpu(gtop)).sum().backward()
    ga, gs = rt.formal_solution_adjoint(G, MU1, to_gpu(a), to_gpu(s), to_gpu(gtop), ckpt_stride=3)
    assert torch.equal(A.grad, ga) and torch.equal(S.grad, gs)


def test_lte_temperature_chain_rule(rt):
    from oracle.physics import dplanck_dT
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(16, 16, 32)
    T, rho = to_gpu(f["T"]), to_gpu(f["rho"])
    rng = np.random.default_rng(6)
    gA, gS = rng.standard_normal(f["T"].size), rng.standard_normal(f["T"].size)
    gT = rt.source_terms_lte_adjoint(T, rho, atm.kappa0, 500e-9, to_gpu(gA), to_gpu(gS))
    ref = gA * 9.0 * a / f["T"] + gS * dplanck_dT(f["T"], 500e-9)
    scale = np.abs(gA * 9.0 * a / f["T"]) + np.abs(gS * dplanck_dT(f["T"], 500e-9))
    err = np.abs(gT.cpu().double().numpy() - ref) / scale
    assert err.max() < 1e-5


def test_nlte_temperature_chain_rule(rt):
    """dalpha/dT, dS/dT of the atom (dual numbers on the GPU) against central differences of the
    oracle's FP64 source terms, at the line core and both continua."""
    from oracle.physics import Atom
    from synth import make_atmosphere, model_atom
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(8, 8, 16, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(8, 8, 16, dx, dy, z, dirs, w)
    rng = np.random.default_rng(7)
    nl = len(data["lam"])
    gA = np.zeros((nl, f["T"].size))
    gS = np.zeros_like(gA)
    for j in (24, 50, 51):
        gA[j] = rng.standard_normal(f["T"].size)
        gS[j] = rng.standard_normal(f["T"].size)
    ga_ = rt.Atom(data, atm.kappa0)
    gm = rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))
    gT = rt.source_terms_adjoint(G, ga_, gm, to_gpu(pops), to_gpu(gA), to_gpu(gS))
    h = 1e-3 * f["T"]
    ap, sp = A.alpha_S(f["T"] + h, f["rho"], f["ne"], pops)
    am, sm = A.alpha_S(f["T"] - h, f["rho"], f["ne"], pops)
    da, ds = (ap - am) / (2 * h), (sp - sm) / (2 * h)
    ref = (gA * da + gS * ds).sum(0)
    scale = (np.abs(gA * da) + np.abs(gS * ds)).sum(0)
    err = np.abs(gT.cpu().double().numpy() - ref) / scale
    assert err.max() < 1e-3


def test_voronoi_adjoint_vs_oracle(rt):
    rng = np.random.default_rng(8)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((600, 3))
    off, code, shift = delaunay_neighbours(xyz, box)
    dirs, w = s4_quadrature()
    G = rt.VoronoiGrid(xyz, off, code, shift, box, dirs, w)
    top = G.top_points()
    n, nlam = 600, 3
    a = f32(10.0 ** rng.uniform(-0.5, 1.5, (nlam, n)))
    s = f32(rng.uniform(0.5, 2.0, (nlam, n)))
    gtop = f32(rng.standard_normal((nlam, len(top))))
    tab = oracle.voronoi_tables(xyz, off, code, shift, box, np.array([MU1]), 7.0)
    _, Ir = oracle.voronoi_fs(tab, np.array([MU1]), np.ones(1), a, s, want_I=True)
    I_top = rt.emergent_intensity(G, MU1, to_gpu(a), to_gpu(s))
    assert_parity(I_top.cpu().numpy(), Ir[0][:, top], what="Voronoi I_top")
    ga, gs = rt.formal_solution_adjoint(G, MU1, to_gpu(a), to_gpu(s), to_gpu(gtop))
    gI = np.zeros((nlam, n))
    gI[:, top] = gtop
    gar, gsr = oracle.voronoi_adjoint(tab, 0, True, a, s, gI)
    assert_parity(ga.cpu().numpy(), gar, rel=1e-4, floor=1e-6, what="Voronoi g_alpha")
    assert_parity(gs.cpu().numpy(), gsr, rel=1e-4, floor=1e-6, what="Voronoi g_S")

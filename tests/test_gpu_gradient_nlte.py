"""Gradient of the vertical (mu = 1) emergent intensity at the line core and the two continuum
wavelengths with respect to T, alpha and S at every point, with the populations held at their
converged NLTE values (Eq. 2 differentiated, through the atom's opacities and source functions
of Sect. 2.2): the GPU's torch.autograd composition SourceTerms -> EmergentIntensity against the
FP64 oracle's adjoint and against central differences of the oracle's whole forward model."""
import functools

import numpy as np
import pytest

import oracle
from helpers import assert_parity, to_gpu
from synth import make_atmosphere, model_atom, s4_quadrature
from synth.atmosphere import regular_fields

pytestmark = pytest.mark.gpu
MU1 = (0.0, 0.0, 1.0)


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _pick(data):
    lam = np.asarray(data["lam"])
    return [int(np.argmin(np.abs(lam - data["lam0"]))), len(lam) - 2, len(lam) - 1]


@functools.lru_cache(maxsize=None)
def _regular_case():
    """12 x 10 x 24 points of the synthetic atmosphere; populations converged by the oracle's
    Lambda iteration (max relative change < 1e-4)."""
    from oracle.physics import Atom
    from oracle.solve import RegularGrid, lambda_iterate
    nx, ny, nz = 12, 10, 24
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    f = {k: f32(v) for k, v in f.items()}
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    pops, it, hist = lambda_iterate(RegularGrid(nx, ny, nz, dx, dy, z, dirs, w), A, f["T"],
                                    f["rho"], f["ne"], f["nH"], max_iter=300, tol=1e-4)
    assert hist[-1] < 1e-4
    return dict(kind="regular", shape=(nx, ny, nz), dx=dx, dy=dy, z=z, f=f, data=data, A=A,
                kappa0=atm.kappa0, pops=f32(pops))


@functools.lru_cache(maxsize=None)
def _voronoi_case():
    """3000 sites (rho^0.3) of the synthetic atmosphere; populations converged by the oracle."""
    from helpers import voronoi_grid
    from oracle.physics import Atom
    from oracle.solve import VoronoiGrid, lambda_iterate
    atm, vg, f = voronoi_grid(3000, "rho03", 3)
    f = {k: f32(v) for k, v in f.items()}
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    dirs, w = s4_quadrature()
    pops, it, hist = lambda_iterate(VoronoiGrid(vg, dirs, w), A, f["T"], f["rho"], f["ne"],
                                    f["nH"], max_iter=300, tol=1e-4)
    assert hist[-1] < 1e-4
    tab = oracle.voronoi_tables(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"],
                                vg["box"], np.array([MU1]), 7.0)
    return dict(kind="voronoi", vg=vg, tab=tab, f=f, data=data, A=A, kappa0=atm.kappa0,
                pops=f32(pops))


def _oracle_top(case, a3, s3):
    """The oracle's mu = 1 intensity at the emergent layer [3][ntop] (and the layer's points)."""
    if case["kind"] == "regular":
        nx, ny, nz = case["shape"]
        from oracle.synthesis import emergent_mu1
        return emergent_mu1(nx, ny, nz, case["dx"], case["dy"], case["z"], a3, s3), \
            np.arange((nz - 1) * nx * ny, nz * nx * ny)
    from oracle.synthesis import top_sites
    top = top_sites(case["vg"]["nbr_off"], case["vg"]["nbr_idx"])
    _, I = oracle.voronoi_fs(case["tab"], np.array([MU1]), np.ones(1), a3, s3, want_I=True)
    return I[0][:, top], top


def _oracle_adjoint(case, a3, s3, gI_full):
    if case["kind"] == "regular":
        nx, ny, nz = case["shape"]
        return oracle.sc_regular_adjoint(nx, ny, nz, case["dx"], case["dy"], case["z"],
                                         np.array(MU1), a3, s3, gI_full)
    return oracle.voronoi_adjoint(case["tab"], 0, True, a3, s3, gI_full)


def _gpu_grid(rt, case):
    dirs, w = s4_quadrature()
    if case["kind"] == "regular":
        nx, ny, nz = case["shape"]
        return rt.RegularGrid(nx, ny, nz, case["dx"], case["dy"], case["z"], dirs, w)
    vg = case["vg"]
    return rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"],
                          dirs, w)


@pytest.mark.parametrize("case_fn", [_regular_case, _voronoi_case])
def test_temperature_gradient_at_converged_populations(rt, case_fn):
    import torch
    case = case_fn()
    f, A, data, pops = case["f"], case["A"], case["data"], case["pops"]
    pick = _pick(data)
    G = _gpu_grid(rt, case)
    ga = rt.Atom(data, case["kappa0"])
    gm = rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))
    rng = np.random.default_rng(3)
    gI = rng.standard_normal((3, G.ntop))
    # GPU: T -> (alpha, S) -> mu = 1 map -> L = sum(gI * I), reverse mode through both Functions
    T = to_gpu(f["T"]).requires_grad_(True)
    alpha, S = rt.SourceTerms.apply(T, G, ga, gm, to_gpu(pops))
    alpha.retain_grad()
    S.retain_grad()
    I = rt.EmergentIntensity.apply(alpha[pick].contiguous(), S[pick].contiguous(), G, MU1)
    (I * to_gpu(gI)).sum().backward()
    gT = T.grad.cpu().double().numpy()
    # oracle: the adjoint sweep of the three wavelengths, then the exact chain to T
    a, s = A.alpha_S(f["T"], f["rho"], f["ne"], pops)
    a3, s3 = a[pick], s[pick]
    I_ref, top = _oracle_top(case, a3, s3)
    assert_parity(I.detach().cpu().numpy(), I_ref, what="mu = 1 map")
    gI_full = np.zeros_like(a3)
    gI_full[:, top] = gI
    g_a3, g_s3 = _oracle_adjoint(case, a3, s3, gI_full)
    assert_parity(alpha.grad[pick].cpu().numpy(), g_a3, rel=1e-4, floor=1e-6, what="dL/dalpha")
    assert_parity(S.grad[pick].cpu().numpy(), g_s3, rel=1e-4, floor=1e-6, what="dL/dS")
    h = 1e-5 * f["T"]
    ap, sp = A.alpha_S(f["T"] + h, f["rho"], f["ne"], pops)
    am, sm = A.alpha_S(f["T"] - h, f["rho"], f["ne"], pops)
    da, ds = (ap[pick] - am[pick]) / (2 * h), (sp[pick] - sm[pick]) / (2 * h)
    ref = (g_a3 * da + g_s3 * ds).sum(0)
    scale = (np.abs(g_a3 * da) + np.abs(g_s3 * ds)).sum(0)
    scale = np.maximum(scale, 1e-6 * scale.max())
    err = np.abs(gT - ref) / scale
    assert err.max() < 1e-4, err.max()

    # central differences of the oracle's whole forward model at 64 random points
    def loss(Tv):
        aa, ss = A.alpha_S(Tv, f["rho"], f["ne"], pops)
        return float((gI * _oracle_top(case, aa[pick], ss[pick])[0]).sum())
    pts = rng.choice(f["T"].size, 64, replace=False)
    for p in pts:
        hp = 1e-4 * f["T"][p]
        Tp, Tm = f["T"].copy(), f["T"].copy()
        Tp[p] += hp
        Tm[p] -= hp
        fd = (loss(Tp) - loss(Tm)) / (2 * hp)
        assert abs(gT[p] - fd) <= 1e-3 * max(scale[p], 1e-3 * np.abs(gT).max()), (p, gT[p], fd)


def _atom_fields_3(A, f, pops, pick, chunk=1 << 17):
    """alpha, S of the atom at the three wavelengths, evaluated in slices of points."""
    n = f["T"].size
    a3 = np.empty((3, n))
    s3 = np.empty((3, n))
    for q in range(0, n, chunk):
        sl = slice(q, q + chunk)
        a, s = A.alpha_S(f["T"][sl], f["rho"][sl], f["ne"][sl], pops[:, sl])
        a3[:, sl], s3[:, sl] = a[pick], s[pick]
    return f32(a3), f32(s3)


@pytest.mark.parametrize("kind", ["regular_128", "voronoi_200k"])
def test_adjoint_full_size_matches_oracle(rt, kind):
    """The adjoint sweeps at the workload sizes: 128^3 points, and the 200 000-site grid sampled
    from |dtau/dz|; the atom's line core and continua at LTE populations, a random weighting of
    the mu = 1 map: dL/dalpha and dL/dS at every point against the oracle's adjoint."""
    from oracle.physics import Atom
    dirs, w = s4_quadrature()
    atm = make_atmosphere(0)
    if kind == "regular_128":
        n = 128
        f, (x, y, z, dx, dy) = regular_fields(n, n, n, atm)
        G = rt.RegularGrid(n, n, n, dx, dy, z, dirs, w)
    else:
        from helpers import voronoi_grid
        atm, vg, f = voronoi_grid(200000, "dtau", 9)
        G = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"],
                           dirs, w)
    f = {k: f32(v) for k, v in f.items()}
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    a3, s3 = _atom_fields_3(A, f, pops, _pick(data))
    top = G.top_points()
    gI = f32(np.random.default_rng(5).standard_normal((3, len(top))))
    ga, gs = rt.formal_solution_adjoint(G, MU1, to_gpu(a3), to_gpu(s3), to_gpu(gI))
    gI_full = np.zeros_like(a3)
    gI_full[:, top] = gI
    if kind == "regular_128":
        ra, rs = oracle.sc_regular_adjoint(n, n, n, dx, dy, z, np.array(MU1), a3, s3, gI_full)
    else:
        tab = oracle.voronoi_tables(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"],
                                    vg["box"], np.array([MU1]), 7.0)
        ra, rs = oracle.voronoi_adjoint(tab, 0, True, a3, s3, gI_full)
    assert_parity(ga.cpu().numpy(), ra, rel=1e-4, floor=1e-6, what=f"{kind} dL/dalpha")
    assert_parity(gs.cpu().numpy(), rs, rel=1e-4, floor=1e-6, what=f"{kind} dL/dS")

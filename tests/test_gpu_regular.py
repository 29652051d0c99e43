"""GPU parity of the regular-grid formal solution (plane-to-plane short characteristics, Sect. 2.6;
linear S, Eq. 2; J, Eq. 4) against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from helpers import assert_parity, lte_regular, to_gpu
from synth import s4_quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def test_lte_continuum_32x32x64(rt):
    """The 32 x 32 x 64 LTE continuum workload (500 nm, 24 directions)."""
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(32, 32, 64)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(32, 32, 64, dx, dy, z, dirs, w)
    alpha, S = rt.source_terms_lte(to_gpu(f["T"]), to_gpu(f["rho"]), atm.kappa0, 500e-9)
    assert_parity(alpha.cpu().numpy(), a, rel=2e-6, what="alpha")
    assert_parity(S.cpu().numpy(), s, rel=2e-6, what="S")
    J, I = rt.formal_solution(g, alpha[None], S[None], want_I=True)
    Jr, Ir = oracle.sc_regular(32, 32, 64, dx, dy, z, dirs, w, a[None], s[None], want_I=True)
    assert_parity(J.cpu().numpy(), Jr, what="J")
    assert_parity(I.cpu().numpy(), Ir, what="I")


@pytest.mark.parametrize("periodic,bc", [(True, 0), (True, 2), (False, 1), (False, 2)])
def test_ragged_random_multi_lambda(rt, periodic, bc):
    """Ragged plane (37 x 23 points, not a multiple of the block), non-uniform z, 3 wavelengths,
    optical depths per step from 1e-6 to 1e3, every boundary condition."""
    rng = np.random.default_rng(11)
    nx, ny, nz, nlam = 37, 23, 19, 3
    z = np.cumsum(np.r_[0.0, 0.3 + rng.random(nz - 1)])
    dirs, w = s4_quadrature()
    npt = nx * ny * nz
    a = 10.0 ** rng.uniform(-6, 3, (nlam, npt))
    s = rng.uniform(0.5, 2.0, (nlam, npt))
    ibc = rng.uniform(0.0, 3.0, (24, nlam, nx * ny)) if bc == 2 else None
    g = rt.RegularGrid(nx, ny, nz, 0.7, 0.9, z, dirs, w, periodic=periodic)
    J, I = rt.formal_solution(g, to_gpu(a), to_gpu(s), bc=bc,
                              I_bc=to_gpu(ibc) if ibc is not None else None, want_I=True)
    Jr, Ir = oracle.sc_regular(nx, ny, nz, 0.7, 0.9, z, dirs, w, a, s, bc=bc, ibc=ibc,
                               periodic=periodic, want_I=True)
    assert_parity(J.cpu().numpy(), Jr, what="J")
    assert_parity(I.cpu().numpy(), Ir, what="I")


def test_constant_source_closed_form(rt):
    """Constant alpha and S on the GPU: I = I0 exp(-tau) + S (1 - exp(-tau)) along every ray."""
    nx, ny, nz = 8, 8, 40
    z = np.linspace(0.0, 4.0, nz)
    dirs, w = s4_quadrature()
    a0, s0, i0 = 1.3, 2.0, 0.5
    al = np.full((1, nx * ny * nz), a0)
    S = np.full((1, nx * ny * nz), s0)
    ibc = np.full((24, 1, nx * ny), i0)
    g = rt.RegularGrid(nx, ny, nz, 0.2, 0.2, z, dirs, w)
    _, I = rt.formal_solution(g, to_gpu(al), to_gpu(S), bc=2, I_bc=to_gpu(ibc), want_I=True)
    I = I.cpu().numpy()
    for d, mu in enumerate(dirs):
        path = (z - (z[0] if mu[2] > 0 else z[-1])) / mu[2]
        ex = i0 * np.exp(-a0 * path) + s0 * (1 - np.exp(-a0 * path))
        np.testing.assert_allclose(I[d, 0].reshape(nz, -1), np.repeat(ex[:, None], nx * ny, 1),
                                   rtol=2e-6)


def test_searchlight_flux_and_peak(rt):
    """Searchlight beam (Sect. 3.1): 51^3, alpha = S = 0, radius 0.2, theta = 20 deg.  Periodic
    sides conserve the beam's flux; the peak is reported against the oracle."""
    n = 51
    h = 1.0 / (n - 1)
    z = np.arange(n) * h
    th = math.radians(20.0)
    mu = np.array([[math.sin(th), 0.0, math.cos(th)]])
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="xy")
    beam = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 <= 0.04).astype(float).ravel()
    zero = np.zeros((1, n ** 3))
    for periodic in (True, False):
        g = rt.RegularGrid(n, n, n, h, h, z, mu, np.ones(1), periodic=periodic)
        _, I = rt.formal_solution(g, to_gpu(zero), to_gpu(zero), bc=2,
                                  I_bc=to_gpu(beam[None, None]), want_I=True)
        top = I[0, 0].reshape(n, -1)[-1].cpu().double().numpy()
        _, Ir = oracle.sc_regular(n, n, n, h, h, z, mu, np.ones(1), zero, zero, bc=2,
                                  ibc=beam[None, None], periodic=periodic, want_I=True)
        assert_parity(top, Ir[0, 0].reshape(n, -1)[-1], rel=1e-5, what="searchlight top")
        if periodic:
            assert top.sum() == pytest.approx(beam.sum(), rel=1e-5)


@pytest.mark.slow
def test_full_size_128cubed_sampled_wavelengths(rt):
    """The 128^3 x 24-direction sweep in the launch configuration of the benchmark, compared
    with the oracle on three sampled wavelengths (line core, line wing, Lyman continuum) of the
    NLTE atom's LTE start."""
    from oracle.physics import Atom
    from synth import model_atom
    from synth.atmosphere import regular_fields
    from synth import make_atmosphere
    atm = make_atmosphere(0)
    nx = ny = nz = 128
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    A = Atom(data, atm.kappa0)
    pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    alpha, S = A.alpha_S(f["T"], f["rho"], f["ne"], pops)
    pick = [24, 10, 50]
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    J = rt.formal_solution(g, to_gpu(alpha[pick]), to_gpu(S[pick]))
    Jr = oracle.sc_regular(nx, ny, nz, dx, dy, z, dirs, w, alpha[pick], S[pick])
    assert_parity(J.cpu().numpy(), Jr, what="J 128^3")


@pytest.mark.parametrize("shape,nlam,zkind", [((64, 64, 40), 4, "rough"), ((32, 48, 17), 3, "rough"),
                                              ((128, 128, 24), 2, "rough"), ((40, 24, 9), 2, "rough"),
                                              ((64, 64, 40), 4, "uniform"), ((36, 48, 17), 3, "uniform"),
                                              ((16, 16, 5), 2, "uniform"), ((96, 40, 33), 5, "uniform"),
                                              ((64, 64, 40), 4, "stretched"),
                                              ((36, 40, 19), 3, "stretched"),
                                              ((128, 64, 33), 3, "stretched"),
                                              ((64, 96, 20), 2, "uniform"),
                                              ((32, 32, 10), 2, "uniform"),
                                              ((64, 65, 12), 2, "uniform"),
                                              ((64, 67, 12), 2, "uniform")])
def test_sweep_variants_match_each_other_and_oracle(rt, monkeypatch, shape, nlam, zkind):
    """The regular-grid sweeps -- the persistent wavefront kernel (default wherever the staged
    tile covers every stencil; constant-bank stencils on uniform z, per-plane stencil tables on
    stretched z; a thread's two points as packed FP32 pairs), shared-memory tiles per plane, and
    the plain per-plane kernel -- compute the same updates: each matches the oracle and the
    others (up to FMA contraction).  "rough" z steps reach beyond the tile halo, where the default falls
    back to the plain kernel.  The uniform steps reach 3 rows: 32 x 32 is a single tile column
    whose ring halo copies wrap onto the tile itself; with 65 rows the last of five tile rows is
    shorter than the reach, so the warp-specialised sweep gives way to the other persistent one,
    and with 67 rows it is not."""
    import torch
    nx, ny, nz = shape
    rng = np.random.default_rng(21)
    if zkind == "uniform":
        z = np.arange(nz) * 0.8
    elif zkind == "stretched":
        z = np.cumsum(np.r_[0.0, 0.3 + 0.3 * rng.random(nz - 1)])
    else:
        z = np.cumsum(np.r_[0.0, 0.3 + rng.random(nz - 1)])
    dirs, w = s4_quadrature()
    npt = nx * ny * nz
    a = 10.0 ** rng.uniform(-5, 2, (nlam, npt))
    s = rng.uniform(0.5, 2.0, (nlam, npt))
    g = rt.RegularGrid(nx, ny, nz, 0.7, 0.9, z, dirs, w)
    Jr = oracle.sc_regular(nx, ny, nz, 0.7, 0.9, z, dirs, w, a, s)
    out = {}
    for mode in ("default", "tile", "plane"):
        if mode == "default":
            monkeypatch.delenv("RT_REGULAR_SWEEP", raising=False)
        else:
            monkeypatch.setenv("RT_REGULAR_SWEEP", mode)
        ag, sg = to_gpu(a), to_gpu(s)
        n0 = rt.kernel_launches()
        J = rt.formal_solution(g, ag, sg)
        launched = rt.kernel_launches() - n0
        torch.cuda.synchronize()
        if mode == "default" and zkind != "rough":
            assert launched == 1, launched   # one persistent launch for both hemispheres
        out[mode] = J.cpu().numpy().astype(np.float64)
        assert_parity(out[mode], Jr, what=f"{mode} J")
    assert_parity(out["default"], out["plane"], rel=2e-6, what="default vs plane")
    assert_parity(out["tile"], out["plane"], rel=2e-6, what="tile vs plane")

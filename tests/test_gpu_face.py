"""GPU parity of the face-hitting short characteristics (Kunasz & Auer, the regular-grid scheme
Sect. 2.6 names; linear S, Eq. 2; J, Eq. 4) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, lte_regular, to_gpu
from oracle.physics import Atom
from oracle.solve import RegularGrid as OrcRegular
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


def _vertical_face_steps(z, dirs, dx, dy):
    dz = np.diff(z)
    n = 0
    for mu in dirs:
        t = min(dx / abs(mu[0]) if mu[0] else np.inf, dy / abs(mu[1]) if mu[1] else np.inf)
        n += int(np.sum(dz / abs(mu[2]) > t))
    return n


@pytest.mark.parametrize("jmode", ["after_sweep", "per_plane"])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_ragged_random_multi_lambda(rt, monkeypatch, bc, jmode):
    """37 x 23 points (neither a multiple of the warp), non-uniform z with both kinds of face,
    lines along x for some rays and along y for others, optical depths per step from 1e-6 to 1e3,
    three wavelengths, every boundary condition; J and every directional intensity.  J formed
    after the sweep from every plane kept (the default where memory allows) and, with a zero
    memory budget for that, per plane step by each block."""
    monkeypatch.setenv("RT_FACE_VOLUME_MB", "0" if jmode == "per_plane" else "100000")
    rng = np.random.default_rng(21)
    nx, ny, nz, nlam = 37, 23, 19, 3
    dx, dy = 0.7, 0.9
    z = np.cumsum(np.r_[0.0, 0.15 + 0.5 * rng.random(nz - 1)])
    dirs, w = s4_quadrature()
    assert 0 < _vertical_face_steps(z, dirs, dx, dy) < len(dirs) * (nz - 1)
    npt = nx * ny * nz
    a = 10.0 ** rng.uniform(-6, 3, (nlam, npt))
    s = rng.uniform(0.5, 2.0, (nlam, npt))
    ibc = rng.uniform(0.0, 3.0, (24, nlam, nx * ny)) if bc == 2 else None
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w, scheme="face")
    J, I = rt.formal_solution(g, to_gpu(a), to_gpu(s), bc=bc,
                              I_bc=to_gpu(ibc) if ibc is not None else None, want_I=True)
    Jr, Ir = oracle.sc_regular_face(nx, ny, nz, dx, dy, z, dirs, w, a, s, bc=bc, ibc=ibc,
                                    want_I=True)
    assert_parity(J.cpu().numpy(), Jr, what="J")
    assert_parity(I.cpu().numpy(), Ir, what="I")


@pytest.mark.parametrize("jmode", ["after_sweep", "per_plane"])
def test_thin_layers_close_the_periodic_cycle(rt, monkeypatch, jmode):
    """Planes far apart (f_z about 0.1): the same-plane chain runs around the box several times,
    and the walk before the first stored line is long; optically thin, so nothing damps it.  J
    after the sweep and per plane step."""
    monkeypatch.setenv("RT_FACE_VOLUME_MB", "0" if jmode == "per_plane" else "100000")
    nx, ny, nz = 20, 16, 6
    z = np.arange(nz) * 4.0
    dirs, w = s4_quadrature()
    rng = np.random.default_rng(22)
    npt = nx * ny * nz
    a = 10.0 ** rng.uniform(-5, -2, (1, npt))
    s = rng.uniform(0.5, 2.0, (1, npt))
    ibc = rng.uniform(0.0, 3.0, (24, 1, nx * ny))
    g = rt.RegularGrid(nx, ny, nz, 1.0, 1.0, z, dirs, w, scheme="face")
    J, I = rt.formal_solution(g, to_gpu(a), to_gpu(s), bc=2, I_bc=to_gpu(ibc), want_I=True)
    Jr, Ir = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, w, a, s, bc=2, ibc=ibc,
                                    want_I=True)
    assert_parity(J.cpu().numpy(), Jr, what="J")
    assert_parity(I.cpu().numpy(), Ir, what="I")


def test_scheme_switch_and_limits(rt):
    """The scheme is a property of the grid; plane to plane again after switching back; closed
    sides are refused."""
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(24, 24, 16)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(24, 24, 16, dx, dy, z, dirs, w)
    J_plane = rt.formal_solution(g, to_gpu(a[None]), to_gpu(s[None])).cpu().numpy()
    g.set_scheme("face")
    J_face = rt.formal_solution(g, to_gpu(a[None]), to_gpu(s[None])).cpu().numpy()
    g.set_scheme("plane")
    J_back = rt.formal_solution(g, to_gpu(a[None]), to_gpu(s[None])).cpu().numpy()
    assert np.array_equal(J_plane, J_back)
    assert_parity(J_face, oracle.sc_regular_face(24, 24, 16, dx, dy, z, dirs, w, a[None], s[None]),
                  what="J face")
    assert_parity(J_plane, oracle.sc_regular(24, 24, 16, dx, dy, z, dirs, w, a[None], s[None]),
                  what="J plane")
    closed = rt.RegularGrid(8, 8, 8, 1.0, 1.0, np.arange(8.0), dirs, w, periodic=False)
    with pytest.raises(rt.RTError):
        closed.set_scheme("face")


def test_128cubed_52_wavelengths_sampled(rt):
    """The 128^3 grid of the NLTE workload with 52 wavelengths in one launch (opacity spread
    10^-2 .. 10^4 times the continuum, as from the far wing to the core of the line); two
    wavelengths, the extremes, against the oracle at every point."""
    nx = ny = nz = 128
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(nx, ny, nz)
    dirs, w = s4_quadrature()
    assert _vertical_face_steps(z, dirs, dx, dy) == 16 * (nz - 1)
    scale = 10.0 ** np.linspace(-2.0, 4.0, 52)
    A = (a[None, :] * scale[:, None]).astype(np.float32)
    S = np.broadcast_to(s[None, :], A.shape).astype(np.float32)
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w, scheme="face")
    J = rt.formal_solution(g, to_gpu(A), to_gpu(S)).cpu().numpy()
    pick = [0, 51]
    Jr = oracle.sc_regular_face(nx, ny, nz, dx, dy, z, dirs, w, A[pick].astype(np.float64),
                                S[pick].astype(np.float64))
    assert_parity(J[pick], Jr, what="J at 128^3")


def test_lambda_iteration_with_the_face_scheme(rt):
    """Six Lambda iterations (52 wavelengths, 24 directions) on a 24 x 24 x 16 grid whose shallow
    rays meet vertical faces (dz / dx = 0.75)."""
    nx, ny, nz, nit = 24, 24, 16, 6
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    dirs, w = s4_quadrature()
    assert _vertical_face_steps(z, dirs, dx, dy) > 0
    A = Atom(data, atm.kappa0)
    ref, it, hist = orc_lambda_iterate(OrcRegular(nx, ny, nz, dx, dy, z, dirs, w, scheme="face"),
                                       A, f["T"], f["rho"], f["ne"], f["nH"], max_iter=nit,
                                       tol=0.0)
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w, scheme="face")
    ga = rt.Atom(data, atm.kappa0)
    gm = rt.Atmos(to_gpu(f["T"]), to_gpu(f["rho"]), to_gpu(f["ne"]), to_gpu(f["nH"]))
    pops = rt.lte_populations(g, ga, gm)
    its, ghist, conv = rt.lambda_iterate(g, ga, gm, pops, max_iter=nit, tol=0.0, use_graph=True)
    assert its == nit and not conv
    assert_parity(pops.cpu().numpy(), ref, rel=1e-4, floor=0.0, what="pops after 6 iterations")
    np.testing.assert_allclose(ghist, hist, rtol=2e-2)

"""Pins of the oracle's face-hitting short characteristics (Kunasz & Auer, the regular-grid scheme
Sect. 2.6 names; CPU only).

What fixes the scheme independently of its code:
* S linear in z with constant alpha: I = S - b mu_z / alpha solves the transfer equation, is
  linear in space (so every interpolation of it is exact) and is integrated exactly by linear-S
  intervals (Eq. 2): the scheme reproduces it at every point, on both kinds of face.
* In vacuum the interpolation weights sum to one and the box is periodic: the beam of a
  searchlight keeps its plane sum, and its centroid moves by exactly dz (mu_x, mu_y) / |mu_z| per
  plane (the mean of every upwind stencil lies on the ray).
* On a vertical face the share of a point's upwind intensity that comes from its own plane is
  1 - f_z, f_z = t |mu_z| / dz: a searchlight's first plane decays along the face-normal axis
  as f_z (1 - f_z)^n, summed over every lap around the periodic box.
* The periodic plane system has one solution: shifting every input by whole cells shifts the
  output identically.
* Where every ray meets the plane face first, the scheme is the plane-to-plane one.
* S = A + c cos(k x), alpha constant: the infinite-medium intensity is closed-form; the error
  halves with the cells (first order, as for every short-characteristics scheme with linear
  interpolation).
"""
import numpy as np
import pytest

import oracle
from synth import s4_quadrature

MU1 = 0.3500212
MU2 = np.sqrt(1.0 - 2.0 * MU1 ** 2)


def _z(nz, lo, hi, seed=4):
    """nz plane heights with spacings drawn uniformly from [lo, hi] (dx = 1)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([[0.0], np.cumsum(rng.uniform(lo, hi, nz - 1))])


def _kinds(z, dirs, dx=1.0, dy=1.0):
    """Number of (direction, plane) steps that meet a vertical face first."""
    dz = np.diff(z)
    n = 0
    for mu in dirs:
        tz = dz / abs(mu[2])
        tx = dx / abs(mu[0]) if mu[0] else np.inf
        ty = dy / abs(mu[1]) if mu[1] else np.inf
        n += int(np.sum(tz > min(tx, ty)))
    return n


def test_linear_source_exact_on_both_faces():
    nx, ny, nz = 7, 6, 12
    z = _z(nz, 0.25, 1.4)
    dirs, w = s4_quadrature()
    lateral = _kinds(z, dirs)
    assert 0 < lateral < len(dirs) * (nz - 1)          # both kinds of face occur
    a0, A, B = 1.7, 2.0, 0.6
    Z = np.repeat(z, nx * ny)
    S = (A + B * Z)[None]
    al = np.full_like(S, a0)
    ibc = np.empty((len(dirs), 1, nx * ny))
    for d, mu in enumerate(dirs):
        zw = z[0] if mu[2] > 0 else z[-1]
        ibc[d, 0] = A + B * zw - B * mu[2] / a0
    J, I = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, w, al, S, bc=2, ibc=ibc,
                                  want_I=True)
    for d, mu in enumerate(dirs):
        np.testing.assert_allclose(I[d, 0], S[0] - B * mu[2] / a0, rtol=1e-12)
    np.testing.assert_allclose(J[0], S[0] - B * np.sum(w * dirs[:, 2]) / a0, rtol=1e-12)


def _searchlight(nx, ny, z, dirs, i0, j0):
    nz = len(z)
    zero = np.zeros((1, nx * ny * nz))
    ibc = np.zeros((len(dirs), 1, nx * ny))
    ibc[:, 0, j0 * nx + i0] = 1.0
    _, I = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, np.full(len(dirs), 1 / len(dirs)),
                                  zero, zero, bc=2, ibc=ibc, want_I=True)
    return I[:, 0].reshape(len(dirs), nz, ny, nx)


def test_searchlight_flux_and_centroid():
    nx = ny = 48
    # dz in [0.3, 0.5]: the shallow rays meet the plane face below dz = 0.403 and a vertical face
    # above, with f_z >= 0.8, so the beam's tail along the face normal stays far inside the box
    z = _z(10, 0.3, 0.5, seed=5)
    dirs, _ = s4_quadrature()
    assert 0 < _kinds(z, dirs) < 8 * 9
    i0, j0 = 24, 24
    I = _searchlight(nx, ny, z, dirs, i0, j0)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    for d, mu in enumerate(dirs):
        planes = range(len(z)) if mu[2] > 0 else range(len(z) - 1, -1, -1)
        zw = z[0] if mu[2] > 0 else z[-1]
        for k in planes:
            P = I[d, k]
            assert P.sum() == pytest.approx(1.0, rel=1e-12)
            cx = i0 + abs(z[k] - zw) * mu[0] / abs(mu[2])
            cy = j0 + abs(z[k] - zw) * mu[1] / abs(mu[2])
            ux = (ii - cx + nx / 2) % nx - nx / 2       # displacement from the expected centre
            uy = (jj - cy + ny / 2) % ny - ny / 2
            assert abs(np.sum(P * ux)) < 1e-9 and abs(np.sum(P * uy)) < 1e-9, (d, k)


def test_first_plane_decays_along_the_face_normal():
    """With f_z = 0.2 the chain runs around the periodic box many times: every column of the
    first plane is fixed, fz (1 - fz)^m / (1 - (1 - fz)^nx) at m cells past the face."""
    nx, ny = 40, 12
    dz = 2.0
    z = np.arange(3) * dz
    mu = np.array([[MU2, MU1, MU1]])                    # meets the x face first: dx/mu_x < dz/mu_z
    t = 1.0 / MU2
    assert t < dz / MU1
    fz = t * MU1 / dz
    i0 = 5
    I = _searchlight(nx, ny, z, mu, i0, 6)[0, 1]       # plane 1
    cols = I.sum(axis=0)                                # sum over y at each x
    m = (np.arange(nx) - (i0 + 1)) % nx
    np.testing.assert_allclose(cols, fz * (1.0 - fz) ** m / (1.0 - (1.0 - fz) ** nx), rtol=1e-12)


def test_periodic_plane_system_is_translation_equivariant():
    nx, ny, nz = 9, 8, 7
    z = _z(nz, 0.3, 1.2, seed=6)
    dirs, w = s4_quadrature()
    rng = np.random.default_rng(7)
    al = rng.uniform(0.05, 3.0, (2, nz, ny, nx))
    S = rng.uniform(0.5, 2.0, (2, nz, ny, nx))
    J0 = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, w, al.reshape(2, -1),
                                S.reshape(2, -1)).reshape(2, nz, ny, nx)
    sh = (5, 3)
    J1 = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, w,
                                np.roll(al, sh, axis=(2, 3)).reshape(2, -1),
                                np.roll(S, sh, axis=(2, 3)).reshape(2, -1)).reshape(2, nz, ny, nx)
    np.testing.assert_allclose(J1, np.roll(J0, sh, axis=(2, 3)), rtol=1e-12)


def test_reduces_to_plane_to_plane_where_no_vertical_face_is_met():
    nx, ny, nz = 8, 7, 10
    z = _z(nz, 0.1, 0.38, seed=8)                      # dz / mu_z < dx / mu_x for every direction
    dirs, w = s4_quadrature()
    assert _kinds(z, dirs) == 0
    rng = np.random.default_rng(9)
    al = rng.uniform(0.05, 3.0, (2, nx * ny * nz))
    S = rng.uniform(0.5, 2.0, (2, nx * ny * nz))
    for bc in (0, 1):
        a = oracle.sc_regular_face(nx, ny, nz, 1.0, 1.0, z, dirs, w, al, S, bc=bc)
        b = oracle.sc_regular(nx, ny, nz, 1.0, 1.0, z, dirs, w, al, S, bc=bc)
        np.testing.assert_allclose(a, b, rtol=1e-13)


def test_cosine_source_converges_at_first_order():
    """S = A + c cos(k x), alpha constant, exact inflow: I(x) = A + c (alpha^2 cos kx +
    alpha k mu_x sin kx) / (alpha^2 + k^2 mu_x^2).  Short characteristics with linear
    interpolation make an O(h^2) error per step and take O(1/h) steps per mean free path: the
    error halves with the cells.  Measured on the shallow rays, which meet vertical faces."""
    dirs, w = s4_quadrature()
    shallow = [d for d, mu in enumerate(dirs) if abs(mu[2]) < 0.5]
    A, c, a0, k = 1.0, 0.5, 8.0, 2.0 * np.pi
    errs = []
    for nx in (16, 32, 64):
        dx = 1.0 / nx
        ny, dz = 2, 0.5 * dx                            # dz / mu_z > dx / mu_x on the shallow rays
        nz = int(round(0.25 / dz)) + 1
        z = np.arange(nz) * dz
        assert _kinds(z, dirs, dx, dx) == len(shallow) * (nz - 1)
        x = np.arange(nx) * dx
        X = np.broadcast_to(x[None, None, :], (nz, ny, nx)).ravel()
        S = (A + c * np.cos(k * X))[None]
        al = np.full_like(S, a0)

        def exact(mu, xx):
            return A + c * (a0 ** 2 * np.cos(k * xx) + a0 * k * mu[0] * np.sin(k * xx)) / (
                a0 ** 2 + (k * mu[0]) ** 2)
        ibc = np.stack([np.broadcast_to(exact(mu, x)[None, :], (ny, nx)).ravel()[None]
                        for mu in dirs])
        _, I = oracle.sc_regular_face(nx, ny, nz, dx, dx, z, dirs, w, al, S, bc=2, ibc=ibc,
                                      want_I=True)
        errs.append(max(np.abs(I[d, 0] - exact(dirs[d], X)).max() for d in shallow))
    r = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(1.8 < v < 2.3 for v in r), (errs, r)
    assert errs[2] < 0.01 * c


def _scheme_difference(n):
    """J and the top-plane intensity of the face-hitting and plane-to-plane schemes on the n^3 LTE
    continuum (500 nm) of the synthetic atmosphere: relative differences (RMS over points)."""
    from oracle.physics import lte_alpha_S
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    dirs, w = s4_quadrature()
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(n, n, n, atm)
    a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    Jp, Ip = oracle.sc_regular(n, n, n, dx, dy, z, dirs, w, a[None], s[None], want_I=True)
    Jf, If = oracle.sc_regular_face(n, n, n, dx, dy, z, dirs, w, a[None], s[None], want_I=True)
    top = slice((n - 1) * n * n, n ** 3)
    steep = [d for d, mu in enumerate(dirs) if mu[2] > 0.8]
    shallow = [d for d, mu in enumerate(dirs) if 0.0 < mu[2] < 0.5]
    rms = lambda r: float(np.sqrt(np.mean(r ** 2)))   # noqa: E731
    dJ = rms((Jf[0] - Jp[0]) / Jp[0])
    dI = rms(np.concatenate([(If[d, 0, top] - Ip[d, 0, top]) / Ip[d, 0, top] for d in shallow]))
    steep_same = max(np.abs(If[d, 0] - Ip[d, 0]).max() / np.abs(Ip[d, 0]).max() for d in steep)
    return dJ, dI, steep_same


def test_the_two_readings_converge_to_each_other():
    """On the LTE continuum of the synthetic atmosphere (dz = dx / 2, so the 16 shallow rays meet
    vertical faces on every plane): the steep rays agree to rounding; the schemes' J differs by
    under 1 % and the shallow rays' emergent intensity by under 2 % (RMS), less on the finer grid
    (both are first-order consistent discretisations of the same transfer equation)."""
    d32 = _scheme_difference(32)
    d64 = _scheme_difference(64)
    assert d32[2] < 1e-12 and d64[2] < 1e-12
    assert d64[0] < d32[0] / 1.3 and d64[1] < d32[1] / 1.3
    assert max(d32[0], d32[1]) < 0.02 and max(d64[0], d64[1]) < 0.012

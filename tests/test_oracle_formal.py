"""Pins of the oracle's formal solution against what the mathematics fixes (CPU only).

Each test names the property it pins and the passage of the paper it follows.
"""
import functools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle.physics import lte_alpha_S
from synth import make_atmosphere, s4_quadrature
from synth.atmosphere import regular_fields


# ---- linear-S interval weights (Sect. 2.5: linear interpolation of S; Eq. 2) -------------------
@pytest.mark.parametrize("d", [1e-9, 3e-7, 9.99e-7, 1.01e-6, 1e-4, 1e-2, 0.3, 1.0, 7.0, 60.0, 700.0])
def test_linear_weights_match_quadrature(d):
    """w0, w1 are the integrals of the two hat functions against exp(-(d - t)) over [0, d]."""
    (ex, w0, w1), (dex, dw0, dw1) = oracle.linear_weights(d)
    k0 = integrate.quad(lambda t: (1.0 - t / d) * math.exp(-(d - t)), 0.0, d, epsabs=0,
                        epsrel=1e-13, limit=200)[0]
    k1 = integrate.quad(lambda t: (t / d) * math.exp(-(d - t)), 0.0, d, epsabs=0, epsrel=1e-13,
                        limit=200)[0]
    assert ex == pytest.approx(math.exp(-d), rel=1e-14, abs=0)
    assert w0 == pytest.approx(k0, rel=1e-9, abs=1e-300)
    assert w1 == pytest.approx(k1, rel=1e-9, abs=1e-300)
    # derivatives against central differences of the quadrature values
    h = 1e-5 * d
    (_, a0, a1), _ = oracle.linear_weights(d + h)
    (_, b0, b1), _ = oracle.linear_weights(d - h)
    assert dw0 == pytest.approx((a0 - b0) / (2 * h), rel=1e-5, abs=1e-12)
    assert dw1 == pytest.approx((a1 - b1) / (2 * h), rel=1e-5, abs=1e-12)
    assert dex == pytest.approx(-math.exp(-d), rel=1e-14)


@pytest.mark.parametrize("d", [50.0, 1e3, 1e6, 1e9, 1e13])
def test_linear_weights_thick_closed_form(d):
    """Optically thick intervals: the hat-function integrals have the closed forms
    w0 = (1 - (1 + d) e^-d) / d and w1 = (1 - e^-d) - w0, so w0 -> 1/d while w1 -> 1.  w0 keeps
    full relative precision however thick the interval (it carries the upwind source function,
    which can exceed the local one by a factor comparable to d)."""
    (ex, w0, w1), _ = oracle.linear_weights(d)
    ref0 = -math.expm1(-d) / d - (1.0 + 1.0 / d) * math.exp(-d) if d < 700 else 1.0 / d
    assert w0 == pytest.approx(ref0, rel=1e-13)
    assert w1 == pytest.approx(-math.expm1(-d) - ref0, rel=1e-15)


def _grid_z(nz, nonuniform=True, L=1.0, seed=3):
    rng = np.random.default_rng(seed)
    dz = np.ones(nz - 1) if not nonuniform else 0.5 + rng.random(nz - 1)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    return z * (L / z[-1])


# ---- constant S and alpha: I = I0 exp(-tau) + S (1 - exp(-tau)) exactly (Eq. 2) ---------------
@pytest.mark.parametrize("bc", [1, 2])
def test_constant_source_exact(bc):
    nx, ny, nz = 5, 4, 9
    z = _grid_z(nz)
    dirs, w = s4_quadrature()
    a0, s0, i0 = 3.7, 2.5, 0.6
    al = np.full((1, nx * ny * nz), a0)
    S = np.full((1, nx * ny * nz), s0)
    ibc = np.full((len(dirs), 1, nx * ny), i0) if bc == 2 else None
    J, I = oracle.sc_regular(nx, ny, nz, 0.3, 0.2, z, dirs, w, al, S, bc=bc, ibc=ibc,
                             want_I=True)
    inflow = i0 if bc == 2 else 0.0
    for d, mu in enumerate(dirs):
        zk = z if mu[2] > 0 else z[::-1]
        s_path = np.abs(z - zk[0]) / abs(mu[2])
        exact = inflow * np.exp(-a0 * s_path) + s0 * (1.0 - np.exp(-a0 * s_path))
        got = I[d, 0].reshape(nz, ny * nx)
        np.testing.assert_allclose(got, np.broadcast_to(exact[:, None], got.shape), rtol=1e-13,
                                   atol=1e-15)


# ---- S linear along every ray is integrated exactly (Eq. 2, linear S) --------------------------
def test_linear_source_exact():
    """S = a + b z, alpha constant: I = S - b mu_z / alpha solves dI/dtau = S - I on every ray;
    with that inflow on both walls the scheme must reproduce it at every point."""
    nx, ny, nz = 6, 5, 11
    z = _grid_z(nz, L=2.0)
    dirs, w = s4_quadrature()
    a0, A, B = 1.3, 2.0, 0.7
    Z = np.repeat(z, nx * ny)
    S = (A + B * Z)[None]
    al = np.full_like(S, a0)
    ibc = np.empty((len(dirs), 1, nx * ny))
    for d, mu in enumerate(dirs):
        zw = z[0] if mu[2] > 0 else z[-1]
        ibc[d, 0] = A + B * zw - B * mu[2] / a0
    J, I = oracle.sc_regular(nx, ny, nz, 0.4, 0.3, z, dirs, w, al, S, bc=2, ibc=ibc, want_I=True)
    for d, mu in enumerate(dirs):
        np.testing.assert_allclose(I[d, 0], S[0] - B * mu[2] / a0, rtol=1e-12)
    np.testing.assert_allclose(J[0], S[0] - B * np.sum(w * dirs[:, 2]) / a0, rtol=1e-12)


# ---- horizontally homogeneous slab = the exact 1D solution on the slanted ray ----------------
def _exact_slab(z, mu, alpha_f, tau_f, S_f, inflow):
    """Exact Eq. 2 along a ray of direction cosine mu through a slab (scipy quadrature)."""
    out = []
    z0 = z[0] if mu > 0 else z[-1]
    for zz in z:
        t_end = abs(tau_f(zz) - tau_f(z0)) / abs(mu)

        def integrand(zp):
            t = abs(tau_f(zz) - tau_f(zp)) / abs(mu)
            return S_f(zp) * alpha_f(zp) / abs(mu) * math.exp(-t)
        lo, hi = (z0, zz) if mu > 0 else (zz, z0)
        val = integrate.quad(integrand, lo, hi, epsabs=0, epsrel=1e-12, limit=400)[0]
        out.append(inflow * math.exp(-t_end) + val)
    return np.array(out)


def test_plane_parallel_reduction_converges():
    alpha_f = lambda z: 2.0 + math.cos(z)               # noqa: E731
    tau_f = lambda z: 2.0 * z + math.sin(z)             # noqa: E731  (integral of alpha)
    S_f = lambda z: 1.0 + 0.5 * math.sin(2.0 * z)       # noqa: E731
    dirs, w = s4_quadrature()
    errs = []
    for nz in (17, 33, 65):
        z = np.linspace(0.0, 4.0, nz)
        al = np.array([alpha_f(v) for v in z])
        S = np.array([S_f(v) for v in z])
        nx = ny = 3
        AL = np.repeat(al, nx * ny)[None]
        SS = np.repeat(S, nx * ny)[None]
        _, I = oracle.sc_regular(nx, ny, nz, 0.7, 0.9, z, dirs, w, AL, SS, bc=0, want_I=True)
        e = 0.0
        for d in (0, 2, 12, 14):                        # both mu_z values, both hemispheres
            mu = dirs[d, 2]
            inflow = S_f(z[0]) if mu > 0 else 0.0
            ex = _exact_slab(z, mu, alpha_f, tau_f, S_f, inflow)
            got = I[d, 0].reshape(nz, nx * ny)
            assert np.ptp(got, axis=1).max() < 1e-13   # horizontally homogeneous
            e = max(e, np.abs(got[:, 0] - ex).max())
        errs.append(e)
    # second-order scheme: each halving of dz cuts the error by about 4
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 2e-3


# ---- J -> B at depth (LTE continuum, 32 x 32 x 64) ---------------------------------------------
def test_J_tends_to_B_at_depth():
    atm = make_atmosphere(0)
    dirs, w = s4_quadrature()
    f, (x, y, z, dx, dy) = regular_fields(32, 32, 64, atm)
    al, S = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    J = oracle.sc_regular(32, 32, 64, dx, dy, z, dirs, w, al[None], S[None])[0]
    A = al.reshape(64, 32 * 32)
    tau = np.zeros_like(A)
    for k in range(62, -1, -1):
        tau[k] = tau[k + 1] + 0.5 * (A[k] + A[k + 1]) * (z[k + 1] - z[k])
    r = np.abs(J / S - 1.0).reshape(64, -1)
    assert r[tau > 100].max() < 1e-3
    assert r[tau > 1000].max() < 1e-4
    # and the bound tightens with depth
    assert r[tau > 1000].max() < r[(tau > 100) & (tau < 1000)].max()


# ---- octant symmetry --------------------------------------------------------------------------
def test_mirror_symmetry_x():
    atm = make_atmosphere(1)
    nx, ny, nz = 16, 8, 24
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    al, S = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    # make the fields symmetric under i -> -i (mod nx)
    def sym(v):
        v = v.reshape(nz, ny, nx)
        return 0.5 * (v + v[:, :, (-np.arange(nx)) % nx]).ravel()
    al, S = sym(al), sym(S)
    dirs, w = s4_quadrature()
    _, I = oracle.sc_regular(nx, ny, nz, dx, dy, z, dirs, w, al[None], S[None], want_I=True)
    mirror = {}
    for d, mu in enumerate(dirs):
        for e, nu in enumerate(dirs):
            if np.allclose(nu, mu * np.array([-1, 1, 1])):
                mirror[d] = e
    assert len(mirror) == 24
    for d, e in mirror.items():
        a = I[d, 0].reshape(nz, ny, nx)
        b = I[e, 0].reshape(nz, ny, nx)[:, :, (-np.arange(nx)) % nx]
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


# ---- brute force per-point recursion on a tiny grid ---------------------------------------------
def test_bruteforce_recursion_tiny():
    rng = np.random.default_rng(7)
    nx, ny, nz = 4, 3, 8
    z = _grid_z(nz, L=1.0, seed=11)
    dx, dy = 0.21, 0.17
    al = rng.uniform(0.2, 5.0, (nz, ny, nx))
    S = rng.uniform(0.5, 2.0, (nz, ny, nx))
    dirs, w = s4_quadrature()
    J, I = oracle.sc_regular(nx, ny, nz, dx, dy, z, dirs, w, al.reshape(1, -1),
                             S.reshape(1, -1), bc=0, want_I=True)

    for d, mu in enumerate(dirs):
        @functools.lru_cache(maxsize=None)
        def intensity(k, j, i):
            kb = 0 if mu[2] > 0 else nz - 1
            if k == kb:
                return S[k, j, i] if mu[2] > 0 else 0.0
            ku = k - 1 if mu[2] > 0 else k + 1
            s = abs(z[k] - z[ku]) / abs(mu[2])
            xu = i * dx - s * mu[0]
            yu = j * dy - s * mu[1]
            gx, gy = xu / dx, yu / dy
            i0, j0 = math.floor(gx), math.floor(gy)
            tx, ty = gx - i0, gy - j0
            corners = [((i0, j0), (1 - tx) * (1 - ty)), ((i0 + 1, j0), tx * (1 - ty)),
                       ((i0, j0 + 1), (1 - tx) * ty), ((i0 + 1, j0 + 1), tx * ty)]
            Iu = Su = Au = 0.0
            for (ci, cj), wt in corners:
                Iu += wt * intensity(ku, cj % ny, ci % nx)
                Su += wt * S[ku, cj % ny, ci % nx]
                Au += wt * al[ku, cj % ny, ci % nx]
            t = 0.5 * (Au + al[k, j, i]) * s
            ex = math.exp(-t)
            e0 = 1.0 - ex
            return Iu * ex + (e0 - (t - e0) / t) * Su + (t - e0) / t * S[k, j, i]

        ref = np.array([[[intensity(k, j, i) for i in range(nx)] for j in range(ny)]
                        for k in range(nz)])
        np.testing.assert_allclose(I[d, 0].reshape(nz, ny, nx), ref, rtol=1e-12)


# ---- searchlight beam on the regular grid (Sect. 3.1) ------------------------------------------
def _searchlight_regular(periodic):
    n = 51
    h = 1.0 / (n - 1)
    z = np.arange(n) * h
    th = math.radians(20.0)
    mu = np.array([[math.sin(th), 0.0, math.cos(th)]])
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="xy")
    beam = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 <= 0.2 ** 2).astype(float).ravel()
    zero = np.zeros((1, n ** 3))
    _, I = oracle.sc_regular(n, n, n, h, h, z, mu, np.ones(1), zero, zero, bc=2,
                             ibc=beam[None, None], periodic=periodic, want_I=True)
    top = I[0, 0].reshape(n, n * n)[-1]
    return beam, top


def test_searchlight_flux_conserved():
    """With alpha = S = 0 and periodic sides the bilinear weights sum to one, so the beam's
    total intensity is carried from the bottom plane to the top plane without loss."""
    beam, top = _searchlight_regular(periodic=True)
    assert top.sum() == pytest.approx(beam.sum(), rel=1e-12)
    assert top.min() >= -1e-15 and top.max() <= 1.0 + 1e-12

"""Seeded synthetic model atmosphere standing in for the paper's Bifrost snapshot (Sect. 2.3).

The recipe (one continuous analytic field, so that every grid samples the same atmosphere):

* box 6 x 6 Mm horizontally (periodic), z in [-0.5, 2.5] Mm, surface at z = 0;
* T0(z) piecewise linear through 10 000 K (z = -0.5 Mm), 4 500 K (z = 0), 8 000 K (z = 2.5 Mm);
* T(x, y, z) = T0(z) * (1 + 0.05 g(x, y)), g a periodic Gaussian random field with zero mean and
  unit variance: a finite Fourier series with modes |m_x|, |m_y| <= 16, power spectrum
  exp(-k^2 l^2 / 2) with l = 1 Mm, coefficients drawn from numpy's PCG64 with the given seed;
* rho = rho0 exp(-z / 150 km), rho0 = 3e-4 kg m^-3; n_H = rho / (1.4 m_H);
* n_e = n_H (1e-4 + 1 / (1 + exp((9000 K - T) / 600 K))), a smooth stand-in for the snapshot's
  electron density (the method takes n_e as given);
* kappa0 (m^2 kg^-1) is the background-opacity scale of the recipe alpha_bg = kappa0 rho (T/5000)^9,
  fixed by the recipe so that the horizontally averaged vertical optical depth at 500 nm is 1 at
  z = 0.  Only this calibration constant is produced here; the opacity and source function
  themselves are computed by the oracle and by the CUDA path.
"""
from __future__ import annotations

import dataclasses

import numpy as np

M_H = 1.6735575e-27  # kg, mass of the hydrogen atom (CODATA/IUPAC)
MM = 1.0e6           # one megametre in metres


@dataclasses.dataclass
class Atmosphere:
    seed: int
    Lx: float = 6.0 * MM
    Ly: float = 6.0 * MM
    zmin: float = -0.5 * MM
    zmax: float = 2.5 * MM
    rho0: float = 3.0e-4
    H: float = 150.0e3
    amp: float = 0.05
    corr_len: float = 1.0 * MM
    nmodes: int = 16
    t_knots_z: tuple = (-0.5 * MM, 0.0, 2.5 * MM)
    t_knots_T: tuple = (10000.0, 4500.0, 8000.0)
    lam_cont: float = 500.0e-9
    kappa0: float = 0.0
    _kx: np.ndarray = dataclasses.field(default=None, repr=False)
    _ky: np.ndarray = dataclasses.field(default=None, repr=False)
    _ca: np.ndarray = dataclasses.field(default=None, repr=False)
    _sa: np.ndarray = dataclasses.field(default=None, repr=False)

    # --- the random horizontal field ------------------------------------------------------
    def _draw_modes(self):
        rng = np.random.Generator(np.random.PCG64(self.seed))
        m = np.arange(-self.nmodes, self.nmodes + 1)
        mx, my = np.meshgrid(m, m, indexing="ij")
        mx, my = mx.ravel(), my.ravel()
        half = (my > 0) | ((my == 0) & (mx > 0))          # one of each +-k pair, no k = 0
        mx, my = mx[half], my[half]
        kx = 2.0 * np.pi * mx / self.Lx
        ky = 2.0 * np.pi * my / self.Ly
        p = np.exp(-0.5 * (kx * kx + ky * ky) * self.corr_len ** 2)
        a = rng.standard_normal(mx.size) * np.sqrt(p)
        b = rng.standard_normal(mx.size) * np.sqrt(p)
        var = 0.5 * np.sum(a * a + b * b)                   # exact variance over the period
        s = 1.0 / np.sqrt(var)
        self._kx, self._ky, self._ca, self._sa = kx, ky, a * s, b * s

    def g(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        ph = np.multiply.outer(x, self._kx) + np.multiply.outer(y, self._ky)
        return np.cos(ph) @ self._ca + np.sin(ph) @ self._sa

    # --- thermodynamic fields ---------------------------------------------------------------
    def T0(self, z):
        return np.interp(np.asarray(z, dtype=np.float64), self.t_knots_z, self.t_knots_T)

    def T(self, x, y, z):
        return self.T0(z) * (1.0 + self.amp * self.g(x, y))

    def rho(self, z):
        return self.rho0 * np.exp(-np.asarray(z, dtype=np.float64) / self.H)

    def n_H(self, z):
        return self.rho(z) / (1.4 * M_H)

    @staticmethod
    def n_e(T, nH):
        return nH * (1.0e-4 + 1.0 / (1.0 + np.exp((9000.0 - T) / 600.0)))

    def fields(self, x, y, z):
        """T, rho, n_e, n_H at points (x, y, z) (arrays of equal shape), float64."""
        x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float),
                                      np.asarray(z, float))
        shape = x.shape
        xr, yr, zr = x.ravel(), y.ravel(), z.ravel()
        T = np.empty(xr.size)
        for s in range(0, xr.size, 1 << 16):              # bounded temporaries
            T[s:s + (1 << 16)] = self.T(xr[s:s + (1 << 16)], yr[s:s + (1 << 16)],
                                        zr[s:s + (1 << 16)])
        rho = self.rho(zr)
        nH = rho / (1.4 * M_H)
        ne = self.n_e(T, nH)
        return {k: v.reshape(shape) for k, v in
                dict(T=T, rho=rho, ne=ne, nH=nH).items()}

    # --- recipe calibration -----------------------------------------------------------------
    def _calibrate_kappa0(self):
        """kappa0 such that < integral_0^zmax rho (T/5000)^9 dz >_xy * kappa0 = 1."""
        n = 128
        xs = np.arange(n) * (self.Lx / n)
        ys = np.arange(n) * (self.Ly / n)
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        gg = self.g(X.ravel(), Y.ravel())
        zs = np.linspace(0.0, self.zmax, 6001)
        t0 = self.T0(zs)
        # <(1 + a g)^9>_xy by direct averaging over a 128^2 grid of the band-limited field
        m9 = np.mean((1.0 + self.amp * gg) ** 9)
        integrand = self.rho(zs) * (t0 / 5000.0) ** 9 * m9
        tau_per_kappa = np.trapezoid(integrand, zs)
        self.kappa0 = 1.0 / tau_per_kappa


def make_atmosphere(seed: int = 0) -> Atmosphere:
    atm = Atmosphere(seed=seed)
    atm._draw_modes()
    atm._calibrate_kappa0()
    return atm


def regular_axes(nx: int, ny: int, nz: int, atm: Atmosphere):
    """Cell-centred regular grid of the box: x_i = i dx (periodic), z_k = zmin + (k + 1/2) dz."""
    dx = atm.Lx / nx
    dy = atm.Ly / ny
    dz = (atm.zmax - atm.zmin) / nz
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    z = atm.zmin + (np.arange(nz) + 0.5) * dz
    return x, y, z, dx, dy


def regular_fields(nx: int, ny: int, nz: int, atm: Atmosphere):
    """Fields on the regular grid, flattened with x fastest: index = (k * ny + j) * nx + i.
    The horizontal field g is evaluated once per column (it does not depend on z)."""
    x, y, z, dx, dy = regular_axes(nx, ny, nz, atm)
    Y2, X2 = np.meshgrid(y, x, indexing="ij")
    g = atm.g(X2.ravel(), Y2.ravel()).reshape(ny, nx)
    T = atm.T0(z)[:, None, None] * (1.0 + atm.amp * g)[None]
    rho = np.broadcast_to(atm.rho(z)[:, None, None], (nz, ny, nx))
    nH = rho / (1.4 * M_H)
    ne = atm.n_e(T, nH)
    f = dict(T=T, rho=rho, ne=ne, nH=nH)
    return {k: np.ascontiguousarray(v).reshape(-1) for k, v in f.items()}, (x, y, z, dx, dy)

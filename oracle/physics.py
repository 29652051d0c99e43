"""Oracle physics (FP64, numpy/scipy): Planck function, LTE populations, opacities and source
functions of the 2 + 1 level hydrogen-like atom, radiative and collisional rates, statistical
equilibrium.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Atom (Sect. 2.2, Table 1): levels 1, 2 and the continuum p; one line 1-2 with oscillator
strength f; bound-free from 1 and from 2.  Every transition i -> j (i lower) is treated alike:
with the LTE ratio g_ij(lambda) = (n_i/n_j)* exp(-hc/(lambda k T)),
    alpha_ij = sigma_ij (n_i - n_j g_ij),   eta_ij = sigma_ij n_j g_ij 2hc^2/lambda^5,
    R_ij = 4pi/(hc) int sigma_ij lambda J dlambda,
    R_ji = 4pi/(hc) int sigma_ij lambda g_ij (2hc^2/lambda^5 + J) dlambda,
so that LTE populations give S = B and detailed balance at every wavelength.
Line cross section: sigma = pi e^2/(4 pi eps0 m_e c) f lambda0^2/c phi_lambda, phi a Voigt
profile (damping a, Doppler width from T and the hydrogen mass), renormalised per point to
sum_j phi_j w_j = 1 over the line nodes.  Bound-free: Kramers' hydrogenic cross section with
Gaunt factor 1, sigma = sigma_edge (lambda/lambda_edge)^3 below the edge, sigma_edge =
64 pi^4 m_e e^10 / (3 sqrt3 c h^6 (4 pi eps0)^5 n^5 nu_edge^3).
Collisions (stand-in for Johnson 1972 x 1e9): C21 = q n_e T^-1/2, C12 by detailed balance;
C_ip = q n_e T^-1/2 exp(-E_ip/kT), C_pi by detailed balance.
Background: alpha_bg = kappa0 rho (T/5000)^9 at every wavelength, with source function B.
"""
from __future__ import annotations

import numpy as np
from scipy.special import voigt_profile

# CODATA 2018 (exact where defined)
H = 6.62607015e-34
C = 299792458.0
KB = 1.380649e-23
ME = 9.1093837015e-31
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
MH = 1.6735575e-27


def planck(T, lam):
    """B_lambda(T) [W m^-2 m^-1 sr^-1]."""
    return 2.0 * H * C ** 2 / lam ** 5 / np.expm1(H * C / (lam * KB * T))


def dplanck_dT(T, lam):
    x = H * C / (lam * KB * T)
    return planck(T, lam) * x / T * np.exp(x) / np.expm1(x)


def lte_alpha_S(T, rho, kappa0, lam):
    """LTE continuum of the synthetic atmosphere: alpha = kappa0 rho (T/5000)^9, S = B(T)."""
    return kappa0 * rho * (T / 5000.0) ** 9, planck(T, lam)


class Atom:
    """Derived constants of the model atom from its data dict (see synth.atom)."""

    def __init__(self, data, kappa0):
        self.E = np.asarray(data["E_cm"], float) * 100.0 * H * C   # J
        self.g = np.asarray(data["g"], float)
        self.f = float(data["f"])
        self.a = float(data["voigt_a"])
        self.q = float(data["q_coll"])
        self.lam = np.asarray(data["lam"], float)
        self.w = np.asarray(data["wlam"], float)
        self.kind = np.asarray(data["kind"], int)
        self.kappa0 = float(kappa0)
        self.lam0 = H * C / (self.E[1] - self.E[0])
        self.edge = np.array([H * C / (self.E[2] - self.E[0]), H * C / (self.E[2] - self.E[1])])
        self.sig_line = np.pi * QE ** 2 / (4.0 * np.pi * EPS0 * ME * C) * self.f * self.lam0 ** 2 / C
        kram = 64.0 * np.pi ** 4 * ME * QE ** 10 / (3.0 * np.sqrt(3.0) * C * H ** 6 *
                                                     (4.0 * np.pi * EPS0) ** 5)
        nu_e = C / self.edge
        self.sig_edge = kram / (np.array([1.0, 2.0]) ** 5 * nu_e ** 3)
        self.line = self.kind == 0

    # --- LTE ratios ------------------------------------------------------------------------
    def saha_phi(self, i, T):
        """Phi_i(T) [m^3]: (n_i / (n_p n_e))* for bound level i (0 or 1)."""
        return (self.g[i] / (2.0 * self.g[2]) * (H * H / (2.0 * np.pi * ME * KB * T)) ** 1.5 *
                np.exp((self.E[2] - self.E[i]) / (KB * T)))

    def lte_pops(self, T, ne, nH):
        """Saha-Boltzmann populations [3][npt] with n1 + n2 + np = nH."""
        r21 = self.g[1] / self.g[0] * np.exp(-(self.E[1] - self.E[0]) / (KB * T))
        rp1 = 1.0 / (ne * self.saha_phi(0, T))
        n1 = nH / (1.0 + r21 + rp1)
        return np.stack([n1, n1 * r21, n1 * rp1])

    def gij(self, tr, T, ne, lam):
        """(n_i/n_j)* exp(-hc/(lambda k T)) for transition tr: 0 line, 1 bf from 1, 2 bf from 2."""
        if tr == 0:
            return self.g[0] / self.g[1] * np.exp((self.E[1] - self.E[0] - H * C / lam) / (KB * T))
        i = tr - 1
        return (ne * self.g[i] / (2.0 * self.g[2]) *
                (H * H / (2.0 * np.pi * ME * KB * T)) ** 1.5 *
                np.exp((self.E[2] - self.E[i] - H * C / lam) / (KB * T)))

    # --- profiles and cross sections -----------------------------------------------------
    def phi(self, T):
        """Voigt profile phi_j(T) [n_line][npt] on the line nodes, renormalised per point."""
        lam = self.lam[self.line][:, None]
        dld = self.lam0 / C * np.sqrt(2.0 * KB * T / MH)[None, :]
        p = voigt_profile(lam - self.lam0, dld / np.sqrt(2.0), self.a * dld)
        norm = (p * self.w[self.line][:, None]).sum(axis=0)
        return p / norm

    def sigma(self, tr, lam, phi_row=None):
        if tr == 0:
            return self.sig_line * phi_row
        e = self.edge[tr - 1]
        return np.where(lam <= e, self.sig_edge[tr - 1] * (lam / e) ** 3, 0.0)

    # --- opacity and source function -------------------------------------------------------
    def alpha_S(self, T, rho, ne, pops):
        """alpha, S [nlam][npt] from the populations (n1, n2, np)."""
        nlam = len(self.lam)
        npt = T.size
        alpha = np.empty((nlam, npt))
        S = np.empty((nlam, npt))
        phi = self.phi(T)
        abg = self.kappa0 * rho * (T / 5000.0) ** 9
        lines = np.nonzero(self.line)[0]
        for j in range(nlam):
            lam = self.lam[j]
            a = abg.copy()
            eta = abg * planck(T, lam)
            b2 = 2.0 * H * C ** 2 / lam ** 5
            trs = []
            if self.kind[j] == 0:
                trs.append((0, self.sigma(0, lam, phi[np.searchsorted(lines, j)]), 0, 1))
            for tr in (1, 2):
                if lam <= self.edge[tr - 1]:
                    trs.append((tr, self.sigma(tr, lam), tr - 1, 2))
            for tr, sig, lo, hi in trs:
                gg = self.gij(tr, T, ne, lam)
                a = a + sig * (pops[lo] - pops[hi] * gg)
                eta = eta + sig * pops[hi] * gg * b2
            alpha[j] = a
            S[j] = eta / a
        return alpha, S

    # --- rates and statistical equilibrium -------------------------------------------------
    def rate_matrix(self, T, ne, J):
        """P[i][j][npt]: total rate (s^-1) from level i to level j (radiative + collisional)."""
        npt = T.size
        P = np.zeros((3, 3, npt))
        phi = self.phi(T)
        fac = 4.0 * np.pi / (H * C)
        lines = np.nonzero(self.line)[0]
        for j in range(len(self.lam)):
            lam = self.lam[j]
            tr = int(self.kind[j])
            sig = self.sigma(tr, lam, phi[np.searchsorted(lines, j)] if tr == 0 else None)
            lo, hi = (0, 1) if tr == 0 else (tr - 1, 2)
            gg = self.gij(tr, T, ne, lam)
            up = fac * self.w[j] * sig * lam * J[j]
            dn = fac * self.w[j] * sig * lam * gg * (2.0 * H * C ** 2 / lam ** 5 + J[j])
            P[lo, hi] += up
            P[hi, lo] += dn
        cbase = self.q * ne / np.sqrt(T)
        c21 = cbase
        c12 = c21 * self.g[1] / self.g[0] * np.exp(-(self.E[1] - self.E[0]) / (KB * T))
        P[1, 0] += c21
        P[0, 1] += c12
        for i in (0, 1):
            cip = cbase * np.exp(-(self.E[2] - self.E[i]) / (KB * T))
            P[i, 2] += cip
            P[2, i] += cip * ne * self.saha_phi(i, T)
        return P

    def statistical_equilibrium(self, P, nH):
        """Solve sum_j n_j P_ji - n_i sum_j P_ij = 0 with n1 + n2 + np = nH (row 1 replaced by
        the conservation equation), by Gaussian elimination with partial pivoting (LAPACK)."""
        npt = nH.size
        A = np.zeros((npt, 3, 3))
        for i in range(3):
            for j in range(3):
                if i != j:
                    A[:, i, j] = P[j, i]
            A[:, i, i] = -(P[i].sum(axis=0) - P[i, i])
        A[:, 0, :] = 1.0
        b = np.zeros((npt, 3))
        b[:, 0] = nH
        return np.linalg.solve(A, b[..., None])[..., 0].T.copy()

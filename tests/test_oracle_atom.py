"""Pins of the oracle's atom physics (Sect. 2.2, Table 1) against textbook values and exact
detailed-balance identities (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle.physics import Atom, H, C, KB, ME, planck
from oracle.solve import RegularGrid, lambda_iterate
from synth import make_atmosphere, model_atom, s4_quadrature
from synth.atmosphere import regular_fields

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _atom(atm=None, f=None):
    if f is None:
        data = model_atom(1.0e10)
    else:
        data = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    return Atom(data, atm.kappa0 if atm is not None else 0.03)


def test_atom_data_matches_table1():
    d = model_atom(1e10)
    np.testing.assert_array_equal(d["E_cm"], GOLD["levels_E_cm"]["value"])
    np.testing.assert_array_equal(d["g"], GOLD["levels_g"]["value"])
    assert d["f"] == GOLD["f_line"]["value"]
    assert d["lam0"] * 1e9 == pytest.approx(GOLD["line_core_nm"]["value"], abs=1e-3)


def test_line_cross_section_reproduces_Aul():
    """The radiative part of R_21 with J = 0 is the Einstein A: (g1/g2) 4pi/(hc) int sigma
    lambda 2hc^2/lambda^5 dlambda must equal the paper's A_ul = 4.7e8 s^-1 given f = 0.41641
    (Sect. 2.2) -- this pins the line cross-section prefactor and the wavelength quadrature."""
    a = _atom()
    T = np.array([4000.0, 6000.0, 9000.0])
    phi = a.phi(T)
    lam = a.lam[a.line]
    w = a.w[a.line]
    A = (a.g[0] / a.g[1] * 4 * np.pi / (H * C) *
         (w[:, None] * a.sig_line * phi * lam[:, None] * 2 * H * C ** 2 / lam[:, None] ** 5).sum(0))
    np.testing.assert_allclose(A, GOLD["A_ul"]["value"], rtol=3e-3)


def test_kramers_edge_cross_section():
    """Kramers' hydrogenic edge cross section is 7.91e-22 n m^2 (textbook, Gaunt factor 1)."""
    a = _atom()
    np.testing.assert_allclose(a.sig_edge, [7.91e-22, 2 * 7.91e-22], rtol=5e-3)


def test_saha_constant():
    """(2 pi m_e k / h^2)^(3/2) = 2.4147e21 m^-3 K^-3/2 (textbook)."""
    a = _atom()
    T = 1.0e4
    # Phi_1 = g1/(2 g_p) (h^2/(2 pi m_e k T))^1.5 exp(chi/kT); strip the level factors
    phi = a.saha_phi(0, T) / (a.g[0] / (2 * a.g[2])) / np.exp((a.E[2] - a.E[0]) / (KB * T))
    assert 1.0 / (phi * T ** 1.5) == pytest.approx(2.4147e21, rel=2e-4)


def test_lte_populations_give_planck_source():
    atm = make_atmosphere(0)
    f, _ = regular_fields(8, 8, 16, atm)
    a = _atom(atm, f)
    pops = a.lte_pops(f["T"], f["ne"], f["nH"])
    np.testing.assert_allclose(pops.sum(0), f["nH"], rtol=1e-13)
    alpha, S = a.alpha_S(f["T"], f["rho"], f["ne"], pops)
    for j, lam in enumerate(a.lam):
        np.testing.assert_allclose(S[j], planck(f["T"], lam), rtol=1e-10)
    assert np.all(alpha > 0)


def test_detailed_balance_fixed_point():
    """J = B at every node makes the LTE populations an exact solution of statistical
    equilibrium (radiative and collisional detailed balance)."""
    atm = make_atmosphere(0)
    f, _ = regular_fields(8, 8, 16, atm)
    a = _atom(atm, f)
    J = np.stack([planck(f["T"], lam) for lam in a.lam])
    P = a.rate_matrix(f["T"], f["ne"], J)
    new = a.statistical_equilibrium(P, f["nH"])
    lte = a.lte_pops(f["T"], f["ne"], f["nH"])
    np.testing.assert_allclose(new, lte, rtol=1e-9)


def _tree_solution(P, nH):
    """Markov-chain-tree formula for the 3-state steady state (independent of elimination)."""
    n1 = P[1, 0] * P[2, 0] + P[1, 2] * P[2, 0] + P[2, 1] * P[1, 0]
    n2 = P[0, 1] * P[2, 1] + P[0, 2] * P[2, 1] + P[2, 0] * P[0, 1]
    n3 = P[0, 2] * P[1, 2] + P[0, 1] * P[1, 2] + P[1, 0] * P[0, 2]
    s = n1 + n2 + n3
    return np.stack([n1, n2, n3]) * (nH / s)


def test_statistical_equilibrium_solver():
    """Elimination agrees with the tree formula on random rates spanning eight decades and on
    the physical rates of the synthetic atmosphere (J from the oracle's formal solution)."""
    rng = np.random.default_rng(5)
    P = 10.0 ** rng.uniform(-2, 6, (3, 3, 500))
    nH = 10.0 ** rng.uniform(10, 23, 500)
    a = _atom()
    n = a.statistical_equilibrium(P, nH)
    np.testing.assert_allclose(n, _tree_solution(P, nH), rtol=1e-8)
    atm = make_atmosphere(0)
    nx, ny, nz = 8, 8, 24
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    a = _atom(atm, f)
    pops = a.lte_pops(f["T"], f["ne"], f["nH"])
    alpha, S = a.alpha_S(f["T"], f["rho"], f["ne"], pops)
    dirs, w = s4_quadrature()
    J = RegularGrid(nx, ny, nz, dx, dy, z, dirs, w).formal_solution(alpha, S)
    P = a.rate_matrix(f["T"], f["ne"], J)
    np.testing.assert_allclose(a.statistical_equilibrium(P, f["nH"]), _tree_solution(P, f["nH"]),
                               rtol=1e-9)


def test_collisional_calibration_eps_min():
    atm = make_atmosphere(0)
    f, _ = regular_fields(32, 32, 64, atm)
    d = model_atom(np.min(f["ne"] / np.sqrt(f["T"])))
    c21 = d["q_coll"] * f["ne"] / np.sqrt(f["T"])
    eps = c21 / (c21 + d["A21"])
    assert eps.min() == pytest.approx(GOLD["eps_min"]["value"], rel=1e-12)


def test_voigt_profile_normalised_and_doppler_core():
    a = _atom()
    T = np.array([4500.0, 8000.0])
    phi = a.phi(T)
    np.testing.assert_allclose((phi * a.w[a.line][:, None]).sum(0), 1.0, rtol=1e-13)
    # at a = 1e-3 the core is Gaussian to O(a): phi(l0) sqrt(pi) dl_D ~ 1 - 2a/sqrt(pi)
    dld = a.lam0 / C * np.sqrt(2 * KB * T / 1.6735575e-27)
    j = np.argmin(np.abs(a.lam[a.line] - a.lam0))
    v = (a.lam[a.line][j] - a.lam0) / dld
    raw = phi[j] * (phi[:, 0] * 0 + 1)[j]
    assert np.all(np.abs(raw * np.sqrt(np.pi) * dld / np.exp(-v * v) - 1) < 0.02)


def test_lambda_iteration_converges_small_grid():
    atm = make_atmosphere(0)
    nx, ny, nz = 8, 8, 24
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    a = _atom(atm, f)
    dirs, w = s4_quadrature()
    g = RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    pops, it, hist = lambda_iterate(g, a, f["T"], f["rho"], f["ne"], f["nH"], max_iter=300,
                                    tol=1e-3)
    assert it < 300 and hist[-1] < 1e-3
    assert hist[0] > 1e-3
    np.testing.assert_allclose(pops.sum(0), f["nH"], rtol=1e-12)
    assert np.all(pops > 0)

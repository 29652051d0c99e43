"""Model-atom data (the paper's Table 1 and Sect. 2.2) and its wavelength nodes, as inputs.

Levels (Table 1): E = 0, 82 258.211, 109 677.617 cm^-1 with g = 2, 8, 1 (the last is the H II
continuum).  Line 1-2: f = 0.41641, A_ul = 4.7e8 s^-1 (Sect. 2.2).  Voigt damping a = 1e-3.

Wavelength nodes (the paper's 50 + 20 + 20 are reduced to 50 + 1 + 1):
* 50 line nodes symmetric about lambda0 = 1/E2, equally spaced in asinh(v / 1 km/s) out to
  +-100 km/s, with trapezoid weights in lambda;
* one node per bound-free edge at 0.9 lambda_edge with weight 0.5 lambda_edge.
``kind`` tags each node with the rate integral it feeds: 0 line, 1 bf from level 1, 2 bf from 2.

Collisional scale q (m^3 s^-1 K^1/2): the recipe's collision law is C21 = q n_e T^-1/2 (and
C_ip = q n_e T^-1/2 exp(-E_ip/kT)); q is fixed by the paper's statement that the smallest
destruction probability is about 0.09 (Sect. 2.2), i.e. min over the atmosphere of
C21 / (C21 + A21) = 0.09.  Only the constant is produced here.
"""
import numpy as np

C_LIGHT = 299792458.0

E_CM = (0.0, 82258.211, 109677.617)
G = (2.0, 8.0, 1.0)
F_LINE = 0.41641
A21 = 4.7e8
VOIGT_A = 1.0e-3
EPS_MIN = 0.09


def line_wavelengths(n_line=50, vmax_kms=100.0, v0_kms=1.0):
    lam0 = 1.0 / (E_CM[1] * 100.0)
    umax = np.arcsinh(vmax_kms / v0_kms)
    u = np.linspace(-umax, umax, n_line)
    v = v0_kms * 1e3 * np.sinh(u)
    lam = lam0 * (1.0 + v / C_LIGHT)
    w = np.empty_like(lam)
    w[1:-1] = 0.5 * (lam[2:] - lam[:-2])
    w[0] = 0.5 * (lam[1] - lam[0])
    w[-1] = 0.5 * (lam[-1] - lam[-2])
    return lam, w


def model_atom(ne_min_over_sqrtT=None, n_line=50):
    """Atom data dict.  ``ne_min_over_sqrtT`` = min over the atmosphere of n_e / sqrt(T)."""
    lam_l, w_l = line_wavelengths(n_line)
    edges = [1.0 / ((E_CM[2] - E_CM[i]) * 100.0) for i in (0, 1)]
    lam = np.concatenate([lam_l, [0.9 * edges[0], 0.9 * edges[1]]])
    w = np.concatenate([w_l, [0.5 * edges[0], 0.5 * edges[1]]])
    kind = np.concatenate([np.zeros(n_line, np.int32), np.array([1, 2], np.int32)])
    q = 0.0
    if ne_min_over_sqrtT is not None:
        c21_min = EPS_MIN / (1.0 - EPS_MIN) * A21
        q = c21_min / ne_min_over_sqrtT
    return dict(E_cm=np.array(E_CM), g=np.array(G), f=F_LINE, A21=A21, voigt_a=VOIGT_A,
                q_coll=q, lam=lam, wlam=w, kind=kind, n_line=n_line,
                lam0=1.0 / (E_CM[1] * 100.0))

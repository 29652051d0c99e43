"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package produces *inputs only*: atmospheres (T, rho, n_e, n_H sampled from one continuous
analytic field), the angle quadrature, the model-atom data of the paper's Table 1 with its
wavelength nodes, and irregular-grid sites with their Delaunay neighbour lists.  It holds none of
the method's arithmetic (no opacity, source function, formal solution, rates or statistical
equilibrium): the oracle and the CUDA path each compute those on their own from these inputs.
"""
from .atmosphere import Atmosphere, make_atmosphere, regular_axes
from .quadrature import s4_quadrature
from .atom import model_atom, line_wavelengths
from .sites import rejection_sample, delaunay_neighbours, make_voronoi_grid

__all__ = [
    "Atmosphere", "make_atmosphere", "regular_axes", "s4_quadrature", "model_atom",
    "line_wavelengths", "rejection_sample", "delaunay_neighbours", "make_voronoi_grid",
]

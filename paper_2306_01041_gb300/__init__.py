"""GB300-native formal solution of 3D radiative transfer on regular and Voronoi grids
(Udnaes & Pereira 2023, arXiv:2306.01041): a thin Python binding over librt.so.

Build the library first (``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_2306_01041_gb300/build.py``); importing the API raises if it is missing.
"""
from ._lib import (RT_BC_ARRAY, RT_BC_THERMAL, RT_BC_ZERO, RT_SC_FACE,  # noqa: F401
                   RT_SC_PLANE, RTError, lib)
from .api import (IDW, Atmos, Atom, Batch, EmergentIntensity, Grid, RegularGrid,  # noqa: F401
                  SourceTerms,
                  VoronoiGrid, emergent_intensity, emergent_map, final_synthesis,
                  formal_solution,
                  formal_solution_adjoint,
                  kernel_launches, lambda_iterate, lambda_iterate_ali, lambda_star,
                  lte_populations, ng_extrapolate, sample_sites, source_terms,
                  source_terms_adjoint, source_terms_lte,
                  source_terms_lte_adjoint, statistical_equilibrium, statistical_equilibrium_ali)

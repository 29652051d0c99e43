"""FP64 CPU oracle of the formal solution, J, opacities, rates and the Lambda iteration.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg
are its only users.  It shares no code with the CUDA path (``paper_2306_01041_gb300``); the two
meet only through the seeded inputs of ``synth``.

Layout: ``orc.c`` (C, OpenMP) holds the sweeps (plane-to-plane and face-hitting short
characteristics on the regular grid, the level sweep on the Voronoi grid) and the Voronoi
tables; ``physics.py`` (numpy, scipy) the atom; ``solve.py`` the Lambda iteration that ties them
together.
"""
from .lib import (build, sc_regular, sc_regular_face, sc_regular_adjoint, linear_weights,
                  voronoi_tables, voronoi_order, voronoi_fs, voronoi_adjoint, num_threads)

__all__ = ["build", "sc_regular", "sc_regular_face", "sc_regular_adjoint", "linear_weights",
           "voronoi_tables", "voronoi_order", "voronoi_fs", "voronoi_adjoint", "num_threads"]

"""The maps behind the grid-accuracy comparison (LTE continuum at 500 nm, mu = 1; Sect. 3.2),
computed on the GPU, against the FP64 oracle's maps of the same grids:

* the 128 x 128 x 256 fine reference and the 32 x 32 x 64 regular grid (the top plane);
* the 20 000-site Voronoi grid sampled from |dtau/dz|: the intensities at its emergent-layer
  sites, resampled to 32 x 32 pixels by two-nearest inverse-distance weighting in (x, y);
* the same grid through the paper's own procedure: the opacity at the sites interpolated back to
  the fine mesh by two-nearest inverse-distance weighting, the mesh's source function, and the
  vertical formal solution there."""
import functools

import numpy as np
import pytest

from helpers import assert_parity, to_gpu, voronoi_grid
from oracle import synthesis as syn
from oracle.physics import lte_alpha_S
from synth import make_atmosphere, s4_quadrature
from synth.atmosphere import regular_fields

pytestmark = pytest.mark.gpu
MU1 = (0.0, 0.0, 1.0)


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


@functools.lru_cache(maxsize=None)
def _regular(nx, ny, nz):
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    return f, z, dx, dy, a, s


@pytest.mark.parametrize("shape", [(32, 32, 64), (128, 128, 256)])
def test_regular_maps_match_oracle(rt, shape):
    nx, ny, nz = shape
    f, z, dx, dy, a, s = _regular(nx, ny, nz)
    dirs, w = s4_quadrature()
    G = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    m = rt.emergent_map(G, MU1, to_gpu(a[None]), to_gpu(s[None]), nx, ny)
    assert_parity(m.cpu().numpy(), syn.emergent_mu1(nx, ny, nz, dx, dy, z, a[None], s[None]),
                  what=f"{nx}x{ny}x{nz} map")


def test_voronoi_maps_match_oracle(rt):
    import oracle
    atm, vg, f = voronoi_grid(20000, "dtau", 10)
    a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    dirs, w = s4_quadrature()
    G = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"], dirs,
                       w)
    top = syn.top_sites(vg["nbr_off"], vg["nbr_idx"])
    np.testing.assert_array_equal(G.top_points(), top)
    # native: emergent-layer sites resampled to 32 x 32 pixels
    m = rt.emergent_map(G, MU1, to_gpu(a[None]), to_gpu(s[None]), 32, 32)
    tab = oracle.voronoi_tables(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"],
                                vg["box"], np.array([MU1]), 7.0)
    _, I = oracle.voronoi_fs(tab, np.array([MU1]), np.ones(1), a[None], s[None], want_I=True)
    ref = syn.resample_map(vg["xyz"][top], I[0][:, top], 32, 32, vg["box"])
    assert_parity(m.cpu().numpy(), ref, what="Voronoi map, 32 x 32 pixels")
    # final synthesis on the fine mesh
    ff, zf, dxf, dyf, af, sf = _regular(128, 128, 256)
    mesh = rt.RegularGrid(128, 128, 256, dxf, dyf, zf, dirs, w)
    idw = rt.IDW(G, mesh)
    a_mesh = idw.interpolate(to_gpu(a[None]))
    fs = rt.emergent_map(mesh, MU1, a_mesh, to_gpu(sf[None]), 128, 128)
    k, d = syn.two_nearest(vg["xyz"], syn.mesh_points(128, 128, dxf, dyf, zf), vg["box"])
    a_ref = syn.interpolate(a[None], k, syn.idw_weights(d))
    fs_ref = syn.emergent_mu1(128, 128, 256, dxf, dyf, zf, a_ref, sf[None])
    assert_parity(fs.cpu().numpy(), fs_ref, what="final synthesis map")

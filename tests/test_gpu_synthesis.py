"""GPU parity of the final synthesis on a Voronoi grid (Sect. 2.5, last paragraphs) against the
FP64 oracle, through the C ABI: the two-nearest table, the inverse-distance interpolation of the
populations to the mesh, and the vertical emergent intensity computed on the mesh."""
import numpy as np
import pytest

from helpers import assert_parity, to_gpu, voronoi_grid
from oracle.physics import Atom
from oracle.synthesis import final_synthesis, idw_weights, interpolate, mesh_points, two_nearest
from synth import model_atom, s4_quadrature
from synth.atmosphere import regular_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def case(rt):
    atm, vg, f = voronoi_grid(3000, "dtau", 4)
    nx, ny, nz = 20, 16, 24
    mf, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    dirs, w = s4_quadrature()
    G = rt.VoronoiGrid(vg["xyz"], vg["nbr_off"], vg["nbr_idx"], vg["nbr_shift"], vg["box"], dirs,
                       w)
    M = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w)
    return dict(atm=atm, vg=vg, f=f, mf=mf, mesh=(nx, ny, nz, dx, dy, z), G=G, M=M)


def test_two_nearest_table_matches_oracle(rt, case):
    nx, ny, nz, dx, dy, z = case["mesh"]
    idw = rt.IDW(case["G"], case["M"])
    k, w = idw.table()
    kr, dr = two_nearest(case["vg"]["xyz"], mesh_points(nx, ny, dx, dy, z), case["vg"]["box"])
    np.testing.assert_array_equal(k, kr)
    np.testing.assert_allclose(w, idw_weights(dr), rtol=1e-6)


def test_interpolation_and_final_synthesis(rt, case):
    import torch
    atm, f, mf = case["atm"], case["f"], case["mf"]
    data = model_atom(np.min(mf["ne"] / np.sqrt(mf["T"])))
    A = Atom(data, atm.kappa0)
    site_pops = A.lte_pops(f["T"], f["ne"], f["nH"])
    site_pops[1] *= 1.0 + 0.3 * np.sin(7.0 * case["vg"]["xyz"][:, 0])   # not LTE
    nx, ny, nz, dx, dy, z = case["mesh"]
    kr, dr = two_nearest(case["vg"]["xyz"], mesh_points(nx, ny, dx, dy, z), case["vg"]["box"])
    ref_pops = interpolate(site_pops, kr, idw_weights(dr))
    idw = rt.IDW(case["G"], case["M"])
    got = idw.interpolate(to_gpu(site_pops))
    assert_parity(got.cpu().numpy(), ref_pops, rel=1e-5, floor=0.0, what="interpolated pops")
    ref_I = final_synthesis(A, site_pops, case["vg"]["xyz"], case["vg"]["box"], case["mesh"], mf)
    matm = rt.Atmos(to_gpu(mf["T"]), to_gpu(mf["rho"]), to_gpu(mf["ne"]), to_gpu(mf["nH"]))
    I = rt.final_synthesis(idw, case["M"], rt.Atom(data, atm.kappa0), matm, to_gpu(site_pops))
    torch.cuda.synchronize()
    assert I.shape == (len(data["lam"]), nx * ny)
    assert_parity(I.cpu().numpy(), ref_I, what="emergent intensity of the mesh")

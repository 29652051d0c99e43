"""CPU-side checks of the C ABI library: it builds for sm_103a, loads without a GPU, exports every
function include/rt.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def librt():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2306_01041_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(librt):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(librt, n), n


def test_rejects_bad_description_without_gpu(librt):
    import paper_2306_01041_gb300 as rt
    from paper_2306_01041_gb300 import _lib as L
    d = L.GridDesc()
    d.kind = L.RT_GRID_REGULAR
    d.ndir = 0
    h = ctypes.c_void_p()
    st = rt.lib().rt_grid_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == L.RT_EINVAL
    assert b"ndir" in rt.lib().rt_last_error()


def test_dawson_series_matches_scipy(librt):
    from scipy.special import dawsn
    librt.rt_debug_G_host.restype = ctypes.c_double
    librt.rt_debug_G_host.argtypes = [ctypes.c_double]
    v = np.array([0.0, 0.01, 0.3, 1.0, 2.5, 4.0, 6.0, 7.99, 9.0, 20.0])
    got = np.array([librt.rt_debug_G_host(x) for x in v])
    ref = 2 * v * dawsn(v) - 1
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)


def _vor_desc(L, xyz, off, idx, shift, box):
    d = L.GridDesc()
    d.kind = L.RT_GRID_VORONOI
    d.nsites = len(xyz)
    d.xyz = xyz.ctypes.data_as(L.PD)
    d.nbr_off = off.ctypes.data_as(L.PI64)
    d.nbr_idx = idx.ctypes.data_as(L.PI32)
    d.nbr_shift = shift.ctypes.data_as(L.PI8) if shift is not None else None
    d.box = (ctypes.c_double * 6)(*box)
    d.periodic_xy = 1
    return d


@pytest.mark.parametrize("fault", ["index", "shift", "outside", "offsets", "direction"])
def test_malformed_descriptions_rejected_on_host(librt, fault):
    """Malformed grids are refused with RT_EINVAL before any device call (runs without a GPU)."""
    import paper_2306_01041_gb300 as rt
    from paper_2306_01041_gb300 import _lib as L
    from synth import delaunay_neighbours, s4_quadrature
    rng = np.random.default_rng(0)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((60, 3))
    off, idx, shift = delaunay_neighbours(xyz, box)
    off, idx, shift = off.copy(), idx.copy(), shift.copy()
    dirs, w = s4_quadrature()
    if fault == "index":
        idx[5] = 60
    elif fault == "shift":
        shift[3] = 9
    elif fault == "outside":
        xyz[7, 2] = 1.5
    elif fault == "offsets":
        off[10] = off[11] + 1
    else:
        dirs = dirs.copy()
        dirs[4] = [1.0, 0.0, 0.0]
    d = _vor_desc(L, xyz, off, idx, shift, box)
    d.ndir = len(dirs)
    dirs = np.ascontiguousarray(dirs)
    d.dirs = dirs.ctypes.data_as(L.PD)
    d.wdir = w.ctypes.data_as(L.PD)
    d.r_exponent = 7.0
    h = ctypes.c_void_p()
    assert rt.lib().rt_grid_create(ctypes.byref(d), None, ctypes.byref(h)) == L.RT_EINVAL
    assert rt.lib().rt_last_error()


def test_launch_counter_without_gpu(librt):
    import paper_2306_01041_gb300 as rt
    a = rt.kernel_launches()
    assert isinstance(a, int) and a >= 0
    # a call rejected on the host launches nothing
    with pytest.raises(rt.RTError):
        rt.Batch([], 4)
    assert rt.kernel_launches() == a


def test_accelerated_and_synthesis_entry_points_reject_bad_arguments_on_host(librt):
    """Null handles and out-of-range knobs come back as RT_EINVAL before any device work."""
    import paper_2306_01041_gb300 as rt
    from paper_2306_01041_gb300 import _lib as L
    lib = rt.lib()
    n0 = rt.kernel_launches()
    assert lib.rt_lambda_star(None, 4, None, 0, None, None) == L.RT_EINVAL
    assert lib.rt_statistical_equilibrium_ali(None, None, None, None, None, None, None, None, 1,
                                              None) == L.RT_EINVAL
    it = ctypes.c_int(0)
    assert lib.rt_lambda_iterate_ali(None, None, None, None, 10, 1e-3, ctypes.byref(it), None, 0,
                                     -1, 1, None) == L.RT_EINVAL
    assert b"newton" in lib.rt_last_error()
    h = ctypes.c_void_p()
    assert lib.rt_idw_create(None, None, ctypes.byref(h)) == L.RT_EINVAL
    assert lib.rt_idw_interpolate(None, 3, None, None, None) == L.RT_EINVAL
    assert rt.kernel_launches() == n0


def test_face_scheme_and_site_sampling_reject_bad_arguments_on_host(librt):
    """rt_grid_set_scheme, rt_grid_build_tables_device and rt_sample_sites validate on the host
    before any device work."""
    import paper_2306_01041_gb300 as rt
    from paper_2306_01041_gb300 import _lib as L
    lib = rt.lib()
    n0 = rt.kernel_launches()
    assert lib.rt_grid_set_scheme(None, L.RT_SC_FACE) == L.RT_EINVAL
    assert lib.rt_grid_build_tables_device(None, None) == L.RT_EINVAL
    z = np.linspace(0.0, 1.0, 4)
    box = np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0])
    fake = ctypes.c_void_p(256)                     # never dereferenced: rejected first
    nprop = ctypes.c_int64()

    def call(nx=2, ny=2, nz=4, zz=z, bx=box, n=10, xyz=fake):
        return lib.rt_sample_sites(nx, ny, nz, zz.ctypes.data_as(L.PD), bx.ctypes.data_as(L.PD),
                                   fake, n, 1, xyz, ctypes.byref(nprop), None)
    assert call(nx=0) == L.RT_EINVAL
    assert call(nz=1) == L.RT_EINVAL
    assert call(n=0) == L.RT_EINVAL
    assert call(zz=z[::-1].copy()) == L.RT_EINVAL
    assert b"ascending" in lib.rt_last_error()
    assert call(bx=np.array([0.0, 1.0, 0.0, 1.0, 1.0, 1.0])) == L.RT_EINVAL
    assert call(xyz=ctypes.c_void_p(260)) == L.RT_EINVAL
    assert b"aligned" in lib.rt_last_error()
    assert rt.kernel_launches() == n0


def test_package_reexports_the_binding():
    """Every public function and class of the binding (api.py) is reachable from the package."""
    import inspect

    import paper_2306_01041_gb300 as rt
    from paper_2306_01041_gb300 import api
    public = [n for n, v in vars(api).items()
              if not n.startswith("_") and (inspect.isfunction(v) or inspect.isclass(v))
              and getattr(v, "__module__", "") == api.__name__]
    missing = [n for n in public if not hasattr(rt, n)]
    assert not missing, missing

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

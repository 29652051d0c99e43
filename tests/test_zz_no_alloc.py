"""The allocation-free regular-grid entry point, called through the C ABI, must give the same J as
rt_formal_solution on the same inputs, on two calls in a row (the calls share one static scratch
array, so the second call must not see anything of the first), and must refuse a problem larger
than its fixed scratch before touching the device."""
import ctypes

import numpy as np
import pytest

from helpers import assert_parity, lte_regular, to_gpu
from synth import s4_quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    fn = rt.lib().rt_formal_solution_regular_noalloc
    P = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P]
    return rt


def _call(rt, nx, ny, nz, dx, dy, z, dirs, w, alpha, S, J, bc=0):
    import torch
    z = np.ascontiguousarray(z, np.float64)
    d = np.ascontiguousarray(dirs, np.float64)
    ww = np.ascontiguousarray(w, np.float64)
    st = torch.cuda.current_stream().cuda_stream
    return rt.lib().rt_formal_solution_regular_noalloc(
        nx, ny, nz, dx, dy, z.ctypes.data, 1, len(d), d.ctypes.data, ww.ctypes.data,
        alpha.shape[0], alpha.data_ptr(), S.data_ptr(), bc, None, J.data_ptr(), st)


def test_noalloc_matches_formal_solution_twice(rt):
    import torch
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(32, 32, 64)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(32, 32, 64, dx, dy, z, dirs, w)
    rng = np.random.default_rng(0)
    inputs = [(np.stack([a, 2.0 * a]), np.stack([s, 0.5 * s])),
              (np.stack([a * rng.uniform(0.5, 2.0, a.size)]), np.stack([s[::-1].copy()]))]
    for al, sv in inputs:
        A, S = to_gpu(al), to_gpu(sv)
        J_ref = rt.formal_solution(g, A, S)
        J = torch.full_like(J_ref, float("nan"))
        assert _call(rt, 32, 32, 64, dx, dy, z, dirs, w, A, S, J) == 0
        torch.cuda.synchronize()
        assert_parity(J.cpu().numpy(), J_ref.cpu().numpy().astype(np.float64), rel=2e-6,
                      what="no-alloc J")


def test_noalloc_rejects_oversized_problem(rt):
    import torch
    dirs, w = s4_quadrature()
    z = np.arange(4, dtype=np.float64)
    A = torch.zeros(1, device="cuda")
    # 2 * 200 wavelengths * 12 directions * 64 * 64 floats exceeds the 4 Mi-float scratch
    st = _call(rt, 64, 64, 4, 1.0, 1.0, z, dirs, w, torch.zeros((200, 1), device="cuda"), A, A)
    assert st == 1
    assert b"static scratch" in rt.lib().rt_last_error()

"""The allocation-free regular-grid entry point (rt_formal_solution_regular_noalloc), called
through the C ABI.

It serves callers that cannot allocate device memory -- code in host callbacks or stream-ordered
regions that must not synchronise the device, plugins whose host application owns every
allocation, processes under a fixed device-memory budget -- by taking its scratch from one static
device array.  It must give the FP64 oracle's J (and rt_formal_solution's) on periodic and closed
sides with every inflow condition, on two calls in a row (the calls share the static array, so the
second must not see anything of the first), with directions in one hemisphere only, without
changing the device's free memory, and must refuse a problem larger than its fixed scratch before
touching the device.  This file is collected last so that a run stopping at the first failure
has run every other test first."""
import ctypes

import numpy as np
import pytest

import oracle
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


def _call(rt, nx, ny, nz, dx, dy, z, dirs, w, alpha, S, J, bc=0, I_bc=None, periodic=1):
    import torch
    z = np.ascontiguousarray(z, np.float64)
    d = np.ascontiguousarray(dirs, np.float64)
    ww = np.ascontiguousarray(w, np.float64)
    st = torch.cuda.current_stream().cuda_stream
    return rt.lib().rt_formal_solution_regular_noalloc(
        nx, ny, nz, dx, dy, z.ctypes.data, int(periodic), len(d), d.ctypes.data, ww.ctypes.data,
        alpha.shape[0], alpha.data_ptr(), S.data_ptr(), bc,
        None if I_bc is None else I_bc.data_ptr(), J.data_ptr(), st)


@pytest.mark.parametrize("periodic", [1, 0])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_noalloc_matches_oracle_twice(rt, periodic, bc):
    """Two calls in a row with different inputs (the second with one wavelength fewer) against the
    FP64 oracle and against rt_formal_solution."""
    import torch
    nx, ny, nz = 24, 20, 40
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(nx, ny, nz)
    dirs, w = s4_quadrature()
    g = rt.RegularGrid(nx, ny, nz, dx, dy, z, dirs, w, periodic=bool(periodic))
    rng = np.random.default_rng(10 * bc + periodic)
    inputs = [(np.stack([a, 2.0 * a]), np.stack([s, 0.5 * s])),
              (np.stack([a * rng.uniform(0.5, 2.0, a.size)]), np.stack([s[::-1].copy()]))]
    for al, sv in inputs:
        nlam = al.shape[0]
        ibc = rng.uniform(0.0, 2.0, (len(dirs), nlam, nx * ny)) * s.max() if bc == 2 else None
        A, S = to_gpu(al), to_gpu(sv)
        Ib = to_gpu(ibc) if ibc is not None else None
        J = torch.full((nlam, nx * ny * nz), float("nan"), device="cuda")
        assert _call(rt, nx, ny, nz, dx, dy, z, dirs, w, A, S, J, bc, Ib, periodic) == 0
        torch.cuda.synchronize()
        J_orc = oracle.sc_regular(nx, ny, nz, dx, dy, z, dirs, w, al, sv, bc=bc, ibc=ibc,
                                  periodic=bool(periodic))
        assert_parity(J.cpu().numpy(), J_orc, what=f"no-alloc J vs oracle, bc {bc}")
        J_ref = rt.formal_solution(g, A, S, bc=bc, I_bc=Ib)
        assert_parity(J.cpu().numpy(), J_ref.cpu().numpy().astype(np.float64), rel=2e-6,
                      what="no-alloc J vs rt_formal_solution")


@pytest.mark.parametrize("hemisphere", [1, -1])
def test_noalloc_one_hemisphere(rt, hemisphere):
    """Directions all upward (or all downward): the single pass writes J on its first plane."""
    import torch
    nx, ny, nz = 16, 16, 24
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(nx, ny, nz)
    dirs, w = s4_quadrature()
    keep = dirs[:, 2] * hemisphere > 0
    d, ww = dirs[keep], w[keep] * 2.0
    A, S = to_gpu(a[None]), to_gpu(s[None])
    J = torch.full((1, nx * ny * nz), float("nan"), device="cuda")
    assert _call(rt, nx, ny, nz, dx, dy, z, d, ww, A, S, J, bc=0) == 0
    torch.cuda.synchronize()
    J_orc = oracle.sc_regular(nx, ny, nz, dx, dy, z, d, ww, a[None], s[None], bc=0)
    assert_parity(J.cpu().numpy(), J_orc, what="one hemisphere")


def test_noalloc_leaves_free_memory_unchanged(rt):
    """After a first call (which may load the device code), further calls allocate nothing: the
    device's free memory is the same before and after."""
    import torch
    nx, ny, nz = 32, 32, 64
    atm, f, (x, y, z, dx, dy), a, s = lte_regular(nx, ny, nz)
    dirs, w = s4_quadrature()
    A, S = to_gpu(np.stack([a, a])), to_gpu(np.stack([s, s]))
    J = torch.empty_like(A)
    assert _call(rt, nx, ny, nz, dx, dy, z, dirs, w, A, S, J) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _call(rt, nx, ny, nz, dx, dy, z, dirs, w, A, S, J) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversized_problem(rt):
    import torch
    dirs, w = s4_quadrature()
    z = np.arange(4, dtype=np.float64)
    A = torch.zeros(1, device="cuda")
    # 2 * 200 wavelengths * 12 directions * 64 * 64 floats exceeds the 4 Mi-float scratch
    st = _call(rt, 64, 64, 4, 1.0, 1.0, z, dirs, w, torch.zeros((200, 1), device="cuda"), A, A)
    assert st == 1
    assert b"static scratch" in rt.lib().rt_last_error()

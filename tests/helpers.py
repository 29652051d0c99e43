"""Shared helpers of the test suite: tolerances and seeded problem set-ups."""
import functools

import numpy as np

REL = 1e-4          # GPU (FP32) vs oracle (FP64), relative
FLOOR = 1e-6        # absolute floor as a fraction of the field's largest magnitude


def assert_parity(got, ref, rel=REL, floor=FLOOR, what=""):
    """|got - ref| <= rel * max(|ref|, floor * max|ref|), element by element."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max())
    err = np.abs(got - ref) / scale
    i = int(np.argmax(err))
    assert err.flat[i] <= rel, (f"{what}: max rel err {err.flat[i]:.3e} at {i}: "
                                f"got {got.flat[i]:.6e} ref {ref.flat[i]:.6e}")
    return float(err.max())


@functools.lru_cache(maxsize=None)
def lte_regular(nx, ny, nz, seed=0):
    from oracle.physics import lte_alpha_S
    from synth import make_atmosphere
    from synth.atmosphere import regular_fields
    atm = make_atmosphere(seed)
    f, (x, y, z, dx, dy) = regular_fields(nx, ny, nz, atm)
    a, s = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    return atm, f, (x, y, z, dx, dy), a, s


@functools.lru_cache(maxsize=None)
def voronoi_grid(nsites, kind, seed, atm_seed=0):
    from synth import make_atmosphere, make_voronoi_grid
    atm = make_atmosphere(atm_seed)
    g = make_voronoi_grid(atm, nsites, kind, seed)
    f = atm.fields(g["xyz"][:, 0], g["xyz"][:, 1], g["xyz"][:, 2])
    return atm, g, f


def to_gpu(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")

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


def tie_directions():
    """The 8 directions (+-1, +-1, +-2)/sqrt(6), weights 1/8: on a cubic lattice the neighbours
    (1, 0, 1) and (0, 1, 1) (mirrored to each direction) tie exactly for second place."""
    d = np.array([(sx, sy, 2.0 * sz) for sz in (1, -1) for sy in (1, -1) for sx in (1, -1)])
    d /= np.sqrt(6.0)
    return d, np.full(8, 1.0 / 8.0)


def lattice_grid(m=4, mz=None):
    """m x m x mz sites (mz = m by default) on a lattice of cubic cells of side 1/m (box 1 x 1 x
    mz/m), each with its 26 lattice neighbours as the neighbour list (periodic images in x and y,
    wall mirrors below the first and above the last layer).  Symmetric directions see exact ties
    in alignment, so the tie rules decide; with m = 1 the tied neighbours are two periodic images
    of one site (every lateral neighbour is an image), whose records agree whichever wins."""
    mz = m if mz is None else mz
    hx = hz = 1.0 / m
    idx = lambda i, j, k: (k * m + j) * m + i          # noqa: E731
    xyz = np.array([((i + 0.5) * hx, (j + 0.5) * hx, (k + 0.5) * hz)
                    for k in range(mz) for j in range(m) for i in range(m)])
    off, code, shift = [0], [], []
    for k in range(mz):
        for j in range(m):
            for i in range(m):
                for dk in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        for di in (-1, 0, 1):
                            if di == dj == dk == 0:
                                continue
                            ii, jj, kk = i + di, j + dj, k + dk
                            sx = -1 if ii < 0 else (1 if ii >= m else 0)
                            sy = -1 if jj < 0 else (1 if jj >= m else 0)
                            s = idx(ii % m, jj % m, min(max(kk, 0), mz - 1))
                            if kk < 0:
                                c = -1 - 2 * s                      # mirror in the bottom wall
                            elif kk >= mz:
                                c = -2 - 2 * s                      # mirror in the top wall
                            else:
                                c = s
                            code.append(c)
                            shift.append((sx + 1) * 3 + (sy + 1))
                off.append(len(code))
    return dict(xyz=xyz, nbr_off=np.array(off, np.int64), nbr_idx=np.array(code, np.int32),
                nbr_shift=np.array(shift, np.int8), box=(0.0, 1.0, 0.0, 1.0, 0.0, mz * hz))

"""Oracle of the rejection sampling of Voronoi sites (Sect. 2.4: a proposal position uniform in
the box is kept when the target function there is at least a uniform random rejection level; repeat
until the wanted number of sites).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The random numbers come from the counter-based generator Philox4x64-10 (Salmon, Moraes, Dror &
Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3"), written here from its published
definition; the CUDA path has its own.  Proposal p (0, 1, 2, ...) draws the block of counter
(p, 0, 0, 0) under key (seed, 0); its four 64-bit words give, through u = (w >> 11) 2^-53, the
position (x0 + u0 Lx, y0 + u1 Ly, z0 + u2 Lz) and the rejection level u3.

The target f is given at the points of a mesh: (x0 + i Lx/nx, y0 + j Ly/ny, z_k), periodic in x
and y, z_k ascending.  At a proposal it is interpolated trilinearly (z clamped to [z_0, z_{nz-1}]),
each linear step written lerp(a, b, t) = a + t (b - a), and the proposal is kept iff
f(r) >= u3 * max f.  Every floating-point step is a single IEEE double operation, in the order
written, so that the decision can be reproduced exactly.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """High and low 64-bit words of the 128-bit products a * b (uint64 arrays)."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    al, ah = a & _MASK32, a >> _S32
    bl, bh = b & _MASK32, b >> _S32
    ll = al * bl
    hl = ah * bl
    lh = al * bh
    hh = ah * bh
    cross = (ll >> _S32) + (hl & _MASK32) + lh          # < 2^64: no wrap
    hi = hh + (hl >> _S32) + (cross >> _S32)
    lo = a * b                                          # wraps mod 2^64
    return hi, lo


def philox4x64(counter, key, rounds=10):
    """Philox4x64 blocks: counter [n, 4] uint64, key (k0, k1) -> [n, 4] uint64."""
    with np.errstate(over="ignore"):
        c = np.array(counter, np.uint64, copy=True).reshape(-1, 4)
        k0 = np.uint64(key[0])
        k1 = np.uint64(key[1])
        for r in range(rounds):
            if r:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = _mulhilo(M0, c[:, 0])
            hi1, lo1 = _mulhilo(M1, c[:, 2])
            c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
        return c


def uniform53(w):
    """[0, 1) doubles from 64-bit words: the top 53 bits times 2^-53 (exact)."""
    return (np.asarray(w, np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def _lerp(a, b, t):
    return a + t * (b - a)


def interpolate(f, z, box, pts):
    """Trilinear value of the mesh function f [nz][ny][nx] at pts [n, 3]."""
    nz, ny, nx = f.shape
    f = np.asarray(f, np.float64)
    x0, x1, y0, y1 = box[0], box[1], box[2], box[3]
    dx = (x1 - x0) / nx
    dy = (y1 - y0) / ny
    fx = (pts[:, 0] - x0) / dx
    fy = (pts[:, 1] - y0) / dy
    i0 = np.floor(fx)
    j0 = np.floor(fy)
    tx = fx - i0
    ty = fy - j0
    i0 = i0.astype(np.int64) % nx
    j0 = j0.astype(np.int64) % ny
    i1 = (i0 + 1) % nx
    j1 = (j0 + 1) % ny
    pz = pts[:, 2]
    # k0: the last plane at or below pz (first plane below z_0, last-but-one above z_{nz-1})
    k0 = np.searchsorted(z, pz, side="right") - 1
    k0 = np.clip(k0, 0, nz - 2)
    zlo = z[k0]
    zhi = z[k0 + 1]
    tz = (pz - zlo) / (zhi - zlo)
    tz = np.where(pz <= z[0], 0.0, np.where(pz >= z[-1], 1.0, tz))
    k1 = k0 + 1
    c00 = _lerp(f[k0, j0, i0], f[k0, j0, i1], tx)
    c10 = _lerp(f[k0, j1, i0], f[k0, j1, i1], tx)
    c01 = _lerp(f[k1, j0, i0], f[k1, j0, i1], tx)
    c11 = _lerp(f[k1, j1, i0], f[k1, j1, i1], tx)
    c0 = _lerp(c00, c10, ty)
    c1 = _lerp(c01, c11, ty)
    return _lerp(c0, c1, tz)


def proposals(seed, first, count, box):
    """Positions [count, 3] and rejection levels [count] of proposals first .. first+count-1."""
    ctr = np.zeros((count, 4), np.uint64)
    ctr[:, 0] = np.arange(first, first + count, dtype=np.uint64)
    w = philox4x64(ctr, (seed, 0))
    u = uniform53(w)
    x0, x1, y0, y1, z0, z1 = box
    pos = np.stack([x0 + u[:, 0] * (x1 - x0), y0 + u[:, 1] * (y1 - y0),
                    z0 + u[:, 2] * (z1 - z0)], axis=1)
    return pos, u[:, 3]


def rejection_sample(f, z, box, nsites, seed, batch=1 << 16, max_proposals=None):
    """The first nsites accepted proposals, in proposal order, and the number of proposals drawn
    up to and including the last accepted one.  Raises after max_proposals (default
    1000 nsites + 2^20) proposals without enough sites."""
    f = np.asarray(f, np.float32).astype(np.float64)
    z = np.asarray(z, np.float64)
    fmax = float(f.max())
    if max_proposals is None:
        max_proposals = 1000 * nsites + (1 << 20)
    out = []
    have = 0
    first = 0
    while have < nsites:
        if first >= max_proposals:
            raise RuntimeError("rejection sampling: too few proposals accepted")
        pos, prej = proposals(seed, first, batch, box)
        keep = interpolate(f, z, box, pos) >= prej * fmax
        idx = np.nonzero(keep)[0][:nsites - have]
        out.append(pos[idx])
        have += idx.size
        if have == nsites:
            last = first + int(idx[-1]) + 1 if idx.size else first
            return np.concatenate(out), last
        first += batch
    return np.concatenate(out), first

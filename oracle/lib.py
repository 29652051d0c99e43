"""ctypes binding of the oracle's C part (orc.c), built with gcc on first use.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i8 = ctypes.POINTER(ctypes.c_int8)


def build(force=False):
    """Compile liborc.so (gcc, -O2, OpenMP) if missing or older than its source."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_linear_weights.argtypes = [ctypes.c_double, _d, _d, _d]
            lib.orc_linear_weights_deriv.argtypes = [ctypes.c_double, _d, _d, _d]
            lib.orc_sc_regular.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                _d, ctypes.c_int, ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, ctypes.c_int, _d,
                _d, _d]
            lib.orc_sc_regular_face.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                _d, ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, _d]
            lib.orc_sc_regular_adjoint.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                _d, ctypes.c_int, _d, ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, _d]
            lib.orc_voronoi_tables.argtypes = [ctypes.c_int64, _d, _i64, _i32, _i8, _d,
                                               ctypes.c_int, _d, ctypes.c_double, _i32, _d, _d,
                                               _i32, _i64]
            lib.orc_voronoi_fs.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d, _i32, _d, _d,
                                           _i64, ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, _d]
            lib.orc_voronoi_adjoint.argtypes = [ctypes.c_int64, _i32, _d, _d, _i64, ctypes.c_int,
                                                ctypes.c_int, _d, _d, ctypes.c_int, _d, _d, _d]
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
        return _lib


def _p(a, t=_d):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return _get().orc_num_threads()


def linear_weights(d):
    """(exp(-d), w0, w1) and their d-derivatives for one optical-depth interval."""
    lib = _get()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_linear_weights(float(d), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    da, db, dc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_linear_weights_deriv(float(d), ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc))
    return (a.value, b.value, c.value), (da.value, db.value, dc.value)


def sc_regular(nx, ny, nz, dx, dy, z, dirs, wdir, alpha, S, bc=0, ibc=None, periodic=True,
               want_I=False):
    """Regular-grid formal solution.  alpha, S: [nlam][npt].  Returns J (and I[ndir][nlam][npt])."""
    alpha = _f64(alpha)
    S = _f64(S)
    nlam = alpha.shape[0]
    npt = nx * ny * nz
    assert alpha.shape == (nlam, npt) and S.shape == (nlam, npt)
    dirs = _f64(dirs)
    wdir = _f64(wdir)
    z = _f64(z)
    ndir = len(dirs)
    J = np.empty((nlam, npt))
    I = np.empty((ndir, nlam, npt)) if want_I else None
    ibc = None if ibc is None else _f64(ibc)
    rc = _get().orc_sc_regular(nx, ny, nz, dx, dy, _p(z), int(periodic), ndir, _p(dirs),
                               _p(wdir), nlam, _p(alpha), _p(S), bc, _p(ibc), _p(J), _p(I))
    if rc:
        raise MemoryError("oracle allocation failed")
    return (J, I) if want_I else J


def sc_regular_face(nx, ny, nz, dx, dy, z, dirs, wdir, alpha, S, bc=0, ibc=None, want_I=False):
    """Regular-grid formal solution by face-hitting short characteristics (periodic x, y).
    alpha, S: [nlam][npt].  Returns J (and I[ndir][nlam][npt])."""
    alpha = _f64(alpha)
    S = _f64(S)
    nlam = alpha.shape[0]
    npt = nx * ny * nz
    assert alpha.shape == (nlam, npt) and S.shape == (nlam, npt)
    dirs = _f64(dirs)
    wdir = _f64(wdir)
    ndir = len(dirs)
    J = np.empty((nlam, npt))
    I = np.empty((ndir, nlam, npt)) if want_I else None
    ibc = None if ibc is None else _f64(ibc)
    rc = _get().orc_sc_regular_face(nx, ny, nz, dx, dy, _p(_f64(z)), ndir, _p(dirs), _p(wdir),
                                    nlam, _p(alpha), _p(S), bc, _p(ibc), _p(J), _p(I))
    if rc:
        raise RuntimeError("oracle: allocation failed or a plane system is singular")
    return (J, I) if want_I else J


def sc_regular_adjoint(nx, ny, nz, dx, dy, z, mu, alpha, S, gI, bc=0, periodic=True):
    """Gradients (g_alpha, g_S) of sum(gI * I_mu) for one direction mu (FP64, exact)."""
    alpha = _f64(alpha)
    S = _f64(S)
    gI = _f64(gI)
    nlam = alpha.shape[0]
    ga = np.zeros_like(alpha)
    gs = np.zeros_like(alpha)
    rc = _get().orc_sc_regular_adjoint(nx, ny, nz, dx, dy, _p(_f64(z)), int(periodic),
                                       _p(_f64(mu)), nlam, _p(alpha), _p(S), bc, _p(gI), _p(ga),
                                       _p(gs))
    if rc:
        raise MemoryError("oracle allocation failed")
    return ga, gs


def voronoi_tables(xyz, nbr_off, nbr_idx, nbr_shift, box, dirs, r_exp=7.0):
    """Upwind tables per (dir, site): k[ndir][n][2], w, len, and level[ndir][n]."""
    xyz = _f64(xyz)
    n = len(xyz)
    dirs = _f64(dirs)
    ndir = len(dirs)
    off = np.ascontiguousarray(nbr_off, np.int64)
    idx = np.ascontiguousarray(nbr_idx, np.int32)
    sh = np.ascontiguousarray(nbr_shift, np.int8)
    k = np.empty((ndir, n, 2), np.int32)
    w = np.empty((ndir, n, 2))
    ln = np.empty((ndir, n, 2))
    lv = np.empty((ndir, n), np.int32)
    nfb = ctypes.c_int64(0)
    rc = _get().orc_voronoi_tables(n, _p(xyz), _p(off, _i64), _p(idx, _i32), _p(sh, _i8),
                                   _p(_f64(box)), ndir, _p(dirs), float(r_exp), _p(k, _i32),
                                   _p(w), _p(ln), _p(lv, _i32), ctypes.byref(nfb))
    if rc:
        raise MemoryError("oracle allocation failed")
    return dict(k=k, w=w, len=ln, level=lv, n_fallback=nfb.value)


def voronoi_order(level):
    """Per direction, the sites sorted by level (stable): a valid upwind visiting order."""
    return np.ascontiguousarray(np.argsort(level, axis=1, kind="stable").astype(np.int64))


def voronoi_fs(tab, dirs, wdir, alpha, S, bc=0, ibc=None, order=None, want_I=False):
    alpha = _f64(alpha)
    S = _f64(S)
    nlam, n = alpha.shape
    ndir = len(dirs)
    if order is None:
        order = voronoi_order(tab["level"])
    J = np.empty((nlam, n))
    I = np.empty((ndir, nlam, n)) if want_I else None
    ibc = None if ibc is None else _f64(ibc)
    rc = _get().orc_voronoi_fs(n, ndir, _p(_f64(dirs)), _p(_f64(wdir)), _p(tab["k"], _i32),
                               _p(_f64(tab["w"])), _p(_f64(tab["len"])),
                               _p(np.ascontiguousarray(order, np.int64), _i64), nlam, _p(alpha),
                               _p(S), bc, _p(ibc), _p(J), _p(I))
    if rc:
        raise MemoryError("oracle allocation failed")
    return (J, I) if want_I else J


def voronoi_adjoint(tab, d, up, alpha, S, gI, bc=0, order=None):
    """Gradients (g_alpha, g_S) of sum(gI * I_d) for direction index d of the tables."""
    alpha = _f64(alpha)
    S = _f64(S)
    nlam, n = alpha.shape
    if order is None:
        order = voronoi_order(tab["level"])
    ga = np.zeros_like(alpha)
    gs = np.zeros_like(alpha)
    k = np.ascontiguousarray(tab["k"][d])
    w = _f64(tab["w"][d])
    ln = _f64(tab["len"][d])
    od = np.ascontiguousarray(order[d], np.int64)
    rc = _get().orc_voronoi_adjoint(n, _p(k, _i32), _p(w), _p(ln), _p(od, _i64), int(up), nlam,
                                    _p(alpha), _p(S), bc, _p(_f64(gI)), _p(ga), _p(gs))
    if rc:
        raise MemoryError("oracle allocation failed")
    return ga, gs

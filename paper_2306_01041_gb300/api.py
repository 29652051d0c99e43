"""Python face of librt.so: the same calls as include/rt.h on torch tensors.

Only argument marshalling happens here -- shapes, dtypes, devices and raw pointers are checked
and passed through; every step of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from ._lib import check, lib


def kernel_launches() -> int:
    """Kernel launches the library has issued in this process (graph captures count once)."""
    return int(lib().rt_kernel_launches())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Grid:
    """A regular or Voronoi grid with its precomputed upwind tables (rt_grid_create)."""

    def __init__(self, desc: L.GridDesc, keep):
        self._keep = keep
        h = ctypes.c_void_p()
        check(lib().rt_grid_create(ctypes.byref(desc), _stream(), ctypes.byref(h)))
        self._h = h
        self.kind = desc.kind
        self.ndir = desc.ndir
        npt, ntop, ml, nfb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        check(lib().rt_grid_info(h, ctypes.byref(npt), ctypes.byref(ntop), ctypes.byref(ml),
                                 ctypes.byref(nfb)))
        self.npt, self.ntop, self.max_levels, self.n_fallback = (npt.value, ntop.value, ml.value,
                                                                 nfb.value)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.rt_grid_destroy(h)
            self._h = None

    def set_scheme(self, scheme):
        """Short-characteristics scheme of a regular grid: "plane" (default) or "face"."""
        code = {"plane": L.RT_SC_PLANE, "face": L.RT_SC_FACE}[scheme]
        check(lib().rt_grid_set_scheme(self._h, code))
        self.scheme = scheme
        return self

    def build_tables_device(self, stream=None):
        """Rebuild a Voronoi grid's upwind tables and levels on the GPU (in place)."""
        check(lib().rt_grid_build_tables_device(self._h, _stream(stream)))
        npt, ntop, ml, nfb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        check(lib().rt_grid_info(self._h, ctypes.byref(npt), ctypes.byref(ntop), ctypes.byref(ml),
                                 ctypes.byref(nfb)))
        self.max_levels, self.n_fallback = ml.value, nfb.value
        return self

    def top_points(self):
        out = np.empty(self.ntop, np.int64)
        check(lib().rt_grid_top_points(self._h, out.ctypes.data_as(L.PI64)))
        return out

    def tables(self):
        """Voronoi upwind tables (k, w, len, level) in site order, as numpy arrays."""
        n, nd = self.npt, self.ndir
        k = np.empty((nd, n, 2), np.int32)
        w = np.empty((nd, n, 2), np.float32)
        ln = np.empty((nd, n, 2), np.float32)
        lv = np.empty((nd, n), np.int32)
        check(lib().rt_grid_tables(self._h, k.ctypes.data_as(L.PI32), w.ctypes.data_as(L.PF),
                                   ln.ctypes.data_as(L.PF), lv.ctypes.data_as(L.PI32)))
        return dict(k=k, w=w, len=ln, level=lv)


def _dirs(dirs, wdir):
    d = _np(dirs, np.float64)
    w = _np(wdir, np.float64)
    if d.ndim != 2 or d.shape[1] != 3 or len(w) != len(d):
        raise ValueError("dirs must be [ndir][3] with ndir weights")
    return d, w


def RegularGrid(nx, ny, nz, dx, dy, z, dirs, wdir, periodic=True, scheme="plane") -> Grid:
    z = _np(z, np.float64)
    d, w = _dirs(dirs, wdir)
    desc = L.GridDesc()
    desc.kind = L.RT_GRID_REGULAR
    desc.nx, desc.ny, desc.nz = nx, ny, nz
    desc.dx, desc.dy = dx, dy
    desc.z = z.ctypes.data_as(L.PD)
    desc.periodic_xy = int(bool(periodic))
    desc.ndir = len(d)
    desc.dirs = d.ctypes.data_as(L.PD)
    desc.wdir = w.ctypes.data_as(L.PD)
    desc.r_exponent = 7.0
    g = Grid(desc, (z, d, w))
    g.shape = (nz, ny, nx)
    g.scheme = "plane"
    if scheme != "plane":
        g.set_scheme(scheme)
    return g


def VoronoiGrid(xyz, nbr_off, nbr_idx, nbr_shift, box, dirs, wdir, r_exponent=7.0,
                periodic=True) -> Grid:
    xyz = _np(xyz, np.float64)
    off = _np(nbr_off, np.int64)
    idx = _np(nbr_idx, np.int32)
    sh = None if nbr_shift is None else _np(nbr_shift, np.int8)
    d, w = _dirs(dirs, wdir)
    desc = L.GridDesc()
    desc.kind = L.RT_GRID_VORONOI
    desc.nsites = len(xyz)
    desc.xyz = xyz.ctypes.data_as(L.PD)
    desc.nbr_off = off.ctypes.data_as(L.PI64)
    desc.nbr_idx = idx.ctypes.data_as(L.PI32)
    desc.nbr_shift = sh.ctypes.data_as(L.PI8) if sh is not None else None
    desc.box = (ctypes.c_double * 6)(*box)
    desc.periodic_xy = int(bool(periodic))
    desc.ndir = len(d)
    desc.dirs = d.ctypes.data_as(L.PD)
    desc.wdir = w.ctypes.data_as(L.PD)
    desc.r_exponent = r_exponent
    return Grid(desc, (xyz, off, idx, sh, d, w))


def formal_solution(grid: Grid, alpha, S, bc=L.RT_BC_THERMAL, I_bc=None, want_I=False,
                    J=None, stream=None):
    """J [nlam][npt] (and I [ndir][nlam][npt] when want_I) from alpha, S [nlam][npt]."""
    nlam = alpha.shape[0]
    shp = (nlam, grid.npt)
    pa, ps = _dev(alpha, shp, "alpha"), _dev(S, shp, "S")
    if J is None:
        J = torch.empty(shp, device=alpha.device, dtype=torch.float32)
    pj = _dev(J, shp, "J")
    I = None
    pI = None
    if want_I:
        I = torch.empty((grid.ndir,) + shp, device=alpha.device, dtype=torch.float32)
        pI = _dev(I)
    pbc = None
    if bc == L.RT_BC_ARRAY:
        pbc = _dev(I_bc, None, "I_bc")
    check(lib().rt_formal_solution(grid.handle, nlam, pa, ps, bc, pbc, pj, pI, _stream(stream)))
    return (J, I) if want_I else J


def source_terms_lte(T, rho, kappa0, lam, stream=None):
    n = T.numel()
    alpha = torch.empty_like(T)
    S = torch.empty_like(T)
    check(lib().rt_source_terms_lte(n, _dev(T), _dev(rho), float(kappa0), float(lam), _dev(alpha),
                                    _dev(S), _stream(stream)))
    return alpha, S


def source_terms_lte_adjoint(T, rho, kappa0, lam, g_alpha, g_S, stream=None):
    gT = torch.empty_like(T)
    check(lib().rt_source_terms_lte_adjoint(T.numel(), _dev(T), _dev(rho), float(kappa0),
                                            float(lam), _dev(g_alpha), _dev(g_S), _dev(gT),
                                            _stream(stream)))
    return gT


class Atom:
    """rt_atom from a model-atom dict (E_cm, g, f, voigt_a, q_coll, lam, wlam, kind)."""

    def __init__(self, data, kappa0):
        self.lam = _np(data["lam"], np.float64)
        self.wlam = _np(data["wlam"], np.float64)
        self.kind = _np(data["kind"], np.int32)
        d = L.AtomDesc()
        d.E_cm = (ctypes.c_double * 3)(*data["E_cm"])
        d.g = (ctypes.c_double * 3)(*data["g"])
        d.f_line = float(data["f"])
        d.voigt_a = float(data["voigt_a"])
        d.q_coll = float(data["q_coll"])
        d.kappa0 = float(kappa0)
        d.nlam = len(self.lam)
        d.lam = self.lam.ctypes.data_as(L.PD)
        d.wlam = self.wlam.ctypes.data_as(L.PD)
        d.kind = self.kind.ctypes.data_as(L.PI32)
        self.desc = d
        self.nlam = len(self.lam)


class Atmos:
    """rt_atmos over float32 CUDA tensors T, rho, ne, nH [npt]."""

    def __init__(self, T, rho, ne, nH):
        self.tensors = (T, rho, ne, nH)
        d = L.AtmosDesc()
        d.T, d.rho, d.ne, d.nH = (_dev(T, None, "T"), _dev(rho, None, "rho"), _dev(ne, None, "ne"),
                                  _dev(nH, None, "nH"))
        self.desc = d


def lte_populations(grid, atom: Atom, atm: Atmos, stream=None):
    pops = torch.empty((3, grid.npt), device="cuda", dtype=torch.float32)
    check(lib().rt_lte_populations(grid.handle, ctypes.byref(atom.desc), ctypes.byref(atm.desc),
                                   _dev(pops), _stream(stream)))
    return pops


def source_terms(grid, atom: Atom, atm: Atmos, pops, stream=None, out=None):
    """alpha, S [nlam][npt] from the populations; ``out`` = (alpha, S) to write in place."""
    shp = (atom.nlam, grid.npt)
    if out is None:
        alpha = torch.empty(shp, device="cuda", dtype=torch.float32)
        S = torch.empty(shp, device="cuda", dtype=torch.float32)
    else:
        alpha, S = out
        _dev(alpha, shp, "alpha")
        _dev(S, shp, "S")
    check(lib().rt_source_terms(grid.handle, ctypes.byref(atom.desc), ctypes.byref(atm.desc),
                                _dev(pops, (3, grid.npt), "pops"), _dev(alpha), _dev(S),
                                _stream(stream)))
    return alpha, S


def source_terms_adjoint(grid, atom: Atom, atm: Atmos, pops, g_alpha, g_S, stream=None):
    gT = torch.empty(grid.npt, device="cuda", dtype=torch.float32)
    check(lib().rt_source_terms_adjoint(grid.handle, ctypes.byref(atom.desc),
                                        ctypes.byref(atm.desc), _dev(pops), _dev(g_alpha),
                                        _dev(g_S), _dev(gT), _stream(stream)))
    return gT


def statistical_equilibrium(grid, atom: Atom, atm: Atmos, J, pops, stream=None):
    """Updates pops in place; returns the device scalar max |dn/n|."""
    dmax = torch.zeros(1, device="cuda", dtype=torch.float32)
    check(lib().rt_statistical_equilibrium(grid.handle, ctypes.byref(atom.desc),
                                           ctypes.byref(atm.desc), _dev(J), _dev(pops),
                                           _dev(dmax), _stream(stream)))
    return dmax


def _iterate_ex(grid, atom, atm, pops, max_iter, tol, use_graph, newton, fixed_lstar, ng_period,
                stream):
    hist = np.zeros(max_iter, np.float32)
    it = ctypes.c_int(0)
    st = lib().rt_lambda_iterate_ex(grid.handle, ctypes.byref(atom.desc), ctypes.byref(atm.desc),
                                    _dev(pops, (3, grid.npt), "pops"), max_iter, float(tol),
                                    ctypes.byref(it), hist.ctypes.data_as(L.PF), int(use_graph),
                                    int(newton), int(bool(fixed_lstar)), int(ng_period),
                                    _stream(stream))
    if st not in (L.RT_OK, L.RT_ENOCONV):
        check(st)
    return it.value, hist[:it.value].copy(), st == L.RT_OK


def ng_extrapolate(x0, x1, x2, x3, stream=None):
    """Ng extrapolation of four iterates (newest first); returns (x, ok)."""
    n = x0.numel()
    out = torch.empty_like(x0)
    scratch = torch.zeros(16, device=x0.device, dtype=torch.float32)
    ok = ctypes.c_int(0)
    check(lib().rt_ng_extrapolate(n, _dev(x0), _dev(x1), _dev(x2), _dev(x3), _dev(out),
                                  _dev(scratch), ctypes.byref(ok), _stream(stream)))
    return out, bool(ok.value)


def lambda_iterate(grid, atom: Atom, atm: Atmos, pops, max_iter=300, tol=1e-3, use_graph=True,
                   ng_period=0, stream=None):
    """Runs the Lambda iteration in place on pops; returns (iterations, history, converged).
    ``ng_period`` > 0: Ng extrapolation after every ng_period-th iteration."""
    if ng_period:
        return _iterate_ex(grid, atom, atm, pops, max_iter, tol, use_graph, -1, True, ng_period,
                           stream)
    hist = np.zeros(max_iter, np.float32)
    it = ctypes.c_int(0)
    st = lib().rt_lambda_iterate(grid.handle, ctypes.byref(atom.desc), ctypes.byref(atm.desc),
                                 _dev(pops, (3, grid.npt), "pops"), max_iter, float(tol),
                                 ctypes.byref(it), hist.ctypes.data_as(L.PF), int(use_graph),
                                 _stream(stream))
    if st not in (L.RT_OK, L.RT_ENOCONV):
        check(st)
    return it.value, hist[:it.value].copy(), st == L.RT_OK


def lambda_star(grid, alpha, bc=L.RT_BC_THERMAL, out=None, stream=None):
    """Lambda* [nlam][npt]: dJ_p/dS_p at fixed opacities (the diagonal of the Lambda operator)."""
    nlam = alpha.shape[0]
    Ls = torch.empty_like(alpha) if out is None else out
    check(lib().rt_lambda_star(grid.handle, nlam, _dev(alpha, (nlam, grid.npt), "alpha"), int(bc),
                               _dev(Ls, (nlam, grid.npt), "Lstar"), _stream(stream)))
    return Ls


def statistical_equilibrium_ali(grid, atom: Atom, atm: Atmos, J, Lstar, S_old, pops, newton=3,
                                stream=None):
    """Accelerated update of pops in place (see rt_statistical_equilibrium_ali); returns the
    device scalar max |dn/n|."""
    dmax = torch.zeros(1, device="cuda", dtype=torch.float32)
    check(lib().rt_statistical_equilibrium_ali(grid.handle, ctypes.byref(atom.desc),
                                               ctypes.byref(atm.desc), _dev(J), _dev(Lstar),
                                               _dev(S_old), _dev(pops), _dev(dmax), int(newton),
                                               _stream(stream)))
    return dmax


def lambda_iterate_ali(grid, atom: Atom, atm: Atmos, pops, max_iter=300, tol=1e-3,
                       use_graph=True, newton=1, fixed_lstar=True, ng_period=0, stream=None):
    """Accelerated Lambda iteration in place on pops; returns (iterations, history, converged).
    ``fixed_lstar``: Lambda* of the starting opacities held fixed (else recomputed per iteration);
    ``ng_period`` > 0: Ng extrapolation after every ng_period-th iteration."""
    if ng_period:
        return _iterate_ex(grid, atom, atm, pops, max_iter, tol, use_graph, newton, fixed_lstar,
                           ng_period, stream)
    hist = np.zeros(max_iter, np.float32)
    it = ctypes.c_int(0)
    st = lib().rt_lambda_iterate_ali(grid.handle, ctypes.byref(atom.desc),
                                     ctypes.byref(atm.desc), _dev(pops, (3, grid.npt), "pops"),
                                     max_iter, float(tol), ctypes.byref(it),
                                     hist.ctypes.data_as(L.PF), int(use_graph), int(newton),
                                     int(bool(fixed_lstar)), _stream(stream))
    if st not in (L.RT_OK, L.RT_ENOCONV):
        check(st)
    return it.value, hist[:it.value].copy(), st == L.RT_OK


class IDW:
    """Two-nearest inverse-distance interpolation from a Voronoi grid's sites to a regular mesh
    (the final synthesis of Sect. 2.5)."""

    def __init__(self, voronoi, mesh):
        h = ctypes.c_void_p()
        check(lib().rt_idw_create(voronoi.handle, mesh.handle, ctypes.byref(h)))
        self._h = h
        self.nsites, self.npt = voronoi.npt, mesh.npt

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.rt_idw_destroy(h)
            self._h = None

    def table(self):
        """(k [npt][2] int32, w [npt][2] float32) on the host."""
        k = np.empty((self.npt, 2), np.int32)
        w = np.empty((self.npt, 2), np.float32)
        check(lib().rt_idw_table(self._h, k.ctypes.data_as(L.PI32), w.ctypes.data_as(L.PF)))
        return k, w

    def interpolate(self, src, out=None, stream=None):
        nf = src.shape[0]
        dst = torch.empty((nf, self.npt), device=src.device, dtype=torch.float32) \
            if out is None else out
        check(lib().rt_idw_interpolate(self._h, nf, _dev(src, (nf, self.nsites), "src"),
                                       _dev(dst, (nf, self.npt), "dst"), _stream(stream)))
        return dst


def sample_sites(f, z, box, nsites, seed, stream=None):
    """Rejection sampling of nsites Voronoi sites (rt_sample_sites): f a float32 CUDA tensor
    [nz][ny][nx] (the target at the mesh points), z the mesh heights, box (x0, x1, y0, y1, z0, z1).
    Returns (xyz, nproposals): float64 CUDA [nsites][3] and the proposals drawn."""
    fp = _dev(f, name="f")
    if f.dim() != 3:
        raise ValueError("f must be [nz][ny][nx]")
    nz, ny, nx = f.shape
    zz = _np(z, np.float64)
    bx = _np(box, np.float64)
    if len(zz) != nz or bx.shape != (6,):
        raise ValueError("z must have nz entries and box six")
    xyz = torch.empty((int(nsites), 3), dtype=torch.float64, device=f.device)
    nprop = ctypes.c_int64()
    check(lib().rt_sample_sites(nx, ny, nz, zz.ctypes.data_as(L.PD), bx.ctypes.data_as(L.PD),
                                fp, int(nsites), int(seed), xyz.data_ptr(),
                                ctypes.byref(nprop), _stream(stream)))
    return xyz, nprop.value


def final_synthesis(idw: IDW, mesh, atom: Atom, mesh_atm: Atmos, site_pops, stream=None):
    """Emergent vertical intensity [nlam][nx ny] of the mesh from converged site populations:
    interpolation to the mesh, opacities and source functions there, long characteristics
    along mu = 1."""
    pops = idw.interpolate(site_pops, stream=stream)
    alpha, S = source_terms(mesh, atom, mesh_atm, pops, stream=stream)
    return emergent_intensity(mesh, (0.0, 0.0, 1.0), alpha, S, stream=stream)


def emergent_intensity(grid, direction, alpha, S, bc=L.RT_BC_THERMAL, stream=None):
    nlam = alpha.shape[0]
    d = (ctypes.c_double * 3)(*[float(v) for v in direction])
    out = torch.empty((nlam, grid.ntop), device=alpha.device, dtype=torch.float32)
    check(lib().rt_emergent_intensity(grid.handle, d, nlam, _dev(alpha), _dev(S), bc, _dev(out),
                                      _stream(stream)))
    return out


def emergent_map(grid, direction, alpha, S, npx, npy, bc=L.RT_BC_THERMAL, stream=None):
    """Emergent intensity along one direction on an npx x npy pixel grid, [nlam][npy * npx]:
    the top plane of a regular grid, or the emergent-layer sites of a Voronoi grid resampled by
    two-nearest inverse-distance weighting in (x, y)."""
    nlam = alpha.shape[0]
    d = (ctypes.c_double * 3)(*[float(v) for v in direction])
    out = torch.empty((nlam, npy * npx), device=alpha.device, dtype=torch.float32)
    check(lib().rt_emergent_map(grid.handle, d, nlam, _dev(alpha, (nlam, grid.npt), "alpha"),
                                _dev(S, (nlam, grid.npt), "S"), bc, int(npx), int(npy), _dev(out),
                                _stream(stream)))
    return out


def formal_solution_adjoint(grid, direction, alpha, S, gI_top, bc=L.RT_BC_THERMAL,
                            ckpt_stride=1, stream=None):
    nlam = alpha.shape[0]
    d = (ctypes.c_double * 3)(*[float(v) for v in direction])
    nbytes = lib().rt_adjoint_workspace_size(grid.handle, nlam, int(ckpt_stride))
    ws = torch.empty(max(nbytes, 16) // 4 + 4, device=alpha.device, dtype=torch.float32)
    ga = torch.empty_like(alpha)
    gs = torch.empty_like(alpha)
    check(lib().rt_formal_solution_adjoint(grid.handle, d, nlam, _dev(alpha), _dev(S), bc,
                                           _dev(gI_top, (nlam, grid.ntop), "gI_top"), _dev(ga),
                                           _dev(gs), int(ckpt_stride), _dev(ws), ws.numel() * 4,
                                           _stream(stream)))
    return ga, gs


class EmergentIntensity(torch.autograd.Function):
    """I_top = emergent intensity of (alpha, S) along one direction; backward runs the library's
    adjoint sweep (level checkpointing with ``ckpt_stride``)."""

    @staticmethod
    def forward(ctx, alpha, S, grid, direction, bc=L.RT_BC_THERMAL, ckpt_stride=1):
        ctx.grid, ctx.direction, ctx.bc, ctx.stride = grid, direction, bc, ckpt_stride
        ctx.save_for_backward(alpha, S)
        return emergent_intensity(grid, direction, alpha, S, bc)

    @staticmethod
    def backward(ctx, g):
        alpha, S = ctx.saved_tensors
        ga, gs = formal_solution_adjoint(ctx.grid, ctx.direction, alpha, S, g.contiguous(), ctx.bc,
                                         ctx.stride)
        return ga, gs, None, None, None, None


class SourceTerms(torch.autograd.Function):
    """(alpha, S) [nlam][npt] of the atom from the temperature T [npt] at fixed populations,
    density and electron density (rt_source_terms); backward gives dL/dT from dL/dalpha and dL/dS
    (rt_source_terms_adjoint).  Composed with EmergentIntensity it gives the gradient of an
    emergent map with respect to T, alpha (the opacity) and S at every point."""

    @staticmethod
    def forward(ctx, T, grid, atom, atm, pops):
        rho, ne, nH = atm.tensors[1:]
        a = Atmos(T.detach().contiguous(), rho, ne, nH)
        ctx.grid, ctx.atom, ctx.atm = grid, atom, a
        ctx.save_for_backward(pops)
        return source_terms(grid, atom, a, pops)

    @staticmethod
    def backward(ctx, g_alpha, g_S):
        (pops,) = ctx.saved_tensors
        ga = torch.zeros_like(pops[:1].expand(ctx.atom.nlam, -1)).contiguous() \
            if g_alpha is None else g_alpha.contiguous()
        gs = torch.zeros_like(ga) if g_S is None else g_S.contiguous()
        gT = source_terms_adjoint(ctx.grid, ctx.atom, ctx.atm, pops, ga, gs)
        return gT, None, None, None, None


class Batch:
    """Several Voronoi grids solved by one persistent level-scheduled launch."""

    def __init__(self, grids, nlam, lam_chunk=None, threads=0):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(grids))(*[g.handle.value for g in grids])
        lc = None
        self._lc = None
        if lam_chunk is not None:
            self._lc = _np(lam_chunk, np.int32)
            lc = self._lc.ctypes.data_as(L.PI32)
        h = ctypes.c_void_p()
        check(lib().rt_batch_create(arr, len(grids), nlam, lc, int(threads), ctypes.byref(h)))
        self._h = h
        self.nlam = nlam

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.rt_batch_destroy(h)
            self._h = None

    def formal_solution(self, alphas, Ss, bc=L.RT_BC_THERMAL, Js=None, stream=None):
        n = len(self.grids)
        if Js is None:
            Js = [torch.empty_like(a) for a in alphas]
        pa = (ctypes.c_void_p * n)(*[_dev(a).value for a in alphas])
        ps = (ctypes.c_void_p * n)(*[_dev(s).value for s in Ss])
        pj = (ctypes.c_void_p * n)(*[_dev(j).value for j in Js])
        check(lib().rt_batch_formal_solution(self._h, pa, ps, bc, pj, _stream(stream)))
        return Js

    def lambda_iterate(self, atom: Atom, atms, pops, max_iter=300, tol=1e-3, use_graph=True,
                       stream=None):
        """Lambda iteration of every atmosphere of the batch together (one model atom), in place on
        pops (one [3][npt] tensor per grid); returns (iterations, history, converged)."""
        n = len(self.grids)
        if len(atms) != n or len(pops) != n:
            raise ValueError("one Atmos and one pops tensor per grid")
        descs = (L.AtmosDesc * n)(*[m.desc for m in atms])
        pp = (ctypes.c_void_p * n)(*[_dev(p, (3, g.npt), "pops").value
                                     for p, g in zip(pops, self.grids)])
        hist = np.zeros(max_iter, np.float32)
        it = ctypes.c_int(0)
        st = lib().rt_batch_lambda_iterate(self._h, ctypes.byref(atom.desc), descs, pp, max_iter,
                                           float(tol), ctypes.byref(it),
                                           hist.ctypes.data_as(L.PF), int(use_graph),
                                           _stream(stream))
        if st not in (L.RT_OK, L.RT_ENOCONV):
            check(st)
        return it.value, hist[:it.value].copy(), st == L.RT_OK

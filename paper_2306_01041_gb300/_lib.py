"""ctypes declarations of include/rt.h (argument marshalling only).

Loading fails loudly when librt.so has not been built: there is no other implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librt.so")

c_int, c_int64, c_double, c_float, c_size_t = (ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_float, ctypes.c_size_t)
P = ctypes.c_void_p
PD = ctypes.POINTER(ctypes.c_double)
PF = ctypes.POINTER(ctypes.c_float)
PI32 = ctypes.POINTER(ctypes.c_int32)
PI64 = ctypes.POINTER(ctypes.c_int64)
PI8 = ctypes.POINTER(ctypes.c_int8)

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ECYCLE, RT_ETIMEOUT, RT_ENAN, RT_ECAPACITY, \
    RT_ENOCONV = range(9)
STATUS_NAMES = ["RT_OK", "RT_EINVAL", "RT_ENOMEM", "RT_ECUDA", "RT_ECYCLE", "RT_ETIMEOUT",
                "RT_ENAN", "RT_ECAPACITY", "RT_ENOCONV"]
RT_GRID_REGULAR, RT_GRID_VORONOI = 0, 1
RT_BC_THERMAL, RT_BC_ZERO, RT_BC_ARRAY = 0, 1, 2
RT_SC_PLANE, RT_SC_FACE = 0, 1


class GridDesc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx", c_double), ("dy", c_double), ("z", PD),
                ("nsites", c_int64), ("xyz", PD), ("nbr_off", PI64), ("nbr_idx", PI32),
                ("nbr_shift", PI8), ("box", c_double * 6), ("periodic_xy", c_int),
                ("ndir", c_int), ("dirs", PD), ("wdir", PD), ("r_exponent", c_double)]


class AtomDesc(ctypes.Structure):
    _fields_ = [("E_cm", c_double * 3), ("g", c_double * 3), ("f_line", c_double),
                ("voigt_a", c_double), ("q_coll", c_double), ("kappa0", c_double),
                ("nlam", c_int), ("lam", PD), ("wlam", PD), ("kind", PI32)]


class AtmosDesc(ctypes.Structure):
    _fields_ = [("T", P), ("rho", P), ("ne", P), ("nH", P)]


class RTError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "rt_grid_create": (c_int, [ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)]),
    "rt_grid_destroy": (None, [P]),
    "rt_grid_info": (c_int, [P, PI64, PI64, ctypes.POINTER(c_int), PI64]),
    "rt_grid_tables": (c_int, [P, PI32, PF, PF, PI32]),
    "rt_grid_top_points": (c_int, [P, PI64]),
    "rt_grid_set_scheme": (c_int, [P, c_int]),
    "rt_grid_build_tables_device": (c_int, [P, P]),
    "rt_formal_solution": (c_int, [P, c_int, P, P, c_int, P, P, P, P]),
    "rt_source_terms_lte": (c_int, [c_int64, P, P, c_double, c_double, P, P, P]),
    "rt_source_terms_lte_adjoint": (c_int, [c_int64, P, P, c_double, c_double, P, P, P, P]),
    "rt_source_terms": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc), P, P, P,
                                P]),
    "rt_source_terms_adjoint": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc),
                                        P, P, P, P, P]),
    "rt_lte_populations": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc), P, P]),
    "rt_statistical_equilibrium": (c_int, [P, ctypes.POINTER(AtomDesc),
                                           ctypes.POINTER(AtmosDesc), P, P, P, P]),
    "rt_lambda_iterate": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc), P, c_int,
                                  c_double, ctypes.POINTER(c_int), PF, c_int, P]),
    "rt_lambda_star": (c_int, [P, c_int, P, c_int, P, P]),
    "rt_statistical_equilibrium_ali": (c_int, [P, ctypes.POINTER(AtomDesc),
                                               ctypes.POINTER(AtmosDesc), P, P, P, P, P, c_int,
                                               P]),
    "rt_lambda_iterate_ali": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc), P,
                                      c_int, c_double, ctypes.POINTER(c_int), PF, c_int, c_int,
                                      c_int, P]),
    "rt_ng_extrapolate": (c_int, [c_int64, P, P, P, P, P, P, ctypes.POINTER(c_int), P]),
    "rt_lambda_iterate_ex": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc), P,
                                     c_int, c_double, ctypes.POINTER(c_int), PF, c_int, c_int,
                                     c_int, c_int, P]),
    "rt_idw_create": (c_int, [P, P, ctypes.POINTER(P)]),
    "rt_idw_destroy": (None, [P]),
    "rt_idw_table": (c_int, [P, PI32, PF]),
    "rt_idw_interpolate": (c_int, [P, c_int, P, P, P]),
    "rt_emergent_intensity": (c_int, [P, PD, c_int, P, P, c_int, P, P]),
    "rt_emergent_map": (c_int, [P, PD, c_int, P, P, c_int, c_int, c_int, P, P]),
    "rt_adjoint_workspace_size": (c_size_t, [P, c_int, c_int]),
    "rt_formal_solution_adjoint": (c_int, [P, PD, c_int, P, P, c_int, P, P, P, c_int, P, c_size_t,
                                           P]),
    "rt_batch_create": (c_int, [ctypes.POINTER(P), c_int, c_int, PI32, c_int, ctypes.POINTER(P)]),
    "rt_batch_destroy": (None, [P]),
    "rt_batch_formal_solution": (c_int, [P, ctypes.POINTER(P), ctypes.POINTER(P), c_int,
                                         ctypes.POINTER(P), P]),
    "rt_batch_lambda_iterate": (c_int, [P, ctypes.POINTER(AtomDesc), ctypes.POINTER(AtmosDesc),
                                        ctypes.POINTER(P), c_int, c_double, ctypes.POINTER(c_int),
                                        PF, c_int, P]),
    "rt_sample_sites": (c_int, [c_int, c_int, c_int, PD, PD, P, c_int64, ctypes.c_uint64, P,
                                PI64, P]),
    "rt_last_error": (ctypes.c_char_p, []),
    "rt_kernel_launches": (ctypes.c_ulonglong, []),
}


def lib():
    """The loaded librt.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"librt.so not found at {LIB_PATH}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != RT_OK:
        msg = lib().rt_last_error()
        raise RTError(status, msg.decode() if msg else "")
    return status

"""EFIE matrix rows (dense MoM and near part) via the oracle's C loops.

Paper Sec. 2, Eq. 1 (field of a surface current), Eq. 2 (weak null-field condition)
and Eq. 3 (matrix entries).  The formulas and the singular-pair rule are stated in
the header of ``efie_oracle.c``.
"""
import ctypes
import math

import numpy as np

from . import build as _build
from .quadrature import WEIGHTS, triangle_points

ETA0 = 4e-7 * math.pi * 299792458.0  # free-space impedance mu0 * c (ohm)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        _lib.orc_efie_rows.restype = ctypes.c_int
        _lib.orc_efie_rows.argtypes = [ctypes.c_int64, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P, P,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int64, P, ctypes.c_int, P,
                                       ctypes.c_int, P]
        _lib.orc_static_integrals.restype = None
        _lib.orc_static_integrals.argtypes = [P, P, P, P]
        _lib.orc_green_matrix.restype = None
        _lib.orc_green_matrix.argtypes = [ctypes.c_double, ctypes.c_int64, P, ctypes.c_int64, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def static_integrals(tri_vertices, r):
    """Closed-form int_T 1/R dS' and int_T (r'-r)/R dS' for a flat triangle."""
    v = np.ascontiguousarray(tri_vertices, dtype=np.float64).reshape(9)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(3)
    i1 = np.zeros(1)
    iv = np.zeros(3)
    lib().orc_static_integrals(_p(v), _p(r), _p(i1), _p(iv))
    return i1[0], iv


def green_matrix(k, a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    G = np.zeros((len(a), len(b)), np.complex128)
    lib().orc_green_matrix(k, len(a), _p(a), len(b), _p(b), _p(G))
    return G


SINGULAR_MODES = {"touching": 0, "self": 1}


def efie_rows(vertices, triangles, rwg, k, rows=None, near_leaf_ijk=None, eta=ETA0, singular_mode="touching"):
    """Rows ``rows`` (default all) of the EFIE matrix Z (complex128 [len(rows), N]).

    ``near_leaf_ijk`` None: the full dense MoM matrix.  Otherwise an int array
    [nt, 7, 3] of the leaf coordinates of every quadrature point, and only the near
    part is returned: point pairs whose leaves touch (|di|,|dj|,|dk| <= 1).
    ``singular_mode`` "touching": singularity extraction for every triangle pair that
    shares a vertex; "self": for T = T' only (see efie_oracle.c)."""
    verts = np.ascontiguousarray(vertices, np.float64)
    tris = np.ascontiguousarray(triangles, np.int32)
    q = np.ascontiguousarray(triangle_points(verts, tris))
    w = np.ascontiguousarray(WEIGHTS)
    n = rwg["n"]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    tri_rwg = np.ascontiguousarray(rwg["tri_rwg"], np.int32)
    tri_sl = np.ascontiguousarray(rwg["tri_sl"], np.float64)
    rwg_tri = np.ascontiguousarray(rwg["tri"], np.int32)
    rwg_free = np.ascontiguousarray(rwg["free"], np.int32)
    out = np.zeros((len(rows), n), np.complex128)
    if near_leaf_ijk is None:
        mode, leaf = 0, np.zeros(3, np.int32)
    else:
        mode, leaf = 1, np.ascontiguousarray(near_leaf_ijk, np.int32)
    st = lib().orc_efie_rows(len(verts), _p(verts), len(tris), _p(tris), _p(q), _p(w), n, _p(tri_rwg), _p(tri_sl),
                             _p(rwg_tri), _p(rwg_free), float(k), float(eta), len(rows), _p(rows), mode, _p(leaf),
                             SINGULAR_MODES[singular_mode], _p(out))
    if st != 0:
        raise ValueError("a singular (touching) triangle pair straddles non-touching leaves: "
                         "triangles too large for the leaf size")
    return out

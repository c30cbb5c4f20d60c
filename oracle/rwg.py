"""RWG (Rao-Wilton-Glisson 1982) basis functions on a triangle mesh.

The paper expands the surface current as j = sum_n j_n phi_n (Sec. 2) without naming
the basis.  Reading used here:
* one function per interior edge, i.e. an edge shared by exactly two triangles; an edge
  shared by more than two triangles is an error, a boundary edge carries none;
* edges numbered in lexicographic order of (smaller vertex id, larger vertex id);
* T+ is the adjacent triangle with the smaller index, T- the other one;
* phi_n = l/(2A+) (r - v+) on T+ and l/(2A-) (v- - r) on T-, with v+- the vertex
  opposite the edge, l the edge length; div phi_n = +l/A+ on T+ and -l/A- on T-.
"""
import numpy as np

from .quadrature import triangle_areas


class MeshError(ValueError):
    pass


def build_rwg(vertices, triangles):
    """Return a dict with
    ``n``            number of RWG functions,
    ``edge``         [n,2] vertex ids (sorted),
    ``tri``          [n,2] (T+, T-),
    ``free``         [n,2] local index (0..2) of the free vertex in T+ and T-,
    ``length``       [n] edge length,
    ``tri_rwg``      [nt,3] RWG attached to the edge opposite local vertex c (or -1),
    ``tri_sl``       [nt,3] sign * length of that RWG on the triangle (0 if none),
    ``area``         [nt] triangle areas.
    """
    tris = np.asarray(triangles, dtype=np.int64)
    nt = len(tris)
    edges = {}
    for t in range(nt):
        for c in range(3):
            a, b = tris[t, (c + 1) % 3], tris[t, (c + 2) % 3]
            key = (min(a, b), max(a, b))
            edges.setdefault(key, []).append((t, c))
    interior = []
    for key in sorted(edges):
        adj = edges[key]
        if len(adj) > 2:
            raise MeshError("non-manifold edge %s shared by %d triangles" % (key, len(adj)))
        if len(adj) == 2:
            interior.append((key, sorted(adj)))
    n = len(interior)
    area = triangle_areas(vertices, tris)
    edge = np.zeros((n, 2), np.int64)
    tri = np.zeros((n, 2), np.int64)
    free = np.zeros((n, 2), np.int64)
    length = np.zeros(n)
    tri_rwg = -np.ones((nt, 3), np.int64)
    tri_sl = np.zeros((nt, 3))
    for i, (key, adj) in enumerate(interior):
        edge[i] = key
        length[i] = np.linalg.norm(vertices[key[1]] - vertices[key[0]])
        for side, (t, c) in enumerate(adj):
            if area[t] <= 0.0:
                raise MeshError("degenerate triangle %d" % t)
            tri[i, side] = t
            free[i, side] = c
            tri_rwg[t, c] = i
            tri_sl[t, c] = (1.0 if side == 0 else -1.0) * length[i]
    return dict(n=n, edge=edge, tri=tri, free=free, length=length, tri_rwg=tri_rwg,
                tri_sl=tri_sl, area=area)

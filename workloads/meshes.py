"""Procedural triangle meshes (lengths in wavelengths).

Every generator returns ``(vertices, triangles)``: float64 ``[nv, 3]`` and int32
``[nt, 3]``, triangles counter-clockwise when seen from outside (outward normal by
the right-hand rule).  Ordering is deterministic.
"""
import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def _orient_outward(v, f):
    """Flip triangles whose right-hand normal points toward the origin (star-shaped bodies)."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c)) < 0
    f = f.copy()
    f[flip] = f[flip][:, [0, 2, 1]]
    return f


def icosphere(subdiv, radius=1.0):
    """Icosahedron split ``subdiv`` times 1->4, vertices projected to the sphere after
    each split.  ``20 * 4**subdiv`` triangles."""
    v, f = _icosahedron()
    verts = [p for p in v]
    for _ in range(subdiv):
        cache = {}
        nf = np.empty((len(f) * 4, 3), dtype=np.int64)

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            m = cache.get(key)
            if m is None:
                p = verts[i] + verts[j]
                verts.append(p / np.linalg.norm(p))
                m = len(verts) - 1
                cache[key] = m
            return m

        for t, (a, b, c) in enumerate(f):
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf[4 * t + 0] = (a, ab, ca)
            nf[4 * t + 1] = (b, bc, ab)
            nf[4 * t + 2] = (c, ca, bc)
            nf[4 * t + 3] = (ab, bc, ca)
        f = nf
    v = np.array(verts) * radius
    return v, _orient_outward(v, f).astype(np.int32)


def geodesic_ellipsoid(freq, semi_axes=(3.0, 1.0, 1.0)):
    """Ellipsoid from a frequency-``freq`` geodesic subdivision of the icosahedron:
    each face is split into ``freq**2`` triangles on a barycentric grid, points are
    projected to the unit sphere and then scaled by the semi-axes.  ``20*freq**2``
    triangles."""
    v0, f0 = _icosahedron()
    verts, index = [], {}

    def vid(key, p):
        m = index.get(key)
        if m is None:
            verts.append(p / np.linalg.norm(p))
            m = len(verts) - 1
            index[key] = m
        return m

    def key_of(face, i, j):
        # canonical key of barycentric grid point (i, j, freq-i-j) on a face, so that
        # points on shared edges and corners get one id
        a, b, c = face
        w = {a: freq - i - j, b: i, c: j}
        items = tuple(sorted((vtx, wt) for vtx, wt in w.items() if wt > 0))
        return items

    tris = []
    for face in f0:
        a, b, c = (v0[face[0]], v0[face[1]], v0[face[2]])
        ids = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                p = (a * (freq - i - j) + b * i + c * j) / freq
                ids[(i, j)] = vid(key_of(face, i, j), p)
        for i in range(freq):
            for j in range(freq - i):
                tris.append((ids[(i, j)], ids[(i + 1, j)], ids[(i, j + 1)]))
                if i + j + 1 < freq:
                    tris.append((ids[(i + 1, j)], ids[(i + 1, j + 1)], ids[(i, j + 1)]))
    v = np.array(verts) * np.asarray(semi_axes, dtype=np.float64)
    f = np.array(tris, dtype=np.int64)
    return v, _orient_outward(v, f).astype(np.int32)


def plate(nx, ny, size_x, size_y, origin=(0.0, 0.0, 0.0)):
    """Flat rectangular plate in the z=const plane, ``nx*ny`` squares each split on
    one diagonal; normals point to +z."""
    xs = np.linspace(0.0, size_x, nx + 1) + origin[0]
    ys = np.linspace(0.0, size_y, ny + 1) + origin[1]
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    v = np.stack([X.ravel(), Y.ravel(), np.full(X.size, origin[2])], 1)
    tris = []
    for i in range(nx):
        for j in range(ny):
            p00 = i * (ny + 1) + j
            p10 = (i + 1) * (ny + 1) + j
            p01 = i * (ny + 1) + j + 1
            p11 = (i + 1) * (ny + 1) + j + 1
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    return v.astype(np.float64), np.array(tris, dtype=np.int32)


def _merge(parts):
    vs, fs, off = [], [], 0
    for v, f in parts:
        vs.append(v)
        fs.append(f.astype(np.int64) + off)
        off += len(v)
    return np.concatenate(vs), np.concatenate(fs).astype(np.int32)


def ring_ellipsoid(a, b, edge):
    """Prolate ellipsoid x^2/a^2 + (y^2 + z^2)/b^2 = 1 meshed by rings: meridian nodes at
    equal arc length (about ``edge`` apart), the same number of points on every ring
    (about ``edge`` apart on the widest one), poles closed by fans."""
    phi = np.linspace(0.0, np.pi, 4001)
    ds = np.sqrt((a * np.sin(phi)) ** 2 + (b * np.cos(phi)) ** 2)
    arc = np.concatenate([[0.0], np.cumsum(0.5 * (ds[1:] + ds[:-1]) * np.diff(phi))])
    nring = max(2, int(round(arc[-1] / edge))) - 1
    phis = np.interp(np.linspace(0.0, arc[-1], nring + 2)[1:-1], arc, phi)
    nth = max(3, int(round(2.0 * np.pi * b / edge)))
    th = 2.0 * np.pi * np.arange(nth) / nth
    verts = [[a, 0.0, 0.0]]
    for p in phis:
        r = b * np.sin(p)
        for t in th:
            verts.append([a * np.cos(p), r * np.cos(t), r * np.sin(t)])
    verts.append([-a, 0.0, 0.0])
    v = np.array(verts)
    f = []
    ring = lambda j, i: 1 + j * nth + (i % nth)
    for i in range(nth):
        f.append([0, ring(0, i), ring(0, i + 1)])
    for j in range(nring - 1):
        for i in range(nth):
            f.append([ring(j, i), ring(j + 1, i), ring(j + 1, i + 1)])
            f.append([ring(j, i), ring(j + 1, i + 1), ring(j, i + 1)])
    last = len(v) - 1
    for i in range(nth):
        f.append([last, ring(nring - 1, i + 1), ring(nring - 1, i)])
    f = np.array(f, dtype=np.int64)
    return v, _orient_outward(v, f).astype(np.int32)


def aircraft(edge=0.1, length=10.0, seed=0):
    """Aircraft-like PEC body: a prolate fuselage ``length`` long, two thin wing plates
    and a tail plate, all separate closed/open surfaces (no junctions), mesh edge about
    ``edge``.  ``seed`` jitters the wing sweep slightly (deterministic)."""
    rng = np.random.default_rng(seed)
    a = length / 2.0
    b = length / 12.0
    fv, ff = ring_ellipsoid(a, b, edge)
    span = 0.45 * length
    chord = 0.12 * length
    sweep = 0.05 * length * (1.0 + 0.1 * rng.standard_normal())
    gap = 2.0 * edge
    nx_w = max(2, int(round(chord / edge)))
    ny_w = max(2, int(round((span - b - gap) / edge)))
    parts = [(fv, ff)]
    for side in (+1, -1):
        v, f = plate(nx_w, ny_w, chord, span - b - gap)
        v = v.copy()
        v[:, 1] = side * (b + gap + v[:, 1])
        v[:, 0] += -0.1 * length + sweep * np.abs(v[:, 1]) / span
        if side < 0:
            f = f[:, [0, 2, 1]]
        parts.append((v, f))
    tail_h = 0.12 * length
    nx_t = max(2, int(round(0.6 * chord / edge)))
    nz_t = max(2, int(round(tail_h / edge)))
    v, f = plate(nx_t, nz_t, 0.6 * chord, tail_h)
    v = np.stack([v[:, 0] + 0.8 * a - 0.3 * chord, np.zeros(len(v)), v[:, 1] + b + gap], 1)
    parts.append((v, f))
    return _merge(parts)

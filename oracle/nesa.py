"""Naive NESA matrix-vector product (paper Sec. 2, Eqs. 4-7, and Sec. 3, Eqs. 9-14).

One box pair at a time, in the paper's order: near field (Eq. 9), radiation (Eq. 10),
source transfer (Eq. 11), translation (Eq. 12), potential transfer (Eq. 13) and
reception (Eq. 14).

How the EFIE is cast into these stages (readings; the construction itself is left to
the paper's NESA reference):

* Far point pairs.  With the quadrature points of the triangles as sources, the far
  part of Z x is (see efie_oracle.c for the matrix entries)
      y_m = -i eta k sum_p w_p sl_m [ (r_p - v_m).F_p/2 - k^-2 F^rho_p ]
      F^c_p = sum_{q far from p} g(r_p, r_q) J^c_q
      J^{x,y,z}_q = w_q sum_n sl_n (r_q - v_n)/2 x_n,   J^rho_q = w_q sum_n sl_n x_n
  (sl = sign * edge length of the RWG on the point's triangle, v its free vertex),
  i.e. four scalar Helmholtz products ("channels" x, y, z, rho) with channel weights
  (1, 1, 1, -1/k^2) on the testing side.  A point pair is far when its leaves do not
  touch.
* Equivalent sources (Fig. 3 of the paper, with Q per group, Sec. 3).  At level l a box
  of side w has circumradius R = sqrt(3)/2 w.  Its Q_l equivalent points E are a
  Fibonacci lattice on the sphere of radius rho_eq R about the box centre, its 2 Q_l test
  points T a Fibonacci lattice on radius rho_test R, rho_test = (2 - sqrt3/2)/(sqrt3/2)
  (the nearest equivalent point of an interacting box is at distance >= 2w - R).
  K_l is the Tikhonov-regularised pseudo-inverse of G(T, E):
  K = (A^H A + eps^2 I)^-1 A^H,  eps = pinv_eps * ||A||_F.
* Operators (Eq. 4-5).  V_beta = K_L G(T_L + c_beta, X_beta) (radiation),
  C_l(delta) = K_{l-1} G(T_{l-1}, E_l + delta) with delta the child centre minus the
  parent centre (source transfer), D_l(off) = G(E_l + off, E_l) with off the centre of
  the observation box minus that of the source box (translation), and, because g is
  symmetric, B = C^T and U = V^T (potential transfer and reception): the incoming
  field of a box is represented by sources at its test points with strengths K^T o.
* Q_l: 'fixed' gives q_fixed in every group (the paper's choice); 'auto' gives
  max(q_fixed, (n_l + 1)^2), n_l = ceil(kR + 1.8 d^(2/3) (kR)^(1/3)), d = q_digits
  (the excess-bandwidth rule of the multilevel fast multipole literature).
"""
import math

import numpy as np

from .efie import ETA0, efie_rows
from .quadrature import WEIGHTS
from .rwg import build_rwg
from .tree import Tree

RHO_TEST_DEFAULT = (2.0 - math.sqrt(3.0) / 2.0) / (math.sqrt(3.0) / 2.0)


def fibonacci_sphere(n, radius):
    """n points z_i = 1 - (2i+1)/n, azimuth i * pi (3 - sqrt 5), on a sphere."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    s = np.sqrt(1.0 - z * z)
    return radius * np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)


def green(k, a, b):
    """G[i, j] = exp(-i k |a_i - b_j|) / (4 pi |a_i - b_j|)  (Eq. 1)."""
    d = a[:, None, :] - b[None, :, :]
    R = np.sqrt(np.einsum("ijx,ijx->ij", d, d))
    return np.exp(-1j * k * R) / (4.0 * math.pi * R)


def tikhonov_pinv(A, pinv_eps):
    eps = pinv_eps * np.linalg.norm(A)
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    return (Vh.conj().T * (s / (s * s + eps * eps))) @ U.conj().T


def q_for_level(k, width, q_mode, q_fixed, q_digits):
    if q_mode == "fixed":
        return int(q_fixed)
    kr = k * math.sqrt(3.0) / 2.0 * width
    nl = math.ceil(kr + 1.8 * q_digits ** (2.0 / 3.0) * kr ** (1.0 / 3.0))
    return max(int(q_fixed), (nl + 1) ** 2)


def channel_sources(vertices, triangles, rwg, points, x):
    """Channel point sources J [npts, 4] (x, y, z current and charge at every quadrature
    point, weights included) from RWG coefficients x [N]; points [7 nt, 3]."""
    r = rwg
    pts = np.asarray(points).reshape(-1, 7, 3)
    J = np.zeros((len(triangles), 7, 4), np.complex128)
    for t in range(len(triangles)):
        for c in range(3):
            n = r["tri_rwg"][t, c]
            if n < 0:
                continue
            sl = r["tri_sl"][t, c]
            v = vertices[triangles[t, c]]
            J[t, :, :3] += (WEIGHTS * sl * x[n] / 2.0)[:, None] * (pts[t] - v)
            J[t, :, 3] += WEIGHTS * sl * x[n]
    return J.reshape(-1, 4)


def apply_testing(vertices, triangles, rwg, points, k, eta, F, rows=None):
    """Testing (Eq. 3) of channel fields F [npts, 4] at the quadrature points:
    y_m = -i eta k sum_p w_p sl [ (r_p - v).F_p/2 - F^rho_p / k^2 ] for m in rows."""
    r = rwg
    pts = np.asarray(points).reshape(-1, 7, 3)
    F = F.reshape(-1, 7, 4)
    rows = range(r["n"]) if rows is None else rows
    y = np.zeros(len(rows), np.complex128)
    for i, m in enumerate(rows):
        acc = 0.0 + 0.0j
        for side in range(2):
            t = r["tri"][m, side]
            c = r["free"][m, side]
            sl = r["tri_sl"][t, c]
            v = vertices[triangles[t, c]]
            acc += np.sum(WEIGHTS * sl * (np.einsum("px,px->p", pts[t] - v, F[t, :, :3]) / 2.0
                                           - F[t, :, 3] / k ** 2))
        y[i] = -1j * eta * k * acc
    return y


class NesaOracle:
    def __init__(self, vertices, triangles, k, leaf_size, n_levels, q_mode="auto", q_fixed=100, q_digits=5.0,
                 rho_eq=1.0, rho_test=RHO_TEST_DEFAULT, pinv_eps=1e-9, eta=ETA0, singular_mode="touching",
                 points_per_leaf=0):
        self.singular_mode = singular_mode
        self.vertices = np.asarray(vertices, np.float64)
        self.triangles = np.asarray(triangles, np.int64)
        self.k = float(k)
        self.eta = float(eta)
        self.rwg = build_rwg(self.vertices, self.triangles)
        self.n = self.rwg["n"]
        self.tree = Tree(self.vertices, self.triangles, leaf_size, n_levels, points_per_leaf)
        t = self.tree
        self.L, self.l0 = t.L, t.l0
        self.Q, self.E, self.T, self.K = {}, {}, {}, {}
        for l in range(self.l0, self.L + 1):
            w = t.width(l)
            R = math.sqrt(3.0) / 2.0 * w
            q = q_for_level(self.k, w, q_mode, q_fixed, q_digits)
            self.Q[l] = q
            self.E[l] = fibonacci_sphere(q, rho_eq * R)
            self.T[l] = fibonacci_sphere(2 * q, rho_test * R)
            self.K[l] = tikhonov_pinv(green(self.k, self.T[l], self.E[l]), pinv_eps)
        self._C = {}
        self._D = {}
        self._near = None

    # ---------------------------------------------------------------- operators
    def C(self, level, octant):
        """Source transfer C_l for the child at octant (bits of its coordinates)."""
        key = (level, octant)
        if key not in self._C:
            w = self.tree.width(level)
            delta = (np.array(octant, np.float64) - 0.5) * w
            self._C[key] = self.K[level - 1] @ green(self.k, self.T[level - 1], self.E[level] + delta)
        return self._C[key]

    def D(self, level, off):
        key = (level, off)
        if key not in self._D:
            shift = np.array(off, np.float64) * self.tree.width(level)
            self._D[key] = green(self.k, self.E[level] + shift, self.E[level])
        return self._D[key]

    # ---------------------------------------------------------------- point maps
    def sources(self, x):
        """Channel point sources J [npts, 4] from RWG coefficients x [N]."""
        return channel_sources(self.vertices, self.triangles, self.rwg, self.tree.points, x)

    def test(self, F, rows=None):
        """y_m = -i eta k sum_p w_p sl [ (r_p - v).F_p/2 - F^rho_p / k^2 ] for m in rows."""
        return apply_testing(self.vertices, self.triangles, self.rwg, self.tree.points, self.k, self.eta, F, rows)

    # ---------------------------------------------------------------- near field
    def near_rows(self, rows=None):
        ijk = self.tree.point_leaf_ijk.reshape(-1, 7, 3)
        return efie_rows(self.vertices, self.triangles, self.rwg, self.k, rows=rows, near_leaf_ijk=ijk, eta=self.eta,
                         singular_mode=self.singular_mode)

    def near_matrix(self):
        if self._near is None:
            self._near = self.near_rows()
        return self._near

    # ---------------------------------------------------------------- far field
    def radiate(self, J, leaf):
        """Eq. 10 for one leaf: s = K_L G(T_L + c, X_leaf) J_leaf  (Q_L x 4)."""
        t = self.tree
        idx = t.leaf_points[leaf]
        c = t.box_center(self.L, leaf)
        return self.K[self.L] @ (green(self.k, self.T[self.L] + c, t.points[idx]) @ J[idx])

    def source_transfer(self, level, child, s_child):
        """Eq. 11 for one child at ``level``: contribution C_l(octant) s_child to its parent."""
        oct_ = (child[0] & 1, child[1] & 1, child[2] & 1)
        return self.C(level, oct_) @ s_child

    def translate(self, level, box, s, o_parent):
        """Eqs. 13 and 12 for one box: o = C_l(octant)^T o_parent + sum_{b in IL} D_l(box - b) s_b."""
        acc = np.zeros((self.Q[level], 4), np.complex128)
        if o_parent is not None:
            oct_ = (box[0] & 1, box[1] & 1, box[2] & 1)
            acc += self.C(level, oct_).T @ o_parent
        for b in self.tree.interaction_list(level, box):
            off = (box[0] - b[0], box[1] - b[1], box[2] - b[2])
            acc += self.D(level, off) @ s[b]
        return acc

    def receive(self, leaf, o_leaf):
        """Eq. 14 for one leaf: field G(X_leaf, T_L + c) K_L^T o at the leaf's points."""
        t = self.tree
        idx = t.leaf_points[leaf]
        c = t.box_center(self.L, leaf)
        return idx, green(self.k, t.points[idx], self.T[self.L] + c) @ (self.K[self.L].T @ o_leaf)

    def far_fields(self, x, needed_leaves=None):
        """Five far-field stages (Eqs. 10-14).  Returns F [npts, 4] at the points of
        ``needed_leaves`` (all leaves by default)."""
        t = self.tree
        L, l0 = self.L, self.l0
        J = self.sources(x)
        s = {l: {} for l in range(l0, L + 1)}
        for b in t.boxes[L]:
            s[L][b] = self.radiate(J, b)
        for l in range(L, l0, -1):
            for b in t.boxes[l]:
                p = t.parent(b)
                s[l - 1][p] = s[l - 1].get(p, 0) + self.source_transfer(l, b, s[l][b])
        if needed_leaves is None:
            need = {l: list(t.boxes[l]) for l in range(l0, L + 1)}
        else:
            need = {L: sorted(set(needed_leaves))}
            for l in range(L - 1, l0 - 1, -1):
                need[l] = sorted({t.parent(b) for b in need[l + 1]})
        o = {l: {} for l in range(l0, L + 1)}
        for l in range(l0, L + 1):
            for a in need[l]:
                o[l][a] = self.translate(l, a, s[l], o[l - 1][t.parent(a)] if l > l0 else None)
            self._D = {key: v for key, v in self._D.items() if key[0] != l}
        F = np.zeros((len(t.points), 4), np.complex128)
        for a in need[L]:
            idx, f = self.receive(a, o[L][a])
            F[idx] = f
        return F

    def far_rows(self, x, rows=None):
        if rows is None:
            return self.test(self.far_fields(x))
        tri = self.rwg["tri"][np.asarray(rows)].ravel()
        leaves = {tuple(c) for c in self.tree.point_leaf_ijk.reshape(-1, 7, 3)[tri].reshape(-1, 3).tolist()}
        return self.test(self.far_fields(x, leaves), rows)

    def matvec(self, x):
        """Z~ x = Z^near x + far part (all rows)."""
        return self.near_matrix() @ x + self.far_rows(x)

    def matvec_rows(self, x, rows):
        """Rows of Z~ x only (near rows computed directly, far part on the needed boxes)."""
        return self.near_rows(rows) @ x + self.far_rows(x, rows)

    # ---------------------------------------------------------------- checks
    def far_exact(self, x):
        """Far part computed point pair by point pair without any approximation:
        F_p = sum over points q in leaves not touching leaf(p) of g(p,q) J_q."""
        t = self.tree
        J = self.sources(x)
        X = t.points
        F = np.zeros((len(X), 4), np.complex128)
        leaves = t.boxes[self.L]
        for a in leaves:
            ia = t.leaf_points[a]
            far = [q for b in leaves if not t.touch(a, b) for q in t.leaf_points[b]]
            if far:
                F[ia] = green(self.k, X[ia], X[far]) @ J[far]
        return self.test(F)

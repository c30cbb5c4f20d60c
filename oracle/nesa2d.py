"""Oracle of the paper's 2D model problem (Sec. 3): the potential of N charges on a
curve in the plane, evaluated at the charges,

    phi = K q,   K_ij = -log|x_i - x_j| (i != j),   K_ii = 0          (Eq. 8),

directly and in the NESA form of Sec. 2 run as Sec. 3 describes it: the near field
between neighbouring finest-level groups (Eq. 9) and the five far-field stages,
radiation (Eq. 10), source transfer (Eq. 11), translation (Eq. 12), potential
transfer (Eq. 13) and reception (Eq. 14).  Real FP64, one group pair at a time.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the CPU legs of bench.py).

Readings (the paper leaves the construction of the operators to its NESA reference,
and the quadtree to its figures):

* Quadtree.  The root square has the side of the largest extent of the points and its
  lower-left corner at their minimum; level l has 2^l x 2^l boxes of side w_l, and a
  point belongs to the box floor((x - lo) / w_l) (the last box on the upper edges).
  The coarsest level is l0 = 2: four groups along the longest dimension.  The finest
  level L is the deepest one whose occupied groups hold on average at least P points
  (L = l0 if none does).
* Lists.  Near groups of alpha: the occupied groups whose integer coordinates differ
  from alpha's by at most one in each direction, alpha included (left, right, top,
  bottom, diagonal and self).  Interaction list at l0: every occupied group that is
  not near; at l > l0: the occupied children of the parent's near groups that are
  not near alpha.  The near field is evaluated at level L only.
* Equivalent points (Fig. 3): Q points on the circle of radius rho_eq R about the
  group centre, R = w / sqrt(2) the circumradius, at angles 2 pi (j + 1/2) / Q.  Test
  points: 2Q points on the circle of radius rho_test R at angles 2 pi j / (2Q), with
  rho_test R = (2 - 1/sqrt(2)) w: an interacting group's centre is at least 2w away,
  so its equivalent circle (radius R) does not reach the test circle.
* K_l is the Tikhonov-regularised pseudo-inverse of G(T_l, E_l), G = -log|.|.
  V_beta = K_L G(T_L + c_beta, X_beta); C_l(delta) = K_{l-1} G(T_{l-1}, E_l + delta),
  delta the child centre minus the parent centre; D_l(off) = G(E_l + off, E_l), off
  the observation centre minus the source centre; and since G is symmetric,
  B = C^T and U = V^T.
"""
import math

import numpy as np

RHO_TEST_2D = (2.0 - 1.0 / math.sqrt(2.0)) / (1.0 / math.sqrt(2.0))


def log_kernel(a, b):
    """G[i, j] = -log|a_i - b_j| for point sets a [m][2], b [n][2] (Eq. 8)."""
    d = a[:, None, :] - b[None, :, :]
    return -0.5 * np.log(np.einsum("ijx,ijx->ij", d, d))


def dense_rows(x, q, rows):
    """phi_i = sum_{j != i} -log|x_i - x_j| q_j for the listed rows (Eq. 8)."""
    x = np.asarray(x, np.float64)
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        d = x - x[i]
        r2 = np.einsum("jx,jx->j", d, d)
        r2[i] = 1.0  # K_ii = 0
        out[t] = -0.5 * np.dot(np.log(r2), q)
    return out


def dense_matvec(x, q, block=512):
    """phi = K q over all rows (Eq. 8), a block of rows at a time."""
    x = np.asarray(x, np.float64)
    q = np.asarray(q, np.float64)
    n = len(x)
    out = np.empty(n)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        d = x[i0:i1, None, :] - x[None, :, :]
        r2 = np.einsum("ijx,ijx->ij", d, d)
        r2[np.arange(i1 - i0), np.arange(i0, i1)] = 1.0  # K_ii = 0
        out[i0:i1] = -0.5 * (np.log(r2) @ q)
    return out


class Tree2D:
    """Quadtree of Sec. 3 (readings in the module docstring)."""

    def __init__(self, x, P, l0=2):
        x = np.asarray(x, np.float64)
        self.x = x
        self.lo = x.min(0)
        self.side = float((x.max(0) - self.lo).max())
        self.l0 = l0
        L = l0
        while L < 40 and len(x) / len(self._occupied(L + 1)) >= P:
            L += 1
        self.L = L
        self.boxes = {l: self._occupied(l) for l in range(l0, L + 1)}
        self.index = {l: {b: i for i, b in enumerate(self.boxes[l])} for l in self.boxes}
        ij = self.coords(L)
        order = np.lexsort((np.arange(len(x)), ij[:, 1], ij[:, 0]))
        self.leaf_points = {}
        for p in order:
            self.leaf_points.setdefault((int(ij[p, 0]), int(ij[p, 1])), []).append(int(p))
        self.leaf_points = {b: np.array(v, np.int64) for b, v in self.leaf_points.items()}

    def width(self, l):
        return self.side / (1 << l)

    def coords(self, l):
        """Integer box coordinates of every point at level l."""
        n = 1 << l
        return np.clip(np.floor((self.x - self.lo) / self.width(l)).astype(np.int64), 0, n - 1)

    def _occupied(self, l):
        ij = self.coords(l)
        return sorted({(int(a), int(b)) for a, b in ij})

    def center(self, l, b):
        return self.lo + (np.array(b, np.float64) + 0.5) * self.width(l)

    def near(self, l, a):
        """Occupied groups within one box of a in each direction, a included."""
        ix = self.index[l]
        return [(a[0] + di, a[1] + dj) for di in (-1, 0, 1) for dj in (-1, 0, 1)
                if (a[0] + di, a[1] + dj) in ix]

    def interaction_list(self, l, a):
        near = set(self.near(l, a))
        if l == self.l0:
            return [b for b in self.boxes[l] if b not in near]
        p = (a[0] >> 1, a[1] >> 1)
        out = []
        for pb in self.near(l - 1, p):
            for ci in (0, 1):
                for cj in (0, 1):
                    b = (2 * pb[0] + ci, 2 * pb[1] + cj)
                    if b in self.index[l] and b not in near:
                        out.append(b)
        return sorted(out)


def _pinv(A, pinv_eps):
    """Tikhonov-regularised pseudo-inverse (A^T A + eps^2 I)^-1 A^T, eps = pinv_eps ||A||_F."""
    eps = pinv_eps * np.linalg.norm(A)
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    return (Vh.T * (s / (s * s + eps * eps))) @ U.T


def circle(n, radius, shift):
    """n points on a circle about the origin at angles 2 pi (j + shift) / n."""
    t = 2.0 * math.pi * (np.arange(n, dtype=np.float64) + shift) / n
    return radius * np.stack([np.cos(t), np.sin(t)], 1)


class Nesa2D:
    """The NESA product of the 2D model problem, one group pair at a time."""

    def __init__(self, x, P, Q, rho_eq=1.0, rho_test=RHO_TEST_2D, pinv_eps=1e-9):
        self.x = np.asarray(x, np.float64)
        self.n = len(self.x)
        self.Q = int(Q)
        self.tree = Tree2D(self.x, P)
        t = self.tree
        self.E, self.T, self.K = {}, {}, {}
        for l in range(t.l0, t.L + 1):
            R = t.width(l) / math.sqrt(2.0)
            self.E[l] = circle(self.Q, rho_eq * R, 0.5)
            self.T[l] = circle(2 * self.Q, rho_test * R, 0.0)
            self.K[l] = _pinv(log_kernel(self.T[l], self.E[l]), pinv_eps)

    # ------------------------------------------------------------------ operators
    def V(self, b):
        """Radiation matrix of leaf b (Q x its points), Eq. 10."""
        t = self.tree
        X = self.x[t.leaf_points[b]]
        return self.K[t.L] @ log_kernel(self.T[t.L] + t.center(t.L, b), X)

    def C(self, l, octant):
        """Source transfer from a child at level l, quadrant bits (x, y), Eq. 11."""
        delta = (np.array(octant, np.float64) - 0.5) * self.tree.width(l)
        return self.K[l - 1] @ log_kernel(self.T[l - 1], self.E[l] + delta)

    def D(self, l, off):
        """Translation between groups whose centres differ by off boxes, Eq. 12."""
        shift = np.array(off, np.float64) * self.tree.width(l)
        return log_kernel(self.E[l] + shift, self.E[l])

    # ------------------------------------------------------------------ product
    def near(self, q):
        """Eq. 9 over every near pair of finest-level groups."""
        t = self.tree
        phi = np.zeros(self.n)
        for a in t.boxes[t.L]:
            ia = t.leaf_points[a]
            for b in t.near(t.L, a):
                ib = t.leaf_points[b]
                G = log_kernel(self.x[ia], self.x[ib]) if a != b else self._self_block(ia)
                phi[ia] += G @ q[ib]
        return phi

    def _self_block(self, ia):
        d = self.x[ia][:, None, :] - self.x[ia][None, :, :]
        r2 = np.einsum("ijx,ijx->ij", d, d)
        np.fill_diagonal(r2, 1.0)  # K_ii = 0
        return -0.5 * np.log(r2)

    def far(self, q):
        """Eqs. 10-14: radiation, source transfer, translation, potential transfer, reception."""
        t = self.tree
        L, l0 = t.L, t.l0
        s = {l: {} for l in range(l0, L + 1)}
        for b in t.boxes[L]:
            s[L][b] = self.V(b) @ q[t.leaf_points[b]]
        for l in range(L, l0, -1):
            for b in t.boxes[l]:
                p = (b[0] >> 1, b[1] >> 1)
                s[l - 1][p] = s[l - 1].get(p, 0.0) + self.C(l, (b[0] & 1, b[1] & 1)) @ s[l][b]
        o = {l: {} for l in range(l0, L + 1)}
        for l in range(l0, L + 1):
            for a in t.boxes[l]:
                acc = np.zeros(self.Q)
                if l > l0:
                    acc += self.C(l, (a[0] & 1, a[1] & 1)).T @ o[l - 1][(a[0] >> 1, a[1] >> 1)]
                for b in t.interaction_list(l, a):
                    acc += self.D(l, (a[0] - b[0], a[1] - b[1])) @ s[l][b]
                o[l][a] = acc
        phi = np.zeros(self.n)
        for a in t.boxes[L]:
            phi[t.leaf_points[a]] += self.V(a).T @ o[L][a]
        return phi

    def matvec(self, q):
        q = np.asarray(q, np.float64)
        return self.near(q) + self.far(q)

"""Oracle of the preconditioners: block-Jacobi and the learned correction of it.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, FP64.

Block-Jacobi: every RWG function belongs to the leaf holding the centroid of its T+
(its "home leaf"); BJ applies the inverses of the near-field diagonal blocks of these
groups.

Overlapping block-Jacobi S (restricted additive Schwarz): the group of a leaf is solved
with the functions of the touching leaves and only its own rows are kept.

Learned preconditioner (not in the paper):  M u = a1 u + a2 S u + a3 S N S u, with
N the near-field matrix and complex coefficients a (6 reals per function) from a
network shared by all functions,
    h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), a = W3 h2 + b3,
on 8 static features x per function: k l, A+/l^2, A-/l^2, Re and Im of Z_mm/|Z_mm|,
log(|Z_mm| / mean |Z_mm|), (near-row length) / mean, (group size) / mean.
Loss over samples (u_s, v_s):  L = sum_s |M u_s - v_s|^2 / sum_s |v_s|^2.
Weights are one vector: W1 (32x8), b1, W2 (32x32), b2, W3 (6x32), b3, row-major.
"""
import numpy as np

NF, NH, NO = 8, 32, 6
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NO, NH)), ("b3", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, p = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[p:p + k], np.float64).reshape(shape)
        p += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SIZES])


def initial_theta():
    """Block-Jacobi start: zero output layer, b3 = (0,0, 1,0, 0,0)."""
    t = np.zeros(NPARAM)
    p = unpack(t)
    p["b3"][2] = 1.0
    return pack(p)


def groups(nesa_oracle):
    """RWG functions grouped by the leaf of the centroid (node 0) of T+."""
    o = nesa_oracle
    leaf = o.tree.point_leaf_ijk.reshape(-1, 7, 3)[o.rwg["tri"][:, 0], 0]
    out = {}
    for m, key in enumerate(map(tuple, leaf.tolist())):
        out.setdefault(key, []).append(m)
    return [np.array(v) for _, v in sorted(out.items())]


def touching(a, b):
    """Leaves with integer coordinates a and b touch (or coincide): every coordinate
    differs by at most one."""
    return max(abs(x - y) for x, y in zip(a, b)) <= 1


def ras_blocks(N, home):
    """Blocks of the overlapping block-Jacobi preconditioner for the functions whose
    home leaves (integer coordinates) are the rows of ``home``: per home leaf c, its
    group g (functions homed in c), the extended set E (functions whose home leaf
    touches c, ascending) and the rows of g in (N restricted to E x E)^-1."""
    by_leaf = {}
    for m, key in enumerate(map(tuple, np.asarray(home).tolist())):
        by_leaf.setdefault(key, []).append(m)
    out = []
    for key, members in by_leaf.items():
        E = np.array(sorted(m for k2, ms in by_leaf.items() if touching(key, k2) for m in ms))
        g = np.array(members)
        rows = np.linalg.inv(N[np.ix_(E, E)])[np.searchsorted(E, g), :]
        out.append((g, E, rows))
    return out


def ras_apply(blocks, u):
    """z = S u: each group's rows of its extended inverse applied to u on E."""
    z = np.zeros_like(u)
    for g, E, rows in blocks:
        z[g] = rows @ u[E]
    return z


class Preconditioner:
    def __init__(self, nesa_oracle):
        self.o = nesa_oracle
        self.N = nesa_oracle.near_matrix()
        self.groups = groups(nesa_oracle)
        self.inv = [np.linalg.inv(self.N[np.ix_(g, g)]) for g in self.groups]
        self._ras = None
        self.features = self._features()

    def bj(self, u):
        """Block-Jacobi on columns of u ([N] or [N, ns])."""
        z = np.zeros_like(u)
        for g, A in zip(self.groups, self.inv):
            z[g] = A @ u[g]
        return z

    def _ras_setup(self):
        """Overlapping block-Jacobi (restricted additive Schwarz) over the home leaves."""
        o = self.o
        home = o.tree.point_leaf_ijk.reshape(-1, 7, 3)[o.rwg["tri"][:, 0], 0]
        self._ras = ras_blocks(self.N, home)

    def ras(self, u):
        if self._ras is None:
            self._ras_setup()
        return ras_apply(self._ras, u)

    def near_row_lengths(self):
        """Structural length of every near-field row: the number of functions n with at
        least one quadrature-point pair (p on a triangle of m, q on a triangle of n) in
        touching leaves."""
        o, r = self.o, self.o.rwg
        leaves = o.tree.point_leaf_ijk.reshape(-1, 7, 3)
        nt = len(leaves)
        near_tri = np.zeros((nt, nt), bool)
        for p in range(7):
            for q in range(7):
                d = np.abs(leaves[:, None, p, :] - leaves[None, :, q, :]).max(-1)
                near_tri |= d <= 1
        tri_of = [[] for _ in range(o.n)]
        for m in range(o.n):
            tri_of[m] = list(r["tri"][m])
        funcs_of_tri = [[] for _ in range(nt)]
        for m in range(o.n):
            for t in r["tri"][m]:
                funcs_of_tri[t].append(m)
        out = np.zeros(o.n)
        for m in range(o.n):
            cols = set()
            for t in tri_of[m]:
                for t2 in np.nonzero(near_tri[t])[0]:
                    cols.update(funcs_of_tri[t2])
            out[m] = len(cols)
        return out

    def _features(self):
        o, r = self.o, self.o.rwg
        n = o.n
        diag = np.diag(self.N)
        mag = np.abs(diag)
        nnz = self.near_row_lengths()
        gs = np.zeros(n)
        for g in self.groups:
            gs[g] = len(g)
        l = r["length"]
        ap = r["area"][r["tri"][:, 0]]
        am = r["area"][r["tri"][:, 1]]
        x = np.stack([o.k * l, ap / l ** 2, am / l ** 2, diag.real / mag, diag.imag / mag,
                      np.log(mag / mag.mean()), nnz / nnz.mean(), gs / gs.mean()], 1)
        return x

    # ------------------------------------------------------------ network
    def forward(self, theta):
        p = unpack(theta)
        x = self.features
        h1 = np.tanh(x @ p["W1"].T + p["b1"])
        h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
        a = h2 @ p["W3"].T + p["b3"]
        return a, (x, h1, h2, p)

    def apply(self, theta, u):
        """M u for columns u [N, ns]."""
        a, _ = self.forward(theta)
        f2 = self.ras(u)
        f3 = self.ras(self.N @ f2)
        c = [(a[:, 2 * k] + 1j * a[:, 2 * k + 1])[:, None] for k in range(3)]
        return c[0] * u + c[1] * f2 + c[2] * f3

    def loss_grad(self, theta, U, V):
        """L and dL/dtheta for samples U = [N, ns] (inputs), V = [N, ns] (targets)."""
        a, (x, h1, h2, p) = self.forward(theta)
        f = [U, self.ras(U)]
        f.append(self.ras(self.N @ f[1]))
        c = [(a[:, 2 * k] + 1j * a[:, 2 * k + 1])[:, None] for k in range(3)]
        e = c[0] * f[0] + c[1] * f[1] + c[2] * f[2] - V
        vn = np.sum(np.abs(V) ** 2)
        L = np.sum(np.abs(e) ** 2) / vn
        # dL/d(Re a_k) = 2 Re(conj(e) f_k)/vn, dL/d(Im a_k) = -2 Im(conj(e) f_k)/vn
        ga = np.zeros_like(a)
        for k in range(3):
            G = np.sum(np.conj(e) * f[k], axis=1)
            ga[:, 2 * k] = 2.0 * G.real / vn
            ga[:, 2 * k + 1] = -2.0 * G.imag / vn
        g = {"W3": ga.T @ h2, "b3": ga.sum(0)}
        gz2 = (ga @ p["W3"]) * (1.0 - h2 ** 2)
        g["W2"], g["b2"] = gz2.T @ h1, gz2.sum(0)
        gz1 = (gz2 @ p["W2"]) * (1.0 - h1 ** 2)
        g["W1"], g["b1"] = gz1.T @ x, gz1.sum(0)
        return L, pack(g)

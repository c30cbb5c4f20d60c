"""Pins of the 2D model-problem oracle (Sec. 3): what the mathematics fixes.

* The dense potential (Eq. 8) against a plain double loop.
* The quadtree rules: four groups along the longest dimension at l0, the finest level
  the deepest whose groups average at least P points, leaves partitioning the points.
* Coverage: every ordered pair of points is handled exactly once, by the near field
  at the finest level or by one interaction list at one level.
* The NESA product (Eqs. 9-14) against the dense one: the error falls steadily with Q
  (a dropped or transposed stage leaves an O(1) error at every Q).
* Bilinear symmetry: U = V^T, B = C^T and D(off)^T = D(-off) make the NESA matrix
  symmetric up to rounding.
* Radiation alone: the equivalent charges of a group reproduce its field far away.
"""
import math

import numpy as np
import pytest

from oracle.nesa2d import Nesa2D, Tree2D, dense_matvec, dense_rows, log_kernel
from workloads.curve2d import charges, curve_points


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_dense_potential_vs_double_loop():
    x = curve_points(50, seed=3)
    q = charges(50, seed=3)
    ref = [sum(-math.log(math.hypot(x[i, 0] - x[j, 0], x[i, 1] - x[j, 1])) * q[j] for j in range(50) if j != i)
           for i in range(50)]
    assert rel(dense_matvec(x, q), ref) < 1e-13
    assert rel(dense_rows(x, q, [0, 17, 49]), [ref[0], ref[17], ref[49]]) < 1e-13


def test_quadtree_rules():
    x = curve_points(3000, seed=1)
    P = 30
    t = Tree2D(x, P)
    assert t.l0 == 2 and t.width(t.l0) == pytest.approx(float((x.max(0) - x.min(0)).max()) / 4)
    assert len(x) / len(t.boxes[t.L]) >= P
    assert len(x) / len(t._occupied(t.L + 1)) < P
    pts = np.sort(np.concatenate(list(t.leaf_points.values())))
    assert np.array_equal(pts, np.arange(len(x)))  # the leaves partition the points
    assert sorted(t.leaf_points) == t.boxes[t.L]
    ij = t.coords(t.L)
    for b, idx in t.leaf_points.items():
        assert (ij[idx] == np.array(b)).all()


def test_every_pair_covered_once():
    x = curve_points(600, seed=5)
    t = Tree2D(x, 10)
    n = len(x)
    count = np.zeros((n, n), np.int64)
    for a in t.boxes[t.L]:
        for b in t.near(t.L, a):
            count[np.ix_(t.leaf_points[a], t.leaf_points[b])] += 1
    for l in range(t.l0, t.L + 1):
        ij = t.coords(l)
        members = {}
        for p in range(n):
            members.setdefault((int(ij[p, 0]), int(ij[p, 1])), []).append(p)
        for a in t.boxes[l]:
            for b in t.interaction_list(l, a):
                count[np.ix_(members[a], members[b])] += 1
    assert t.L > t.l0 + 1
    assert (count == 1).all()


def test_nesa_converges_to_dense():
    x = curve_points(3000, seed=1)
    q = charges(3000, seed=1)
    ref = dense_matvec(x, q)
    errs = [rel(Nesa2D(x, 30, Q, pinv_eps=1e-9).matvec(q), ref) for Q in (6, 10, 16, 24)]
    print("2D NESA vs dense, Q = 6, 10, 16, 24:", ["%.2e" % e for e in errs])
    assert all(e2 < e1 / 5 for e1, e2 in zip(errs, errs[1:]))
    assert errs[1] < 1e-3 and errs[-1] < 1e-6


def test_regulariser_reading_does_not_change_the_accuracy():
    """The equivalent-charge fit is Tikhonov-regularised at eps = 1e-9 ||G(T, E)||_F (the
    same rule as the 3D fit).  The error against the dense product at 1e-9 is that of
    the nearly unregularised fit (1e-12) to within 10 %, at every Q of the table."""
    x = curve_points(3000, seed=1)
    q = charges(3000, seed=1)
    ref = dense_matvec(x, q)
    for Q in (10, 16, 24):
        e9 = rel(Nesa2D(x, 30, Q, pinv_eps=1e-9).matvec(q), ref)
        e12 = rel(Nesa2D(x, 30, Q, pinv_eps=1e-12).matvec(q), ref)
        assert abs(e9 - e12) <= 0.1 * e12, (Q, e9, e12)


def test_nesa_matrix_is_symmetric():
    x = curve_points(2000, seed=2)
    o = Nesa2D(x, 25, 12)
    q1, q2 = charges(2000, seed=11), charges(2000, seed=12)
    a, b = float(q1 @ o.matvec(q2)), float(q2 @ o.matvec(q1))
    assert abs(a - b) <= 1e-12 * np.linalg.norm(q1) * np.linalg.norm(o.matvec(q2))
    # the far part alone, and its stages: D(off)^T = D(-off)
    assert rel(o.D(o.tree.L, (2, -3)).T, o.D(o.tree.L, (-2, 3))) < 1e-15


def test_equivalent_charges_reproduce_far_field():
    x = curve_points(3000, seed=4)
    o = Nesa2D(x, 30, 16)
    t = o.tree
    rng = np.random.default_rng(0)
    for b in t.boxes[t.L][::7]:
        qb = rng.uniform(-1, 1, len(t.leaf_points[b]))
        c = t.center(t.L, b)
        w = t.width(t.L)
        ang = rng.uniform(0, 2 * math.pi, 50)
        Y = c + (2.0 + rng.uniform(0, 2, 50))[:, None] * w * np.stack([np.cos(ang), np.sin(ang)], 1)
        far = log_kernel(Y, x[t.leaf_points[b]]) @ qb
        eq = log_kernel(Y, o.E[t.L] + c) @ (o.V(b) @ qb)
        assert rel(eq, far) < 1e-4, b

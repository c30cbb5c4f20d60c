"""Pins of the oracle's EFIE matrix, its near/far split and the naive NESA product.
CPU only; nothing here uses the CUDA path."""
import math

import numpy as np
import pytest

from oracle.efie import efie_rows
from oracle.nesa import NesaOracle, green
from workloads import get_config, random_coefficients


@pytest.fixture(scope="module")
def tiny():
    c = get_config("tiny")
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    Z = efie_rows(c["vertices"], c["triangles"], o.rwg, c["k"])
    return c, o, Z


def test_dense_matrix_is_symmetric(tiny):
    # reciprocity: Z = Z^T (no conjugation) for the Galerkin EFIE
    _, _, Z = tiny
    assert np.abs(Z - Z.T).max() <= 1e-13 * np.abs(Z).max()


def test_near_plus_exact_far_equals_dense(tiny):
    # the near/far split by quadrature-point leaves loses and doubles nothing
    _, o, Z = tiny
    x = random_coefficients(o.n, 1, seed=3)[0]
    y = o.near_matrix() @ x + o.far_exact(x)
    assert np.linalg.norm(y - Z @ x) <= 1e-13 * np.linalg.norm(Z @ x)


def test_near_matrix_sparsity_and_symmetry(tiny):
    _, o, Z = tiny
    N = o.near_matrix()
    assert np.abs(N - N.T).max() <= 1e-13 * np.abs(N).max()
    # entries of pairs whose quadrature points all touch equal the dense entries
    assert np.count_nonzero(N) < N.size


def test_nesa_matches_dense(tiny):
    _, o, Z = tiny
    x = random_coefficients(o.n, 1, seed=4)[0]
    err = np.linalg.norm(o.matvec(x) - Z @ x) / np.linalg.norm(Z @ x)
    assert err < 1e-4


def test_nesa_error_decreases_with_q():
    c = get_config("tiny")
    x = random_coefficients(480, 1, seed=5)[0]
    errs = []
    Z = None
    for q in (36, 64, 100, 144):
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"], q_mode="fixed",
                       q_fixed=q)
        if Z is None:
            Z = efie_rows(c["vertices"], c["triangles"], o.rwg, c["k"])
        far_exact = o.far_exact(x)
        errs.append(np.linalg.norm(o.far_rows(x) - far_exact) / np.linalg.norm(far_exact))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs


def test_nesa_bilinear_symmetry(tiny):
    # U = V^T, B = C^T and D(-o) = D(o)^T make the NESA operator symmetric too
    _, o, _ = tiny
    x = random_coefficients(o.n, 1, seed=6)[0]
    y = random_coefficients(o.n, 1, seed=7)[0]
    a = y @ o.matvec(x)
    b = x @ o.matvec(y)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_pseudo_inverse_and_translation_operator(tiny):
    _, o, _ = tiny
    l = o.L
    A = green(o.k, o.T[l], o.E[l])
    assert np.abs(o.K[l] @ A - np.eye(o.Q[l])).max() < 1e-8
    # D(-off) = D(off)^T
    D1 = o.D(l, (2, 0, -1))
    D2 = o.D(l, (-2, 0, 1))
    assert np.abs(D1 - D2.T).max() <= 1e-15 * np.abs(D1).max()
    # outgoing representation reproduces the field of a point source at a far box
    rng = np.random.default_rng(0)
    w = o.tree.width(l)
    src = (rng.random((5, 3)) - 0.5) * w
    q = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    s = o.K[l] @ (green(o.k, o.T[l], src) @ q)
    far = o.E[l] + np.array([2.0 * w, 0, 0])
    exact = green(o.k, far, src) @ q
    assert np.linalg.norm(green(o.k, far, o.E[l]) @ s - exact) < 1e-3 * np.linalg.norm(exact)


def test_sampled_rows_equal_full_product(tiny):
    _, o, _ = tiny
    x = random_coefficients(o.n, 1, seed=8)[0]
    rows = [0, 17, 250, o.n - 1]
    full = o.matvec(x)
    assert np.abs(o.matvec_rows(x, rows) - full[rows]).max() <= 1e-14 * np.abs(full).max()


@pytest.mark.slow
def test_nesa_matches_dense_c1b_rows():
    c = get_config("C1b")
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    assert o.l0 < o.L  # transfers are exercised
    rows = np.arange(0, o.n, 397)
    x = random_coefficients(o.n, 1, seed=9)[0]
    dense = efie_rows(c["vertices"], c["triangles"], o.rwg, c["k"], rows=rows) @ x
    err = np.linalg.norm(o.matvec_rows(x, rows) - dense) / np.linalg.norm(dense)
    assert err < 1e-4


def test_self_only_singular_mode():
    """singular_mode 'self' (extraction for T = T' only) changes exactly the entries whose
    supports contain two distinct triangles sharing a vertex; every other entry is the
    same number.  Z stays symmetric to rounding, and the plain 7x7 rule on adjacent
    triangles stays within a few per cent of the extracted value overall."""
    from oracle.rwg import build_rwg
    c = get_config("tiny")
    r = build_rwg(c["vertices"], c["triangles"])
    Zt = efie_rows(c["vertices"], c["triangles"], r, c["k"])
    Zs = efie_rows(c["vertices"], c["triangles"], r, c["k"], singular_mode="self")
    T = c["triangles"]
    shares = [[len(set(T[a]) & set(T[b])) > 0 and a != b for b in range(len(T))] for a in range(len(T))]
    n = r["n"]
    adj = np.array([[any(shares[a][b] for a in r["tri"][m] for b in r["tri"][k]) for k in range(n)] for m in range(n)])
    d = np.abs(Zs - Zt)
    assert d[~adj].max() == 0.0
    assert np.count_nonzero(d[adj]) > 0.9 * adj.sum()
    assert np.abs(Zs - Zs.T).max() <= 1e-13 * np.abs(Zs).max()
    assert np.linalg.norm(Zs - Zt) / np.linalg.norm(Zt) < 0.1
